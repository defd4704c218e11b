"""Adjoint of one implicit step for the oracle (TEST INFRASTRUCTURE ONLY,
see ``oracle/__init__.py``).

The step solves f(q_{n+1}; q_n, qdot_n, kappabar) = 0 (Sec. III-C, Eq. 15)
and sets qdot_{n+1} = (q_{n+1} - q_n)/dt.  For a loss L(q_{n+1}, qdot_{n+1}),
by the implicit function theorem with J = df/dq_{n+1}:
    J^T lambda = dL/dq_{n+1} + dL/dqdot_{n+1} / dt,
    dL/dp = -lambda . df/dp  for p in (kappabar, q_n, qdot_n),
plus -dL/dqdot_{n+1} / dt on q_n from the velocity update.  The committed
reference frames are held fixed.  J is the oracle's autograd Jacobian;
lambda . df/dp is a vector-Jacobian product of the oracle's residual.
Fixed DOFs keep q_{n+1} = q_n: they pass dL/dq_{n+1} through and get no
velocity gradient.

Implicit midpoint (the textbook rule, f = 2M/dt^2 (q_{n+1} - q_n - dt qdot_n)
- F((q_n + q_{n+1})/2), qdot_{n+1} = 2 (q_{n+1} - q_n)/dt - qdot_n): the same
with dL/dqdot_{n+1} entering as 2/dt, and the velocity update adding
-2/dt dL/dqdot_{n+1} on q_n and -dL/dqdot_{n+1} on qdot_n.
"""
import numpy as np
import torch

DT = torch.float64


def step_adjoint(osys, q_next, gq, gv):
    """osys holds step n (state and frames); q_next, gq, gv in the
    get_state layout.  Returns (dL/dkappabar [slots, 2], dL/dq_n, dL/dqdot_n)
    with the kappabar slots in the set_natural_curvature layout.  A joint
    node appears once per rod in the layout: its loss gradients are summed
    over the copies and its output gradients go to its first copy (zeros in
    the others).  Backward Euler or implicit midpoint."""
    dt = osys.dt
    cv = 2.0 / dt if osys.midpoint else 1.0 / dt  # dqdot_{n+1} / dq_{n+1}
    maps = osys._rod_maps()
    n_slots = int(np.sum(osys.npr - 2))
    gk = np.zeros((n_slots, 2))
    gq0 = np.zeros(len(q_next))
    gv0 = np.zeros(len(q_next))
    slot0 = np.concatenate([[0], np.cumsum(osys.npr - 2)])
    # layout slices per system
    offs = {}
    off = 0
    for (r, si, idx) in maps:
        offs.setdefault(si, []).append((off, idx))
        off += len(idx)
    for si, parts in offs.items():
        s = osys.systems[si]
        q = s.q.clone()
        g_q = torch.zeros(s.n, dtype=DT)
        g_v = torch.zeros(s.n, dtype=DT)
        seen = np.zeros(s.n, bool)
        for (o, idx) in parts:
            k = len(idx)
            new = ~seen[idx]
            ti = torch.as_tensor(idx[new])
            q[ti] = torch.as_tensor(q_next[o:o + k][new], dtype=DT)
            # a loss on a shared node counts once per copy in the layout
            g_q.index_add_(0, torch.as_tensor(idx), torch.as_tensor(gq[o:o + k], dtype=DT))
            g_v.index_add_(0, torch.as_tensor(idx), torch.as_tensor(gv[o:o + k], dtype=DT))
            seen[idx] = True
        _, _, J = osys.residual(s, q, s.q, s.v, need_jac=True)
        gbar = torch.where(s.fixed, torch.zeros_like(g_q), g_q + cv * g_v)
        lam = torch.as_tensor(np.linalg.solve(J.numpy().T, gbar.numpy()))
        keep = (s.kbar1, s.kbar2)
        kb1 = s.kbar1.clone().requires_grad_(True)
        kb2 = s.kbar2.clone().requires_grad_(True)
        qn = s.q.clone().requires_grad_(True)
        vn = s.v.clone().requires_grad_(True)
        s.kbar1, s.kbar2 = kb1, kb2
        try:
            f, _, _ = osys.residual(s, q, qn, vn, need_jac=False)
            d1, d2, dqn, dvn = torch.autograd.grad(f, [kb1, kb2, qn, vn], grad_outputs=lam,
                                                   allow_unused=True)
        finally:
            s.kbar1, s.kbar2 = keep
        z = torch.zeros(s.n, dtype=DT)
        dqn = z if dqn is None else dqn
        dvn = z if dvn is None else dvn
        a_q0 = torch.where(s.fixed, g_q, -dqn - cv * g_v)
        a_v0 = torch.where(s.fixed, torch.zeros_like(g_v),
                           -dvn - g_v if osys.midpoint else -dvn)
        done = np.zeros(s.n, bool)
        for (o, idx) in parts:
            k = len(idx)
            ti = torch.as_tensor(idx)
            firstc = ~done[idx]
            gq0[o:o + k] = np.where(firstc, a_q0[ti].numpy(), 0.0)
            gv0[o:o + k] = np.where(firstc, a_v0[ti].numpy(), 0.0)
            done[idx] = True
        for kk, gst in enumerate(s.st):
            slot = osys.st_rodslot[gst]
            if slot == -1:
                continue
            rr, j = slot
            gk[slot0[rr] + j, 0] = -float(d1[kk]) if d1 is not None else 0.0
            gk[slot0[rr] + j, 1] = -float(d2[kk]) if d2 is not None else 0.0
    return gk, gq0, gv0
