"""Differentiable rollouts of the implicit step: per-step natural-curvature
controls and the initial state -> the trajectory of node positions, with the
gradient by the library's step adjoint (dm_step_adjoint) and checkpoints.

The forward pass stores the state and frames every ``checkpoint_every``
steps; the backward pass re-simulates each segment from its checkpoint,
keeping the per-step states of that segment only, and runs the step adjoint
backwards through it.  Any system the step adjoint accepts: single rods,
rods in edge-edge contact without pair friction, rod networks and rods on
the ground.

The frame chain: the step adjoint holds the committed reference frames
fixed, but each step's frames come from the earlier tangents by
time-parallel transport (Sec. III).  A rotation of edge e's committed
director acts on the energy like a shift of its twist angle, so its adjoint
sigma_e = -lambda . K[:, theta_e] = -(gbar_theta - M_theta/dt^2 lambda_theta)
needs only the step adjoint's own quantities, and moving a tangent rotates
the directors transported from or to it by -w . dt with
w(a, b) = (a x b)/(1 + a . b) (the holonomy of the geodesic triangle; both
for the source and the target of a transport).  With Phi_n the committed
frame angles of step n:  Phibar_n = Phibar_{n+1} + sigma_{n+1} and
dL/dt_n = -Phibar_n [w(t_n, t_{n+1}) + w(t_{n-1}, t_n)], carried to the
node positions through t = e/|e|.  The directors of the initial state are
taken as transported along with its tangents.
"""
import numpy as np
import torch

from . import dismech as dmx


def _edge_tangents(q, npr):
    """Unit tangents [E, 3] and inverse lengths [E] of every edge, from a
    state in the dm_get_state layout."""
    ts, ils = [], []
    off = 0
    for N in npr:
        x = q[off:off + 4 * N - 1]
        X = np.stack([x[4 * i:4 * i + 3] for i in range(N)])
        e = X[1:] - X[:-1]
        l = np.linalg.norm(e, axis=1)
        ts.append(e / l[:, None])
        ils.append(1.0 / l)
        off += 4 * N - 1
    return np.concatenate(ts), np.concatenate(ils)


def _hol(a, b):
    """w(a, b) = (a x b) / (1 + a . b) per edge."""
    return np.cross(a, b) / (1.0 + np.sum(a * b, axis=1))[:, None]


def _theta_index(npr):
    """Layout index of every edge's twist angle."""
    idx = []
    off = 0
    for N in npr:
        idx.append(off + 4 * np.arange(N - 1) + 3)
        off += 4 * N - 1
    return np.concatenate(idx)


def _tangent_to_positions(gt, il, t, npr, n):
    """dL/dt per edge -> dL/dq on the node positions (t = e/|e|)."""
    g = gt - np.sum(gt * t, axis=1)[:, None] * t
    g = g * il[:, None]
    out = np.zeros(n)
    off = 0
    e0 = 0
    for N in npr:
        for i in range(N - 1):
            out[off + 4 * (i + 1):off + 4 * (i + 1) + 3] += g[e0 + i]
            out[off + 4 * i:off + 4 * i + 3] -= g[e0 + i]
        e0 += N - 1
        off += 4 * N - 1
    return out


def _layout_positions(npr):
    """Boolean mask of the position entries in the dm_get_state layout."""
    mask = []
    for N in npr:
        m = np.ones(4 * N - 1, bool)
        m[3::4] = False
        mask.append(m)
    return np.concatenate(mask)


class Rollout(torch.autograd.Function):
    """x = Rollout.apply(kbar_seq, q0, v0, system, frames0, checkpoint_every)

    kbar_seq: [T, slots, 2] float64 (natural curvature applied before each
    step), q0, v0: [n] float64 (dm_get_state layout), frames0: (d1, beta) of
    the initial state.  Returns the states q_1..q_T as [T, n] float64; the
    gradient flows to kbar_seq, q0 and v0."""

    @staticmethod
    def forward(ctx, kbar_seq, q0, v0, system, frames0, checkpoint_every):
        T = kbar_seq.shape[0]
        R = system.n_rods
        kb = kbar_seq.detach().cpu().numpy()
        q = q0.detach().cpu().numpy().copy()
        v = v0.detach().cpu().numpy().copy()
        system.set_state(q, v)
        system.set_frames(*frames0)
        ckpt = {}
        out = np.zeros((T, len(q)))
        qprev = None
        for t in range(T):
            if t % checkpoint_every == 0:
                ckpt[t] = (q.copy(), v.copy()) + tuple(a.copy() for a in system.get_frames()) \
                    + (None if qprev is None else qprev.copy(),)
            system.set_natural_curvature(0, R, kb[t])
            system.step(1, stats=False)
            qprev = q
            q, v = system.get_state()
            out[t] = q
        ctx.system = system
        ctx.kb = kb
        ctx.ckpt = ckpt
        ctx.every = checkpoint_every
        ctx.T = T
        return torch.from_numpy(out)

    @staticmethod
    def backward(ctx, gx):
        system, kb, T, every = ctx.system, ctx.kb, ctx.T, ctx.every
        R = system.n_rods
        gx = gx.detach().cpu().numpy()
        n = gx.shape[1]
        npr = np.asarray(system._npr)
        dt = system.dt
        th = _theta_index(npr)
        thfree = ~system.fixed_mask()[th]
        gk = np.zeros_like(kb)
        carry_q = np.zeros(n)
        carry_v = np.zeros(n)
        carry_phi = np.zeros(len(th))
        starts = sorted(ctx.ckpt)
        for s0 in reversed(starts):
            s1 = min(s0 + every, T)
            q, v, d1, beta, qprev = ctx.ckpt[s0]
            # re-simulate the segment, keeping its per-step states
            seg = []
            system.set_state(q, v)
            system.set_frames(d1, beta)
            for t in range(s0, s1):
                frames = system.get_frames()
                qs, vs = system.get_state()
                system.set_natural_curvature(0, R, kb[t])
                system.step(1, stats=False)
                qn, _ = system.get_state()
                seg.append((qs, vs, frames, qn, qprev))
                qprev = qs
            for t in range(s1 - 1, s0 - 1, -1):
                qs, vs, frames, qn, qp = seg[t - s0]
                system.set_state(qs, vs)
                system.set_frames(*frames)
                system.set_natural_curvature(0, R, kb[t])
                gq = gx[t] + carry_q
                gv = carry_v
                gkt, gq0, gv0 = system.step_adjoint(qn, gq, gv)
                gk[t] = gkt
                # frame chain (module docstring)
                sigma = np.where(thfree, -((gq[th] + gv[th] / dt) - gv0[th] / dt), 0.0)
                phibar = carry_phi + sigma
                tt, il = _edge_tangents(qs, npr)
                t1, _ = _edge_tangents(qn, npr)
                w = _hol(tt, t1)
                if qp is not None:
                    w = w + _hol(_edge_tangents(qp, npr)[0], tt)
                gq0 = gq0 + _tangent_to_positions(-phibar[:, None] * w, il, tt, npr, n)
                carry_q, carry_v, carry_phi = gq0, gv0, phibar
        return torch.from_numpy(gk), torch.from_numpy(carry_q), torch.from_numpy(carry_v), \
            None, None, None


def rollout(system, kbar_seq, q0, v0, frames0, checkpoint_every=50):
    """Differentiable trajectory q_1..q_T (see Rollout)."""
    return Rollout.apply(kbar_seq, q0, v0, system, frames0, checkpoint_every)


def calibrate(system, target, kbar_init, q0, v0, frames0, iters=20, lr=None,
              checkpoint_every=50):
    """Gradient descent on the per-step natural curvatures so that the node
    positions follow `target` ([T, n], layout order; positions only enter
    the loss): the calibration loop of the paper with adjoint gradients in
    place of finite differences, with a backtracking step length (lr = None:
    the first trial step is loss / |grad|^2).  Returns (kbar, losses)."""
    pos = torch.from_numpy(_layout_positions(
        np.asarray(system._npr)).astype(np.float64))
    kb = torch.tensor(np.asarray(kbar_init, np.float64), requires_grad=True)
    q0t = torch.as_tensor(q0, dtype=torch.float64)
    v0t = torch.as_tensor(v0, dtype=torch.float64)
    tgt = torch.as_tensor(target, dtype=torch.float64)
    losses = []

    def evaluate(k):
        x = rollout(system, k, q0t, v0t, frames0, checkpoint_every)
        return (((x - tgt) ** 2) * pos).sum()

    step = lr
    for _ in range(iters):
        loss = evaluate(kb)
        losses.append(float(loss.detach()))
        g, = torch.autograd.grad(loss, [kb])
        gg = float((g * g).sum())
        if gg == 0.0:
            break
        if step is None:
            step = losses[-1] / gg  # first trial: the Gauss-Newton scale of a quadratic loss
        # backtracking on the step length (halving until the loss decreases)
        with torch.no_grad():
            for _ in range(20):
                trial = kb - step * g
                try:
                    lt = float(evaluate(trial))
                except dmx.DismechError:  # too long a step for Newton: shorter
                    lt = float("inf")
                if lt < losses[-1]:
                    kb.copy_(trial)
                    step *= 1.5
                    break
                step *= 0.5
    return kb.detach().numpy(), losses
