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
taken as transported along with its tangents.  Implicit midpoint takes each
step's energy at (q_n + q_{n+1})/2, with the frames transported to its
tangents; the library's frame chain splits the transport out of t_n
accordingly (dm_adjoint_frame_chain).
"""
import numpy as np
import torch

from . import dismech as dmx


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
    the initial state.  Returns the states q_1..q_T as [T, n] float64 on the
    device of q0; the gradient flows to kbar_seq, q0 and v0.  Every state,
    checkpoint and gradient of the forward and backward passes stays in GPU
    memory; the frame chain runs in the library (dm_adjoint_frame_chain)."""

    @staticmethod
    def forward(ctx, kbar_seq, q0, v0, system, frames0, checkpoint_every):
        dev = torch.device("cuda")
        f64 = dict(device=dev, dtype=torch.float64)
        T = kbar_seq.shape[0]
        R = system.n_rods
        kb = kbar_seq.detach().to(**f64).contiguous()
        q = q0.detach().to(**f64).clone()
        v = v0.detach().to(**f64).clone()
        d1 = torch.as_tensor(np.asarray(frames0[0]), **f64).contiguous()
        beta = torch.as_tensor(np.asarray(frames0[1]), **f64).contiguous()
        system.set_state(q, v)
        system.set_frames(d1, beta)
        ckpt = {}
        out = torch.empty((T, q.numel()), **f64)
        qprev = None
        for t in range(T):
            if t % checkpoint_every == 0:
                fr = system.get_frames(torch.empty_like(d1), torch.empty_like(beta))
                ckpt[t] = (q, v) + fr + (qprev,)
            system.set_natural_curvature(0, R, kb[t])
            system.step(1, stats=False)
            qprev = q
            q, v = system.get_state(torch.empty_like(q), torch.empty_like(v))
            out[t] = q
        ctx.system = system
        ctx.kb = kb
        ctx.ckpt = ckpt
        ctx.every = checkpoint_every
        ctx.T = T
        ctx.devices = (kbar_seq.device, q0.device, v0.device)
        ctx.frame_shapes = (d1.shape, beta.shape)
        return out.to(q0.device)

    @staticmethod
    def backward(ctx, gx):
        system, kb, T, every = ctx.system, ctx.kb, ctx.T, ctx.every
        R = system.n_rods
        gx = gx.detach().to(device="cuda", dtype=torch.float64)
        n = gx.shape[1]
        gk = torch.zeros_like(kb)
        carry_q = torch.zeros(n, dtype=torch.float64, device="cuda")
        carry_v = torch.zeros_like(carry_q)
        carry_phi = torch.zeros(system.n_edges, dtype=torch.float64, device="cuda")
        d1_shape, beta_shape = ctx.frame_shapes
        for s0 in reversed(sorted(ctx.ckpt)):
            s1 = min(s0 + every, T)
            q, v, d1, beta, qprev = ctx.ckpt[s0]
            # re-simulate the segment, keeping its per-step states and frames
            seg = []
            system.set_state(q, v)
            system.set_frames(d1, beta)
            for t in range(s0, s1):
                fr = system.get_frames(torch.empty(d1_shape, dtype=torch.float64, device="cuda"),
                                       torch.empty(beta_shape, dtype=torch.float64,
                                                   device="cuda"))
                system.set_natural_curvature(0, R, kb[t])
                system.step(1, stats=False)
                qn, vn = system.get_state(torch.empty_like(q), torch.empty_like(v))
                seg.append((q, v, fr, qn, qprev))
                qprev, q, v = q, qn, vn
            for t in range(s1 - 1, s0 - 1, -1):
                qs, vs, frames, qn, qp = seg[t - s0]
                system.set_state(qs, vs)
                system.set_frames(*frames)
                system.set_natural_curvature(0, R, kb[t])
                gq = gx[t] + carry_q
                gv = carry_v
                gkt, gq0, gv0 = system.step_adjoint(qn, gq, gv)
                gk[t] = gkt
                # frame chain (module docstring): carry_phi and gq0 in place
                system.adjoint_frame_chain(qp, qs, qn, gq, gv, gv0, carry_phi, gq0)
                carry_q, carry_v = gq0, gv0
        dk, dq, dv = ctx.devices
        return gk.to(dk), carry_q.to(dq), carry_v.to(dv), None, None, None


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
