"""Adjoint of the implicit step on the GPU (dm_step_adjoint) against the
oracle's adjoint and against central differences of the GPU step, for a
batch of uneven rods with natural curvature (committed frames held fixed)."""
import numpy as np
import pytest

import workloads
from oracle import OracleSystems
from oracle.adjoint import step_adjoint
from test_gpu_parity import _gpu

pytestmark = pytest.mark.gpu


def _batch(integrator="be"):
    desc, params, kbar = workloads.uneven_rods(n_rods=64, seed=2)
    sub, kb = workloads.subset(desc, [3, 17, 40], kbar)
    return sub, dict(params, integrator=integrator), kb


@pytest.mark.parametrize("integrator", ["be", "midpoint"])
def test_step_adjoint_matches_oracle_adjoint(integrator):
    """The GPU adjoint (for implicit midpoint: over dt/2 at the midpoint
    configuration) against the oracle's (for implicit midpoint: in q_{n+1})."""
    desc, params, kb = _batch(integrator)
    gpu = _gpu(desc, params)
    ora = OracleSystems(desc, params)
    R = len(desc["nodes_per_rod"])
    gpu.set_natural_curvature(0, R, kb)
    ora.set_natural_curvature(0, R, kb)
    for _ in range(3):
        ora.step(1)
    q0, v0 = ora.get_state()
    d1, beta = ora.get_frames()
    ora.step(1)
    q1, _ = ora.get_state()
    rng = np.random.default_rng(0)
    wq, wv = rng.normal(size=len(q0)), rng.normal(size=len(q0))
    ora.set_state(q0, v0)
    ora.set_frames(d1, beta)
    ok, oq, ov = step_adjoint(ora, q1, wq, wv)
    gpu.set_state(q0, v0)
    gpu.set_frames(d1, beta)
    gk, gq, gv = gpu.step_adjoint(q1, wq, wv)
    for a, b in ((gk, ok), (gq, oq), (gv, ov)):
        scale = max(1.0, float(np.abs(b).max()))
        assert np.abs(a - b).max() <= 1e-8 * scale, np.abs(a - b).max() / scale


def test_step_adjoint_kappabar_matches_central_differences():
    desc, params, kb = _batch()
    gpu = _gpu(desc, params)
    R = len(desc["nodes_per_rod"])
    gpu.set_natural_curvature(0, R, kb)
    for _ in range(3):
        gpu.step(1)
    q0, v0 = gpu.get_state()
    d1, beta = gpu.get_frames()
    rng = np.random.default_rng(1)
    wq, wv = rng.normal(size=len(q0)), rng.normal(size=len(q0))

    def loss(k):
        gpu.set_state(q0, v0)
        gpu.set_frames(d1, beta)
        gpu.set_natural_curvature(0, R, k)
        gpu.step(1)
        q1, v1 = gpu.get_state()
        return float(wq @ q1 + wv @ v1), q1

    _, q1 = loss(kb)
    gpu.set_state(q0, v0)
    gpu.set_frames(d1, beta)
    gpu.set_natural_curvature(0, R, kb)
    gk, _, _ = gpu.step_adjoint(q1, wq, wv)
    h = 1e-6
    for i in rng.choice(len(kb), size=8, replace=False):
        for c in (0, 1):
            kp, km = kb.copy(), kb.copy()
            kp[i, c] += h
            km[i, c] -= h
            fd = (loss(kp)[0] - loss(km)[0]) / (2 * h)
            assert abs(fd - gk[i, c]) <= 1e-5 * max(1.0, abs(fd)), (i, c, fd, gk[i, c])


def _rollout_case(T=8, integrator="be"):
    from paper_2311_18126_gb300 import dismech as dmx
    desc, params, kb = _batch(integrator)
    gpu = dmx.System(desc, params)
    R = len(desc["nodes_per_rod"])
    gpu.set_natural_curvature(0, R, kb)
    for _ in range(2):
        gpu.step(1)
    q0, v0 = gpu.get_state()
    frames = gpu.get_frames()
    rng = np.random.default_rng(2)
    kseq = np.repeat(kb[None], T, axis=0) + rng.normal(scale=0.01, size=(T,) + kb.shape)
    return gpu, q0, v0, frames, kseq


@pytest.mark.parametrize("integrator", ["be", "midpoint"])
def test_rollout_gradient_against_central_differences(integrator):
    """Gradient of a trajectory loss through 8 steps (checkpoints every 3
    steps, the frame chain included) against central differences of the GPU
    rollout.  Without the frame chain the errors were 18-26 %."""
    import torch
    from paper_2311_18126_gb300.adjoint import rollout
    gpu, q0, v0, frames, kseq = _rollout_case(integrator=integrator)
    rng = np.random.default_rng(3)
    w = rng.normal(size=(kseq.shape[0], len(q0)))

    def loss_np(k, q, v):
        x = rollout(gpu, torch.from_numpy(k), torch.from_numpy(q), torch.from_numpy(v), frames, 3)
        return float((x.numpy() * w).sum())

    kt = torch.tensor(kseq, requires_grad=True)
    qt = torch.tensor(q0, requires_grad=True)
    vt = torch.tensor(v0, requires_grad=True)
    x = rollout(gpu, kt, qt, vt, frames, 3)
    (x * torch.from_numpy(w)).sum().backward()
    gk = kt.grad.numpy()
    errs = []
    h = 1e-6
    for (t, i, c) in [(0, 5, 0), (2, 40, 1), (5, 100, 0), (7, 7, 1)]:
        kp, km = kseq.copy(), kseq.copy()
        kp[t, i, c] += h
        km[t, i, c] -= h
        fd = (loss_np(kp, q0, v0) - loss_np(km, q0, v0)) / (2 * h)
        errs.append(abs(fd - gk[t, i, c]) / max(abs(fd), 1e-3 * np.abs(gk).max()))
    # initial velocities of free DOFs (the frames of the initial state stay
    # as given: positions would move its tangents under fixed directors)
    gv0 = vt.grad.numpy()
    for i in rng.choice(np.flatnonzero(~gpu.fixed_mask()), size=4, replace=False):
        vp, vm = v0.copy(), v0.copy()
        vp[i] += 1e-5
        vm[i] -= 1e-5
        fd = (loss_np(kseq, q0, vp) - loss_np(kseq, q0, vm)) / 2e-5
        errs.append(abs(fd - gv0[i]) / max(abs(fd), 1e-3 * np.abs(gv0).max()))
    print("rollout gradient relative errors vs central differences (%s):" % integrator,
          ["%.2e" % e for e in errs])
    assert max(errs) < 2e-4


def test_calibration_reduces_trajectory_loss():
    """Gradient descent on per-step natural curvatures towards a target
    trajectory made by the solver itself from other controls."""
    from paper_2311_18126_gb300.adjoint import calibrate
    gpu, q0, v0, frames, kseq = _rollout_case(T=10)
    R = gpu.n_rods
    gpu.set_state(q0, v0)
    gpu.set_frames(*frames)
    target = []
    for t in range(kseq.shape[0]):
        gpu.set_natural_curvature(0, R, kseq[t])
        gpu.step(1, stats=False)
        target.append(gpu.get_state()[0])
    target = np.array(target)
    k0 = np.zeros_like(kseq)
    kfit, losses = calibrate(gpu, target, k0, q0, v0, frames, iters=8, lr=None,
                             checkpoint_every=4)
    print("calibration losses:", ["%.3e" % l for l in losses])
    assert losses[-1] < 0.1 * losses[0]


def _stars():
    desc, params, gait = workloads.star_robots(n_robots=3, seed=3, nodes_per_limb=8)
    return desc, params, gait


@pytest.mark.parametrize("integrator", ["be", "midpoint"])
def test_step_adjoint_star_robots_matches_oracle_adjoint(integrator):
    """Limbed robots on the ground (joints, contact, friction: J not
    symmetric, solved transposed by the condensation kernels)."""
    desc, params, gait = _stars()
    params = dict(params, integrator=integrator)
    R = len(desc["nodes_per_rod"])
    gpu = _gpu(desc, params)
    ora = OracleSystems(desc, params)
    for k in range(4):
        kb = workloads.gait_kbar(gait, k * params["dt"])
        ora.set_natural_curvature(0, R, kb)
        ora.step(1)
    kb = workloads.gait_kbar(gait, 4 * params["dt"])
    ora.set_natural_curvature(0, R, kb)
    gpu.set_natural_curvature(0, R, kb)
    q0, v0 = ora.get_state()
    d1, beta = ora.get_frames()
    ora.step(1)
    q1, _ = ora.get_state()
    rng = np.random.default_rng(5)
    wq, wv = rng.normal(size=len(q0)), rng.normal(size=len(q0))
    ora.set_state(q0, v0)
    ora.set_frames(d1, beta)
    ok, oq, ov = step_adjoint(ora, q1, wq, wv)
    gpu.set_state(q0, v0)
    gpu.set_frames(d1, beta)
    gk, gq, gv = gpu.step_adjoint(q1, wq, wv)
    for a, b in ((gk, ok), (gq, oq), (gv, ov)):
        scale = max(1.0, float(np.abs(b).max()))
        assert np.abs(a - b).max() <= 1e-8 * scale, np.abs(a - b).max() / scale


def test_star_robot_rollout_gradient_against_central_differences():
    """Six steps of star robots on the ground with the gait as controls:
    rollout gradient (frame chain, friction, joints) against central
    differences of the GPU rollout."""
    import torch
    from paper_2311_18126_gb300 import dismech as dmx
    from paper_2311_18126_gb300.adjoint import rollout
    desc, params, gait = _stars()
    R = len(desc["nodes_per_rod"])
    gpu = dmx.System(desc, params)
    dt = params["dt"]
    for k in range(3):
        gpu.set_natural_curvature(0, R, workloads.gait_kbar(gait, k * dt))
        gpu.step(1)
    q0, v0 = gpu.get_state()
    frames = gpu.get_frames()
    T = 6
    kseq = np.stack([workloads.gait_kbar(gait, (3 + t) * dt) for t in range(T)])
    rng = np.random.default_rng(6)
    w = rng.normal(size=(T, len(q0)))
    kt = torch.tensor(kseq, requires_grad=True)
    x = rollout(gpu, kt, torch.from_numpy(q0), torch.from_numpy(v0), frames, 4)
    (x * torch.from_numpy(w)).sum().backward()
    gk = kt.grad.numpy()

    def loss_np(k):
        x = rollout(gpu, torch.from_numpy(k), torch.from_numpy(q0), torch.from_numpy(v0),
                    frames, 4)
        return float((x.numpy() * w).sum())

    errs = []
    h = 1e-6
    for (t, i, c) in [(0, 2, 0), (2, 20, 1), (4, 40, 0), (5, 9, 0)]:
        kp, km = kseq.copy(), kseq.copy()
        kp[t, i, c] += h
        km[t, i, c] -= h
        fd = (loss_np(kp) - loss_np(km)) / (2 * h)
        errs.append(abs(fd - gk[t, i, c]) / max(abs(fd), 1e-3 * np.abs(gk).max()))
    print("star-robot rollout gradient relative errors:", ["%.2e" % e for e in errs])
    assert max(errs) < 1e-3


@pytest.mark.parametrize("integrator", ["be", "midpoint"])
def test_step_adjoint_coil_with_contact_matches_oracle_adjoint(integrator):
    """A self-contacting coil (edge-edge IMC contact, no friction): the
    transposed dense-band LU on the GPU against the oracle's adjoint, at a
    step where turns touch."""
    from test_gpu_contact import _short_coil, _oracle_active_pairs
    desc, params = _short_coil()
    params = dict(params, integrator=integrator)
    gpu = _gpu(desc, params)
    ora = OracleSystems(desc, params)
    for _ in range(36):
        ora.step(1)
    q0, v0 = ora.get_state()
    d1, beta = ora.get_frames()
    ora.step(1)
    assert _oracle_active_pairs(ora, params) > 0
    q1, _ = ora.get_state()
    rng = np.random.default_rng(7)
    wq, wv = rng.normal(size=len(q0)), rng.normal(size=len(q0))
    ora.set_state(q0, v0)
    ora.set_frames(d1, beta)
    ok, oq, ov = step_adjoint(ora, q1, wq, wv)
    gpu.set_state(q0, v0)
    gpu.set_frames(d1, beta)
    gk, gq, gv = gpu.step_adjoint(q1, wq, wv)
    for a, b in ((gk, ok), (gq, oq), (gv, ov)):
        scale = max(1.0, float(np.abs(b).max()))
        assert np.abs(a - b).max() <= 1e-8 * scale, np.abs(a - b).max() / scale


@pytest.mark.parametrize("integrator", ["be", "midpoint"])
def test_frame_chain_kernel_matches_a_numpy_restatement(integrator):
    """dm_adjoint_frame_chain (the rollout adjoint's frame chain on the GPU)
    against the same chain written out in NumPy: sigma at every free twist
    angle, the carried frame adjoint, and the tangent term on the node
    positions, on random states of three rods (one with fixed DOFs).  For
    implicit midpoint the step energy sees the frames transported to the
    tangents of (q + q_next)/2."""
    import torch
    desc, params, _ = workloads.uneven_rods(n_rods=3, seed=9, n_min=6, n_max=9)
    params = dict(params, integrator=integrator)
    gpu = _gpu(desc, params)
    npr = np.asarray(desc["nodes_per_rod"])
    fixed = gpu.fixed_mask()
    n = gpu.n_state
    rng = np.random.default_rng(3)
    q = gpu.get_state()[0]
    pos = np.ones(n, bool)
    off = 0
    for N in npr:
        pos[off + 4 * np.arange(N - 1) + 3] = False
        off += 4 * N - 1
    jitter = lambda s: q + s * rng.standard_normal(n) * pos
    q_prev, q_next = jitter(0.01), jitter(0.01)
    gq, gv, gv0 = rng.standard_normal((3, n))
    phi0 = rng.standard_normal(int(np.sum(npr - 1)))
    gq0 = rng.standard_normal(n)
    mid = integrator == "midpoint"
    dt = params["dt"] / 2 if mid else params["dt"]

    # NumPy restatement
    def tangents(x):
        ts, ils, off = [], [], 0
        for N in npr:
            X = np.stack([x[off + 4 * i:off + 4 * i + 3] for i in range(N)])
            e = X[1:] - X[:-1]
            l = np.linalg.norm(e, axis=1)
            ts.append(e / l[:, None])
            ils.append(1.0 / l)
            off += 4 * N - 1
        return np.concatenate(ts), np.concatenate(ils)

    hol = lambda a, b: np.cross(a, b) / (1.0 + np.sum(a * b, axis=1))[:, None]
    th = np.concatenate([o + 4 * np.arange(N - 1) + 3
                         for o, N in zip(np.concatenate([[0], np.cumsum(4 * npr - 1)])[:-1], npr)])
    if mid:
        sigma = np.where(~fixed[th], -(2 * gq[th] + (gv[th] - gv0[th]) / dt), 0.0)
    else:
        sigma = np.where(~fixed[th], -((gq[th] + gv[th] / dt) - gv0[th] / dt), 0.0)
    phi = phi0 + sigma
    t, il = tangents(q)
    if mid:
        # phi0 on the committed transport t -> t(q_next), sigma on the
        # transport t -> t((q + q_next)/2) the step energy sees
        gt = -(phi0[:, None] * hol(t, tangents(q_next)[0])
               + sigma[:, None] * hol(t, tangents(0.5 * (q + q_next))[0])
               + phi[:, None] * hol(tangents(q_prev)[0], t))
    else:
        w = hol(t, tangents(q_next)[0]) + hol(tangents(q_prev)[0], t)
        gt = -phi[:, None] * w
    g = (gt - np.sum(gt * t, axis=1)[:, None] * t) * il[:, None]
    want = gq0.copy()
    off, e0 = 0, 0
    for N in npr:
        for i in range(N - 1):
            want[off + 4 * (i + 1):off + 4 * (i + 1) + 3] += g[e0 + i]
            want[off + 4 * i:off + 4 * i + 3] -= g[e0 + i]
        e0 += N - 1
        off += 4 * N - 1

    T = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    tphi, tgq0 = T(phi0), T(gq0)
    gpu.adjoint_frame_chain(T(q_prev), T(q), T(q_next), T(gq), T(gv), T(gv0), tphi, tgq0)
    torch.cuda.synchronize()
    np.testing.assert_allclose(tphi.cpu().numpy(), phi, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(tgq0.cpu().numpy(), want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    assert np.any(fixed[th])  # the clamped first twist angles are exercised


def test_step_adjoint_rods_in_contact_on_the_ground_matches_oracle_adjoint():
    """Two rods of one contact group lying across each other on the ground
    (edge-edge contact without pair friction, ground contact with friction):
    the transposed contact LU with the ground terms, and the ground
    friction's dependence on x_n, against the oracle's adjoint."""
    from test_gpu_contact import _crossing_rods_on_ground, _oracle_active_pairs
    desc, params = _crossing_rods_on_ground()
    params = dict(params, pair_mu=0.0)
    gpu = _gpu(desc, params)
    ora = OracleSystems(desc, params)
    for _ in range(5):
        ora.step(1)
    q0, v0 = ora.get_state()
    d1, beta = ora.get_frames()
    ora.step(1)
    assert _oracle_active_pairs(ora, params) > 0
    q1, _ = ora.get_state()
    rng = np.random.default_rng(11)
    wq, wv = rng.normal(size=len(q0)), rng.normal(size=len(q0))
    ora.set_state(q0, v0)
    ora.set_frames(d1, beta)
    ok, oq, ov = step_adjoint(ora, q1, wq, wv)
    gpu.set_state(q0, v0)
    gpu.set_frames(d1, beta)
    gk, gq, gv = gpu.step_adjoint(q1, wq, wv)
    for a, b in ((gk, ok), (gq, oq), (gv, ov)):
        scale = max(1.0, float(np.abs(b).max()))
        assert np.abs(a - b).max() <= 1e-8 * scale, np.abs(a - b).max() / scale
