"""GPU vs oracle for the general path: rods joined at elastic joints
(Sec. III-D), ground contact with smooth Coulomb friction (Sec. III-B,
Eq. 10-13), and the limb/border block solve.  Identical initial states,
element-by-element comparison of the per-rod state after every step."""
import math

import numpy as np
import pytest

import workloads
from oracle import OracleSystems
from test_gpu_parity import _assert_close, _gpu

pytestmark = pytest.mark.gpu


def _run(desc, params, steps, rel, kbar_fn=None, nrods=None):
    gpu = _gpu(desc, params)
    ora = OracleSystems(desc, params)
    npr = desc["nodes_per_rod"]
    L = max(1.0, float(np.max(np.abs(desc["x0"]))))
    for k in range(steps):
        if kbar_fn is not None:
            kb = kbar_fn(k * params["dt"])
            gpu.set_natural_curvature(0, nrods, kb)
            ora.set_natural_curvature(0, nrods, kb)
        gpu.step(1)
        st = ora.step(1)
        assert all(x[0] == 0 for x in st), st
        qg, vg = gpu.get_state()
        qo, vo = ora.get_state()
        _assert_close(qg, qo, npr, L, rel)
        # identical states for the next step (per-step parity)
        d1, beta = ora.get_frames()
        gpu.set_state(qo, vo)
        gpu.set_frames(d1, beta)
    return gpu, ora


def test_star_robots_on_ground_with_gait():
    desc, params, gait = workloads.star_robots(n_robots=3, seed=3, nodes_per_limb=8)
    R = len(desc["nodes_per_rod"])
    _run(desc, params, 6, 1e-10, lambda t: workloads.gait_kbar(gait, t), R)


def test_joined_chain_without_ground():
    # two rods joined end to end plus a rod joined to their junction: a
    # T-shaped network with a free end swinging under gravity
    N = 7
    a = np.c_[np.linspace(0, 0.3, N), np.zeros(N), np.zeros(N)]
    b = np.c_[np.linspace(0.3, 0.6, N), np.zeros(N), np.zeros(N)]
    c = np.c_[np.full(N, 0.3), np.linspace(0, 0.25, N), np.zeros(N)]
    fixed = np.zeros(3 * (4 * N - 1), np.uint8)
    fixed[0:8] = 1
    desc = dict(nodes_per_rod=[N, N, N], x0=np.concatenate([a, b, c]),
                E=[1e6, 2e6, 1.5e6], nu=[0.5] * 3, rho=[1e3] * 3, radius=[2e-3, 2.5e-3, 2e-3],
                joints=[[(0, N - 1), (1, 0), (2, 0)]], fixed=fixed)
    params = dict(dt=2e-3, tol=1e-10, max_iter=60, g=(0, 0, -9.81), eta=0.05)
    _run(desc, params, 6, 1e-10)


def test_rod_sliding_on_ground_with_friction():
    N = 9
    h = 0.01
    x = np.c_[np.linspace(0, 0.5, N), np.zeros(N), np.full(N, h)]
    m = 1000.0 * math.pi * h * h * 0.5
    kc = 50.0 * m / (N - 1) * 9.81 / 5e-4
    desc = dict(nodes_per_rod=[N], x0=x, E=[1e6], nu=[0.5], rho=[1e3], radius=[h],
                ground_mu=[0.4], ground_kc=[kc],
                v0=np.c_[np.full(N, 0.05), np.full(N, 0.02), np.zeros(N)])
    params = dict(dt=2e-3, tol=1e-10, max_iter=60, g=(2.0, 0.0, -9.81), eta=0.0,
                  ground=True, ground_z=0.0, delta=5e-4, nu_slip=1e-3)
    _run(desc, params, 8, 1e-10)


def test_star_robots_trajectory():
    # free-running trajectory (no per-step reset): contact-rich, so the
    # tolerance is looser than the contact-free 1e-7 rule
    desc, params, gait = workloads.star_robots(n_robots=2, seed=7, nodes_per_limb=6)
    R = len(desc["nodes_per_rod"])
    gpu = _gpu(desc, params)
    ora = OracleSystems(desc, params)
    for k in range(12):
        kb = workloads.gait_kbar(gait, k * params["dt"])
        gpu.set_natural_curvature(0, R, kb)
        ora.set_natural_curvature(0, R, kb)
        gpu.step(1)
        ora.step(1)
    qg, _ = gpu.get_state()
    qo, _ = ora.get_state()
    _assert_close(qg, qo, desc["nodes_per_rod"], 1.0, 1e-7)


def test_chain_with_two_jointed_ends_and_mixed_batch():
    # a chain of three rods (the middle rod is jointed at both ends, which
    # takes the limb/Schur path) batched with a T of three rods attached at
    # one end each (the condensation path)
    N = 9
    xs, npr, joints = [], [], []
    for k in range(3):
        xs.append(np.c_[np.linspace(0.3 * k, 0.3 * (k + 1), N), np.zeros(N), np.zeros(N)])
    joints += [[(0, N - 1), (1, 0)], [(1, N - 1), (2, 0)]]
    y0 = 1.0
    xs.append(np.c_[np.linspace(0, 0.3, N), np.full(N, y0), np.zeros(N)])
    xs.append(np.c_[np.linspace(0.3, 0.6, N), np.full(N, y0), np.zeros(N)])
    xs.append(np.c_[np.full(N, 0.3), y0 + np.linspace(0, 0.25, N), np.zeros(N)])
    joints += [[(3, N - 1), (4, 0), (5, 0)]]
    nd = 4 * N - 1
    fixed = np.zeros(6 * nd, np.uint8)
    fixed[0:8] = 1            # chain clamped at its first rod's start
    fixed[3 * nd:3 * nd + 8] = 1
    desc = dict(nodes_per_rod=[N] * 6, x0=np.concatenate(xs),
                E=[1e6, 2e6, 1.5e6, 1e6, 2e6, 1.5e6], nu=[0.5] * 6, rho=[1e3] * 6,
                radius=[2e-3, 2.5e-3, 2e-3] * 2, joints=joints, fixed=fixed)
    params = dict(dt=2e-3, tol=1e-10, max_iter=60, g=(0, 0, -9.81), eta=0.05)
    _run(desc, params, 6, 1e-10)


def _robot_subset(desc, robots, gait):
    """Descriptor of whole robots (their limbs and joints) of a star-robot
    batch, rods renumbered in order."""
    owner = np.asarray(gait["robot"])
    rods = [r for r in range(len(owner)) if owner[r] in set(robots)]
    newid = {r: k for k, r in enumerate(rods)}
    npr = np.asarray(desc["nodes_per_rod"])
    noff = np.concatenate([[0], np.cumsum(npr)])
    foff = np.concatenate([[0], np.cumsum(4 * npr - 1)])
    out = dict(nodes_per_rod=npr[rods].astype(np.int32))
    out["x0"] = np.concatenate([desc["x0"].reshape(-1, 3)[noff[r]:noff[r + 1]] for r in rods])
    for k in ("E", "nu", "rho", "radius", "ground_mu", "ground_kc"):
        out[k] = np.asarray(desc[k])[rods]
    out["fixed"] = np.concatenate([desc["fixed"][foff[r]:foff[r + 1]] for r in rods])
    out["joints"] = [[(newid[r], i) for (r, i) in grp] for grp in desc["joints"]
                     if grp[0][0] in newid]
    return out, rods


def test_star_robots_full_batch_sampled_robots_in_bench_configuration():
    """1024 star robots (the star_robots bench workload) autotuned with
    graph rounds; three sampled robots against the oracle run on those
    robots alone (robots are independent systems), 3 gait steps."""
    desc, params, gait = workloads.star_robots(n_robots=1024, seed=3)
    R = len(desc["nodes_per_rod"])
    gpu = _gpu(desc, params)
    dt = params["dt"]
    gpu.set_natural_curvature(0, R, workloads.gait_kbar(gait, 0.0))
    gpu.autotune(steps=2)
    robots = [0, 517, 1023]
    sub, rods = _robot_subset(desc, robots, gait)
    ora = OracleSystems(sub, params)
    npr = np.asarray(desc["nodes_per_rod"])
    off = np.concatenate([[0], np.cumsum(4 * npr - 1)])
    nint = gait["nodes_per_limb"] - 2
    for k in range(3):
        kb = workloads.gait_kbar(gait, k * dt)
        gpu.set_natural_curvature(0, R, kb)
        ora.set_natural_curvature(0, len(rods),
                                  np.concatenate([kb[r * nint:(r + 1) * nint] for r in rods]))
        gpu.step(1)
        st = ora.step(1)
        assert all(x[0] == 0 for x in st), st
    qg, _ = gpu.get_state()
    qo, _ = ora.get_state()
    qs = np.concatenate([qg[off[r]:off[r + 1]] for r in rods])
    # the first steps settle the robots onto the ground (many line-search
    # iterations): Newton ends just under the tolerance on both sides
    _assert_close(qs, qo, sub["nodes_per_rod"], 1.0, 1e-7)


def test_star_robots_30_node_limbs_per_step_tight_newton():
    """The star-robot configuration of the bench (limbs of 30 nodes, 0.1 m,
    on the ground, line search, gait), backward Euler per step from identical
    states at 1e-10, with Newton run to 1e-13 on both sides.  On the step in
    which the robots settle onto the ground the twist angles of the
    converged state move about 400 times the scaled residual at which
    Newton stops (the oracle alone: stopping at 5e-12 instead of 2e-15
    moves them by 2e-9), so two correct solvers that stop at different
    points under a 1e-10 or 1e-12 tolerance can differ by more than 1e-10;
    under 1e-13 that term stays below 4e-11."""
    desc, params, gait = workloads.star_robots(n_robots=2, seed=3)
    R = len(desc["nodes_per_rod"])
    _run(desc, dict(params, tol=1e-13), 4, 1e-10, lambda t: workloads.gait_kbar(gait, t), R)
