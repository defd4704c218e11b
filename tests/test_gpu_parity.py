"""GPU (CUDA library through the C ABI) vs the CPU oracle, element by element,
from identical states.

Tolerances (spec parity rule): per step, positions within
1e-10 * max(|x|_inf, L) and angles within 1e-10 * max(1, |theta|_inf);
over contact-free trajectories 1e-7 relative.
"""
import numpy as np
import pytest

import workloads
from oracle import OracleSystems

pytestmark = pytest.mark.gpu


def _gpu(desc, params):
    from paper_2311_18126_gb300 import ensure_built, System
    ensure_built()
    return System(desc, params)


def _split(q, npr):
    """Masks of position and angle entries in the per-rod layout."""
    pos = np.ones(len(q), bool)
    off = 0
    for N in npr:
        idx = off + 4 * np.arange(N - 1) + 3
        pos[idx] = False
        off += 4 * N - 1
    return pos


def _assert_close(qg, qo, npr, L, rel):
    pos = _split(qo, npr)
    sx = max(np.max(np.abs(qo[pos])), L)
    th = ~pos
    st = max(1.0, np.max(np.abs(qo[th])) if th.any() else 1.0)
    ex = np.max(np.abs(qg[pos] - qo[pos])) / sx
    et = np.max(np.abs(qg[th] - qo[th])) / st if th.any() else 0.0
    assert ex <= rel and et <= rel, (ex, et)
    return ex, et


def test_cantilever_per_step_and_trajectory():
    desc, params = workloads.cantilever()
    gpu = _gpu(desc, params)
    ora = OracleSystems(desc, params)
    npr = desc["nodes_per_rod"]
    for k in range(20):
        gpu.step(1)
        ora.step(1)
        qg, vg = gpu.get_state()
        qo, vo = ora.get_state()
        if k < 5:
            # per-step parity from identical states: reset the GPU to the oracle
            _assert_close(qg, qo, npr, 1.0, 1e-10)
            d1, beta = ora.get_frames()
            gpu.set_state(qo, vo)
            gpu.set_frames(d1, beta)
        else:
            _assert_close(qg, qo, npr, 1.0, 1e-7)


def test_iterations_match_oracle():
    desc, params = workloads.cantilever(N=30)
    gpu = _gpu(desc, params)
    ora = OracleSystems(desc, params)
    for _ in range(3):
        gpu.step(1)
        st = ora.step(1)
        assert int(gpu.iterations[0]) == st[0][1]


@pytest.mark.parametrize("n_rods,seed", [(24, 2), (7, 5)])
def test_uneven_rods_batch(n_rods, seed):
    desc, params, kbar = workloads.uneven_rods(n_rods=n_rods, seed=seed)
    gpu = _gpu(desc, params)
    ora = OracleSystems(desc, params)
    gpu.set_natural_curvature(0, n_rods, kbar)
    ora.set_natural_curvature(0, n_rods, kbar)
    L = float(np.max(np.linalg.norm(desc["x0"], axis=1)))
    for _ in range(3):
        gpu.step(1)
        ora.step(1)
        qg, _ = gpu.get_state()
        qo, _ = ora.get_state()
        _assert_close(qg, qo, desc["nodes_per_rod"], L, 1e-9)


def test_degenerate_sizes_and_free_rod():
    # rods of 2 and 3 nodes (no / one stencil), a free rod with spin, a clamped rod
    rng = np.random.default_rng(0)
    xs, npr, fixed = [], [2, 3, 9, 5], []
    for N in npr:
        x = np.zeros((N, 3))
        x[:, 0] = np.linspace(0, 0.3, N)
        x[:, 1] = 0.01 * rng.standard_normal(N)
        xs.append(x)
        fixed.append(np.zeros(4 * N - 1, np.uint8))
    fixed[3][:8] = 1
    v0 = 0.1 * rng.standard_normal((sum(npr), 3))
    desc = dict(nodes_per_rod=npr, x0=np.concatenate(xs), v0=v0,
                theta_dot0=rng.standard_normal(sum(npr) - len(npr)),
                E=[1e6, 2e6, 5e6, 1e7], nu=[0.5, 0.3, 0.5, 0.4], rho=[1e3] * 4,
                radius=[1e-3, 2e-3, 1.5e-3, 1e-3], fixed=np.concatenate(fixed))
    params = dict(dt=1e-3, tol=1e-10, max_iter=50, g=(0, 0, -9.81), eta=0.05)
    gpu = _gpu(desc, params)
    ora = OracleSystems(desc, params)
    for _ in range(4):
        gpu.step(1)
        ora.step(1)
        qg, vg = gpu.get_state()
        qo, vo = ora.get_state()
        _assert_close(qg, qo, npr, 0.3, 1e-10)


def test_full_batch_sampled_rods_in_bench_configuration():
    """The 4096-rod bench batch in the launch configuration bench.py times
    (autotuned shapes, Newton rounds as one graph per step): six sampled
    rods, the longest and the shortest among them, against the oracle run on
    those rods alone (the rods are independent systems), 3 steps."""
    desc, params, kbar = workloads.uneven_rods(n_rods=4096, seed=2)
    gpu = _gpu(desc, params)
    gpu.set_natural_curvature(0, 4096, kbar)
    gpu.autotune(steps=2)
    npr = np.asarray(desc["nodes_per_rod"])
    rng = np.random.default_rng(123)
    rods = sorted({int(np.argmax(npr)), int(np.argmin(npr))} |
                  set(rng.choice(4096, 4, replace=False).tolist()))
    sub, kb = workloads.subset(desc, rods, kbar)
    ora = OracleSystems(sub, params)
    ora.set_natural_curvature(0, len(rods), kb)
    off = np.concatenate([[0], np.cumsum(4 * npr - 1)])
    for _ in range(3):
        gpu.step(1)
        st = ora.step(1)
        assert all(x[0] == 0 for x in st), st
    qg, _ = gpu.get_state()
    qo, _ = ora.get_state()
    qs = np.concatenate([qg[off[r]:off[r + 1]] for r in rods])
    L = max(1.0, float(np.max(np.abs(sub["x0"]))))
    _assert_close(qs, qo, sub["nodes_per_rod"], L, 1e-9)


@pytest.mark.parametrize("n_rods,seed", [(24, 2), (7, 5)])
def test_uneven_rods_projected_predictor_per_step(n_rods, seed):
    """The length-projected Newton guess on both sides: per step from
    identical states at 1e-10, and no more Newton iterations than the
    extrapolated guess takes from the same states."""
    desc, params, kbar = workloads.uneven_rods(n_rods=n_rods, seed=seed)
    pp = dict(params, predictor="projected")
    gpu = _gpu(desc, pp)
    ref = _gpu(desc, params)
    ora = OracleSystems(desc, pp)
    for s in (gpu, ref, ora):
        s.set_natural_curvature(0, n_rods, kbar)
    L = max(1.0, float(np.max(np.abs(desc["x0"]))))
    its_p, its_e = 0, 0
    for _ in range(4):
        gpu.step(1)
        ref.step(1)
        st = ora.step(1)
        assert all(x[0] == 0 for x in st), st
        its_p += int(gpu.iterations.sum())
        its_e += int(ref.iterations.sum())
        qg, _ = gpu.get_state()
        qo, vo = ora.get_state()
        _assert_close(qg, qo, desc["nodes_per_rod"], L, 1e-10)
        d1, beta = ora.get_frames()
        for s in (gpu, ref):
            s.set_state(qo, vo)
            s.set_frames(d1, beta)
    assert its_p <= its_e, (its_p, its_e)
