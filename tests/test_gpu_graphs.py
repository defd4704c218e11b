"""Newton rounds as one CUDA graph per step (a device-side while loop over
rounds) against the host-driven loop.  Both launch the same kernels in the
same order, so the results agree: bit for bit on single rods (banded
LDL^T); to rounding on star robots on the ground (line search,
condensation solve: the limbs add their Schur-complement contributions to
the border block with float atomics, in an order that varies from run to
run) and on a self-contacting coil (contact forces summed the same way)."""
import time

import numpy as np
import pytest

import workloads
from test_gpu_parity import _gpu

pytestmark = pytest.mark.gpu


def _compare(desc, params, steps, controls=None, rel=0.0):
    runs = []
    for graphs in (True, False):
        s = _gpu(desc, params)
        s.set_graphs(graphs)
        its, qs = [], []
        for k in range(steps):
            if controls is not None:
                s.set_natural_curvature(0, s.n_rods, controls(k))
            s.step(1)
            its.append(s.iterations)
            qs.append(np.concatenate(s.get_state()))
        runs.append((np.array(its), np.array(qs), s.residual))
        s.close()
    (ia, qa, ra), (ib, qb, rb) = runs
    assert ia.sum() > 0
    if rel == 0.0:
        assert np.array_equal(ia, ib)
        assert np.array_equal(qa, qb)
        assert np.array_equal(ra, rb)
    else:
        scale = np.maximum(1.0, np.abs(qb).max(axis=1, keepdims=True))
        assert np.abs(qa - qb).max() <= rel * scale.max()
        assert abs(int(ia.sum()) - int(ib.sum())) <= 1
    return ia


def test_graph_rounds_single_rods():
    desc, params, kbar = workloads.uneven_rods(n_rods=96, seed=2)
    its = _compare(desc, params, 6, controls=lambda k: kbar)
    assert its.max() >= 2


def test_graph_rounds_star_robots_line_search():
    desc, params, gait = workloads.star_robots(n_robots=12, seed=3)
    dt = params["dt"]
    _compare(desc, params, 8, controls=lambda k: workloads.gait_kbar(gait, k * dt), rel=1e-12)


def test_graph_rounds_contact_coil():
    desc, params, _ = workloads.coil(N=60)
    params = dict(params, dt=1e-3, line_search=False)
    _compare(desc, params, 40, rel=1e-12)


def test_graph_rounds_launch_accounting_and_speed():
    """Launch counts in graph mode (rounds counted on the device) equal the
    host loop's, and the per-step time of a small system (one 50-node
    cantilever, every kernel latency-bound) is printed for both."""
    desc, params = workloads.cantilever(N=50)
    out = {}
    for graphs in (True, False):
        s = _gpu(desc, params)
        s.set_graphs(graphs)
        for _ in range(5):
            s.step(1, stats=False)
        s.set_profiling(False)  # resets the counters, events stay off
        import torch
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(200):
            s.step(1, stats=False)
        torch.cuda.synchronize()
        out[graphs] = ((time.perf_counter() - t0) / 200 * 1e6,
                       {k: v[0] for k, v in s.get_profile().items()})
        s.close()
    print("cantilever N=50: %.1f us/step with the round graph, %.1f us/step host-driven"
          % (out[True][0], out[False][0]))
    g, h = out[True][1], out[False][1]
    # the graph adds one loop-control kernel per round, counted as step_begin
    assert {k: v for k, v in g.items() if k != "step_begin"} == \
        {k: v for k, v in h.items() if k != "step_begin"}
    assert g["step_begin"] > h["step_begin"]


def _state(s):
    q, v = s.get_state()
    d1, beta = s.get_frames()
    return np.concatenate([q, v, np.ravel(d1), np.ravel(beta)])


@pytest.mark.parametrize("kind", ["rods", "stars"])
def test_autotune_keeps_state_and_results(kind):
    """The autotuner leaves the committed state as it found it, returns
    launch shapes within the candidate sets, and the tuned system steps
    like an untuned one (bit for bit on single rods: every shape does the
    same arithmetic per system)."""
    if kind == "rods":
        desc, params, kbar = workloads.uneven_rods(n_rods=512, seed=2)
        controls = lambda k: kbar
    else:
        desc, params, gait = workloads.star_robots(n_robots=48, seed=3)
        controls = lambda k: workloads.gait_kbar(gait, k * params["dt"])
    a, b = _gpu(desc, params), _gpu(desc, params)
    for s in (a, b):
        s.set_natural_curvature(0, s.n_rods, controls(0))
        s.step(1)
    before = _state(a)
    tune = a.autotune(steps=2)
    print(kind, tune)
    assert np.array_equal(before, _state(a))
    assert tune["stencil_threads"] in (32, 64, 128) and tune["stencil_per_thread"] in (1, 2)
    assert tune["solve_warps"] in (1, 2, 4) and tune["solve_blocks_per_sm"] in (1, 2, 3, 4)
    assert all(v > 0 for k, v in tune["us_per_launch"].items()
               if k in ("edge", "stencil"))
    for k in range(1, 5):
        for s in (a, b):
            s.set_natural_curvature(0, s.n_rods, controls(k))
            s.step(1)
        qa, qb = a.get_state()[0], b.get_state()[0]
        if kind == "rods":
            assert np.array_equal(qa, qb)
            assert np.array_equal(a.iterations, b.iterations)
        else:
            assert np.abs(qa - qb).max() <= 1e-12 * max(1.0, np.abs(qb).max())
    a.close()
    b.close()


def test_set_tuning_applies_shapes_and_rejects_others():
    """dm_set_tuning: an autotuned shape applied to a second system of the
    same workload steps it bit for bit like the tuned one; a shape outside
    the candidate sets is rejected and changes nothing."""
    from paper_2311_18126_gb300 import DismechError
    desc, params, kbar = workloads.uneven_rods(n_rods=512, seed=2)
    a, b = _gpu(desc, params), _gpu(desc, params)
    for s in (a, b):
        s.set_natural_curvature(0, s.n_rods, kbar)
        s.step(1)
    tune = a.autotune(steps=2)
    b.set_tuning(tune)
    bad = dict(tune, stencil_threads=96)
    with pytest.raises(DismechError):
        b.set_tuning(bad)
    for k in range(3):
        a.step(1)
        b.step(1)
        assert np.array_equal(a.get_state()[0], b.get_state()[0])
    a.close()
    b.close()


@pytest.mark.parametrize("graphs", [True, False])
def test_split_first_round_matches_fused(graphs):
    """The first Newton round by the split passes (gradient pass, then the
    Hessian pass) against the fused passes: the same arithmetic per entry in
    another kernel grouping, so the same iteration counts and states to
    rounding."""
    desc, params, kbar = workloads.uneven_rods(n_rods=48, seed=6, n_min=20, n_max=90)
    runs = []
    for fused in (True, False):
        s = _gpu(desc, params)
        s.set_graphs(graphs)
        s.set_fused_first(fused)
        s.set_natural_curvature(0, s.n_rods, kbar)
        its, qs = [], []
        for _ in range(4):
            s.step(1)
            its.append(s.iterations)
            qs.append(np.concatenate(s.get_state()))
        runs.append((np.array(its), np.array(qs)))
        s.close()
    (ia, qa), (ib, qb) = runs
    assert ia.sum() > 0 and np.array_equal(ia, ib)
    scale = np.maximum(1.0, np.abs(qb).max(axis=1, keepdims=True))
    assert np.max(np.abs(qa - qb) / scale) < 1e-12
