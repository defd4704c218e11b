"""Implicit midpoint (Sec. III-C offers it beside backward Euler) on the GPU
against the oracle's midpoint: per step from identical states (1e-10
relative) on single rods with gravity and damping, star robots on the
ground (friction, line search, condensation solve) and a self-contacting
coil (contact-band LU), and a free trajectory on a batch of uneven rods
(1e-7).  The GPU solves backward Euler over dt/2 for the midpoint
configuration; the oracle takes the midpoint residual as written, so the
two formulations check each other."""
import numpy as np
import pytest

import workloads
from oracle import OracleSystems
from test_gpu_general import _run
from test_gpu_parity import _assert_close, _gpu

pytestmark = pytest.mark.gpu


def test_midpoint_cantilever_per_step():
    desc, params = workloads.cantilever(N=30)
    _run(desc, dict(params, integrator="midpoint"), 25, 1e-10)


def test_midpoint_star_robots_per_step():
    # the configuration of the backward-Euler star-robot parity test, with
    # Newton run to 1e-12 on both sides: at 1e-10 the settling first step
    # (line search, many iterations) ends just under the tolerance at points
    # whose twist angles differ by a few 1e-10
    desc, params, gait = workloads.star_robots(n_robots=3, seed=3, nodes_per_limb=8)
    _run(desc, dict(params, integrator="midpoint", tol=1e-12), 8, 1e-10,
         kbar_fn=lambda t: workloads.gait_kbar(gait, t), nrods=len(desc["nodes_per_rod"]))


def test_midpoint_star_robots_30_node_limbs():
    # 30-node limbs: the first step (the robots settle from rest onto the
    # ground, ~20 line-search iterations) ends just under the tolerance on
    # both sides, at points 1e-8 apart (backward Euler: 1e-9); every later
    # step from identical states agrees to rounding
    desc, params, gait = workloads.star_robots(n_robots=4, seed=3)
    params = dict(params, integrator="midpoint")
    R = len(desc["nodes_per_rod"])
    gpu = _gpu(desc, params)
    ora = OracleSystems(desc, params)
    for k in range(10):
        kb = workloads.gait_kbar(gait, k * params["dt"])
        gpu.set_natural_curvature(0, R, kb)
        ora.set_natural_curvature(0, R, kb)
        gpu.step(1)
        st = ora.step(1)
        assert all(x[0] == 0 for x in st), st
        qg, _ = gpu.get_state()
        qo, vo = ora.get_state()
        _assert_close(qg, qo, desc["nodes_per_rod"], 1.0, 2e-8 if k == 0 else 1e-10)
        d1, beta = ora.get_frames()
        gpu.set_state(qo, vo)
        gpu.set_frames(d1, beta)


def test_midpoint_contact_coil_per_step():
    desc, params, _ = workloads.coil(N=60)
    params = dict(params, dt=1e-3, line_search=False, integrator="midpoint")
    gpu = _gpu(desc, params)
    ora = OracleSystems(desc, params)
    npr = desc["nodes_per_rod"]
    touched = 0
    for k in range(44):
        gpu.step(1)
        st = ora.step(1)
        assert all(x[0] == 0 for x in st), st
        qg, _ = gpu.get_state()
        qo, vo = ora.get_state()
        _assert_close(qg, qo, npr, 1.0, 1e-10)
        touched += gpu.contact_pairs() > 0
        d1, beta = ora.get_frames()
        gpu.set_state(qo, vo)
        gpu.set_frames(d1, beta)
    assert touched >= 3


@pytest.mark.parametrize("predictor", ["extrapolate", "projected"])
def test_midpoint_uneven_rods_trajectory(predictor):
    desc, params, kbar = workloads.uneven_rods(n_rods=4096, seed=2)
    sub, kb = workloads.subset(desc, [5, 77, 1031, 2500, 4000], kbar)
    params = dict(params, integrator="midpoint", predictor=predictor)
    gpu = _gpu(sub, params)
    ora = OracleSystems(sub, params)
    R = len(sub["nodes_per_rod"])
    gpu.set_natural_curvature(0, R, kb)
    ora.set_natural_curvature(0, R, kb)
    for _ in range(20):
        gpu.step(1)
        st = ora.step(1)
        assert all(x[0] == 0 for x in st), st
    qg, vg = gpu.get_state()
    qo, vo = ora.get_state()
    L = max(1.0, float(np.max(np.abs(sub["x0"]))))
    _assert_close(qg, qo, sub["nodes_per_rod"], L, 1e-7)
    # velocities: qdot_{n+1} = 2 (q_{n+1} - q_n)/dt - qdot_n on both sides
    scale = max(1.0, float(np.abs(vo).max()))
    assert np.abs(vg - vo).max() <= 1e-6 * scale


def test_midpoint_divergence_matches_oracle_and_line_search_recovers():
    """Rod 379 of the headline batch (N = 151, E = 1.26e7): without the
    numerical damping of backward Euler, plain Newton diverges at the 5th
    midpoint step on both sides; the GPU reports DM_ERR_NOT_CONVERGED and
    keeps the last good state, which equals the oracle's.  With the line
    search both converge and agree."""
    from paper_2311_18126_gb300 import DismechError
    desc, params, kbar = workloads.uneven_rods(n_rods=4096, seed=2)
    sub, kb = workloads.subset(desc, [379], kbar)
    npr = sub["nodes_per_rod"]
    L = max(1.0, float(np.max(np.abs(sub["x0"]))))
    for ls in (False, True):
        p = dict(params, integrator="midpoint", line_search=ls)
        gpu = _gpu(sub, p)
        ora = OracleSystems(sub, p)
        gpu.set_natural_curvature(0, 1, kb)
        ora.set_natural_curvature(0, 1, kb)
        for k in range(6):
            st = ora.step(1)
            if st[0][0] != 0:
                assert not ls and k == 4
                with pytest.raises(DismechError) as ei:
                    gpu.step(1)
                assert ei.value.code == 2  # DM_ERR_NOT_CONVERGED
                break
            gpu.step(1)
        qg, _ = gpu.get_state()
        qo, _ = ora.get_state()
        _assert_close(qg, qo, npr, L, 1e-8)
