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


def _batch():
    desc, params, kbar = workloads.uneven_rods(n_rods=64, seed=2)
    sub, kb = workloads.subset(desc, [3, 17, 40], kbar)
    return sub, params, kb


def test_step_adjoint_matches_oracle_adjoint():
    desc, params, kb = _batch()
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
