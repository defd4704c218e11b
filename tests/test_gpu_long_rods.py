"""Long rods in the Newton step: single rods with at least
2048 DOFs are solved by the partitioned band solve inside dm_step.  Per
step from identical states against the oracle (1e-10 relative) on a batch
that mixes long and short rods, and the same trajectory with every rod on
the sequential twisted LDL^T (long_rod_dofs < 0)."""
import numpy as np
import pytest

import workloads
from oracle import OracleSystems
from test_gpu_parity import _assert_close, _gpu

pytestmark = pytest.mark.gpu


def _batch():
    # N = 748, 394, 311, 989: two long (>= 2048 DOFs) and two short rods
    desc, params, kbar = workloads.uneven_rods(n_rods=4, seed=8, n_min=100, n_max=1000)
    return desc, params, kbar


def test_long_rods_per_step():
    desc, params, kbar = _batch()
    npr = np.asarray(desc["nodes_per_rod"])
    assert (4 * npr - 1 >= 2048).any() and (4 * npr - 1 < 2048).any()
    gpu = _gpu(desc, params)
    ora = OracleSystems(desc, params)
    R = len(npr)
    gpu.set_natural_curvature(0, R, kbar)
    ora.set_natural_curvature(0, R, kbar)
    L = max(1.0, float(np.max(np.abs(desc["x0"]))))
    for k in range(5):
        gpu.step(1)
        st = ora.step(1)
        assert all(x[0] == 0 for x in st), st
        qg, _ = gpu.get_state()
        qo, vo = ora.get_state()
        _assert_close(qg, qo, npr, L, 1e-10)
        d1, beta = ora.get_frames()
        gpu.set_state(qo, vo)
        gpu.set_frames(d1, beta)


def test_long_rods_partitioned_vs_sequential_trajectory():
    desc, params, kbar = _batch()
    R = len(desc["nodes_per_rod"])
    out = []
    for long_dofs in (0, -1):
        s = _gpu(desc, dict(params, long_rod_dofs=long_dofs))
        s.set_natural_curvature(0, R, kbar)
        its = []
        for _ in range(15):
            s.step(1)
            its.append(s.iterations)
        out.append((s.get_state()[0], np.array(its)))
        s.close()
    (qa, ia), (qb, ib) = out
    assert np.array_equal(ia, ib)
    scale = max(1.0, float(np.abs(qb).max()))
    assert np.abs(qa - qb).max() <= 1e-9 * scale
