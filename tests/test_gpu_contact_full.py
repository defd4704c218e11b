"""Edge-edge contact at full size (Sec. III-B, Eq. 10-13): the 500-node coil
once its turns have collapsed onto each other, and the five 60-node gripper
fingers (Sec. IV) once they touch, per step from identical states against
the oracle (1e-10), with equal numbers of edge pairs in contact.

The starting states come from the oracle alone (tests/golden/
make_contact_states.py): the GPU path contributes no input."""
import os

import numpy as np
import pytest

import workloads
from oracle import OracleSystems
from test_gpu_contact import _oracle_active_pairs
from test_gpu_parity import _assert_close, _gpu

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _per_step(desc, params, state, steps, kbar=None):
    gpu = _gpu(desc, params)
    ora = OracleSystems(desc, params)
    R = len(desc["nodes_per_rod"])
    q, v, d1, beta = state["q"], state["qdot"], state["d1"], state["beta"]
    npr = desc["nodes_per_rod"]
    L = max(1.0, float(np.max(np.abs(desc["x0"]))))
    pairs = []
    for k in range(steps):
        for side in (gpu, ora):
            side.set_state(q, v)
            side.set_frames(d1, beta)
            if kbar is not None:
                side.set_natural_curvature(0, R, kbar)
        gpu.step(1)
        st = ora.step(1)
        assert all(x[0] == 0 for x in st), st
        qg, _ = gpu.get_state()
        q, v = ora.get_state()
        d1, beta = ora.get_frames()
        _assert_close(qg, q, npr, L, 1e-10)
        ng, no = gpu.contact_pairs(), _oracle_active_pairs(ora, params)
        assert ng == no, (k, ng, no)
        pairs.append(no)
    gpu.close()
    return pairs


def test_collapsed_500_node_coil_per_step():
    desc, params, _ = workloads.coil(N=500)
    state = np.load(os.path.join(GOLD, "coil500_state.npz"))
    pairs = _per_step(desc, params, state, 3)
    assert min(pairs) >= 500, pairs


def test_5x60_gripper_in_contact_per_step():
    desc, params, kfn = workloads.gripper()
    state = np.load(os.path.join(GOLD, "gripper5x60_state.npz"))
    kb = kfn(int(state["step"]) * params["dt"])
    pairs = _per_step(desc, params, state, 3, kbar=kb)
    assert min(pairs) >= 1, pairs
