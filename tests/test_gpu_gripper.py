"""Edge-edge contact with friction between rods (the paper's active
entanglement gripper, Sec. IV): fingers of one contact group solved
as one system, per step from identical states against the oracle (1e-10
relative) through contacts between different fingers."""
import numpy as np
import pytest
import torch

import workloads
from oracle import OracleSystems
from oracle.contact import segment_distance
from test_gpu_parity import _assert_close, _gpu

pytestmark = pytest.mark.gpu


def _cross_rod_pairs(ora, params):
    s = ora.systems[0]
    cand = s.pair_cand
    nd = torch.as_tensor(s.node_dof)
    nl = torch.as_tensor(s.edge_nl)
    i, j = torch.as_tensor(cand[:, 0]), torch.as_tensor(cand[:, 1])
    idx = torch.stack([nd[nl[i, 0]], nd[nl[i, 1]], nd[nl[j, 0]], nd[nl[j, 1]]], 1)
    x = s.q[(idx[:, :, None] + torch.arange(3)).reshape(-1, 12)]
    D, _, _ = segment_distance(x[:, 0:3], x[:, 3:6], x[:, 6:9], x[:, 9:12])
    C = torch.as_tensor(s.h_edge[cand[:, 0]] + s.h_edge[cand[:, 1]])
    act = (D < C + params["delta"]).numpy()
    cross = s.edge_rod[cand[:, 0]] != s.edge_rod[cand[:, 1]]
    return int(act.sum()), int((act & cross).sum())


def test_gripper_fingers_in_frictional_contact_per_step():
    desc, params, kfn = workloads.gripper(n_rods=3, N=16, L=0.08, ring=0.012, ramp=0.02,
                                          dt=2e-3)
    gpu = _gpu(desc, params)
    ora = OracleSystems(desc, params)
    assert len(ora.systems) == 1
    npr = desc["nodes_per_rod"]
    R = len(npr)
    crossed = 0
    for k in range(40):
        kb = kfn(k * params["dt"])
        gpu.set_natural_curvature(0, R, kb)
        ora.set_natural_curvature(0, R, kb)
        gpu.step(1)
        st = ora.step(1)
        assert all(x[0] == 0 for x in st), st
        qg, _ = gpu.get_state()
        qo, vo = ora.get_state()
        _assert_close(qg, qo, npr, 1.0, 1e-10)
        total, cross = _cross_rod_pairs(ora, params)
        assert gpu.contact_pairs() == total, (k, gpu.contact_pairs(), total)
        crossed += cross > 0
        d1, beta = ora.get_frames()
        gpu.set_state(qo, vo)
        gpu.set_frames(d1, beta)
    assert crossed >= 5


def test_contact_group_rules():
    from paper_2311_18126_gb300 import System, DismechError
    desc, params, _ = workloads.gripper(n_rods=3, N=8, L=0.04)
    # a group needs edge-edge contact on
    with pytest.raises(DismechError):
        System(desc, dict(params, self_contact=False))
    # the rods of a group must be consecutive
    bad = dict(desc, contact_groups=[[0, 2]])
    with pytest.raises(DismechError):
        System(bad, params)
    s = System(desc, params)
    assert s.n_systems == 1
    s.close()
