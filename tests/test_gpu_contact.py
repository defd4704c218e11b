"""GPU vs oracle for edge-edge contact (Sec. III-B, Eq. 10-11): a helical rod
collapsing under gravity until its turns touch.  Per step from identical
states (1e-10 relative) with the active pair counts of both sides compared,
and a free trajectory through the first contacts."""
import numpy as np
import pytest
import torch

import workloads
from oracle import OracleSystems
from oracle.contact import segment_distance
from test_gpu_parity import _assert_close, _gpu

pytestmark = pytest.mark.gpu


def _oracle_active_pairs(ora, params):
    s = ora.systems[0]
    cand = s.pair_cand
    nd = torch.as_tensor(s.node_dof)
    nl = torch.as_tensor(s.edge_nl)
    i, j = torch.as_tensor(cand[:, 0]), torch.as_tensor(cand[:, 1])
    idx = torch.stack([nd[nl[i, 0]], nd[nl[i, 1]], nd[nl[j, 0]], nd[nl[j, 1]]], 1)
    x = s.q[(idx[:, :, None] + torch.arange(3)).reshape(-1, 12)]
    D, _, _ = segment_distance(x[:, 0:3], x[:, 3:6], x[:, 6:9], x[:, 9:12])
    C = torch.as_tensor(s.h_edge[cand[:, 0]] + s.h_edge[cand[:, 1]])
    return int((D < C + params["delta"]).sum())


def _short_coil():
    # 60 nodes at dt = 1 ms without line search: the turns touch from step 30
    desc, params, _ = workloads.coil(N=60)
    return desc, dict(params, dt=1e-3, line_search=False)


def test_coil_contact_per_step():
    desc, params = _short_coil()
    gpu = _gpu(desc, params)
    ora = OracleSystems(desc, params)
    npr = desc["nodes_per_rod"]
    touched = 0
    for k in range(44):
        gpu.step(1)
        st = ora.step(1)
        assert all(x[0] == 0 for x in st), st
        qg, vg = gpu.get_state()
        qo, vo = ora.get_state()
        _assert_close(qg, qo, npr, 1.0, 1e-10)
        # pairs in contact at the converged state: the GPU counts them at
        # its last evaluated iterate, which is the converged one
        ng = gpu.contact_pairs()
        no = _oracle_active_pairs(ora, params)
        assert ng == no, (k, ng, no)
        touched += no > 0
        d1, beta = ora.get_frames()
        gpu.set_state(qo, vo)
        gpu.set_frames(d1, beta)
    assert touched >= 5


def test_coil_contact_trajectory():
    desc, params = _short_coil()
    gpu = _gpu(desc, params)
    ora = OracleSystems(desc, params)
    for k in range(40):
        gpu.step(1)
        ora.step(1)
    assert gpu.contact_pairs() > 0
    qg, _ = gpu.get_state()
    qo, _ = ora.get_state()
    _assert_close(qg, qo, desc["nodes_per_rod"], 1.0, 1e-7)


def test_contact_options_rejected():
    from paper_2311_18126_gb300 import System, DismechError
    desc, params, _ = workloads.coil(N=20)
    with pytest.raises(DismechError):
        System(desc, dict(params, pair_mu=-0.3))


def test_coil_contact_with_friction_per_step():
    """Friction at the closest points of touching edges (Eq. 12-13, pair_mu
    > 0): per-step parity through the first contacts, line search on."""
    desc, params = _short_coil()
    params = dict(params, pair_mu=0.3, line_search=True)
    gpu = _gpu(desc, params)
    ora = OracleSystems(desc, params)
    npr = desc["nodes_per_rod"]
    touched = 0
    for k in range(40):
        gpu.step(1)
        st = ora.step(1)
        assert all(x[0] == 0 for x in st), st
        qg, vg = gpu.get_state()
        qo, vo = ora.get_state()
        _assert_close(qg, qo, npr, 1.0, 1e-10)
        touched += _oracle_active_pairs(ora, params) > 0
        d1, beta = ora.get_frames()
        gpu.set_state(qo, vo)
        gpu.set_frames(d1, beta)
    assert touched >= 5


def _crossing_rods_on_ground(N=12, h=1e-3, delta=5e-4):
    # two free rods of one contact group dropped on the ground, the upper one
    # crossing the lower one and sliding along it: ground contact with
    # friction and edge-edge contact with friction act together
    import math
    L = 0.1
    s = np.linspace(-L / 2, L / 2, N)
    xa = np.stack([s, np.zeros(N), np.full(N, h + 1e-4)], 1)
    xb = np.stack([np.full(N, 0.01), s, np.full(N, 3 * h + 2e-4)], 1)
    v0 = np.zeros((2 * N, 3))
    v0[N:, 0] = 0.05
    rho, E = 1000.0, 1e6
    kc = 50.0 * rho * math.pi * h * h * (L / (N - 1)) * 9.81 / delta  # reading C11
    desc = dict(nodes_per_rod=[N, N], x0=np.concatenate([xa, xb]), v0=v0, E=[E, E],
                nu=[0.5, 0.5], rho=[rho, rho], radius=[h, h],
                fixed=np.zeros(2 * (4 * N - 1), np.uint8), ground_mu=[0.5, 0.5],
                ground_kc=[kc, kc], contact_groups=[[0, 1]])
    params = dict(dt=1e-3, tol=1e-10, max_iter=100, g=(0.0, 0.0, -9.81), eta=0.05,
                  ground=True, ground_z=0.0, delta=delta, nu_slip=1e-3, self_contact=True,
                  pair_kc=E * h, pair_mu=0.4, line_search=True)
    return desc, params


def test_edge_contact_together_with_ground_contact_per_step():
    desc, params = _crossing_rods_on_ground()
    gpu = _gpu(desc, params)
    ora = OracleSystems(desc, params)
    npr = desc["nodes_per_rod"]
    touching = 0
    for k in range(20):
        gpu.step(1)
        st = ora.step(1)
        assert all(x[0] == 0 for x in st), st
        qg, _ = gpu.get_state()
        qo, vo = ora.get_state()
        _assert_close(qg, qo, npr, 1.0, 1e-10)
        ng, no = gpu.contact_pairs(), _oracle_active_pairs(ora, params)
        assert ng == no, (k, ng, no)
        touching += no > 0
        d1, beta = ora.get_frames()
        gpu.set_state(qo, vo)
        gpu.set_frames(d1, beta)
    assert touching >= 10
