"""Pins of the oracle's joint stencils (Sec. III-D, reading C18) and of its
contact Jacobians (Sec. III-B, Eq. 10-13), CPU only.

* A rod split at a node into two rods joined there, the second listed in
  reverse, is the same mechanical system as the unsplit rod: energy, forces
  (twist signs included), Jacobian and one backward-Euler step must agree.
  This fails if a reversed edge's t, d2 or theta sign is wrong.
* Joint stencils of a planar star: the curvature of each edge pair is the
  kink curvature 2 tan(phi/2) of Eq. 5, with phi the turning angle between
  the edge entering the joint and the one leaving it.
* The bending and twisting energy of a kinked or twisted joint between two
  different rods is the closed form with the averaged EI and GJ.
* Node masses: half the mass of every incident edge (the joint node of a
  star included), and the masses add up to the rods' total mass.
* Contact Jacobians (ground with friction, edge pairs with friction) equal
  central differences of the oracle's forces.
"""
import math

import numpy as np
import pytest
import torch

from oracle import OracleSystems, der

DT = torch.float64


def _desc(rod_points, E, nu, rho, h, joints=(), theta0=None, **extra):
    npr = [len(p) for p in rod_points]
    R = len(npr)
    d = dict(nodes_per_rod=npr, x0=np.concatenate(rod_points), E=list(E), nu=list(nu),
             rho=list(rho), radius=list(h),
             fixed=np.zeros(int(sum(4 * n - 1 for n in npr)), np.uint8),
             joints=[list(j) for j in joints])
    if theta0 is not None:
        d["theta0"] = np.asarray(theta0, np.float64)
    d.update(extra)
    assert len(d["E"]) == R
    return d


def _elastic_energy(o, s, q):
    """Stretching + bending + twisting of one system at q, with the reference
    frames time-transported from the committed step (Sec. III)."""
    idx = torch.as_tensor(s.st_dofs)
    e6 = torch.as_tensor(s.edge_dofs6)
    Es = der.stretch_energy(q[e6], torch.as_tensor(s.EA), torch.as_tensor(s.lbar)).sum()
    Eb = der.time_transported_energy(q[idx], *o._stencil_history(s)).sum() \
        if len(s.st) else torch.zeros((), dtype=DT)
    return Es + Eb


# ---------------------------------------------------------------------------
# A reversed rod joined to its other half is the unsplit rod
# ---------------------------------------------------------------------------

def _dof_map(o1, s1, o2, s2):
    """For every DOF of system s1: the DOF of s2 that describes the same
    coordinate and the sign relating them (-1 for the twist angle of an edge
    stored in the opposite direction).  Nodes are matched by position."""
    x1 = s1.q[torch.as_tensor(s1.node_dof)[:, None] + torch.arange(3)].numpy()
    x2 = s2.q[torch.as_tensor(s2.node_dof)[:, None] + torch.arange(3)].numpy()
    node12 = np.array([int(np.argmin(np.linalg.norm(x2 - p, axis=1))) for p in x1])
    assert np.allclose(x2[node12], x1)
    perm = np.zeros(s1.n, np.int64)
    sign = np.ones(s1.n)
    for k in range(len(s1.nodes)):
        for c in range(3):
            perm[s1.node_dof[k] + c] = s2.node_dof[node12[k]] + c
    pos2 = {}
    for k in range(len(s2.edges)):
        a, b = s2.edge_nl[k]
        pos2[(a, b)] = (k, 1.0)
        pos2[(b, a)] = (k, -1.0)
    for k in range(len(s1.edges)):
        a, b = s1.edge_nl[k]
        k2, sg = pos2[(node12[a], node12[b])]
        perm[s1.edge_dof[k]] = s2.edge_dof[k2]
        sign[s1.edge_dof[k]] = sg
    return perm, sign, node12


def _split_pair(seed, planar):
    rng = np.random.default_rng(seed)
    N, k = 9, 4
    x = np.zeros((N, 3))
    x[:, 0] = np.linspace(0.0, 0.4, N)
    if planar:
        x[:, 1] = 0.03 * np.sin(np.linspace(0.0, 3.0, N)) + 0.004 * rng.standard_normal(N)
    else:
        x[:, 1:] = 0.03 * rng.standard_normal((N, 2))
    th = 0.4 * rng.standard_normal(N - 1)
    mat = dict(E=[2e7], nu=[0.45], rho=[1100.0], h=[2e-3])
    one = OracleSystems(_desc([x], theta0=th, **mat), dict(g=(0.0, -3.0, -9.81), eta=0.2))
    # rod A = nodes 0..k, rod B = nodes N-1 .. k (reversed); B's edge j runs
    # from node N-1-j to N-2-j: the original edge N-2-j reversed
    thB = -th[::-1][:N - 1 - k]
    two = OracleSystems(_desc([x[:k + 1], x[k:][::-1]], theta0=np.concatenate([th[:k], thB]),
                              joints=[[(0, k), (1, N - 1 - k)]],
                              **{key: v * 2 for key, v in mat.items()}),
                        dict(g=(0.0, -3.0, -9.81), eta=0.2))
    s1, s2 = one.systems[0], two.systems[0]
    perm, sign, node12 = _dof_map(one, s1, two, s2)
    if not planar:
        # the initial reference directors of the reversed rod come from its
        # own first tangent; give it those of the unsplit rod (the director
        # vector is the same for either storage direction) and recompute the
        # reference twist and natural strains from them
        d1 = s2.d1.clone()
        for kk in range(len(s1.edges)):
            a, b = s1.edge_nl[kk]
            for k2 in range(len(s2.edges)):
                if set(s2.edge_nl[k2]) == {node12[a], node12[b]}:
                    d1[k2] = s1.d1[kk]
        s2.d1 = d1
        two._init_stencil_rest(s2)
    return one, s1, two, s2, perm, sign, rng


@pytest.mark.parametrize("seed,planar", [(0, True), (1, False), (2, False)])
def test_reversed_half_joined_at_a_node_equals_the_unsplit_rod(seed, planar):
    one, s1, two, s2, perm, sign, rng = _split_pair(seed, planar)
    P = torch.as_tensor(perm)
    S = torch.as_tensor(sign)
    # committed step and an iterate away from it
    q1 = s1.q + torch.as_tensor(0.004 * rng.standard_normal(s1.n))
    q2 = torch.zeros(s2.n, dtype=DT)
    q2[P] = S * q1
    E1 = float(_elastic_energy(one, s1, q1))
    E2 = float(_elastic_energy(two, s2, q2))
    assert E1 > 1e-6
    assert E2 == pytest.approx(E1, rel=1e-12)
    F1, _, J1 = one.forces(s1, q1, s1.v, s1.q)
    F2, _, J2 = two.forces(s2, q2, s2.v, s2.q)
    sc = float(F1.abs().max())
    np.testing.assert_allclose((S * F2[P]).numpy(), F1.numpy(), rtol=0, atol=1e-12 * sc)
    J2m = (S[:, None] * J2[P][:, P] * S[None, :]).numpy()
    np.testing.assert_allclose(J2m, J1.numpy(), rtol=0, atol=1e-12 * float(J1.abs().max()))
    # one backward-Euler step from the same state (masses included)
    v1 = torch.as_tensor(0.05 * rng.standard_normal(s1.n))
    s1.v = v1.clone()
    s2.v = torch.zeros(s2.n, dtype=DT)
    s2.v[P] = S * v1
    for s in (s1, s2):
        s.q = s.q.clone()
    assert one.step_system(s1)[0] == 0
    assert two.step_system(s2)[0] == 0
    np.testing.assert_allclose((S * s2.q[P]).numpy(), s1.q.numpy(), rtol=0, atol=1e-12)
    np.testing.assert_allclose((S * s2.v[P]).numpy(), s1.v.numpy(), rtol=0,
                               atol=1e-10 * float(s1.v.abs().max()))


# ---------------------------------------------------------------------------
# Joint-stencil curvature of a star: 2 tan(phi / 2) per edge pair
# ---------------------------------------------------------------------------

def _star(angles, n=4, L=0.1, R=None):
    pts = []
    for a in angles:
        s = np.linspace(0.0, L, n)
        pts.append(np.stack([s * math.cos(a), s * math.sin(a), np.zeros(n)], 1))
    if R is not None:
        pts = [p @ R.T for p in pts]
    k = len(angles)
    return _desc(pts, E=[1e6] * k, nu=[0.5] * k, rho=[1000.0] * k, h=[1e-3] * k,
                 joints=[[(r, 0) for r in range(k)]])


@pytest.mark.parametrize("angles_deg", [(0.0, 100.0, 230.0), (10.0, 75.0, 160.0, 290.0)])
def test_star_joint_curvature_is_the_kink_curvature(angles_deg):
    ang = np.deg2rad(angles_deg)
    o = OracleSystems(_star(ang))
    s = o.systems[0]
    joint = [k for k, g in enumerate(s.st) if o.st_rodslot[g] == -1]
    assert len(joint) == len(ang) * (len(ang) - 1) // 2
    for k in joint:
        a, b = o.st_edges[s.st[k]]
        ra, rb = o.edge_rod[a], o.edge_rod[b]
        # every limb leaves the joint: edge a enters it reversed, so the
        # turning angle is pi - (alpha_b - alpha_a); with d1 = z the kink
        # bends about d1 and kappa2 = 2 cot((alpha_b - alpha_a) / 2)
        dlt = ang[rb] - ang[ra]
        assert float(s.kbar2[k]) == pytest.approx(2.0 / math.tan(0.5 * dlt), rel=1e-13)
        assert abs(float(s.kbar1[k])) < 1e-13
        assert abs(float(s.taubar[k])) < 1e-13
    # the same star turned out of the plane: each limb's reference director
    # is z projected off its own tangent, so the two frames of a pair differ
    # by the reference twist beta (= taubar, theta being 0); averaging the
    # two material frames (Eq. 5) then gives
    # kappa1^2 + kappa2^2 = (2 tan(phi/2))^2 cos^2(beta/2)
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    o2 = OracleSystems(_star(ang, R=Q))
    s2 = o2.systems[0]
    twisted = 0
    for k in [k for k, g in enumerate(s2.st) if o2.st_rodslot[g] == -1]:
        a, b = o2.st_edges[s2.st[k]]
        phi = math.pi - math.acos(math.cos(ang[o2.edge_rod[b]] - ang[o2.edge_rod[a]]))
        beta = float(s2.taubar[k])
        twisted += abs(beta) > 1e-3
        kap = math.hypot(float(s2.kbar1[k]), float(s2.kbar2[k]))
        assert kap == pytest.approx(2.0 * math.tan(0.5 * phi) * abs(math.cos(0.5 * beta)),
                                    rel=1e-12)
    assert twisted > 0


# ---------------------------------------------------------------------------
# Averaged EI and GJ at a joint between different rods
# ---------------------------------------------------------------------------

def _two_rod_joint():
    # rod A (E_a, h_a, nu_a) ends at the joint, rod B (E_b, h_b, nu_b) starts
    # there; straight along +x at rest, different edge lengths
    la, lb = 0.02, 0.035
    xa = np.stack([np.linspace(-4 * la, 0.0, 5), np.zeros(5), np.zeros(5)], 1)
    xb = np.stack([np.linspace(0.0, 3 * lb, 4), np.zeros(4), np.zeros(4)], 1)
    E, nu, h = [3e6, 8e6], [0.5, 0.3], [1.5e-3, 1e-3]
    o = OracleSystems(_desc([xa, xb], E=E, nu=nu, rho=[1000.0, 1500.0], h=h,
                            joints=[[(0, 4), (1, 0)]]), dict(g=(0.0, 0.0, 0.0)))
    EI = [E[r] * math.pi * h[r] ** 4 / 4.0 for r in range(2)]
    GJ = [E[r] / (2.0 * (1.0 + nu[r])) * math.pi * h[r] ** 4 / 2.0 for r in range(2)]
    V = 0.5 * (la + lb)
    return o, o.systems[0], EI, GJ, V


@pytest.mark.parametrize("phi", [0.2, 0.9, 1.6])
def test_joint_kink_energy_uses_the_averaged_bending_stiffness(phi):
    o, s, EI, _, V = _two_rod_joint()
    # turn rod B rigidly about the joint in the x-y plane (d1 = z is kept
    # by the time-parallel transport): a kink of angle phi at the joint only
    q = s.q.clone()
    joint_x = q[s.node_dof[4]:s.node_dof[4] + 3].clone()
    c, sn = math.cos(phi), math.sin(phi)
    for k in range(len(s.nodes)):
        d = s.node_dof[k]
        p = q[d:d + 3] - joint_x
        if float(p[0]) > 1e-12:
            q[d:d + 3] = joint_x + torch.tensor([c * p[0] - sn * p[1], sn * p[0] + c * p[1],
                                                 p[2]], dtype=DT)
    kap = 2.0 * math.tan(0.5 * phi)
    expect = 0.5 * (0.5 * (EI[0] + EI[1]) / V) * kap ** 2
    assert float(_elastic_energy(o, s, q)) == pytest.approx(expect, rel=1e-12)


def test_joint_twist_energy_uses_the_averaged_twist_stiffness():
    o, s, _, GJ, V = _two_rod_joint()
    # uniform twist angle c on rod B's edges, none on rod A's: only the
    # joint stencil twists, by c (Eq. 7 with zero reference twist)
    cth = 0.37
    q = s.q.clone()
    for k, e in enumerate(s.edges):
        if o.edge_rod[e] == 1:
            q[s.edge_dof[k]] = cth
    expect = 0.5 * (0.5 * (GJ[0] + GJ[1]) / V) * cth ** 2
    assert float(_elastic_energy(o, s, q)) == pytest.approx(expect, rel=1e-12)


# ---------------------------------------------------------------------------
# Node masses at joints
# ---------------------------------------------------------------------------

def test_joint_node_mass_is_half_the_incident_edge_masses():
    ang = np.deg2rad([0.0, 80.0, 200.0])
    pts, lens = [], [0.03, 0.05, 0.02]
    for a, l in zip(ang, lens):
        s_ = np.arange(5) * l
        pts.append(np.stack([s_ * math.cos(a), s_ * math.sin(a), np.zeros(5)], 1))
    rho, h = [900.0, 1200.0, 2000.0], [1e-3, 2e-3, 1.5e-3]
    o = OracleSystems(_desc(pts, E=[1e6] * 3, nu=[0.5] * 3, rho=rho, h=h,
                            joints=[[(0, 0), (1, 0), (2, 0)]]))
    s = o.systems[0]
    edge_mass = [rho[r] * math.pi * h[r] ** 2 * lens[r] for r in range(3)]
    centre = [k for k in range(len(s.nodes)) if np.allclose(s.q[s.node_dof[k]:s.node_dof[k] + 3], 0)]
    assert len(centre) == 1
    d = s.node_dof[centre[0]]
    expect = 0.5 * sum(edge_mass)
    np.testing.assert_allclose(s.mass[d:d + 3].numpy(), expect, rtol=1e-14)
    # total translational mass = mass of the rods (nothing counted twice)
    total = float(s.mass[torch.as_tensor(np.concatenate([s.node_dof + c for c in range(3)]))].sum()) / 3
    assert total == pytest.approx(4 * sum(edge_mass), rel=1e-13)
    # twist inertia per edge: rho A h^2 l / 2 (reading C7)
    for k, e in enumerate(s.edges):
        r = o.edge_rod[e]
        assert float(s.mass[s.edge_dof[k]]) == pytest.approx(
            0.5 * rho[r] * math.pi * h[r] ** 4 * lens[r], rel=1e-13)


# ---------------------------------------------------------------------------
# Contact Jacobians by central differences (Eq. 10-13, readings C11-C15, C28)
# ---------------------------------------------------------------------------

def _fd_jacobian(o, s, q, qn, hstep):
    n = s.n
    fd = np.zeros((n, n))
    for j in range(n):
        dq = torch.zeros(n, dtype=DT)
        dq[j] = hstep
        Fp, _, _ = o.forces(s, q + dq, s.v, qn, need_jac=False)
        Fm, _, _ = o.forces(s, q - dq, s.v, qn, need_jac=False)
        fd[:, j] = -(Fp - Fm).numpy() / (2 * hstep)
    return fd


def test_ground_contact_and_friction_jacobian_matches_central_differences():
    # a 7-node rod lying on the ground, sliding: nodes in the quadratic
    # branch (D <= C - delta), in the softplus band and above it
    N, h, delta = 7, 1e-3, 5e-4
    x = np.zeros((N, 3))
    x[:, 0] = np.linspace(0.0, 0.06, N)
    x[:, 1] = 0.002 * np.sin(np.arange(N))
    z = np.array([h - 7e-4, h - 2e-4, h + 1e-4, h + 3e-4, h - 1e-4, h + 8e-4, h - 6e-4])
    x[:, 2] = z
    kc = 50.0 * 1000.0 * math.pi * h * h * 0.01 * 9.81 / delta
    d = _desc([x], E=[1e6], nu=[0.5], rho=[1000.0], h=[h], ground_mu=[0.6], ground_kc=[kc])
    prm = dict(dt=1e-2, ground=True, ground_z=0.0, delta=delta, nu_slip=1e-2, eta=0.1)
    o = OracleSystems(d, prm)
    s = o.systems[0]
    rng = np.random.default_rng(4)
    q = s.q.clone()
    qn = s.q.clone()
    nd = torch.as_tensor(s.node_dof)
    # previous positions: slips of 0.1-20 tangential speed units in random
    # directions, so every node slides (gamma away from its limit)
    for k in range(N):
        ang = rng.uniform(0, 2 * math.pi)
        sp = prm["nu_slip"] * 10 ** rng.uniform(-1, 1.3) * prm["dt"]
        qn[nd[k]] -= sp * math.cos(ang)
        qn[nd[k] + 1] -= sp * math.sin(ang)
        qn[nd[k] + 2] -= 1e-5 * rng.standard_normal()
    F, _, J = o.forces(s, q, s.v, qn, need_jac=True)
    # the contact terms are switched on at this state
    assert float(F[nd + 2].abs().max()) > 1e-3
    fd = _fd_jacobian(o, s, q, qn, 1e-9)
    sc = np.max(np.abs(fd))
    np.testing.assert_allclose(J.numpy(), fd, rtol=0, atol=2e-6 * sc)
    # friction makes J nonsymmetric, and the FD sees the same asymmetry
    asym = J.numpy() - J.numpy().T
    assert np.max(np.abs(asym)) > 1e-3 * sc
    np.testing.assert_allclose(asym, fd - fd.T, rtol=0, atol=4e-6 * sc)


def test_edge_pair_contact_and_friction_jacobian_matches_central_differences():
    # two crossing rods of one contact group: rod 1 along x, rod 2 along y
    # just above it, one pair in the softplus band and one inside C - delta
    h, delta = 1e-3, 2e-4
    x1 = np.stack([np.linspace(-0.03, 0.03, 4), np.zeros(4), np.zeros(4)], 1)
    gap = 2 * h - 0.5 * delta
    x2 = np.stack([np.full(4, 0.001), np.linspace(-0.03, 0.03, 4), np.full(4, gap)], 1)
    x2[1, 2] -= 0.9 * delta       # tilt: the crossing pair sits at varying depth
    d = _desc([x1, x2], E=[1e6] * 2, nu=[0.5] * 2, rho=[1000.0] * 2, h=[h] * 2,
              contact_groups=[[0, 1]])
    prm = dict(dt=1e-2, self_contact=True, delta=delta, pair_kc=1e3, pair_mu=0.4,
               nu_slip=1e-2, g=(0.0, 0.0, 0.0))
    o = OracleSystems(d, prm)
    s = o.systems[0]
    rng = np.random.default_rng(9)
    q = s.q.clone()
    # slip: rod 2 moved along x relative to rod 1 during the step
    qn = s.q.clone() - torch.as_tensor(2e-4 * rng.standard_normal(s.n))
    F, _, J = o.forces(s, q, s.v, qn, need_jac=True)
    from oracle.contact import pair_terms
    act = list(pair_terms(o, s, q, qn, False))
    assert act and len(act[0][0]) >= 1
    fd = _fd_jacobian(o, s, q, qn, 1e-10)
    sc = np.max(np.abs(fd))
    np.testing.assert_allclose(J.numpy(), fd, rtol=0, atol=2e-6 * sc)
