"""Pins of the CPU oracle against closed forms, invariances, finite
differences and textbook results (DisMech, arXiv 2311.18126, Sec. III-IV).

These run on the CPU only.  Each test is chosen so that a plausible mistake
in the oracle (a dropped term, a wrong sign or index, a transposed operand)
fails at least one of them."""
import json
import math
import os

import numpy as np
import pytest
import torch
from torch.func import grad, hessian, vmap

from oracle import OracleSystems, der

GOLD = os.path.join(os.path.dirname(__file__), "golden")
DT = torch.float64


def rod_desc(x, E=1e7, nu=0.5, rho=1000.0, h=1e-3, fixed=None, v0=None, theta0=None):
    x = np.asarray(x, dtype=np.float64)
    N = len(x)
    d = dict(nodes_per_rod=[N], x0=x, E=[E], nu=[nu], rho=[rho], radius=[h],
             fixed=np.zeros(4 * N - 1, np.uint8) if fixed is None else fixed)
    if v0 is not None:
        d["v0"] = v0
    if theta0 is not None:
        d["theta0"] = theta0
    return d


def clamp(N):
    m = np.zeros(4 * N - 1, np.uint8)
    m[0:8] = 1
    return m


def straight(N, L=1.0):
    x = np.zeros((N, 3))
    x[:, 0] = np.linspace(0, L, N)
    return x


def random_rod(N, seed, amp=0.2):
    rng = np.random.default_rng(seed)
    x = straight(N) + amp * rng.standard_normal((N, 3)) / N
    return x


# ---------------------------------------------------------------------------
# Eq. 4-5: kappa = 2 tan(phi/2) for a kink of turning angle phi
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("phi", [0.1, 0.7, 1.5, 2.5, 3.0])
def test_kink_curvature_closed_form(phi):
    # kink in the x-y plane: d1 = z stays normal to the plane
    x = np.array([[-1.0, 0, 0], [0, 0, 0], [math.cos(phi), math.sin(phi), 0]])
    o = OracleSystems(rod_desc(x))
    s = o.systems[0]
    k1, k2 = float(s.kbar1[0]), float(s.kbar2[0])
    assert abs(k1) < 1e-14
    # material frame m1 = d1 = z, m2 = t x z: in-plane bending is kappa2
    assert k2 == pytest.approx(-2.0 * math.tan(phi / 2.0), rel=1e-13)
    # kink in the x-z plane: bending about the d2 axis is kappa1
    x = np.array([[-1.0, 0, 0], [0, 0, 0], [math.cos(phi), 0, math.sin(phi)]])
    s = OracleSystems(rod_desc(x)).systems[0]
    assert abs(float(s.kbar2[0])) < 1e-13
    assert abs(float(s.kbar1[0])) == pytest.approx(2.0 * math.tan(phi / 2.0), rel=1e-13)


def test_arc_bending_energy_closed_form():
    # straight rest shape bent into an arc of turning angle phi per node:
    # E_b = sum 1/2 EI/V (2 tan(phi/2))^2 with V the rest Voronoi length
    N, phi, h, E = 9, 0.2, 1e-3, 1e7
    L = 1.0
    desc = rod_desc(straight(N, L), E=E, h=h)
    o = OracleSystems(desc)
    s = o.systems[0]
    ell = L / (N - 1)
    ang = phi * np.arange(N - 1)
    pts = np.concatenate([[[0, 0, 0]], np.cumsum(ell * np.stack(
        [np.cos(ang), np.sin(ang), np.zeros(N - 1)], 1), 0)])
    q = s.q.clone()
    for i in range(N):
        q[4 * i:4 * i + 3] = torch.as_tensor(pts[i])
    _, t = o._stencil_geometry(s, q)
    d1 = o._time_parallel_frames(s, t)
    sa, sb, ta, d1a, tb, d1b = o._oriented(s, t, d1)
    beta = der.reference_twist(ta, d1a, tb, d1b, s.beta)
    q11 = q[torch.as_tensor(s.st_dofs)]
    Eb = der.bend_energy_only(q11, sa, sb, ta, d1a, tb, d1b, beta,
                              torch.as_tensor(s.st_kb), s.kbar1, s.kbar2).sum()
    EI = E * math.pi * h ** 4 / 4
    expect = (N - 2) * 0.5 * EI / ell * (2 * math.tan(phi / 2)) ** 2
    assert float(Eb) == pytest.approx(expect, rel=1e-12)


# ---------------------------------------------------------------------------
# Eq. 7-8: uniform twist of a straight rod
# ---------------------------------------------------------------------------

def test_uniform_twist_end_moments():
    N, c, E, nu, h = 7, 0.3, 2e6, 0.25, 2e-3
    L = 0.6
    o = OracleSystems(rod_desc(straight(N, L), E=E, nu=nu, h=h))
    s = o.systems[0]
    q = s.q.clone()
    th = c * np.arange(N - 1)
    q[torch.as_tensor(s.edge_dof)] = torch.as_tensor(th)
    F, _, _ = o.forces(s, q, s.v, s.q, need_jac=False)
    G = E / (2 * (1 + nu))
    GJ = G * math.pi * h ** 4 / 2
    V = L / (N - 1)
    Mth = F[torch.as_tensor(s.edge_dof)].numpy()
    expect = np.zeros(N - 1)
    expect[0] = GJ * c / V          # -dE/dtheta^0 = +GJ tau / V
    expect[-1] = -GJ * c / V
    np.testing.assert_allclose(Mth, expect, rtol=1e-12, atol=1e-12 * GJ * c / V)
    # straight rod: twist exerts no force on the nodes, gravity aside
    Fx = F[torch.as_tensor(s.node_dof)[:, None] + torch.arange(3)].numpy()
    grav = s.mnode[:, None] * np.array([0, 0, -9.81])
    np.testing.assert_allclose(Fx, grav, atol=1e-12 * GJ * c / V)


# ---------------------------------------------------------------------------
# Forces are the negative gradients (Eq. 9): central finite differences
# ---------------------------------------------------------------------------

def _stencil_setup(seed):
    N = 6
    rng = np.random.default_rng(seed)
    x = random_rod(N, seed, amp=0.6)
    o = OracleSystems(rod_desc(x, theta0=0.3 * rng.standard_normal(N - 1)))
    s = o.systems[0]
    s.kbar1 = torch.as_tensor(rng.uniform(-0.3, 0.3, len(s.st)))
    s.kbar2 = torch.as_tensor(rng.uniform(-0.3, 0.3, len(s.st)))
    # move the rod away from its committed state
    q = s.q + torch.as_tensor(0.05 * rng.standard_normal(s.n) / N)
    return o, s, q


def _total_energy(o, s, qq):
    """Stretching + bending + twisting (frames time-transported from the
    committed step) + gravity potential of one system at DOF vector qq."""
    idx = torch.as_tensor(s.st_dofs)
    e6 = torch.as_tensor(s.edge_dofs6)
    Eb = der.time_transported_energy(qq[idx], *o._stencil_history(s)).sum()
    Es = der.stretch_energy(qq[e6], torch.as_tensor(s.EA), torch.as_tensor(s.lbar)).sum()
    x = qq[torch.as_tensor(s.node_dof)[:, None] + torch.arange(3)]
    Eg = -(torch.as_tensor(s.mnode)[:, None] * torch.tensor(o.p["g"], dtype=DT) * x).sum()
    return Eb + Es + Eg


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_forces_match_central_differences(seed):
    # Eq. 9: forces are minus the gradient of the energy
    o, s, q = _stencil_setup(seed)
    F, _, _ = o.forces(s, q, s.v, s.q, need_jac=False)
    hstep = 1e-6
    fd = np.zeros(s.n)
    for i in range(s.n):
        dq = torch.zeros(s.n, dtype=DT)
        dq[i] = hstep
        fd[i] = -(float(_total_energy(o, s, q + dq)) - float(_total_energy(o, s, q - dq))) / (2 * hstep)
    scale = np.max(np.abs(fd))
    np.testing.assert_allclose(F.numpy(), fd, atol=1e-7 * scale)


@pytest.mark.parametrize("seed", [3, 4])
def test_jacobian_matches_central_differences_and_is_symmetric(seed):
    # Eq. 16: J = -dF/dq, by central differences of the forces; it is the
    # Hessian of the energy, hence symmetric
    o, s, q = _stencil_setup(seed)
    _, _, J = o.forces(s, q, s.v, s.q, need_jac=True)
    hstep = 1e-6
    fd = np.zeros((s.n, s.n))
    for j in range(s.n):
        dq = torch.zeros(s.n, dtype=DT)
        dq[j] = hstep
        Fp, _, _ = o.forces(s, q + dq, s.v, s.q, need_jac=False)
        Fm, _, _ = o.forces(s, q - dq, s.v, s.q, need_jac=False)
        fd[:, j] = -(Fp - Fm).numpy() / (2 * hstep)
    sc = np.max(np.abs(fd))
    np.testing.assert_allclose(J.numpy(), fd, atol=1e-6 * sc)
    assert np.allclose(J.numpy(), J.numpy().T, atol=1e-12 * sc)


# ---------------------------------------------------------------------------
# Invariances: rigid motions
# ---------------------------------------------------------------------------

def _rotation(seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((3, 3))
    Q, R = np.linalg.qr(A)
    Q = Q * np.sign(np.diag(R))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


def test_rigid_motion_invariance():
    o, s, q = _stencil_setup(7)
    o.p["g"] = (0.0, 0.0, 0.0)
    F, _, _ = o.forces(s, q, s.v, s.q, need_jac=False)
    nd = torch.as_tensor(s.node_dof)[:, None] + torch.arange(3)
    x = q[nd].numpy()
    Fx = F[nd].numpy()
    M = F[torch.as_tensor(s.edge_dof)].numpy()
    _, t = o._stencil_geometry(s, q)
    # translation invariance: the nodal forces sum to zero
    assert np.allclose(Fx.sum(0), 0, atol=1e-10 * np.abs(Fx).max())
    E0 = float(_total_energy(o, s, q))
    # rotate everything (state, committed frames): forces rotate with it
    Rm = _rotation(1)
    R = torch.as_tensor(Rm)
    q2 = q.clone()
    q2[nd] = q[nd] @ R.T + torch.tensor([0.3, -1.0, 2.0], dtype=DT)
    s.d1 = s.d1 @ R.T
    s.tn = s.tn @ R.T
    F2, _, _ = o.forces(s, q2, s.v, s.q, need_jac=False)
    # the energy (with the committed frames rotated too) is unchanged
    assert float(_total_energy(o, s, q2)) == pytest.approx(E0, rel=1e-12, abs=1e-14)
    np.testing.assert_allclose(F2[nd].numpy(), Fx @ Rm.T, atol=1e-10 * np.abs(Fx).max())
    np.testing.assert_allclose(F2[torch.as_tensor(s.edge_dof)].numpy(), M,
                               atol=1e-10 * np.abs(Fx).max())


def test_linear_momentum_conserved():
    # no gravity, damping, contact or fixed DOFs: backward Euler keeps
    # sum m v exactly, because internal forces sum to zero
    N = 8
    rng = np.random.default_rng(11)
    x = random_rod(N, 11, amp=0.5)
    v0 = rng.standard_normal((N, 3))
    o = OracleSystems(rod_desc(x, v0=v0), dict(g=(0, 0, 0), dt=1e-3, eta=0.0))
    s = o.systems[0]
    nd = torch.as_tensor(s.node_dof)[:, None] + torch.arange(3)

    def mom():
        return (torch.as_tensor(s.mnode)[:, None] * s.v[nd]).sum(0).numpy()

    p0 = mom()
    for _ in range(5):
        st = o.step_system(s)
        assert st[0] == 0
    np.testing.assert_allclose(mom(), p0, atol=1e-12 * np.abs(p0).max())


# ---------------------------------------------------------------------------
# Time-parallel transport and reference twist: holonomy of a closed loop
# ---------------------------------------------------------------------------

def _ode_transport(d, path):
    """Parallel transport along a sampled unit-vector path by integrating
    dd/ds = -(d . dt/ds) t with RK4 on a fine reparametrisation."""
    for k in range(len(path) - 1):
        a, b = path[k], path[k + 1]
        for sub in range(2):
            def tt(u):
                v = a + u * (b - a)
                return v / np.linalg.norm(v)

            def rhs(u, dv):
                t = tt(u)
                h = 1e-6
                tdot = (tt(u + h) - tt(u - h)) / (2 * h)
                return -np.dot(dv, tdot) * t
            u0, du = sub / 2, 0.5
            k1 = rhs(u0, d)
            k2 = rhs(u0 + du / 2, d + du / 2 * k1)
            k3 = rhs(u0 + du / 2, d + du / 2 * k2)
            k4 = rhs(u0 + du, d + du * k3)
            d = d + du / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return d


def test_reference_twist_holonomy():
    # edge a fixed along x; edge b's tangent goes once around a cone about z
    # (half-angle alpha).  Time-parallel transport carries d1^b around the
    # loop; the continued reference twist must change by exactly the angle
    # that the transported director has turned, which is the enclosed solid
    # angle 2 pi (1 - cos alpha) (mod 2 pi) of the traced loop.
    alpha = 0.6
    n = 2000
    ph = np.linspace(0, 2 * math.pi, n + 1)
    path = np.stack([np.sin(alpha) * np.cos(ph), np.sin(alpha) * np.sin(ph),
                     np.full_like(ph, math.cos(alpha))], 1)
    ta = torch.tensor([1.0, 0, 0], dtype=DT)
    d1a = torch.tensor([0, 0, 1.0], dtype=DT)
    tb = torch.as_tensor(path[0])
    d1b = torch.as_tensor(np.cross(path[0], [0, 1.0, 0]))
    d1b = d1b / torch.linalg.vector_norm(d1b)
    beta = der.reference_twist(ta, d1a, tb, d1b, torch.tensor(0.0, dtype=DT))
    beta0 = float(beta)
    d1b_start = d1b.clone()
    for k in range(1, n + 1):
        tnew = torch.as_tensor(path[k])
        d1b = der.parallel_transport(d1b, tb, tnew)
        tb = tnew
        beta = der.reference_twist(ta, d1a, tb, d1b, beta)
    # independent ODE transport agrees with the minimal-rotation steps
    d_ode = _ode_transport(d1b_start.numpy(), path)
    assert np.allclose(d_ode, d1b.numpy(), atol=1e-7)
    turned = math.atan2(np.dot(path[0], np.cross(d1b_start.numpy(), d1b.numpy())),
                        np.dot(d1b_start.numpy(), d1b.numpy()))
    assert float(beta) - beta0 == pytest.approx(turned, abs=1e-9)
    solid = 2 * math.pi * (1 - math.cos(alpha))
    wrapped = (abs(turned) - solid + math.pi) % (2 * math.pi) - math.pi
    assert abs(wrapped) < 1e-4


# ---------------------------------------------------------------------------
# Newton: quadratic convergence with the exact Jacobian; banded == dense LU
# ---------------------------------------------------------------------------

def test_newton_quadratic_convergence():
    # one Newton step from q* + eps w has error O(eps^2) (exact Jacobian,
    # Eq. 16 in full): err/eps^2 stays constant as eps shrinks.  A dropped or
    # wrong Jacobian term makes it grow like 1/eps.
    N = 10
    rng = np.random.default_rng(5)
    desc = rod_desc(straight(N, 0.5), E=1e6, h=2e-3, fixed=clamp(N),
                    v0=np.c_[np.zeros(N), 0.5 * rng.standard_normal(N), rng.standard_normal(N)])
    p = dict(dt=0.01, tol=1e-15, max_iter=40, eta=0.0)
    o = OracleSystems(desc, p)
    s = o.systems[0]
    s.kbar1 = torch.full((N - 2,), 0.05, dtype=DT)
    q_n, v_n = s.q.clone(), s.v.clone()
    hist = (s.tn.clone(), s.d1.clone(), s.beta.clone())
    assert o.step_system(s)[0] == 0
    qstar = s.q.clone()
    # the step committed its frames: restore the history of the step that
    # produced q* before evaluating its residual
    s.q, s.v = q_n, v_n
    s.tn, s.d1, s.beta = hist
    w = torch.as_tensor(rng.standard_normal(s.n))
    w = torch.where(s.fixed, torch.zeros_like(w), w)
    w = w / torch.linalg.vector_norm(w)
    ratios = []
    for eps in (1e-3, 1e-4, 1e-5):
        q0 = qstar + eps * w
        f, _, J = o.residual(s, q0, q_n, v_n, need_jac=True)
        q1 = q0 + o.solve(s, J, -f)
        ratios.append(float(torch.linalg.vector_norm(q1 - qstar)) / eps ** 2)
    assert ratios[2] < 2.0 * ratios[1] and ratios[1] < 2.0 * ratios[0]


def test_banded_and_dense_solves_agree():
    o, s, q = _stencil_setup(9)
    f, _, J = o.residual(s, q, s.q, s.v, need_jac=True)
    x_band = o.solve(s, J, -f).numpy()
    x_dense = np.linalg.solve(J.numpy(), -f.numpy())
    np.testing.assert_allclose(x_band, x_dense, rtol=1e-10, atol=1e-14 * np.abs(x_dense).max())


# ---------------------------------------------------------------------------
# Euler-Bernoulli statics and the first cantilever mode (Sec. IV-A)
# ---------------------------------------------------------------------------

def _static_tip(N, E=1e11, h=1e-2, L=1.0, rho=1000.0):
    desc = rod_desc(straight(N, L), E=E, h=h, rho=rho, fixed=clamp(N))
    o = OracleSystems(desc, dict(dt=1e3, g=(0, 0, -9.81), eta=0.0, tol=1e-12))
    s = o.systems[0]
    for _ in range(3):
        st = o.step_system(s)
        assert st[0] == 0
        s.v.zero_()
    return -float(s.q[4 * (N - 1) + 2])


def test_euler_bernoulli_static_cantilever():
    E, h, L, rho, g = 1e11, 1e-2, 1.0, 1000.0, 9.81
    A, I = math.pi * h * h, math.pi * h ** 4 / 4
    errs = []
    for N in (11, 21):
        # nodes 0 and 1 clamped: the beam is built in at the middle of the
        # clamped edge, where the first free stencil's Voronoi cell begins
        Leff = L - 0.5 * L / (N - 1)
        w = rho * A * g * Leff ** 4 / (8 * E * I)
        errs.append(abs(_static_tip(N) - w) / w)
    assert errs[1] < 0.003
    assert errs[1] < errs[0]


def test_cantilever_first_mode_frequency():
    gold = json.load(open(os.path.join(GOLD, "table2_cantilever.json")))
    h, rho, L, E = gold["radius"], gold["rho"], gold["length"], gold["a1"]["E"]
    N = 21
    ell = L / (N - 1)
    Leff = L - 0.5 * ell                     # built in mid clamped edge
    A, I = math.pi * h * h, math.pi * h ** 4 / 4
    omega = (gold["beta1_L"] / Leff) ** 2 * math.sqrt(E * I / (rho * A))
    # initial velocity in the first mode shape, tip speed from the paper
    bl = gold["beta1_L"]
    sig = (math.sinh(bl) - math.sin(bl)) / (math.cosh(bl) + math.cos(bl))
    s_ = np.clip(np.linspace(0, L, N) - 0.5 * ell, 0, None) * bl / Leff

    def phi(u):
        return np.cosh(u) - np.cos(u) - sig * (np.sinh(u) - np.sin(u))
    v0 = np.zeros((N, 3))
    v0[:, 2] = gold["tip_velocity"] * phi(s_) / phi(bl)
    v0[:2] = 0
    desc = rod_desc(straight(N, L), E=E, h=h, rho=rho, fixed=clamp(N), v0=v0)
    dt = 0.05
    o = OracleSystems(desc, dict(dt=dt, g=(0, 0, 0), eta=0.0))
    s = o.systems[0]
    zs = [0.0]
    half = math.pi / omega
    for _ in range(int(1.3 * half / dt)):
        assert o.step_system(s)[0] == 0
        zs.append(float(s.q[4 * (N - 1) + 2]))
    zs = np.array(zs)
    k = np.nonzero((zs[1:-1] > 0) & (zs[2:] <= 0))[0][0] + 1
    tz = dt * (k + zs[k] / (zs[k] - zs[k + 1]))
    assert tz == pytest.approx(half, rel=0.02)


# ---------------------------------------------------------------------------
# Ground contact with friction: the closed form of Sec. IV-C
# ---------------------------------------------------------------------------

def _sliding_energy(push, T, integ="be"):
    gold = json.load(open(os.path.join(GOLD, "friction_validation.json")))
    h, rho, L, E, mu = gold["radius"], gold["rho"], gold["length"], gold["E"], gold["mu"]
    g = gold["g"]
    N = 11                                   # rigid sliding: N does not matter
    x = straight(N, L)
    x[:, 2] = h
    m = rho * math.pi * h * h * L
    mnode = m / (N - 1)
    kc = 50.0 * mnode * g / gold["delta"]    # reading C11
    desc = rod_desc(x, E=E, h=h, rho=rho, nu=gold["nu"])
    desc["ground_mu"] = [mu]
    desc["ground_kc"] = [kc]
    p = dict(dt=gold["dt"], g=(0.0, 0.0, -g), eta=0.0, ground=True, ground_z=0.0,
             delta=gold["delta"], nu_slip=gold["slip_nu"], integrator=integ)
    o = OracleSystems(desc, p)
    s = o.systems[0]
    for _ in range(40):                      # settle onto the floor at rest
        assert o.step_system(s)[0] == 0
        s.v.zero_()
    # the push is a uniform body force: gravity gains an x component
    o.p["g"] = (push / m, 0.0, -g)
    for _ in range(int(round(T / gold["dt"]))):
        assert o.step_system(s)[0] == 0
    nd = torch.as_tensor(s.node_dof)[:, None] + torch.arange(3)
    v = s.v[nd].numpy()
    Ek = 0.5 * float(np.sum(s.mnode[:, None] * v * v))
    return Ek, m, mu, g


@pytest.mark.parametrize("push,integ", [(10.5, "be"), (3.0, "be"), (10.5, "midpoint")])
def test_friction_kinetic_energy_closed_form(push, integ):
    # (the midpoint takes the friction at the mid-step velocity; under a
    # constant net force both schemes follow the closed form)
    T = 0.5
    Ek, m, mu, g = _sliding_energy(push, T, integ)
    if push <= mu * m * g:
        assert Ek < 1e-6
    else:
        expect = T * T / (2 * m) * (push - mu * m * g) ** 2
        assert Ek == pytest.approx(expect, rel=0.03)


# ---------------------------------------------------------------------------
# Warm-start network reference: backward pass = finite differences of the loss
# ---------------------------------------------------------------------------

def test_mlp_reference_gradient_matches_central_differences():
    from oracle import mlp
    rng = np.random.default_rng(0)
    n = sum(fo * fi + fo for fi, fo in zip(mlp.DIN, mlp.DOUT))
    params = rng.standard_normal(n) * 0.05
    X = np.zeros((6, 64))
    X[:, :20] = rng.standard_normal((6, 20))
    Y = rng.standard_normal((6, 4))
    loss, g = mlp.loss_and_grad(params, X, Y, 4)
    idx = rng.choice(n, size=40, replace=False)
    h = 1e-6
    for i in idx:
        p1 = params.copy()
        p1[i] += h
        p2 = params.copy()
        p2[i] -= h
        fd = (mlp.loss_and_grad(p1, X, Y, 4)[0] - mlp.loss_and_grad(p2, X, Y, 4)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9


def test_segment_distance_matches_brute_force():
    """Eq. 10's D: the clamped closest-point rule against a brute-force
    minimum over the two segment parameters (grid, then local refinement)."""
    from scipy.optimize import minimize
    from oracle.contact import segment_distance
    rng = np.random.default_rng(11)
    for _ in range(40):
        p = rng.normal(size=(4, 3))
        if rng.random() < 0.3:  # nearly parallel pairs too
            p[3] = p[2] + (p[1] - p[0]) * rng.uniform(0.5, 2) + 1e-3 * rng.normal(size=3)
        P = torch.as_tensor(p)
        D, s, t = segment_distance(P[0], P[1], P[2], P[3])
        f = lambda st: np.linalg.norm(p[0] + st[0] * (p[1] - p[0]) - p[2] - st[1] * (p[3] - p[2]))
        g = np.linspace(0, 1, 101)
        best = min(((f((a, b)), a, b) for a in g for b in g))
        r = minimize(f, x0=[best[1], best[2]], bounds=[(0, 1), (0, 1)], method="L-BFGS-B",
                     options=dict(ftol=1e-15, gtol=1e-12))
        ref = min(best[0], r.fun)
        assert float(D) <= ref + 1e-9
        assert float(D) >= ref - 1e-6 * max(1.0, ref)


def test_imc_energy_branches():
    """Eq. 10: zero beyond C + delta, (C - D)^2 below C - delta, and the
    smooth branch joining both (to the accuracy K1 = 15/delta allows)."""
    from oracle.der import imc_energy
    C, delta = 2e-3, 1e-4
    D = torch.tensor([C + 1.01 * delta, C - 1.5 * delta, C - delta * (1 + 1e-9),
                      C - delta * (1 - 1e-9), C + delta * (1 - 1e-9)], dtype=torch.float64)
    E = imc_energy(D, torch.full_like(D, C), delta)
    assert float(E[0]) == 0.0
    assert abs(float(E[1]) - (1.5 * delta) ** 2) < 1e-20
    assert abs(float(E[2]) - float(E[3])) <= 1e-6 * float(E[2])
    assert float(E[4]) <= 1e-12 * delta ** 2


def test_edge_pair_friction_closed_form():
    """Eq. 12-13 at touching edges: two crossing segments (a along x at
    z = 0, b along y at height D < C - delta), b sliding fast along x.  The
    net friction on b is -mu |F_con| x (gamma -> 1), +mu |F_con| x on a, split
    equally between the nodes of each edge at a midpoint crossing, with
    |F_con| = k_c 2 (C - D) on the quadratic branch of Eq. 10."""
    from oracle.contact import _pair_friction
    C, delta, kc, mu, nu, dt = 2e-3, 1e-4, 1e4, 0.3, 1e-3, 1e-3
    D = 1.5e-3
    x = torch.tensor([-1.0, 0, 0, 1.0, 0, 0, 0, -1.0, D, 0, 1.0, D], dtype=torch.float64) * \
        torch.tensor([1e-2, 1, 1, 1e-2, 1, 1, 1, 1e-2, 1, 1, 1e-2, 1], dtype=torch.float64)
    v = 0.5  # m/s along x for edge b: K2 |u| = 7500, gamma = 1 to rounding
    xn = x.clone()
    xn[6] -= v * dt
    xn[9] -= v * dt
    T = lambda z: torch.tensor(z, dtype=torch.float64)
    F = _pair_friction(x, xn, T(C), T(delta), T(kc), T(mu), T(nu), T(dt))
    Fn = kc * 2.0 * (C - D)
    Fa = F[0:3] + F[3:6]
    Fb = F[6:9] + F[9:12]
    np.testing.assert_allclose(Fb.numpy(), [-mu * Fn, 0, 0], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Fa.numpy(), [mu * Fn, 0, 0], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(F[0:3].numpy(), F[3:6].numpy(), rtol=1e-12, atol=1e-15)
    # no friction without relative motion
    F0 = _pair_friction(x, x + 1e-30, T(C), T(delta), T(kc), T(mu), T(nu), T(dt))
    assert float(torch.abs(F0).max()) < 1e-20


@pytest.mark.parametrize("integ", ["be", "midpoint"])
def test_step_adjoint_matches_central_differences(integ):
    """The oracle's one-step adjoint (implicit function theorem) against
    central differences of the oracle's own step, for natural curvatures and
    the initial state, the committed frames (directors, reference twist and
    tangents) held fixed: every evaluation restarts from the same step-n
    frames.  Backward Euler and implicit midpoint."""
    import workloads
    from oracle import OracleSystems
    from oracle.adjoint import step_adjoint
    desc, params = workloads.cantilever(N=10)
    o = OracleSystems(desc, dict(params, integrator=integ))
    rng = np.random.default_rng(4)
    kb0 = rng.uniform(-0.02, 0.02, size=(8, 2))
    o.set_natural_curvature(0, 1, kb0)
    for _ in range(3):
        o.step(1)
    q0, v0 = o.get_state()
    d1, beta = o.get_frames()
    tn = [s.tn.clone() for s in o.systems]  # committed tangents, held fixed too
    wq = rng.normal(size=len(q0))
    wv = rng.normal(size=len(q0))

    def loss(kb, q, v):
        o.set_state(q, v)
        o.set_frames(d1, beta)
        for s, t in zip(o.systems, tn):
            s.tn = t.clone()
        o.set_natural_curvature(0, 1, kb)
        out = o.step(1)
        assert out[0][0] == 0
        q1, v1 = o.get_state()
        return float(wq @ q1 + wv @ v1), q1

    _, q1 = loss(kb0, q0, v0)
    o.set_state(q0, v0)
    o.set_frames(d1, beta)
    o.set_natural_curvature(0, 1, kb0)
    gk, gq0, gv0 = step_adjoint(o, q1, wq, wv)
    h = 1e-6
    for (i, c) in [(0, 0), (3, 1), (7, 0)]:
        kp = kb0.copy(); kp[i, c] += h
        km = kb0.copy(); km[i, c] -= h
        fd = (loss(kp, q0, v0)[0] - loss(km, q0, v0)[0]) / (2 * h)
        assert abs(fd - gk[i, c]) <= 1e-5 * max(1.0, abs(fd)), (i, c, fd, gk[i, c])
    for j in [9, 14, 30]:  # free DOFs (positions and a twist angle)
        for vec, g in ((0, gq0), (1, gv0)):
            qp, vp = q0.copy(), v0.copy()
            qm, vm = q0.copy(), v0.copy()
            hh = 1e-7
            if vec == 0:
                qp[j] += hh; qm[j] -= hh
            else:
                vp[j] += hh; vm[j] -= hh
            fd = (loss(kb0, qp, vp)[0] - loss(kb0, qm, vm)[0]) / (2 * hh)
            assert abs(fd - g[j]) <= 1e-4 * max(1.0, abs(fd)), (vec, j, fd, g[j])


# ---------------------------------------------------------------------------
# Implicit midpoint (Sec. III-C offers it beside backward Euler; the
# textbook rule): exact on a linear oscillator, energy-conserving where
# backward Euler dissipates
# ---------------------------------------------------------------------------

def test_midpoint_linear_oscillator_closed_form():
    # one edge along x, node 0 and the twist clamped, node 1 moving axially:
    # the stretch force -EA y / l is linear in the extension y, so the
    # midpoint rule is the linear map y' = ((1 - a^2 w) y + 2 a v)/(1 + a^2 w),
    # v' = v - a w (y + y') with a = dt/2, w = EA/(l m1), m1 = rho A l / 2,
    # which keeps w y^2 + v^2 exactly
    E, h, rho, l, dt, v0 = 1e7, 1e-3, 1000.0, 0.1, 2e-5, 0.3
    x = np.array([[0.0, 0.0, 0.0], [l, 0.0, 0.0]])
    fixed = np.zeros(7, np.uint8)
    fixed[0:4] = 1
    vel = np.zeros((2, 3))
    vel[1, 0] = v0
    o = OracleSystems(rod_desc(x, E=E, h=h, rho=rho, fixed=fixed, v0=vel),
                      dict(g=(0, 0, 0), dt=dt, eta=0.0, integrator="midpoint"))
    s = o.systems[0]
    A = math.pi * h * h
    w = E * A / (l * rho * A * l / 2)
    a = dt / 2
    y, v = 0.0, v0
    amp = v0 / math.sqrt(w)
    for _ in range(240):  # about one period (222 steps)
        yn = ((1 - a * a * w) * y + 2 * a * v) / (1 + a * a * w)
        v = v - a * w * (y + yn)
        y = yn
        st = o.step_system(s)
        assert st[0] == 0
        assert abs(float(s.q[4]) - l - y) <= 1e-9 * amp
        assert abs(float(s.v[4]) - v) <= 1e-9 * v0
    assert abs(w * y * y + v * v - v0 * v0) <= 1e-12 * v0 * v0


def test_midpoint_momentum_and_energy():
    # free rod with a natural curvature released straight, no gravity or
    # damping: both schemes keep sum m v; the midpoint keeps the total
    # energy (kinetic + elastic) to 0.1 % while backward Euler dissipates
    # more than 10 % of it in the same 150 steps
    N = 12
    out = {}
    for integ in ("midpoint", "be"):
        rng = np.random.default_rng(3)
        vel = 0.01 * rng.standard_normal((N, 3))
        o = OracleSystems(rod_desc(straight(N, 0.2), E=1e6, h=2e-3, v0=vel),
                          dict(g=(0, 0, 0), dt=1e-3, eta=0.0, integrator=integ))
        s = o.systems[0]
        s.kbar1 = torch.full((len(s.st),), 0.15, dtype=DT)
        nd = torch.as_tensor(s.node_dof)[:, None] + torch.arange(3)

        def energy():
            return 0.5 * float((s.mass * s.v * s.v).sum()) + float(_total_energy(o, s, s.q))

        def mom():
            return (torch.as_tensor(s.mnode)[:, None] * s.v[nd]).sum(0).numpy()

        E0, p0 = energy(), mom()
        Es = []
        for _ in range(150):
            assert o.step_system(s)[0] == 0
            Es.append(energy())
        np.testing.assert_allclose(mom(), p0, atol=1e-12 * np.abs(p0).max())
        out[integ] = (E0, np.array(Es))
    E0, Es = out["midpoint"]
    assert np.abs(Es - E0).max() <= 1e-3 * E0
    E0, Es = out["be"]
    assert Es[-1] < 0.9 * E0


def test_contact_group_pair_candidates_brute_force():
    # two 6-node rods declared one contact group: one system, and the
    # candidate edge pairs (reading C16) are every pair of edges of
    # different rods plus the pairs of one rod at least three edges apart,
    # enumerated here by brute force
    from oracle.contact import pair_candidates_all
    x0 = np.concatenate([straight(6, 0.05), straight(6, 0.05) + [0.0, 0.01, 0.0]])
    desc = dict(nodes_per_rod=[6, 6], x0=x0, E=[1e6] * 2, nu=[0.5] * 2, rho=[1e3] * 2,
                radius=[1e-3] * 2, contact_groups=[[0, 1]])
    o = OracleSystems(desc, dict(self_contact=True, pair_kc=1.0, delta=1e-4))
    assert len(o.systems) == 1
    s = o.systems[0]
    got = {tuple(p) for p in pair_candidates_all(o, s).tolist()}
    want = set()
    ne = len(s.edges)
    for i in range(ne):
        for j in range(i + 1, ne):
            ri, rj = s.edge_rod[i], s.edge_rod[j]
            if ri != rj or abs(i - j) >= 3:
                want.add((i, j))
    assert got == want and len(want) == 25 + 2 * 3
    # without the group the rods are two systems
    desc.pop("contact_groups")
    assert len(OracleSystems(desc, dict(self_contact=True, pair_kc=1.0)).systems) == 2


@pytest.mark.parametrize("integ", ["be", "midpoint"])
def test_damped_axial_oscillator_exact_step_map(integ):
    # one edge along x, node 0 and the twist clamped: node 1 is a linear
    # oscillator m y'' = -k y - c y' with k = EA/l, m = rho A l/2 and the
    # viscous damping of reading C8, c = eta V = eta l/2, taken at the
    # implicit (backward Euler) or mid-step (midpoint) velocity.  Each step
    # of either scheme is a 2x2 linear map of (y, v), solved here directly.
    E, h, rho, l, dt, v0, eta = 1e7, 1e-3, 1000.0, 0.1, 2e-5, 0.3, 0.05
    x = np.array([[0.0, 0.0, 0.0], [l, 0.0, 0.0]])
    fixed = np.zeros(7, np.uint8)
    fixed[0:4] = 1
    vel = np.zeros((2, 3))
    vel[1, 0] = v0
    o = OracleSystems(rod_desc(x, E=E, h=h, rho=rho, fixed=fixed, v0=vel),
                      dict(g=(0, 0, 0), dt=dt, eta=eta, integrator=integ))
    s = o.systems[0]
    A = math.pi * h * h
    m, k, c = rho * A * l / 2, E * A / l, eta * l / 2
    if integ == "be":
        # y' = y + dt v', m (v' - v) = dt (-k y' - c v')
        Mx = np.array([[1.0, -dt], [dt * k, m + dt * c]])
        rhs = lambda y, v: np.array([y, m * v])
    else:
        # y' = y + dt (v + v')/2, m (v' - v) = dt (-k (y + y')/2 - c (y' - y)/dt)
        Mx = np.array([[1.0, -dt / 2], [dt * k / 2 + c, m]])
        rhs = lambda y, v: np.array([y + dt * v / 2, m * v - dt * k * y / 2 + c * y])
    y, v = 0.0, v0
    amp = v0 * math.sqrt(m / k)
    for _ in range(150):
        y, v = np.linalg.solve(Mx, rhs(y, v))
        assert o.step_system(s)[0] == 0
        assert abs(float(s.q[4]) - l - y) <= 1e-9 * amp
        assert abs(float(s.v[4]) - v) <= 1e-9 * v0


def test_mlp_gradient_error_scale_bounds_and_matches_positive_terms():
    # the element-wise error scale of the network gradients (sum of the
    # absolute values of the terms) is at least |gradient| everywhere, and
    # equals the gradient where every term is non-negative: positive inputs
    # and weights, outputs above their targets
    from oracle import mlp
    rng = np.random.default_rng(3)
    n = sum(fo * fi + fo for fi, fo in zip(mlp.DIN, mlp.DOUT))
    X = mlp.bf16(rng.standard_normal((64, 64)))
    Y = rng.standard_normal((64, 64))
    p = 0.05 * rng.standard_normal(n)
    _, g = mlp.loss_and_grad(p, X, Y, 4, rounding=True)
    S = mlp.grad_abs_scale(p, X, Y, 4)
    assert np.all(S >= np.abs(g) * (1 - 2.0 ** -6) - 1e-30)
    assert np.max(S) > 0
    Xp = mlp.bf16(np.abs(X))
    pp = np.abs(p)
    Yp = np.full_like(Y, -10.0)
    _, gp = mlp.loss_and_grad(pp, Xp, Yp, 4, rounding=True)
    Sp = mlp.grad_abs_scale(pp, Xp, Yp, 4)
    np.testing.assert_allclose(gp, Sp, rtol=2.0 ** -6, atol=1e-30)


def test_length_projected_guess_keeps_committed_lengths_and_the_root():
    # the optional length-projected starting guess: every free edge takes
    # its committed length along the extrapolated direction, fixed nodes
    # stay, and Newton from it reaches the root Newton reaches from the
    # extrapolation (within what the 1e-10 tolerance allows)
    import workloads
    desc, params, kbar = workloads.uneven_rods(n_rods=3, seed=4)
    outs = []
    for pred in ("extrapolate", "projected"):
        o = OracleSystems(desc, dict(params, predictor=pred))
        o.set_natural_curvature(0, 3, kbar)
        for _ in range(3):
            o.step(1)
        outs.append(o)
    o = outs[1]
    for s in o.systems:
        q_n = s.q
        rng = np.random.default_rng(0)
        guess = q_n + torch.as_tensor(0.01 * rng.standard_normal(s.n))
        guess = torch.where(s.fixed, q_n, guess)
        p = o._project_lengths(s, guess, q_n)
        nd = s.node_dof
        for k in range(1, len(nd)):
            a, b = nd[k - 1], nd[k]
            if bool(s.fixed[b:b + 3].any()):
                assert torch.equal(p[b:b + 3], q_n[b:b + 3])
                continue
            ln = torch.linalg.vector_norm(q_n[b:b + 3] - q_n[a:a + 3])
            e = p[b:b + 3] - p[a:a + 3]
            assert float(torch.linalg.vector_norm(e)) == pytest.approx(float(ln), rel=1e-14)
            g = guess[b:b + 3] - guess[a:a + 3]
            cosang = float(der.dot(e, g) / (torch.linalg.vector_norm(e) * torch.linalg.vector_norm(g)))
            assert cosang == pytest.approx(1.0, abs=1e-14)
        # twist angles are left as guessed
        assert torch.equal(p[torch.as_tensor(s.edge_dof)], guess[torch.as_tensor(s.edge_dof)])
    qa, _ = outs[0].get_state()
    qb, _ = outs[1].get_state()
    assert np.max(np.abs(qa - qb)) <= 1e-8 * max(1.0, np.max(np.abs(qa)))
