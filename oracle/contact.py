"""Ground and edge-edge contact with smooth Coulomb friction for the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. III-B of the DisMech paper (arXiv 2311.18126):
* Eq. 10: IMC contact energy of the minimum distance D, with K1 = 15/delta.
* Eq. 11: contact force = -(dE/dD) (dD/dq).
* Eq. 12-13: friction gamma(|u|) with K2 = 15/nu, F_fr = -mu gamma u_hat |F_con|,
  on the ground and at the closest points of touching edge pairs.

Readings (design notes): the energy is multiplied by a stiffness k_c (C11);
the quadratic branch extends to D <= 0 for the ground (C12); the tangential
velocity is the implicit one (x - x_n)/dt (C26); at u = 0 the friction force
is its limit 0 and its Jacobian the limit of the smooth law (C14); the
Jacobian includes the derivative of |F_con| (C15).
"""
import numpy as np
import torch
from torch.func import grad, jacfwd, vmap

from . import der

DT = torch.float64


def _ground_energy(z, C, delta, zg):
    return der.imc_energy(z - zg, C, delta)


def ground_terms(osys, s, x, xn, need_jac):
    """Per node: contact force along +z and friction in the ground plane.
    Yields (F [Nn,3], Jint [Nn,3,3]) pairs where Jint = -dF/dx."""
    p = osys.p
    dt = osys.dt_vel  # velocity interval (the step; half of it at the midpoint)
    delta = float(p["delta"])
    zg = float(p["ground_z"])
    kc = torch.as_tensor(s.gkc, dtype=DT)
    C = torch.as_tensor(s.hnode, dtype=DT)
    mu = torch.as_tensor(s.gmu, dtype=DT)
    z = x[:, 2]
    dE = vmap(grad(_ground_energy))(z, C, torch.full_like(z, delta),
                                    torch.full_like(z, zg))
    d2E = vmap(grad(grad(_ground_energy)))(z, C, torch.full_like(z, delta),
                                           torch.full_like(z, zg))
    Fn = -kc * dE                                     # Eq. 11, along +z
    Fc = torch.zeros_like(x)
    Fc[:, 2] = Fn
    Jc = None
    if need_jac:
        Jc = torch.zeros(x.shape[0], 3, 3, dtype=DT)
        Jc[:, 2, 2] = kc * d2E
    yield Fc, Jc

    # friction (Eq. 12-13) with the implicit tangential velocity
    nu = float(p["nu_slip"])
    K2 = 15.0 / nu

    def fr_force(xi, xni, kci, Ci, mui):
        u = (xi - xni) / dt
        u = torch.stack([u[0], u[1], torch.zeros_like(u[0])])
        sp = torch.linalg.vector_norm(u)
        fn = torch.abs(kci * grad(_ground_energy)(xi[2], Ci, torch.tensor(delta, dtype=DT),
                                                  torch.tensor(zg, dtype=DT)))
        gam = der.friction_gamma(sp, nu)
        return -mui * gam * u / sp * fn

    u = (x - xn) / dt
    sp = torch.linalg.vector_norm(u[:, 0:2], dim=1)
    moving = (sp > 0) & (mu > 0) & (Fn != 0)
    Ff = torch.zeros_like(x)
    Jf = torch.zeros(x.shape[0], 3, 3, dtype=DT) if need_jac else None
    idx = torch.nonzero(moving).reshape(-1)
    if len(idx):
        args = (x[idx], xn[idx], kc[idx], C[idx], mu[idx])
        Ff[idx] = vmap(fr_force)(*args)
        if need_jac:
            Jf[idx] = -vmap(jacfwd(fr_force))(*args)
    if need_jac:
        still = torch.nonzero((sp == 0) & (mu > 0) & (Fn != 0)).reshape(-1)
        if len(still):
            # limit of -mu |Fn| gamma(|u|) u/|u| as u -> 0: -mu |Fn| K2/2 u
            c = mu[still] * torch.abs(Fn[still]) * K2 / (2.0 * dt)
            Jf[still, 0, 0] = c
            Jf[still, 1, 1] = c
    yield Ff, Jf


# ---------------------------------------------------------------------------
# edge-edge contact
# ---------------------------------------------------------------------------

def segment_distance(p0, p1, q0, q1):
    """Minimum distance between segments [p0,p1] and [q0,q1] (Eq. 10's D).

    Closest parameters by the clamp-s-then-t rule (reading C17): the
    unconstrained minimiser is clamped in s, t is recomputed for that s and
    clamped, and s is recomputed for the clamped t and clamped again.  Near
    parallel segments (|a x b|^2 < 1e-12 |a|^2 |b|^2) take s = 0."""
    a = p1 - p0
    b = q1 - q0
    r = p0 - q0
    A = der.dot(a, a)
    B = der.dot(a, b)
    Cc = der.dot(b, b)
    Dd = der.dot(a, r)
    Ee = der.dot(b, r)
    den = A * Cc - B * B
    par = den < 1e-12 * A * Cc
    s = torch.where(par, torch.zeros_like(A),
                    torch.clamp((B * Ee - Cc * Dd) / torch.where(par, torch.ones_like(den), den), 0.0, 1.0))
    t = torch.clamp((B * s + Ee) / Cc, 0.0, 1.0)
    s = torch.clamp((B * t - Dd) / A, 0.0, 1.0)
    d = (p0 + s[..., None] * a) - (q0 + t[..., None] * b)
    return torch.linalg.vector_norm(d, dim=-1), s, t


def pair_candidates_all(osys, s):
    """Edge pairs that may touch (reading C16): on one rod, pairs that share a
    node or are one edge apart are excluded; on different rods, pairs that
    share a (joint) node are excluded."""
    ne = len(s.edges)
    nl = s.edge_nl
    rods = s.edge_rod
    idx = s.edges - osys.edge_off[rods]          # edge index within its rod
    pairs = []
    for i in range(ne):
        for j in range(i + 1, ne):
            if len({nl[i, 0], nl[i, 1], nl[j, 0], nl[j, 1]}) < 4:
                continue
            if rods[i] == rods[j] and abs(int(idx[j]) - int(idx[i])) <= 2:
                continue
            pairs.append((i, j))
    return np.array(pairs, dtype=np.int64).reshape(-1, 2)


def _pair_energy(x12, C, delta, kc):
    D, _, _ = segment_distance(x12[0:3], x12[3:6], x12[6:9], x12[9:12])
    return kc * der.imc_energy(D, C, delta)


def pair_terms(osys, s, q, q_n, need_jac):
    """Contact forces between edge pairs closer than C + delta at the
    current iterate (the active set is a pure function of q)."""
    p = osys.p
    delta = float(p["delta"])
    kc = float(p["pair_kc"])
    cand = s.pair_cand
    if len(cand) == 0:
        return
    nd = torch.as_tensor(s.node_dof)
    nl = torch.as_tensor(s.edge_nl)
    i, j = torch.as_tensor(cand[:, 0]), torch.as_tensor(cand[:, 1])
    dofs = torch.stack([nd[nl[i, 0]], nd[nl[i, 1]], nd[nl[j, 0]], nd[nl[j, 1]]], 1)
    dofs = (dofs[:, :, None] + torch.arange(3)).reshape(-1, 12)
    x12 = q[dofs]
    C = torch.as_tensor(s.h_edge[cand[:, 0]] + s.h_edge[cand[:, 1]], dtype=DT)
    D, _, _ = segment_distance(x12[:, 0:3], x12[:, 3:6], x12[:, 6:9], x12[:, 9:12])
    if torch.any(D <= 0):
        raise FloatingPointError("edge-edge penetration (reading C12)")
    act = torch.nonzero(D < C + delta).reshape(-1)
    if len(act) == 0:
        return
    xa = x12[act]
    Ca = C[act]
    dl = torch.full_like(Ca, delta)
    kk = torch.full_like(Ca, kc)
    g = vmap(grad(_pair_energy))(xa, Ca, dl, kk)
    H = vmap(jacfwd(grad(_pair_energy)))(xa, Ca, dl, kk) if need_jac else None
    yield dofs[act].numpy(), -g, H
    mu = float(p.get("pair_mu", 0.0))
    if mu == 0.0:
        return
    # friction at the closest points (Eq. 12-13, reading C28)
    xn = q_n[dofs[act]]
    nu = float(p["nu_slip"])
    mm = torch.full_like(Ca, mu)
    nn = torch.full_like(Ca, nu)
    dtt = torch.full_like(Ca, float(osys.dt_vel))
    sig = torch.linalg.vector_norm(vmap(_pair_slip)(xa, xn, dtt), dim=-1)
    moving = torch.nonzero(sig > 0).reshape(-1)
    still = torch.nonzero(sig == 0).reshape(-1)
    for idx, fn in ((moving, _pair_friction), (still, _pair_friction_limit)):
        if len(idx) == 0:
            continue
        args = (xa[idx], xn[idx], Ca[idx], dl[idx], kk[idx], mm[idx], nn[idx], dtt[idx])
        F = vmap(fn)(*args)
        J = -vmap(jacfwd(fn))(*args) if need_jac else None
        yield dofs[act][idx].numpy(), F, J


def _pair_slip(x12, xn12, dt):
    """Tangential relative velocity of the closest points of a pair, with
    the implicit velocities (x - x_n)/dt (reading C26 for the ground)."""
    D, s, t = segment_distance(x12[0:3], x12[3:6], x12[6:9], x12[9:12])
    d = (x12[0:3] + s * (x12[3:6] - x12[0:3])) - (x12[6:9] + t * (x12[9:12] - x12[6:9]))
    n = d / D
    v = (x12 - xn12) / dt
    va = (1.0 - s) * v[0:3] + s * v[3:6]
    vb = (1.0 - t) * v[6:9] + t * v[9:12]
    vr = va - vb
    return vr - der.dot(vr, n) * n


def _pair_normal_force(x12, C, delta, kc):
    """|F_con| of the pair: the net contact force on either edge,
    k_c |dE/dD| (Eq. 11 with |dD/dx| summed over an edge's nodes = 1)."""
    D, _, _ = segment_distance(x12[0:3], x12[3:6], x12[6:9], x12[9:12])
    return torch.abs(kc * grad(der.imc_energy)(D, C, delta))


def _distribute(x12, Fa):
    _, s, t = segment_distance(x12[0:3], x12[3:6], x12[6:9], x12[9:12])
    return torch.cat([(1.0 - s) * Fa, s * Fa, -(1.0 - t) * Fa, -t * Fa])


def _pair_friction(x12, xn12, C, delta, kc, mu, nu, dt):
    """Eq. 13 on edge a (and its opposite on edge b), spread to the nodes
    by the closest-point weights."""
    u = _pair_slip(x12, xn12, dt)
    sp = torch.linalg.vector_norm(u)
    gam = der.friction_gamma(sp, nu)
    Fa = -mu * gam * u / sp * _pair_normal_force(x12, C, delta, kc)
    return _distribute(x12, Fa)


def _pair_friction_limit(x12, xn12, C, delta, kc, mu, nu, dt):
    """The u -> 0 limit of the friction law, -mu |F_con| (K2 / 2) u, whose
    value is 0 at u = 0 and whose Jacobian is the limit of the smooth one."""
    u = _pair_slip(x12, xn12, dt)
    Fa = -mu * (7.5 / nu) * u * _pair_normal_force(x12, C, delta, kc)
    return _distribute(x12, Fa)
