"""Discrete Elastic Rods kinematics and energies, written as plain FP64 torch code.

TEST INFRASTRUCTURE ONLY: this module belongs to the CPU oracle.  Only tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; the product path never does.

Every function here follows a passage of the DisMech paper (arXiv 2311.18126):

* Sec. III, Eq. 1  -- DOF vector of node positions and edge twist angles.
* Sec. III         -- reference frame {d1, d2, t}, material frame {m1, m2, t}
                      obtained by rotating the reference frame by theta about t,
                      reference frames updated between steps by time-parallel
                      transport.
* Sec. III-A Eq. 2-3  -- stretching strain and energy.
* Sec. III-A Eq. 4-6  -- curvature binormal, material curvatures, bending energy.
* Sec. III-A Eq. 7-8  -- twisting strain with reference twist, twisting energy.

Derivatives are never hand-derived here: forces and Jacobians come from
automatic differentiation (``torch.func``) of the energies below, so that the
oracle is the energy definitions and nothing else.
"""
import torch

DT = torch.float64


def dot(a, b):
    return (a * b).sum(-1)


def cross(a, b):
    return torch.linalg.cross(a, b, dim=-1)


def parallel_transport(v, a, b):
    """Minimal rotation that carries unit vector ``a`` onto unit vector ``b``,
    applied to ``v`` (Rodrigues form of the rotation about a x b).

    This is the transport used for the reference frame (Sec. III: "updated
    between time steps via time parallel transport").  The rotation is
    undefined for antiparallel a, b; callers check 1 + a.b first."""
    c = cross(a, b)
    d = dot(a, b)
    return (d[..., None] * v + cross(c, v)
            + c * (dot(c, v) / (1.0 + d))[..., None])


def rotate_about(v, axis, angle):
    """Right-handed rotation of ``v`` by ``angle`` about unit ``axis``."""
    c = torch.cos(angle)[..., None]
    s = torch.sin(angle)[..., None]
    return c * v + s * cross(axis, v) + (1.0 - c) * dot(axis, v)[..., None] * axis


def signed_angle(u, v, n):
    """Angle that rotates ``u`` onto ``v`` about the unit normal ``n``."""
    return torch.atan2(dot(n, cross(u, v)), dot(u, v))


def material_frame(d1, t, theta):
    """Sec. III: the material frame is the reference frame {d1, d2 = t x d1}
    rotated by the signed angle theta about t."""
    d2 = cross(t, d1)
    c = torch.cos(theta)[..., None]
    s = torch.sin(theta)[..., None]
    m1 = c * d1 + s * d2
    m2 = -s * d1 + c * d2
    return m1, m2


def curvature_binormal(ta, tb):
    """Eq. 4: (kappa b)_i = 2 t^{i-1} x t^i / (1 + t^{i-1} . t^i)."""
    return 2.0 * cross(ta, tb) / (1.0 + dot(ta, tb))[..., None]


def reference_twist(ta, d1a, tb, d1b, beta_prev):
    """Eq. 7 reference twist beta: the signed angle, about t^i, from the
    parallel-transported d1^{i-1} to d1^i.  It is continued from the previous
    value ``beta_prev`` so that it carries no 2*pi jumps: the transported
    director is first rotated by beta_prev and the small remaining angle is
    added (reading C24 of the design notes: recomputed at every iterate)."""
    u = rotate_about(parallel_transport(d1a, ta, tb), tb, beta_prev)
    return beta_prev + signed_angle(u, d1b, tb)


# ---------------------------------------------------------------------------
# Stretching (Eq. 2-3)
# ---------------------------------------------------------------------------

def stretch_energy(x6, EA, lbar):
    """Eq. 2-3 for one edge: 1/2 EA (|e|/|ebar| - 1)^2 |ebar|.
    ``x6`` = [x_start (3), x_end (3)]."""
    e = x6[..., 3:6] - x6[..., 0:3]
    eps = torch.linalg.vector_norm(e, dim=-1) / lbar - 1.0
    return 0.5 * EA * eps * eps * lbar


# ---------------------------------------------------------------------------
# Bending and twisting at one node stencil (Eq. 4-8)
# ---------------------------------------------------------------------------

def stencil_strains(q11, sa, sb, ta_ref, d1a_ref, tb_ref, d1b_ref, beta_ref):
    """Material curvatures (Eq. 5) and twist (Eq. 7) of one bend-twist stencil.

    ``q11`` = [x_{i-1} (3), theta^{i-1}, x_i (3), theta^i, x_{i+1} (3)] in the
    interleaved order of Eq. 1.  Edge a runs x_{i-1} -> x_i, edge b runs
    x_i -> x_{i+1}.  At a joint (Sec. III-D) an incident edge may be stored in
    the opposite direction; ``sa``/``sb`` = -1 mark that, and the edge's
    twist angle then enters with the opposite sign (reversing an edge maps
    t -> -t, d2 -> -d2, theta -> -theta and leaves m1 unchanged).

    The reference directors at the evaluation point are the reference
    directors (``d1*_ref`` with tangents ``t*_ref``) carried by parallel
    transport to the current tangents, and the reference twist is continued
    from ``beta_ref``.  Called with the frames of the iterate itself this is
    the at-point gauge (reading C6); called with the frames of the previous
    step it is time-parallel transport (Sec. III)."""
    xa, tha, xm, thb, xb = (q11[..., 0:3], q11[..., 3], q11[..., 4:7],
                            q11[..., 7], q11[..., 8:11])
    ea = xm - xa
    eb = xb - xm
    ta = ea / torch.linalg.vector_norm(ea, dim=-1)[..., None]
    tb = eb / torch.linalg.vector_norm(eb, dim=-1)[..., None]
    d1a = parallel_transport(d1a_ref, ta_ref, ta)
    d1b = parallel_transport(d1b_ref, tb_ref, tb)
    m1a, m2a = material_frame(d1a, ta, sa * tha)
    m1b, m2b = material_frame(d1b, tb, sb * thb)
    kb = curvature_binormal(ta, tb)
    kappa1 = 0.5 * dot(kb, m2a + m2b)
    kappa2 = -0.5 * dot(kb, m1a + m1b)
    beta = reference_twist(ta, d1a, tb, d1b, beta_ref)
    tau = sb * thb - sa * tha + beta
    return kappa1, kappa2, tau


def bend_twist_energy(q11, sa, sb, ta_ref, d1a_ref, tb_ref, d1b_ref, beta_ref,
                      kb_stiff, kt_stiff, kbar1, kbar2, taubar):
    """Eq. 6 + Eq. 8 for one stencil:
    1/2 EI/V (kappa - kappabar)^2 + 1/2 GJ/V (tau - taubar)^2, with
    ``kb_stiff`` = EI/V and ``kt_stiff`` = GJ/V (V the rest Voronoi length,
    reading C1)."""
    k1, k2, tau = stencil_strains(q11, sa, sb, ta_ref, d1a_ref, tb_ref,
                                  d1b_ref, beta_ref)
    return (0.5 * kb_stiff * ((k1 - kbar1) ** 2 + (k2 - kbar2) ** 2)
            + 0.5 * kt_stiff * (tau - taubar) ** 2)


def time_transported_energy(q11, sa, sb, ta_n, d1a_n, tb_n, d1b_n, beta_n,
                            kb_stiff, kt_stiff, kbar1, kbar2, taubar):
    """Eq. 6 + Eq. 8 of one stencil as a function of its 11 DOFs alone: the
    reference directors are those of the committed step (``d1*_n`` on the
    committed oriented tangents ``t*_n``) carried to the current tangents by
    time-parallel transport (Sec. III), and the reference twist is continued
    from ``beta_n``.  Forces and Jacobians are its exact derivatives."""
    xa, xm, xb = q11[..., 0:3], q11[..., 4:7], q11[..., 8:11]
    ta = (xm - xa) / torch.linalg.vector_norm(xm - xa, dim=-1)[..., None]
    tb = (xb - xm) / torch.linalg.vector_norm(xb - xm, dim=-1)[..., None]
    d1a = parallel_transport(d1a_n, ta_n, ta)
    d1b = parallel_transport(d1b_n, tb_n, tb)
    return bend_twist_energy(q11, sa, sb, ta, d1a, tb, d1b, beta_n, kb_stiff,
                             kt_stiff, kbar1, kbar2, taubar)


def bend_energy_only(q11, sa, sb, ta_ref, d1a_ref, tb_ref, d1b_ref, beta_ref,
                     kb_stiff, kbar1, kbar2):
    k1, k2, _ = stencil_strains(q11, sa, sb, ta_ref, d1a_ref, tb_ref,
                                d1b_ref, beta_ref)
    return 0.5 * kb_stiff * ((k1 - kbar1) ** 2 + (k2 - kbar2) ** 2)


def twist_energy_only(q11, sa, sb, ta_ref, d1a_ref, tb_ref, d1b_ref, beta_ref,
                      kt_stiff, taubar):
    _, _, tau = stencil_strains(q11, sa, sb, ta_ref, d1a_ref, tb_ref,
                                d1b_ref, beta_ref)
    return 0.5 * kt_stiff * (tau - taubar) ** 2


# ---------------------------------------------------------------------------
# Contact (Sec. III-B, Eq. 10-13)
# ---------------------------------------------------------------------------

def softplus(x):
    """log(1 + e^x) evaluated without overflow."""
    return torch.clamp(x, min=0.0) + torch.log1p(torch.exp(-torch.abs(x)))


def imc_energy(D, C, delta):
    """Eq. 10 with K1 = 15/delta: (C-D)^2 for D <= C-delta (extended to D <= 0
    for the ground, reading C12), the squared softplus on the open interval
    (C-delta, C+delta) and 0 for D >= C+delta (reading C13)."""
    K1 = 15.0 / delta
    quad = (C - D) ** 2
    smooth = (softplus(K1 * (C - D)) / K1) ** 2
    zero = torch.zeros_like(D)
    return torch.where(D <= C - delta, quad,
                       torch.where(D < C + delta, smooth, zero))


def friction_gamma(speed, nu_slip):
    """Eq. 12: gamma = 2 / (1 + exp(-K2 |u|)) - 1 with K2 = 15/nu."""
    K2 = 15.0 / nu_slip
    return 2.0 / (1.0 + torch.exp(-K2 * speed)) - 1.0
