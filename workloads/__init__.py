"""Seeded synthetic inputs shaped like the DisMech paper's workloads.

This module only draws and lays out input data (rod geometry, materials,
boundary conditions, actuation tables).  It holds none of the method's
arithmetic, and both the CUDA library's tests/bench and the CPU oracle take
their inputs from it.

Workloads (all SI units, FP64):

* ``cantilever``  -- one clamped rod, 50 nodes, L = 1 m, h = 1e-3 m,
  rho = 1000, E = 1e7, nu = 0.5, straight, nodes 0-1 and theta^0 fixed,
  g = -9.81 z, damping 0.1, dt = 1e-3.
* ``uneven_rods`` -- 4096 independent clamped rods, N ~ U{20..200},
  L ~ U(0.2, 1.5), h ~ U(5e-4, 3e-3), log10 E ~ U(6, 8), per-rod natural
  curvature (c1, c2) ~ U[-5, 5]^2 1/m, dt = 1e-3.
* ``star_robots`` -- limbed robots on the ground: k ~ U{3..8} limbs of 30
  nodes / 0.1 m sharing a centre node, E = 1e6, h = 2e-3, sinusoidal limb
  curvature A sin(2 pi t / T + 2 pi j / k), A ~ U[0, 20] 1/m,
  T ~ U[0.5, 2] s, mu ~ U[0.3, 0.8], dt = 5e-3.
* ``coil``        -- one 500-node helical rod, h = 1e-3 m, helix radius
  0.02 m, pitch 2.2 h, stress-free at rest (natural strains = initial),
  clamped at its lower end and collapsing under gravity until its turns
  touch, edge-edge self-contact on, dt = 2.5e-4.
* ``gripper``     -- five 60-node fingers hanging from a 3 cm ring, actuated
  by random natural curvatures, edge-edge contact with friction between all
  fingers (one contact group), dt = 1e-3.

Integrated natural curvature (the library's input) is the physical curvature
times the rest Voronoi length; for a uniformly spaced rod that length is the
generator's own spacing L/(N-1).
"""
import math

import numpy as np

CANTILEVER_PARAMS = dict(dt=1e-3, tol=1e-10, max_iter=100, g=(0.0, 0.0, -9.81),
                         eta=0.1)


def _rod_desc(nodes_per_rod, x0, E, nu, rho, radius, fixed, **extra):
    d = dict(nodes_per_rod=np.asarray(nodes_per_rod, dtype=np.int32),
             x0=np.ascontiguousarray(x0, dtype=np.float64),
             E=np.asarray(E, dtype=np.float64), nu=np.asarray(nu, dtype=np.float64),
             rho=np.asarray(rho, dtype=np.float64),
             radius=np.asarray(radius, dtype=np.float64),
             fixed=np.asarray(fixed, dtype=np.uint8))
    d.update(extra)
    return d


def _clamp_mask(N):
    """Paper layout of one rod (Eq. 1): nodes 0 and 1 and theta^0 fixed."""
    m = np.zeros(4 * N - 1, dtype=np.uint8)
    m[0:3] = 1
    m[3] = 1
    m[4:7] = 1
    return m


def cantilever(N=50, L=1.0, h=1e-3, rho=1000.0, E=1e7, nu=0.5):
    """Single clamped cantilever rod along +x at z = 0."""
    x = np.zeros((N, 3))
    x[:, 0] = np.linspace(0.0, L, N)
    desc = _rod_desc([N], x, [E], [nu], [rho], [h], _clamp_mask(N))
    return desc, dict(CANTILEVER_PARAMS)


def uneven_rods(n_rods=4096, seed=2, n_min=20, n_max=200):
    """Batched uneven clamped rods with per-rod natural curvature.

    Returns (desc, params, kbar) where kbar holds (kappabar1, kappabar2) per
    interior node of every rod, concatenated by rod."""
    rng = np.random.default_rng(seed)
    N = rng.integers(n_min, n_max + 1, size=n_rods)
    L = rng.uniform(0.2, 1.5, size=n_rods)
    h = rng.uniform(5e-4, 3e-3, size=n_rods)
    E = 10.0 ** rng.uniform(6.0, 8.0, size=n_rods)
    c = rng.uniform(-5.0, 5.0, size=(n_rods, 2))
    ang = rng.uniform(0.0, 2.0 * math.pi, size=n_rods)
    side = int(math.ceil(math.sqrt(n_rods)))
    xs, masks, kb = [], [], []
    for r in range(n_rods):
        base = np.array([3.2 * (r % side), 3.2 * (r // side), 0.0])
        s = np.linspace(0.0, L[r], N[r])
        dirv = np.array([math.cos(ang[r]), math.sin(ang[r]), 0.0])
        xs.append(base[None, :] + s[:, None] * dirv[None, :])
        masks.append(_clamp_mask(N[r]))
        spacing = L[r] / (N[r] - 1)
        kb.append(np.tile(c[r] * spacing, (N[r] - 2, 1)))
    desc = _rod_desc(N, np.concatenate(xs), E, np.full(n_rods, 0.5),
                     np.full(n_rods, 1000.0), h, np.concatenate(masks))
    params = dict(dt=1e-3, tol=1e-10, max_iter=100, g=(0.0, 0.0, -9.81), eta=0.1)
    return desc, params, np.concatenate(kb)


def subset(desc, rods, kbar=None):
    """Descriptor of the listed rods only (for sampled parity checks on
    independent rods; joints are not carried over)."""
    rods = np.asarray(rods, dtype=np.int64)
    npr = np.asarray(desc["nodes_per_rod"], dtype=np.int64)
    noff = np.concatenate([[0], np.cumsum(npr)])
    foff = np.concatenate([[0], np.cumsum(4 * npr - 1)])
    koff = np.concatenate([[0], np.cumsum(npr - 2)])
    out = dict(nodes_per_rod=npr[rods].astype(np.int32))
    out["x0"] = np.concatenate([desc["x0"].reshape(-1, 3)[noff[r]:noff[r + 1]] for r in rods])
    for k in ("E", "nu", "rho", "radius", "ground_mu", "ground_kc"):
        if k in desc:
            out[k] = np.asarray(desc[k])[rods]
    out["fixed"] = np.concatenate([desc["fixed"][foff[r]:foff[r + 1]] for r in rods])
    kb = None
    if kbar is not None:
        kb = np.concatenate([kbar[koff[r]:koff[r + 1]] for r in rods])
    return out, kb


def star_robots(n_robots=1024, seed=3, k_min=3, k_max=8, nodes_per_limb=30,
                limb_len=0.1, E=1e6, h=2e-3, rho=1000.0, delta=5e-4,
                nu_slip=1e-3, fixed_limbs=None):
    """Limbed star robots resting on the ground plane z = 0.

    Returns (desc, params, gait).  ``gait`` holds per limb (rod) the
    amplitude A [1/m], period T [s] and phase 2 pi j / k of its natural
    curvature kappa1(t) = A sin(2 pi t / T + phase)."""
    rng = np.random.default_rng(seed)
    ks = (np.full(n_robots, fixed_limbs) if fixed_limbs
          else rng.integers(k_min, k_max + 1, size=n_robots))
    amp = rng.uniform(0.0, 20.0, size=n_robots)
    per = rng.uniform(0.5, 2.0, size=n_robots)
    mu = rng.uniform(0.3, 0.8, size=n_robots)
    side = int(math.ceil(math.sqrt(n_robots)))
    spacing = limb_len / (nodes_per_limb - 1)
    mnode = rho * math.pi * h * h * spacing
    kc = 50.0 * mnode * 9.81 / delta                    # reading C11
    npr, xs, joints, gm, gk = [], [], [], [], []
    gait_A, gait_T, gait_ph, robot_of = [], [], [], []
    rod = 0
    for b in range(n_robots):
        centre = np.array([0.5 * (b % side), 0.5 * (b // side), h])
        k = int(ks[b])
        grp = []
        for j in range(k):
            a = 2.0 * math.pi * j / k
            dirv = np.array([math.cos(a), math.sin(a), 0.0])
            s = np.linspace(0.0, limb_len, nodes_per_limb)
            xs.append(centre[None, :] + s[:, None] * dirv[None, :])
            npr.append(nodes_per_limb)
            grp.append((rod, 0))
            gm.append(mu[b])
            gk.append(kc)
            gait_A.append(amp[b])
            gait_T.append(per[b])
            gait_ph.append(2.0 * math.pi * j / k)
            robot_of.append(b)
            rod += 1
        joints.append(grp)
    R = rod
    desc = _rod_desc(npr, np.concatenate(xs), np.full(R, E), np.full(R, 0.5),
                     np.full(R, rho), np.full(R, h),
                     np.zeros(int(np.sum(4 * np.asarray(npr) - 1)), dtype=np.uint8),
                     joints=joints, ground_mu=np.array(gm), ground_kc=np.array(gk))
    params = dict(dt=5e-3, tol=1e-10, max_iter=100, g=(0.0, 0.0, -9.81), eta=0.1,
                  ground=True, ground_z=0.0, delta=delta, nu_slip=nu_slip,
                  line_search=True)
    gait = dict(A=np.array(gait_A), T=np.array(gait_T), phase=np.array(gait_ph),
                robot=np.array(robot_of), spacing=spacing,
                nodes_per_limb=nodes_per_limb)
    return desc, params, gait


def gait_kbar(gait, t):
    """Integrated natural curvature (kappabar1, kappabar2) per interior node of
    every limb at time t: kappa1 follows the limb's sinusoid, kappa2 = 0."""
    c1 = gait["A"] * np.sin(2.0 * math.pi * t / gait["T"] + gait["phase"])
    n_int = gait["nodes_per_limb"] - 2
    kb = np.zeros((len(c1), n_int, 2))
    kb[:, :, 0] = (c1 * gait["spacing"])[:, None]
    return kb.reshape(-1, 2)


def coil(N=500, h=1e-3, radius=0.02, pitch_factor=2.2, E=1e7, rho=1000.0,
         delta=1e-4, mu=0.0):
    """Helical rod standing on its clamped lower end, stress-free at rest
    (natural strains = initial), collapsing under gravity so that its turns
    come into contact (edge-edge self-contact).  The turns start a gap of
    (pitch_factor - 2) h apart.  Returns (desc, params, None)."""
    pitch = pitch_factor * h
    turn_len = math.sqrt((2.0 * math.pi * radius) ** 2 + pitch ** 2)
    spacing = 2.5e-3
    s = np.arange(N) * spacing
    phi = 2.0 * math.pi * s / turn_len
    x = np.stack([radius * np.cos(phi), radius * np.sin(phi),
                  pitch * phi / (2.0 * math.pi)], 1)
    mask = _clamp_mask(N)
    desc = _rod_desc([N], x, [E], [0.5], [rho], [h], mask)
    kc = E * h                                           # reading C11 (~E h)
    # dt = 0.25 ms and the line search keep Newton at 2-3 iterations through
    # the collapse of the 500-node coil (at 1 ms it stalls once the turns pile up)
    params = dict(dt=2.5e-4, tol=1e-10, max_iter=100, g=(0.0, 0.0, -9.81), eta=0.1,
                  self_contact=True, delta=delta, pair_kc=kc, pair_mu=mu,
                  line_search=True)
    return desc, params, None


def gripper(n_rods=5, N=60, L=0.3, h=2.5e-3, rho=1200.0, E=0.3e6, ring=0.03, mu=0.5,
            delta=5e-4, nu_slip=1e-3, phi_max_deg=40.0, ramp=0.2, dt=1e-3, seed=11):
    """Active entanglement gripper (Sec. IV): `n_rods` fingers hanging from a
    ring of radius `ring`, clamped at the top, actuated by natural
    curvatures 2 tan(phibar/2) per stencil with phibar ~ U[0, phi_max] (the
    bending plane turns by a random angle per rod), ramped in over `ramp`
    seconds; edge-edge contact with friction between all fingers (one
    contact group).  The paper's radius is 5 mm; with N = 60 the edge length
    then equals the radius and edges three apart along a finger would lie
    within C + delta at rest, so h defaults to 2.5 mm.  Returns (desc,
    params, kbar_fn) with kbar_fn(t) the (kappabar1, kappabar2) per interior
    node of every finger."""
    rng = np.random.default_rng(seed)
    xs = []
    for j in range(n_rods):
        a = 2.0 * math.pi * j / n_rods
        top = np.array([ring * math.cos(a), ring * math.sin(a), 0.0])
        z = -np.linspace(0.0, L, N)
        xs.append(top[None, :] + np.stack([np.zeros(N), np.zeros(N), z], 1))
    mask = np.concatenate([_clamp_mask(N) for _ in range(n_rods)])
    desc = _rod_desc([N] * n_rods, np.concatenate(xs), [E] * n_rods, [0.5] * n_rods,
                     [rho] * n_rods, [h] * n_rods, mask,
                     contact_groups=[list(range(n_rods))])
    phi = np.deg2rad(rng.uniform(0.0, phi_max_deg, size=(n_rods, N - 2)))
    psi = rng.uniform(0.0, 2.0 * math.pi, size=n_rods)
    k = 2.0 * np.tan(0.5 * phi)
    kb = np.stack([k * np.cos(psi)[:, None], k * np.sin(psi)[:, None]], -1).reshape(-1, 2)

    def kbar_fn(t):
        return min(max(t / ramp, 0.0), 1.0) * kb

    params = dict(dt=dt, tol=1e-10, max_iter=100, g=(0.0, 0.0, -9.81), eta=0.1,
                  self_contact=True, delta=delta, pair_kc=E * h, pair_mu=mu,
                  nu_slip=nu_slip, line_search=True)
    return desc, params, kbar_fn
