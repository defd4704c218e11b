"""Topology, state and the backward-Euler Newton step of the CPU oracle.

TEST INFRASTRUCTURE ONLY: the oracle is a plain, slow, FP64 restatement of the
DisMech implicit step (arXiv 2311.18126, Sec. III).  Only tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
it.  It shares no code with the CUDA library.

Passages followed (paper sections; readings C1..C27 are listed in the design
notes of the repository):

* Sec. III, Eq. 1 -- DOF vector [q_0, theta^0, q_1, ..., q_{N-1}] per rod.
* Sec. III-A      -- elastic energies (``der.py``); forces are their negative
                     gradients (Eq. 9).
* Sec. III-B      -- IMC contact energy (Eq. 10), contact force by the chain
                     rule (Eq. 11), smooth Coulomb friction (Eq. 12-13),
                     gravity and viscous damping.
* Sec. III-C      -- Eq. 14-15 backward-Euler residual with a diagonal mass
                     matrix, Newton's method with the Jacobian of Eq. 16
                     (taken in full: M/dt^2 - dF/dq, reading C10), velocity
                     update q_dot = (q_{n+1} - q_n)/dt.  The implicit
                     midpoint scheme the section also offers (no formula in
                     the paper; the textbook rule): q_{n+1} - q_n =
                     dt (q_dot_n + q_dot_{n+1})/2 and M (q_dot_{n+1} -
                     q_dot_n)/dt = F at the midpoint configuration
                     (q_n + q_{n+1})/2, velocity-dependent forces taking the
                     mid-step velocity (q_{n+1} - q_n)/dt.
* Sec. III-D      -- elastic joints: bending and twisting for every pair of
                     edges meeting at a joint node.
* Sec. III-E      -- natural curvatures as the control input.

Every derivative is automatic differentiation of the energies; the linear
solve is LAPACK (banded LU with partial pivoting for single rods, dense LU
otherwise).
"""
import math

import numpy as np
import scipy.linalg
import torch
from torch.func import grad, hessian, jacfwd, vmap

from . import der
from .contact import (ground_terms, pair_candidates_all, pair_terms)

DT = torch.float64

# Status codes shared with the C-ABI's documented values.
OK, ERR_INVALID_ARG, ERR_NOT_CONVERGED, ERR_NONFINITE, ERR_DEGENERATE, \
    ERR_PENETRATION = 0, 1, 2, 3, 4, 5


def _t(a):
    return torch.as_tensor(np.asarray(a), dtype=DT)


DEFAULT_PARAMS = dict(dt=1e-3, tol=1e-10, max_iter=100,
                      g=(0.0, 0.0, -9.81), eta=0.0,
                      ground=False, ground_z=0.0, delta=5e-4, nu_slip=1e-3,
                      self_contact=False, pair_kc=0.0, pair_mu=0.0,
                      line_search=False, integrator="be", predictor="extrapolate")


class _Sys:
    """One independent system: the rods connected through joints."""
    pass


class OracleSystems:
    """Batch of independent rod systems built from a descriptor.

    ``desc`` keys (host arrays, SI units):
      nodes_per_rod [R]; x0 [sum N, 3]; optional theta0 [sum (N-1)],
      v0 [sum N, 3], theta_dot0 [sum (N-1)]; E, nu, rho, radius [R];
      joints: list of groups [(rod, node), ...] merged into one node;
      fixed: bool [sum (4N-1)] in the per-rod layout of Eq. 1;
      ground_mu, ground_kc [R] (optional).
    """

    def __init__(self, desc, params=None):
        p = dict(DEFAULT_PARAMS)
        if params:
            p.update(params)
        self.p = p
        self.dt = float(p["dt"])
        if p["integrator"] not in ("be", "midpoint"):
            raise ValueError("integrator must be 'be' or 'midpoint'")
        self.midpoint = p["integrator"] == "midpoint"
        # interval over which velocity-dependent forces (damping, friction)
        # take the velocity of the point where forces are evaluated: the
        # step for backward Euler, half of it at the midpoint, where
        # (x_mid - x_n)/(dt/2) = (x_{n+1} - x_n)/dt
        self.dt_vel = 0.5 * self.dt if self.midpoint else self.dt
        self._build(desc)

    # ------------------------------------------------------------------
    # topology
    # ------------------------------------------------------------------
    def _build(self, desc):
        npr = np.asarray(desc["nodes_per_rod"], dtype=np.int64)
        R = len(npr)
        if R == 0 or np.any(npr < 2):
            raise ValueError("every rod needs at least two nodes")
        self.R = R
        self.npr = npr
        node_off = np.concatenate([[0], np.cumsum(npr)])
        edge_off = np.concatenate([[0], np.cumsum(npr - 1)])
        self.node_off, self.edge_off = node_off, edge_off
        nflat = int(node_off[-1])
        x0 = np.asarray(desc["x0"], dtype=np.float64).reshape(nflat, 3)
        v0 = np.asarray(desc.get("v0", np.zeros((nflat, 3))),
                        dtype=np.float64).reshape(nflat, 3)
        ne = int(edge_off[-1])
        th0 = np.asarray(desc.get("theta0", np.zeros(ne)), dtype=np.float64)
        thd0 = np.asarray(desc.get("theta_dot0", np.zeros(ne)),
                          dtype=np.float64)
        E = np.asarray(desc["E"], dtype=np.float64)
        nu = np.asarray(desc["nu"], dtype=np.float64)
        rho = np.asarray(desc["rho"], dtype=np.float64)
        h = np.asarray(desc["radius"], dtype=np.float64)
        gmu = np.asarray(desc.get("ground_mu", np.zeros(R)), dtype=np.float64)
        gkc = np.asarray(desc.get("ground_kc", np.zeros(R)), dtype=np.float64)

        # --- merge joint nodes: flat (rod,node) index -> global node id
        parent = np.arange(nflat)

        def find(a):
            while parent[a] != a:
                parent[a] = parent[parent[a]]
                a = parent[a]
            return a

        for grp in desc.get("joints", []):
            ids = [int(node_off[r] + i) for (r, i) in grp]
            root = min(find(a) for a in ids)
            for a in ids:
                parent[find(a)] = root
        roots = np.array([find(a) for a in range(nflat)])
        uniq, gid = np.unique(roots, return_inverse=True)
        self.flat2node = gid                      # flat -> global node
        Nn = len(uniq)
        self.Nn = Nn

        # --- edges with their rod's material
        ea = np.zeros(ne, dtype=np.int64)
        eb = np.zeros(ne, dtype=np.int64)
        erod = np.zeros(ne, dtype=np.int64)
        for r in range(R):
            for i in range(npr[r] - 1):
                e = edge_off[r] + i
                ea[e] = gid[node_off[r] + i]
                eb[e] = gid[node_off[r] + i + 1]
                erod[e] = r
        self.edge_nodes = np.stack([ea, eb], 1)
        self.edge_rod = erod
        xnode = np.zeros((Nn, 3))
        vnode = np.zeros((Nn, 3))
        xnode[gid] = x0
        vnode[gid] = v0
        lbar = np.linalg.norm(xnode[eb] - xnode[ea], axis=1)
        if np.any(lbar <= 0):
            raise ValueError("zero-length edge in the rest shape")
        he = h[erod]
        A = math.pi * he ** 2
        EA = E[erod] * A
        EI = E[erod] * math.pi * he ** 4 / 4.0
        G = E[erod] / (2.0 * (1.0 + nu[erod]))          # reading C3
        GJ = G * math.pi * he ** 4 / 2.0
        rhoA = rho[erod] * A

        # --- node masses, Voronoi lengths, contact radius, owner rod
        mnode = np.zeros(Nn)
        vor = np.zeros(Nn)
        hnode = np.zeros(Nn)
        owner = np.full(Nn, R, dtype=np.int64)
        for e in range(ne):
            for n in (ea[e], eb[e]):
                mnode[n] += 0.5 * rhoA[e] * lbar[e]
                vor[n] += 0.5 * lbar[e]
                hnode[n] = max(hnode[n], he[e])
                owner[n] = min(owner[n], erod[e])
        mtheta = 0.5 * rhoA * he ** 2 * lbar            # reading C7

        # --- bend-twist stencils: every unordered pair of incident edges
        inc = [[] for _ in range(Nn)]
        for e in range(ne):
            inc[ea[e]].append(e)
            inc[eb[e]].append(e)
        st_nodes, st_edges, st_sign, st_rodslot = [], [], [], []
        for v in range(Nn):
            es = sorted(inc[v])
            for i in range(len(es)):
                for j in range(i + 1, len(es)):
                    a, b = es[i], es[j]
                    sa = 1 if eb[a] == v else -1          # a oriented into v
                    sb = 1 if ea[b] == v else -1          # b oriented out of v
                    na = ea[a] if sa == 1 else eb[a]
                    nb = eb[b] if sb == 1 else ea[b]
                    st_nodes.append((na, v, nb))
                    st_edges.append((a, b))
                    st_sign.append((sa, sb))
                    # a rod stencil: consecutive edges of one rod
                    slot = -1
                    if erod[a] == erod[b] and b == a + 1 and sa == 1 and sb == 1:
                        r = erod[a]
                        slot = int(a - edge_off[r])       # interior node index - 1
                        slot = (r, slot)
                    st_rodslot.append(slot)
        self.st_nodes = np.array(st_nodes, dtype=np.int64).reshape(-1, 3)
        self.st_edges = np.array(st_edges, dtype=np.int64).reshape(-1, 2)
        self.st_sign = np.array(st_sign, dtype=np.float64).reshape(-1, 2)
        self.st_rodslot = st_rodslot
        Ns = len(st_nodes)
        sa_, sb_ = self.st_edges[:, 0], self.st_edges[:, 1]
        Vbar = 0.5 * (lbar[sa_] + lbar[sb_])             # reading C1
        self.st_kb = 0.5 * (EI[sa_] + EI[sb_]) / Vbar     # reading C18 (avg)
        self.st_kt = 0.5 * (GJ[sa_] + GJ[sb_]) / Vbar

        # --- initial reference frames (reading C5): per rod, z projected
        #     off the first tangent, then space-parallel transport
        t0 = (xnode[eb] - xnode[ea]) / lbar[:, None]
        d1 = np.zeros((ne, 3))
        for r in range(R):
            e0 = edge_off[r]
            t = t0[e0]
            z = np.array([0.0, 0.0, 1.0])
            if np.linalg.norm(np.cross(z, t)) < 1e-6:
                z = np.array([1.0, 0.0, 0.0])
            d = z - np.dot(z, t) * t
            d1[e0] = d / np.linalg.norm(d)
            for i in range(1, npr[r] - 1):
                e = e0 + i
                d1[e] = der.parallel_transport(
                    _t(d1[e - 1]), _t(t0[e - 1]), _t(t0[e])).numpy()

        # --- systems = connected components of the node graph
        comp = np.arange(Nn)

        def cfind(a):
            while comp[a] != a:
                comp[a] = comp[comp[a]]
                a = comp[a]
            return a

        for e in range(ne):
            ra, rb = cfind(ea[e]), cfind(eb[e])
            if ra != rb:
                comp[max(ra, rb)] = min(ra, rb)
        # contact groups: rods solved as one system so that their edges can
        # touch each other (reading C26: contact acts within a system)
        for grp in desc.get("contact_groups", []):
            for r in grp[1:]:
                ra, rb = cfind(gid[node_off[grp[0]]]), cfind(gid[node_off[r]])
                if ra != rb:
                    comp[max(ra, rb)] = min(ra, rb)
        ncomp = np.array([cfind(a) for a in range(Nn)])
        rod_comp = np.array([ncomp[gid[node_off[r]]] for r in range(R)])
        comps = []
        for r in range(R):
            if not comps or rod_comp[r] not in [c[0] for c in comps]:
                comps.append((rod_comp[r], []))
            for c in comps:
                if c[0] == rod_comp[r]:
                    c[1].append(r)
        fixed_flat = np.asarray(desc.get("fixed", np.zeros(int(np.sum(4 * npr - 1)), bool)),
                                dtype=bool)
        fix_off = np.concatenate([[0], np.cumsum(4 * npr - 1)])

        self.systems = []
        for _, rods in comps:
            s = _Sys()
            s.rods = rods
            # DOF numbering: Eq. 1 order per rod, shared nodes numbered once
            node_dof, edge_dof = {}, {}
            n = 0
            for r in rods:
                for i in range(npr[r]):
                    g = gid[node_off[r] + i]
                    if g not in node_dof:
                        node_dof[g] = n
                        n += 3
                    if i < npr[r] - 1:
                        edge_dof[edge_off[r] + i] = n
                        n += 1
            s.n = n
            s.nodes = np.array(sorted(node_dof.keys()), dtype=np.int64)
            s.edges = np.array(sorted(edge_dof.keys()), dtype=np.int64)
            nl = {g: k for k, g in enumerate(s.nodes)}
            el = {e: k for k, e in enumerate(s.edges)}
            s.node_dof = np.array([node_dof[g] for g in s.nodes])
            s.edge_dof = np.array([edge_dof[e] for e in s.edges])
            s.edge_nl = np.array([[nl[ea[e]], nl[eb[e]]] for e in s.edges],
                                 dtype=np.int64).reshape(-1, 2)
            sts = [k for k in range(Ns) if ncomp[self.st_nodes[k, 1]] == ncomp[gid[node_off[rods[0]]]]]
            s.st = np.array(sts, dtype=np.int64)
            s.st_nl = np.array([[nl[g] for g in self.st_nodes[k]] for k in sts],
                               dtype=np.int64).reshape(-1, 3)
            s.st_el = np.array([[el[e] for e in self.st_edges[k]] for k in sts],
                               dtype=np.int64).reshape(-1, 2)
            s.st_sign = self.st_sign[sts] if sts else np.zeros((0, 2))
            s.st_kb = self.st_kb[sts] if sts else np.zeros(0)
            s.st_kt = self.st_kt[sts] if sts else np.zeros(0)
            # 11 DOF indices per stencil in Eq. 1 order
            idx = []
            for k in range(len(sts)):
                a0, m, b1 = s.st_nl[k]
                ea_, eb_ = s.st_el[k]
                nd = s.node_dof
                idx.append([nd[a0], nd[a0] + 1, nd[a0] + 2, s.edge_dof[ea_],
                            nd[m], nd[m] + 1, nd[m] + 2, s.edge_dof[eb_],
                            nd[b1], nd[b1] + 1, nd[b1] + 2])
            s.st_dofs = np.array(idx, dtype=np.int64).reshape(-1, 11)
            s.edge_dofs6 = np.array(
                [[s.node_dof[i], s.node_dof[i] + 1, s.node_dof[i] + 2,
                  s.node_dof[j], s.node_dof[j] + 1, s.node_dof[j] + 2]
                 for (i, j) in s.edge_nl], dtype=np.int64).reshape(-1, 6)
            # materials and masses
            s.EA = EA[s.edges]
            s.lbar = lbar[s.edges]
            s.h_edge = he[s.edges]
            s.edge_rod = erod[s.edges]
            mass = np.zeros(n)
            for k, g in enumerate(s.nodes):
                mass[s.node_dof[k]:s.node_dof[k] + 3] = mnode[g]
            mass[s.edge_dof] = mtheta[s.edges]
            s.mass = _t(mass)
            s.mnode = mnode[s.nodes]
            s.vor = vor[s.nodes]
            s.hnode = hnode[s.nodes]
            s.gmu = gmu[owner[s.nodes]]
            s.gkc = gkc[owner[s.nodes]]
            # fixed DOFs (reading C19)
            fixed = np.zeros(n, dtype=bool)
            for r in rods:
                for k in range(4 * npr[r] - 1):
                    if fixed_flat[fix_off[r] + k]:
                        i, c = divmod(k, 4)
                        if c < 3:
                            fixed[node_dof[gid[node_off[r] + i]] + c] = True
                        else:
                            fixed[edge_dof[edge_off[r] + i]] = True
            s.fixed = torch.as_tensor(fixed)
            # residual scale (convergence reading C9'): a characteristic
            # stiffness per DOF from rest quantities, and a length per DOF
            # (midpoint: the stiffness of the residual with respect to the
            # midpoint configuration, inertia 4 M / dt^2)
            dscale = mass / self.dt_vel ** 2
            for k, e in enumerate(s.edges):
                i, j = s.edge_nl[k]
                kst = EA[e] / lbar[e]
                dscale[s.node_dof[i]:s.node_dof[i] + 3] += kst
                dscale[s.node_dof[j]:s.node_dof[j] + 3] += kst
            for k in range(len(sts)):
                ea_, eb_ = s.st_el[k]
                dscale[s.edge_dof[ea_]] += s.st_kt[k]
                dscale[s.edge_dof[eb_]] += s.st_kt[k]
            lscale = np.ones(n)
            lscale[np.concatenate([s.node_dof + c for c in range(3)])] = float(np.sum(lbar[s.edges]))
            s.rscale = _t(1.0 / (dscale * lscale))
            # state
            q = np.zeros(n)
            v = np.zeros(n)
            for k, g in enumerate(s.nodes):
                q[s.node_dof[k]:s.node_dof[k] + 3] = xnode[g]
                v[s.node_dof[k]:s.node_dof[k] + 3] = vnode[g]
            q[s.edge_dof] = th0[s.edges]
            v[s.edge_dof] = thd0[s.edges]
            s.q = _t(q)
            s.v = _t(v)
            s.d1 = _t(d1[s.edges])
            s.tn = _t(t0[s.edges])
            s.ground_on = bool(self.p["ground"])
            self.systems.append(s)
            # initial reference twist, natural strains (readings C4, C5)
            self._init_stencil_rest(s)
            # edge-edge contact exclusions (reading C16)
            s.pair_excl = None
            if self.p["self_contact"]:
                s.pair_cand = pair_candidates_all(self, s)

    def _stencil_geometry(self, s, q):
        """Oriented tangents per stencil and per-edge tangents at q."""
        x = q[torch.as_tensor(s.node_dof)[:, None] + torch.arange(3)]
        e = x[torch.as_tensor(s.edge_nl[:, 1])] - x[torch.as_tensor(s.edge_nl[:, 0])]
        t = e / torch.linalg.vector_norm(e, dim=1, keepdim=True)
        return x, t

    def _time_parallel_frames(self, s, t):
        """Sec. III: reference directors carried from the committed tangents
        to the current ones by time-parallel transport."""
        c = 1.0 + der.dot(s.tn, t)
        if torch.any(c <= 1e-12):
            raise FloatingPointError("edge reversed within one step")
        return der.parallel_transport(s.d1, s.tn, t)

    def _oriented(self, s, t, d1):
        sa = _t(s.st_sign[:, 0])
        sb = _t(s.st_sign[:, 1])
        ea = torch.as_tensor(s.st_el[:, 0])
        eb = torch.as_tensor(s.st_el[:, 1])
        ta = sa[:, None] * t[ea]
        tb = sb[:, None] * t[eb]
        return sa, sb, ta, d1[ea], tb, d1[eb]

    def _init_stencil_rest(self, s):
        ns = len(s.st)
        x, t = self._stencil_geometry(s, s.q)
        sa, sb, ta, d1a, tb, d1b = self._oriented(s, t, s.d1)
        if ns:
            if torch.any(1.0 + der.dot(ta, tb) <= 1e-12):
                raise ValueError("antiparallel edges at a stencil (reading C25)")
            beta0 = der.reference_twist(ta, d1a, tb, d1b, torch.zeros(ns, dtype=DT))
        else:
            beta0 = torch.zeros(0, dtype=DT)
        s.beta = beta0
        q11 = s.q[torch.as_tensor(s.st_dofs)] if ns else torch.zeros(0, 11, dtype=DT)
        if ns:
            k1, k2, tau = der.stencil_strains(q11, sa, sb, ta, d1a, tb, d1b, beta0)
        else:
            k1 = k2 = tau = torch.zeros(0, dtype=DT)
        s.kbar1 = k1.clone()
        s.kbar2 = k2.clone()
        s.taubar = tau.clone()

    # ------------------------------------------------------------------
    # control input (Sec. III-E)
    # ------------------------------------------------------------------
    def set_natural_curvature(self, rod_begin, rod_end, kbar):
        """kbar: (kappabar1, kappabar2) per interior node of each rod in
        [rod_begin, rod_end), integrated curvature as in Eq. 5 (reading C2).
        Joint stencils keep their initial natural strains."""
        kbar = np.asarray(kbar, dtype=np.float64).reshape(-1, 2)
        need = int(np.sum(self.npr[rod_begin:rod_end] - 2))
        if kbar.shape[0] != need:
            raise ValueError("kbar has %d pairs, expected %d" % (kbar.shape[0], need))
        base = {}
        off = 0
        for r in range(rod_begin, rod_end):
            base[r] = off
            off += self.npr[r] - 2
        for s in self.systems:
            for k, gk in enumerate(s.st):
                slot = self.st_rodslot[gk]
                if slot != -1 and slot[0] in base:
                    s.kbar1[k] = kbar[base[slot[0]] + slot[1], 0]
                    s.kbar2[k] = kbar[base[slot[0]] + slot[1], 1]

    # ------------------------------------------------------------------
    # forces and Jacobian at an iterate
    # ------------------------------------------------------------------
    def forces(self, s, q, v_n, q_n, need_jac=True):
        """Total generalized force F(q) (Eq. 9 plus external forces), the
        per-DOF sum of absolute term contributions (scale of reading C9), and
        (optionally) the matrix Jint = -dF/dq (the force part of Eq. 16,
        reading C10)."""
        n = s.n
        dt = self.dt
        F = torch.zeros(n, dtype=DT)
        Sabs = torch.zeros(n, dtype=DT)
        Jint = torch.zeros(n, n, dtype=DT) if need_jac else None

        def scatter(idx, contrib, jac):
            idx = torch.as_tensor(idx)
            F.index_add_(0, idx.reshape(-1), contrib.reshape(-1))
            Sabs.index_add_(0, idx.reshape(-1), contrib.abs().reshape(-1))
            if need_jac and jac is not None:
                k = idx.shape[-1]
                rows = idx[:, :, None].expand(-1, k, k).reshape(-1)
                cols = idx[:, None, :].expand(-1, k, k).reshape(-1)
                Jint.index_put_((rows, cols), jac.reshape(-1), accumulate=True)

        x, t = self._stencil_geometry(s, q)
        # -- stretching (Eq. 2-3)
        if len(s.edges):
            x6 = q[torch.as_tensor(s.edge_dofs6)]
            EA = _t(s.EA)
            lb = _t(s.lbar)
            g = vmap(grad(der.stretch_energy))(x6, EA, lb)
            H = vmap(hessian(der.stretch_energy))(x6, EA, lb) if need_jac else None
            scatter(s.edge_dofs6, -g, H)
        # -- bending and twisting (Eq. 4-8): the energy of the configuration
        #    q with reference frames carried from the committed step by
        #    time-parallel transport (Sec. III), differentiated exactly
        #    (Eq. 9, reading C6)
        if len(s.st):
            _ = self._time_parallel_frames(s, t)      # checks 1 + t_n.t > 0
            q11 = q[torch.as_tensor(s.st_dofs)]
            args = self._stencil_history(s)
            if torch.any(1.0 + der.dot(*self._oriented_tangents(s, t)) <= 1e-12):
                raise FloatingPointError("antiparallel edges (reading C25)")
            g = vmap(grad(der.time_transported_energy))(q11, *args)
            H = vmap(hessian(der.time_transported_energy))(q11, *args) if need_jac else None
            scatter(s.st_dofs, -g, H)
        # -- gravity and viscous damping (Sec. III-B misc forces, reading C8)
        nd = torch.as_tensor(s.node_dof)[:, None] + torch.arange(3)
        grav = _t(s.mnode)[:, None] * _t(self.p["g"])[None, :]
        scatter(nd, grav, None)
        eta = float(self.p["eta"])
        if eta != 0.0:
            xn = q_n[nd]
            cdamp = eta * _t(s.vor) / self.dt_vel
            Fd = -cdamp[:, None] * (x - xn)
            Jd = cdamp[:, None, None] * torch.eye(3, dtype=DT)[None]
            scatter(nd, Fd, Jd)
        # -- ground contact and friction (Eq. 10-13)
        if s.ground_on:
            xn = q_n[nd]
            for (Fk, Jk) in ground_terms(self, s, x, xn, need_jac):
                scatter(nd, Fk, Jk)
        # -- edge-edge contact (Eq. 10-11)
        if self.p["self_contact"]:
            for (idx, Fk, Jk) in pair_terms(self, s, q, q_n, need_jac):
                scatter(idx, Fk, Jk)
        return F, Sabs, Jint

    def _stencil_history(self, s):
        """Per-stencil committed data: orientation signs, oriented committed
        tangents and reference directors, committed reference twist, and the
        stiffnesses and natural strains."""
        sa = _t(s.st_sign[:, 0])
        sb = _t(s.st_sign[:, 1])
        ea = torch.as_tensor(s.st_el[:, 0])
        eb = torch.as_tensor(s.st_el[:, 1])
        return (sa, sb, sa[:, None] * s.tn[ea], s.d1[ea], sb[:, None] * s.tn[eb], s.d1[eb],
                s.beta, _t(s.st_kb), _t(s.st_kt), s.kbar1, s.kbar2, s.taubar)

    def _oriented_tangents(self, s, t):
        sa = _t(s.st_sign[:, 0])
        sb = _t(s.st_sign[:, 1])
        ea = torch.as_tensor(s.st_el[:, 0])
        eb = torch.as_tensor(s.st_el[:, 1])
        return sa[:, None] * t[ea], sb[:, None] * t[eb]

    # ------------------------------------------------------------------
    # residual, Newton, commit (Sec. III-C)
    # ------------------------------------------------------------------
    def residual(self, s, q, q_n, v_n, need_jac=True):
        """Eq. 15: f = M/dt ((q - q_n)/dt - q_dot_n) - F_int - F_ext, with the
        scale S of reading C9 and (optionally) J = M/dt^2 - dF/dq.  Implicit
        midpoint: f = 2 M/dt^2 (q - q_n - dt q_dot_n) - F(q_mid), q_mid =
        (q + q_n)/2, J = 2 M/dt^2 - (1/2) dF/dx at q_mid."""
        dt = self.dt
        if self.midpoint:
            qm = 0.5 * (q + q_n)
            F, Sabs, Jint = self.forces(s, qm, v_n, q_n, need_jac)
            inert = 2.0 * s.mass / dt ** 2 * (q - q_n)
            mom = 2.0 * s.mass / dt * v_n
            f = inert - mom - F
            S = inert.abs() + mom.abs() + Sabs
            f = torch.where(s.fixed, torch.zeros_like(f), f)
            S = torch.where(s.fixed, torch.zeros_like(S), S)
            J = None
            if need_jac:
                J = 0.5 * Jint + torch.diag(2.0 * s.mass / dt ** 2)
                fx = s.fixed
                J[fx, :] = 0.0
                J[:, fx] = 0.0
                J[fx, fx] = 1.0
            return f, S, J
        F, Sabs, Jint = self.forces(s, q, v_n, q_n, need_jac)
        inert = s.mass / dt ** 2 * (q - q_n)
        mom = s.mass / dt * v_n
        f = inert - mom - F
        S = inert.abs() + mom.abs() + Sabs
        f = torch.where(s.fixed, torch.zeros_like(f), f)
        S = torch.where(s.fixed, torch.zeros_like(S), S)
        J = None
        if need_jac:
            J = Jint + torch.diag(s.mass / dt ** 2)
            fx = s.fixed
            J[fx, :] = 0.0
            J[:, fx] = 0.0
            J[fx, fx] = 1.0
        return f, S, J

    def solve(self, s, J, rhs):
        """J x = rhs by LAPACK: banded LU with partial pivoting when the
        matrix is banded (single rods), dense LU otherwise."""
        Jn = J.numpy()
        b = rhs.numpy()
        nz = np.nonzero(Jn)
        bw = int(np.max(np.abs(nz[0] - nz[1]))) if len(nz[0]) else 0
        n = Jn.shape[0]
        if bw <= 16 and n > 4 * bw:
            ab = np.zeros((2 * bw + 1, n))
            for d in range(-bw, bw + 1):
                diag = np.diagonal(Jn, offset=d)
                if d >= 0:
                    ab[bw - d, d:] = diag
                else:
                    ab[bw - d, :n + d] = diag
            return torch.as_tensor(scipy.linalg.solve_banded((bw, bw), ab, b))
        return torch.as_tensor(np.linalg.solve(Jn, b))

    def step_system(self, s, record=None):
        """One implicit step (backward Euler or implicit midpoint) of one
        system; all-or-nothing."""
        dt = self.dt
        tol = float(self.p["tol"])
        max_iter = int(self.p["max_iter"])
        q_n, v_n = s.q.clone(), s.v.clone()
        q = q_n + dt * v_n                                 # reading C23
        q = torch.where(s.fixed, q_n, q)
        if self.p.get("predictor", "extrapolate") == "projected":
            q = self._project_lengths(s, q, q_n)
        status, it = ERR_NOT_CONVERGED, 0
        res = scale = float("nan")
        ls = bool(self.p["line_search"])
        trial, nback, alpha, q_acc, m_acc = False, 0, 1.0, q, float("inf")
        try:
            while True:
                f, S, _ = self.residual(s, q, q_n, v_n, need_jac=False)
                res = float(torch.max(torch.abs(f) * s.rscale))
                merit = float(torch.linalg.vector_norm(f * s.rscale))
                scale = float(torch.linalg.vector_norm(f))
                if record is not None:
                    record.append(res)
                # backtracking (Sec. III-C optional line search): Armijo test
                # on the 2-norm of the scaled residual, for which the Newton
                # direction is a descent direction; a trial point without
                # sufficient decrease moves halfway back to the last accepted
                # iterate
                if (ls and trial and nback < 12
                        and not (merit <= (1.0 - 1e-4 * alpha) * m_acc)):
                    q = 0.5 * (q + q_acc)
                    alpha *= 0.5
                    nback += 1
                    continue
                trial, nback, alpha, q_acc, m_acc = False, 0, 1.0, q, merit
                if not math.isfinite(res):
                    status = ERR_NONFINITE
                    break
                if res <= tol:
                    status = OK
                    break
                if it >= max_iter:
                    break
                _, _, J = self.residual(s, q, q_n, v_n, need_jac=True)
                dq = self.solve(s, J, -f)
                if not bool(torch.all(torch.isfinite(dq))):
                    status = ERR_NONFINITE
                    break
                q = q + dq
                trial = True
                it += 1
        except FloatingPointError:
            status = ERR_DEGENERATE
        if status == OK:
            self._commit(s, q, q_n)
        return status, it, res, scale

    def _project_lengths(self, s, q, q_n):
        """The length-projected starting guess (an option; Newton's root does
        not depend on it): on a system of one rod, each edge of the guess q
        takes its length in q_n, node positions rebuilt from the first node
        along the guess's edge directions; nodes with a fixed position DOF
        keep their value.  Other systems keep q."""
        if len(s.rods) != 1 or self.p["self_contact"]:
            return q
        out = q.clone()
        nd = s.node_dof
        for k in range(1, len(nd)):
            a, b = nd[k - 1], nd[k]
            if bool(s.fixed[b:b + 3].any()):
                continue
            e = q[b:b + 3] - q[a:a + 3]
            l_n = torch.linalg.vector_norm(q_n[b:b + 3] - q_n[a:a + 3])
            out[b:b + 3] = out[a:a + 3] + l_n * e / torch.linalg.vector_norm(e)
        return out

    def _commit(self, s, q, q_n):
        """Velocity update (Sec. III-C) and commit of the reference frames
        and reference twist carried to the new configuration (reading C24)."""
        _, t = self._stencil_geometry(s, q)
        d1 = self._time_parallel_frames(s, t)
        if len(s.st):
            _, _, ta, d1a, tb, d1b = self._oriented(s, t, d1)
            s.beta = der.reference_twist(ta, d1a, tb, d1b, s.beta)
        s.d1 = d1
        s.tn = t
        if self.midpoint:
            v = 2.0 * (q - q_n) / self.dt - s.v
            s.v = torch.where(s.fixed, torch.zeros_like(v), v)
        else:
            s.v = (q - q_n) / self.dt
        s.q = q

    def step(self, nsteps=1):
        """Advance every system; returns per-system (status, iterations,
        residual, scale) of the last step."""
        out = []
        for _ in range(nsteps):
            out = [self.step_system(s) for s in self.systems]
            bad = [k for k, o in enumerate(out) if o[0] != OK]
            if bad:
                break
        return out

    # ------------------------------------------------------------------
    # state in the per-rod layout of Eq. 1
    # ------------------------------------------------------------------
    def _rod_maps(self):
        """(system, DOF index) for every entry of the per-rod layout."""
        maps = []
        for si, s in enumerate(self.systems):
            nl = {g: k for k, g in enumerate(s.nodes)}
            el = {e: k for k, e in enumerate(s.edges)}
            for r in s.rods:
                idx = []
                for i in range(self.npr[r]):
                    g = self.flat2node[self.node_off[r] + i]
                    d = s.node_dof[nl[g]]
                    idx += [d, d + 1, d + 2]
                    if i < self.npr[r] - 1:
                        idx.append(s.edge_dof[el[self.edge_off[r] + i]])
                maps.append((r, si, np.array(idx)))
        maps.sort(key=lambda m: m[0])
        return maps

    def get_state(self):
        """q and q_dot concatenated per rod in the layout of Eq. 1; a joint
        node appears in every rod that contains it."""
        qs, vs = [], []
        for (_, si, idx) in self._rod_maps():
            s = self.systems[si]
            qs.append(s.q[torch.as_tensor(idx)].numpy())
            vs.append(s.v[torch.as_tensor(idx)].numpy())
        return np.concatenate(qs), np.concatenate(vs)

    def set_state(self, q, v):
        off = 0
        for (r, si, idx) in self._rod_maps():
            s = self.systems[si]
            k = len(idx)
            s.q[torch.as_tensor(idx)] = _t(q[off:off + k])
            s.v[torch.as_tensor(idx)] = _t(v[off:off + k])
            off += k
        for s in self.systems:
            _, s.tn = self._stencil_geometry(s, s.q)

    def get_frames(self):
        """Reference director d1 per edge (edge order of the descriptor) and
        reference twist per stencil, the history a resume needs."""
        d1 = np.zeros((int(self.edge_off[-1]), 3))
        beta = np.zeros(len(self.st_nodes))
        for s in self.systems:
            d1[s.edges] = s.d1.numpy()
            beta[s.st] = s.beta.numpy()
        return d1, beta

    def set_frames(self, d1, beta):
        for s in self.systems:
            s.d1 = _t(np.asarray(d1)[s.edges])
            s.beta = _t(np.asarray(beta)[s.st])
