// Host-side topology builder: joint merging, DOF numbering, rest quantities,
// masses, initial frames and natural strains (DisMech, arXiv 2311.18126,
// Sec. III, Eq. 1-8; Sec. III-D joints; Sec. III-E natural curvature).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <tuple>
#include <utility>

#include "dm_internal.h"

namespace dm {

namespace {

struct V3 {
  double x, y, z;
};
inline V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 add(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 mul(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }

// Minimal rotation from unit a to unit b applied to v (v normal to a):
// v - (v.b)/(1 + a.b) (a + b).
inline V3 transport(V3 v, V3 a, V3 b) {
  double c = dot(v, b) / (1.0 + dot(a, b));
  return sub(v, mul(c, add(a, b)));
}

// Material curvatures and twist strain of one stencil at the rest shape
// (Eq. 4, 5, 7) given oriented tangents, reference directors and angles.
void rest_strains(V3 ta, V3 d1a, double tha, V3 tb, V3 d1b, double thb,
                  double beta, double *k1, double *k2, double *tau) {
  V3 d2a = cross(ta, d1a), d2b = cross(tb, d1b);
  double ca = std::cos(tha), sa = std::sin(tha);
  double cb = std::cos(thb), sb = std::sin(thb);
  V3 m1a = add(mul(ca, d1a), mul(sa, d2a)), m2a = add(mul(-sa, d1a), mul(ca, d2a));
  V3 m1b = add(mul(cb, d1b), mul(sb, d2b)), m2b = add(mul(-sb, d1b), mul(cb, d2b));
  V3 kb = mul(2.0 / (1.0 + dot(ta, tb)), cross(ta, tb));
  *k1 = 0.5 * dot(kb, add(m2a, m2b));
  *k2 = -0.5 * dot(kb, add(m1a, m1b));
  *tau = thb - tha + beta;
}

}  // namespace

bool build_topology(const dm_system_desc *D, const dm_params *P, HostTopology &T) {
  if (!D || D->n_rods <= 0 || !D->nodes_per_rod || !D->x0 || !D->E || !D->nu ||
      !D->rho || !D->radius) {
    set_error("descriptor: n_rods > 0, nodes_per_rod, x0, E, nu, rho, radius required");
    return false;
  }
  if (!P || !(P->dt > 0) || !(P->newton_tol > 0) || P->max_iter < 1) {
    set_error("params: dt > 0, newton_tol > 0, max_iter >= 1 required");
    return false;
  }
  const int R = D->n_rods;
  T.n_rods = R;
  T.npr.assign(D->nodes_per_rod, D->nodes_per_rod + R);
  T.rod_node0.assign(R + 1, 0);
  T.rod_edge0.assign(R + 1, 0);
  T.rod_layout0.assign(R + 1, 0);
  for (int r = 0; r < R; ++r) {
    if (T.npr[r] < 2) {
      set_error("rod " + std::to_string(r) + " has fewer than 2 nodes");
      return false;
    }
    if (!(D->E[r] > 0) || !(D->rho[r] > 0) || !(D->radius[r] > 0) ||
        !(D->nu[r] > -1.0)) {
      set_error("rod " + std::to_string(r) + ": E, rho, radius > 0 and nu > -1 required");
      return false;
    }
    T.rod_node0[r + 1] = T.rod_node0[r] + T.npr[r];
    T.rod_edge0[r + 1] = T.rod_edge0[r] + T.npr[r] - 1;
    T.rod_layout0[r + 1] = T.rod_layout0[r] + 4 * (int64_t)T.npr[r] - 1;
  }
  const int64_t nflat = T.rod_node0[R];
  const int64_t ne = T.rod_edge0[R];

  // --- joints: union-find with the smallest flat index as the root
  std::vector<int64_t> parent(nflat);
  std::iota(parent.begin(), parent.end(), 0);
  auto find = [&](int64_t a) {
    while (parent[a] != a) {
      parent[a] = parent[parent[a]];
      a = parent[a];
    }
    return a;
  };
  if (D->n_joints > 0) {
    if (!D->joint_offsets || !D->joint_members) {
      set_error("joints: joint_offsets and joint_members required");
      return false;
    }
    for (int j = 0; j < D->n_joints; ++j) {
      int32_t b = D->joint_offsets[j], e = D->joint_offsets[j + 1];
      if (e - b < 2 || b < 0) {
        set_error("joint " + std::to_string(j) + " needs at least two members");
        return false;
      }
      int64_t root = -1;
      std::vector<int64_t> ids;
      for (int k = b; k < e; ++k) {
        int32_t r = D->joint_members[2 * k], i = D->joint_members[2 * k + 1];
        if (r < 0 || r >= R || i < 0 || i >= T.npr[r]) {
          set_error("joint member out of range");
          return false;
        }
        ids.push_back(T.rod_node0[r] + i);
      }
      for (int64_t a : ids) {
        int64_t ra = find(a);
        root = (root < 0) ? ra : std::min(root, ra);
      }
      for (int64_t a : ids) {
        int64_t ra = find(a);
        if (ra < root) std::swap(ra, root);
        parent[ra] = root;
      }
    }
  }
  // node id = rank of the root among distinct roots
  std::vector<int64_t> root(nflat);
  for (int64_t a = 0; a < nflat; ++a) root[a] = find(a);
  std::vector<int64_t> rank(nflat, -1);
  int64_t nn = 0;
  for (int64_t a = 0; a < nflat; ++a)
    if (root[a] == a) rank[a] = nn++;
  T.n_nodes = nn;
  T.flat2node.resize(nflat);
  for (int64_t a = 0; a < nflat; ++a) T.flat2node[a] = rank[root[a]];

  // node positions (first member's coordinates)
  std::vector<V3> X(nn), Vn(nn);
  std::vector<char> seen(nn, 0);
  for (int64_t a = 0; a < nflat; ++a) {
    int64_t v = T.flat2node[a];
    if (seen[v]) continue;
    seen[v] = 1;
    X[v] = {D->x0[3 * a], D->x0[3 * a + 1], D->x0[3 * a + 2]};
    Vn[v] = D->v0 ? V3{D->v0[3 * a], D->v0[3 * a + 1], D->v0[3 * a + 2]} : V3{0, 0, 0};
  }

  // --- edges
  T.n_edges = ne;
  T.edge_a.resize(ne);
  T.edge_b.resize(ne);
  T.edge_rod.resize(ne);
  T.edge_lbar.resize(ne);
  T.edge_EA.resize(ne);
  T.edge_EI.resize(ne);
  T.edge_GJ.resize(ne);
  T.edge_rhoA.resize(ne);
  T.edge_h.resize(ne);
  T.t_init.resize(3 * ne);
  for (int r = 0; r < R; ++r) {
    const double h = D->radius[r], E = D->E[r];
    const double A = M_PI * h * h;
    const double G = E / (2.0 * (1.0 + D->nu[r]));  // reading C3
    for (int i = 0; i + 1 < T.npr[r]; ++i) {
      int64_t e = T.rod_edge0[r] + i;
      int64_t a = T.flat2node[T.rod_node0[r] + i], b = T.flat2node[T.rod_node0[r] + i + 1];
      if (a == b) {
        set_error("an edge joins a node to itself");
        return false;
      }
      T.edge_a[e] = (int32_t)a;
      T.edge_b[e] = (int32_t)b;
      T.edge_rod[e] = r;
      V3 ev = sub(X[b], X[a]);
      double l = norm(ev);
      if (!(l > 0)) {
        set_error("zero-length edge in the rest shape");
        return false;
      }
      T.edge_lbar[e] = l;
      T.edge_EA[e] = E * A;
      T.edge_EI[e] = E * M_PI * h * h * h * h / 4.0;
      T.edge_GJ[e] = G * M_PI * h * h * h * h / 2.0;
      T.edge_rhoA[e] = D->rho[r] * A;
      T.edge_h[e] = h;
      T.t_init[3 * e] = ev.x / l;
      T.t_init[3 * e + 1] = ev.y / l;
      T.t_init[3 * e + 2] = ev.z / l;
    }
  }

  // --- node masses, Voronoi lengths, contact radius, owner rod
  T.node_mass.assign(nn, 0.0);
  T.node_vor.assign(nn, 0.0);
  T.node_h.assign(nn, 0.0);
  std::vector<int32_t> owner(nn, R);
  for (int64_t e = 0; e < ne; ++e) {
    for (int32_t v : {T.edge_a[e], T.edge_b[e]}) {
      T.node_mass[v] += 0.5 * T.edge_rhoA[e] * T.edge_lbar[e];
      T.node_vor[v] += 0.5 * T.edge_lbar[e];
      T.node_h[v] = std::max(T.node_h[v], T.edge_h[e]);
      owner[v] = std::min(owner[v], T.edge_rod[e]);
    }
  }
  T.node_mu.resize(nn);
  T.node_kc.resize(nn);
  for (int64_t v = 0; v < nn; ++v) {
    T.node_mu[v] = D->ground_mu ? D->ground_mu[owner[v]] : 0.0;
    T.node_kc[v] = D->ground_kc ? D->ground_kc[owner[v]] : 0.0;
  }

  // --- initial reference frames (reading C5)
  T.d1_init.resize(3 * ne);
  auto tvec = [&](int64_t e) {
    return V3{T.t_init[3 * e], T.t_init[3 * e + 1], T.t_init[3 * e + 2]};
  };
  for (int r = 0; r < R; ++r) {
    int64_t e0 = T.rod_edge0[r];
    V3 t = tvec(e0);
    V3 z{0, 0, 1};
    if (norm(cross(z, t)) < 1e-6) z = {1, 0, 0};
    V3 d = sub(z, mul(dot(z, t), t));
    d = mul(1.0 / norm(d), d);
    V3 prev = d;
    T.d1_init[3 * e0] = d.x;
    T.d1_init[3 * e0 + 1] = d.y;
    T.d1_init[3 * e0 + 2] = d.z;
    for (int i = 1; i + 1 < T.npr[r]; ++i) {
      int64_t e = e0 + i;
      V3 ta = tvec(e - 1), tb = tvec(e);
      if (1.0 + dot(ta, tb) <= 1e-12) {
        set_error("antiparallel consecutive edges in the rest shape");
        return false;
      }
      prev = transport(prev, ta, tb);
      T.d1_init[3 * e] = prev.x;
      T.d1_init[3 * e + 1] = prev.y;
      T.d1_init[3 * e + 2] = prev.z;
    }
  }
  auto d1vec = [&](int64_t e) {
    return V3{T.d1_init[3 * e], T.d1_init[3 * e + 1], T.d1_init[3 * e + 2]};
  };

  // --- systems: connected components of rods (rods must be consecutive)
  std::vector<int32_t> rod_sys(R, -1);
  {
    std::vector<int64_t> comp(nn);
    std::iota(comp.begin(), comp.end(), 0);
    auto cf = [&](int64_t a) {
      while (comp[a] != a) {
        comp[a] = comp[comp[a]];
        a = comp[a];
      }
      return a;
    };
    for (int64_t e = 0; e < ne; ++e) {
      int64_t ra = cf(T.edge_a[e]), rb = cf(T.edge_b[e]);
      if (ra != rb) comp[std::max(ra, rb)] = std::min(ra, rb);
    }
    // contact groups: their rods form one system (edge-edge contact between
    // rods, reading C26)
    if (D->n_contact_groups > 0) {
      if (!P->self_contact || !D->contact_group_offsets || !D->contact_group_rods) {
        set_error("contact groups need self_contact and the group arrays");
        return false;
      }
      for (int g = 0; g < D->n_contact_groups; ++g) {
        const int32_t b = D->contact_group_offsets[g], e = D->contact_group_offsets[g + 1];
        if (b < 0 || e < b) {
          set_error("contact groups: bad offsets");
          return false;
        }
        for (int32_t k = b; k < e; ++k) {
          const int32_t r = D->contact_group_rods[k];
          if (r < 0 || r >= R || (k > b && r != D->contact_group_rods[k - 1] + 1)) {
            set_error("contact group " + std::to_string(g) +
                      ": rods must be valid and consecutive in the descriptor");
            return false;
          }
          const int64_t ra = cf(T.flat2node[T.rod_node0[D->contact_group_rods[b]]]);
          const int64_t rb = cf(T.flat2node[T.rod_node0[r]]);
          if (ra != rb) comp[std::max(ra, rb)] = std::min(ra, rb);
        }
      }
    }
    std::vector<int64_t> rootsys;
    for (int r = 0; r < R; ++r) {
      int64_t c = cf(T.flat2node[T.rod_node0[r]]);
      if (!rootsys.empty() && rootsys.back() == c) {
        rod_sys[r] = (int32_t)rootsys.size() - 1;
      } else {
        for (size_t k = 0; k + 1 < rootsys.size() + 1 && k < rootsys.size(); ++k)
          if (rootsys[k] == c) {
            set_error("rods of one joined system must be consecutive in the descriptor");
            return false;
          }
        rootsys.push_back(c);
        rod_sys[r] = (int32_t)rootsys.size() - 1;
      }
    }
    T.n_systems = (int32_t)rootsys.size();
  }
  const int S = T.n_systems;
  T.sys_rod0.assign(S, -1);
  T.sys_nrods.assign(S, 0);
  for (int r = 0; r < R; ++r) {
    if (T.sys_rod0[rod_sys[r]] < 0) T.sys_rod0[rod_sys[r]] = r;
    T.sys_nrods[rod_sys[r]]++;
  }
  T.edge_sys.resize(ne);
  for (int64_t e = 0; e < ne; ++e) T.edge_sys[e] = rod_sys[T.edge_rod[e]];
  T.node_sys.resize(nn);
  for (int64_t e = 0; e < ne; ++e) {
    T.node_sys[T.edge_a[e]] = T.edge_sys[e];
    T.node_sys[T.edge_b[e]] = T.edge_sys[e];
  }

  // --- joints may only merge rod end nodes
  std::vector<int32_t> mult(nn, 0);
  for (int64_t a = 0; a < nflat; ++a) mult[T.flat2node[a]]++;
  for (int r = 0; r < R; ++r)
    for (int i = 1; i + 1 < T.npr[r]; ++i)
      if (mult[T.flat2node[T.rod_node0[r] + i]] > 1) {
        set_error("joints must join rod end nodes (rod " + std::to_string(r) + ", node " +
                  std::to_string(i) + ")");
        return false;
      }
  T.ground = P->ground != 0;

  // --- DOF numbering.  Single rods without contact: Eq. 1 order.  General
  // systems (joints or ground contact): every rod's interior DOFs in Eq. 1
  // order, then the border: joint nodes, the nodes next to them along each
  // attached rod, and the twist angles of the edges at joint nodes.
  T.node_dof.assign(nn, -1);
  T.edge_thdof.assign(ne, -1);
  T.sys_dof0.assign(S, 0);
  T.sys_ndof.assign(S, 0);
  T.sys_kind.assign(S, SOLVE_ROD_BAND);
  std::vector<char> bnode(nn, 0), bedge(ne, 0);
  std::vector<int32_t> limb_sys, limb_rod, limb_d0, limb_n;
  std::vector<std::vector<int32_t>> sys_border(S);
  int32_t ndof = 0;
  for (int s = 0; s < S; ++s) {
    T.sys_dof0[s] = ndof;
    const int r0 = T.sys_rod0[s], r1 = T.sys_rod0[s] + T.sys_nrods[s];
    // a contact group: several rods without joints, each in Eq. 1 order,
    // solved together on the contact path
    bool jointless = true;
    for (int r = r0; r < r1 && jointless; ++r)
      for (int i = 0; i < T.npr[r]; ++i)
        if (mult[T.flat2node[T.rod_node0[r] + i]] > 1) jointless = false;
    // (with edge-edge contact, jointless systems stay on the contact path
    // also on the ground: the ground terms join their dense matrix)
    const bool group = T.sys_nrods[s] > 1 && P->self_contact && jointless;
    const bool general = (T.sys_nrods[s] > 1 || T.ground) && !group &&
                         !(P->self_contact && jointless);
    T.sys_kind[s] = group ? SOLVE_CONTACT : general ? SOLVE_GENERAL : SOLVE_ROD_BAND;
    if (!general) {
      for (int r = r0; r < r1; ++r)
        for (int i = 0; i < T.npr[r]; ++i) {
          T.node_dof[T.flat2node[T.rod_node0[r] + i]] = ndof;
          ndof += 3;
          if (i + 1 < T.npr[r]) T.edge_thdof[T.rod_edge0[r] + i] = ndof++;
        }
      T.sys_ndof[s] = ndof - T.sys_dof0[s];
      continue;
    }
    for (int r = r0; r < r1; ++r) {
      const int N = T.npr[r];
      for (int end = 0; end < 2; ++end) {
        const int i = end ? N - 1 : 0, nb = end ? N - 2 : 1;
        const int64_t v = T.flat2node[T.rod_node0[r] + i];
        if (mult[v] > 1) {
          bnode[v] = 1;
          bnode[T.flat2node[T.rod_node0[r] + nb]] = 1;
          bedge[T.rod_edge0[r] + (end ? N - 2 : 0)] = 1;
        }
      }
    }
    for (int r = r0; r < r1; ++r) {
      const int N = T.npr[r];
      int first = -1, last = -1, count = 0;
      for (int k = 0; k < 4 * N - 1; ++k) {
        const int i = k / 4, c = k % 4;
        const bool isb = c < 3 ? bnode[T.flat2node[T.rod_node0[r] + i]] != 0
                               : bedge[T.rod_edge0[r] + i] != 0;
        if (isb) continue;
        if (first < 0) first = k;
        if (last >= 0 && k != last + 1) {
          set_error("rod " + std::to_string(r) + ": border DOFs inside the rod");
          return false;
        }
        last = k;
        ++count;
      }
      if (count > 0) {
        limb_sys.push_back(s);
        limb_rod.push_back(r);
        limb_d0.push_back(ndof);
        limb_n.push_back(count);
      }
      for (int k = first; count > 0 && k <= last; ++k) {
        const int i = k / 4, c = k % 4;
        if (c < 3) {
          if (c == 0) T.node_dof[T.flat2node[T.rod_node0[r] + i]] = ndof;
          ++ndof;
        } else {
          T.edge_thdof[T.rod_edge0[r] + i] = ndof++;
        }
      }
    }
    for (int r = r0; r < r1; ++r) {
      const int N = T.npr[r];
      for (int i = 0; i < N; ++i) {
        const int64_t v = T.flat2node[T.rod_node0[r] + i];
        if (bnode[v] && T.node_dof[v] < 0) {
          T.node_dof[v] = ndof;
          for (int c = 0; c < 3; ++c) sys_border[s].push_back(ndof++);
        }
        if (i + 1 < N && bedge[T.rod_edge0[r] + i] && T.edge_thdof[T.rod_edge0[r] + i] < 0) {
          T.edge_thdof[T.rod_edge0[r] + i] = ndof;
          sys_border[s].push_back(ndof++);
        }
      }
    }
    T.sys_ndof[s] = ndof - T.sys_dof0[s];
  }
  T.n_dofs = ndof;
  T.sys_edge0.assign(S, 0);
  T.sys_nedge.assign(S, 0);
  for (int s = 0; s < S; ++s) {
    T.sys_edge0[s] = (int32_t)T.rod_edge0[T.sys_rod0[s]];
    T.sys_nedge[s] = (int32_t)(T.rod_edge0[T.sys_rod0[s] + T.sys_nrods[s]] - T.sys_edge0[s]);
  }

  // --- bend-twist stencils: every unordered pair of edges at a node
  std::vector<std::vector<int32_t>> inc(nn);
  for (int64_t e = 0; e < ne; ++e) {
    inc[T.edge_a[e]].push_back((int32_t)e);
    inc[T.edge_b[e]].push_back((int32_t)e);
  }
  std::vector<int64_t> kslot0(R + 1, 0);
  for (int r = 0; r < R; ++r) kslot0[r + 1] = kslot0[r] + (T.npr[r] - 2);
  for (int64_t v = 0; v < nn; ++v) {
    auto &es = inc[v];
    std::sort(es.begin(), es.end());
    for (size_t i = 0; i < es.size(); ++i)
      for (size_t j = i + 1; j < es.size(); ++j) {
        int32_t a = es[i], b = es[j];
        int32_t sa = (T.edge_b[a] == v) ? 1 : -1;
        int32_t sb = (T.edge_a[b] == v) ? 1 : -1;
        int32_t na = (sa == 1) ? T.edge_a[a] : T.edge_b[a];
        int32_t nb = (sb == 1) ? T.edge_b[b] : T.edge_a[b];
        T.st_node[0].push_back(na);
        T.st_node[1].push_back((int32_t)v);
        T.st_node[2].push_back(nb);
        T.st_edge[0].push_back(a);
        T.st_edge[1].push_back(b);
        T.st_sign[0].push_back(sa);
        T.st_sign[1].push_back(sb);
        T.st_sys.push_back(T.edge_sys[a]);
        int32_t slot = -1;
        if (T.edge_rod[a] == T.edge_rod[b] && b == a + 1 && sa == 1 && sb == 1) {
          int r = T.edge_rod[a];
          slot = (int32_t)(kslot0[r] + (a - T.rod_edge0[r]));
        }
        T.st_rod_slot.push_back(slot);
        // rest Voronoi length (reading C1), averaged stiffness (reading C18)
        double V = 0.5 * (T.edge_lbar[a] + T.edge_lbar[b]);
        T.st_kb.push_back(0.5 * (T.edge_EI[a] + T.edge_EI[b]) / V);
        T.st_kt.push_back(0.5 * (T.edge_GJ[a] + T.edge_GJ[b]) / V);
        // initial reference twist and natural strains (readings C4, C5)
        V3 ta = mul((double)sa, tvec(a)), tb = mul((double)sb, tvec(b));
        if (1.0 + dot(ta, tb) <= 1e-12) {
          set_error("antiparallel edges at a stencil in the rest shape");
          return false;
        }
        V3 d1a = d1vec(a), d1b = d1vec(b);
        V3 u = transport(d1a, ta, tb);
        double beta = std::atan2(dot(tb, cross(u, d1b)), dot(u, d1b));
        double th_a = D->theta0 ? D->theta0[a] : 0.0;
        double th_b = D->theta0 ? D->theta0[b] : 0.0;
        double k1, k2, tau;
        rest_strains(ta, d1a, sa * th_a, tb, d1b, sb * th_b, beta, &k1, &k2, &tau);
        T.st_beta0.push_back(beta);
        T.st_kbar1.push_back(k1);
        T.st_kbar2.push_back(k2);
        T.st_taubar.push_back(tau);
      }
  }
  T.n_stencils = (int64_t)T.st_kb.size();
  T.sys_st0.assign(S, 0);
  T.sys_nst.assign(S, 0);
  {
    int64_t k = 0;
    for (int s = 0; s < S; ++s) {
      T.sys_st0[s] = (int32_t)k;
      while (k < T.n_stencils && T.st_sys[k] == s) ++k;
      T.sys_nst[s] = (int32_t)(k - T.sys_st0[s]);
    }
    if (k != T.n_stencils) {
      set_error("internal: stencils not grouped by system");
      return false;
    }
  }

  // (general-path storage and gather maps are built after the fixed DOFs)
  // --- per-DOF masses (reading C7), state, fixed DOFs
  T.dof_mass.assign(ndof, 0.0);
  T.q0.assign(ndof, 0.0);
  T.v0.assign(ndof, 0.0);
  T.dof_fixed.assign(ndof, 0);
  for (int64_t v = 0; v < nn; ++v)
    for (int c = 0; c < 3; ++c) {
      T.dof_mass[T.node_dof[v] + c] = T.node_mass[v];
      T.q0[T.node_dof[v] + c] = (&X[v].x)[c];
      T.v0[T.node_dof[v] + c] = (&Vn[v].x)[c];
    }
  for (int64_t e = 0; e < ne; ++e) {
    int32_t d = T.edge_thdof[e];
    T.dof_mass[d] = 0.5 * T.edge_rhoA[e] * T.edge_h[e] * T.edge_h[e] * T.edge_lbar[e];
    T.q0[d] = D->theta0 ? D->theta0[e] : 0.0;
    T.v0[d] = D->theta_dot0 ? D->theta_dot0[e] : 0.0;
  }
  T.layout2dof.resize(T.rod_layout0[R]);
  for (int r = 0; r < R; ++r)
    for (int i = 0; i < T.npr[r]; ++i) {
      int64_t base = T.rod_layout0[r] + 4 * i;
      int32_t nd = T.node_dof[T.flat2node[T.rod_node0[r] + i]];
      for (int c = 0; c < 3; ++c) T.layout2dof[base + c] = nd + c;
      if (i + 1 < T.npr[r]) T.layout2dof[base + 3] = T.edge_thdof[T.rod_edge0[r] + i];
    }
  if (D->fixed)
    for (int64_t k = 0; k < T.rod_layout0[R]; ++k)
      if (D->fixed[k]) T.dof_fixed[T.layout2dof[k]] = 1;

  // --- residual scale: 1 / (D_i l_i)
  std::vector<double> dsc(ndof), lsys(S, 0.0);
  for (int32_t i = 0; i < ndof; ++i) dsc[i] = T.dof_mass[i] / (P->dt * P->dt);
  for (int64_t e = 0; e < ne; ++e) {
    double k = T.edge_EA[e] / T.edge_lbar[e];
    for (int c = 0; c < 3; ++c) {
      dsc[T.node_dof[T.edge_a[e]] + c] += k;
      dsc[T.node_dof[T.edge_b[e]] + c] += k;
    }
    lsys[T.edge_sys[e]] += T.edge_lbar[e];
  }
  for (int64_t k = 0; k < T.n_stencils; ++k) {
    dsc[T.edge_thdof[T.st_edge[0][k]]] += T.st_kt[k];
    dsc[T.edge_thdof[T.st_edge[1][k]]] += T.st_kt[k];
  }
  T.dof_rscale.assign(ndof, 0.0);
  for (int64_t v = 0; v < nn; ++v)
    for (int c = 0; c < 3; ++c) {
      int32_t i = T.node_dof[v] + c;
      T.dof_rscale[i] = 1.0 / (dsc[i] * lsys[T.node_sys[v]]);
    }
  for (int64_t e = 0; e < ne; ++e) {
    int32_t i = T.edge_thdof[e];
    T.dof_rscale[i] = 1.0 / dsc[i];
  }

  // --- force gather lists (per DOF: stencil slots and edge slots)
  std::vector<std::vector<int32_t>> lists(ndof);
  for (int64_t k = 0; k < T.n_stencils; ++k) {
    int32_t slots[11];
    for (int n = 0; n < 3; ++n)
      for (int c = 0; c < 3; ++c) slots[4 * n + c] = T.node_dof[T.st_node[n][k]] + c;
    slots[3] = T.edge_thdof[T.st_edge[0][k]];
    slots[7] = T.edge_thdof[T.st_edge[1][k]];
    for (int l = 0; l < 11; ++l) lists[slots[l]].push_back((int32_t)((k << 5) | l));
  }
  for (int64_t e = 0; e < ne; ++e)
    for (int c = 0; c < 3; ++c) {
      lists[T.node_dof[T.edge_a[e]] + c].push_back((int32_t)((e << 5) | 16 | c));
      lists[T.node_dof[T.edge_b[e]] + c].push_back((int32_t)((e << 5) | 16 | (3 + c)));
    }
  T.gat_ptr.assign(ndof + 1, 0);
  for (int32_t i = 0; i < ndof; ++i) T.gat_ptr[i + 1] = T.gat_ptr[i] + (int32_t)lists[i].size();
  T.gat_ent.resize(T.gat_ptr[ndof]);
  for (int32_t i = 0; i < ndof; ++i)
    std::copy(lists[i].begin(), lists[i].end(), T.gat_ent.begin() + T.gat_ptr[i]);
  if (T.n_stencils >= (1 << 26) || ne >= (1 << 26)) {
    set_error("too many stencils or edges for one handle (limit 2^26)");
    return false;
  }

  // --- per-DOF node and component
  T.dof_node.assign(ndof, -1);
  T.dof_comp.assign(ndof, 3);
  for (int64_t v = 0; v < nn; ++v)
    for (int c = 0; c < 3; ++c) {
      T.dof_node[T.node_dof[v] + c] = (int32_t)v;
      T.dof_comp[T.node_dof[v] + c] = c;
    }

  // --- general systems: storage layout and the assembly gather map
  std::vector<int32_t> dof_limb(ndof, -1), dof_row(ndof, -1), dof_bidx(ndof, -1);
  int64_t off = 0;
  std::vector<std::pair<int64_t, uint32_t>> pairs;
  size_t li = 0;
  for (int s = 0; s < S; ++s) {
    if (T.sys_kind[s] != SOLVE_GENERAL) continue;
    T.any_general = true;
    const int gid = (int)T.gen_sys.size();
    T.gen_sys.push_back(s);
    const int nB = (int)sys_border[s].size();
    T.gs_nB.push_back(nB);
    T.gs_border0.push_back((int32_t)T.border_dof.size());
    for (int b = 0; b < nB; ++b) {
      T.border_dof.push_back(sys_border[s][b]);
      dof_bidx[sys_border[s][b]] = b;
    }
    T.gs_limb0.push_back((int32_t)T.lb_dof0.size());
    int nl = 0;
    std::vector<int> mylimbs;
    while (li < limb_sys.size() && limb_sys[li] == s) {
      const int L = (int)T.lb_dof0.size();
      T.lb_dof0.push_back(limb_d0[li]);
      T.lb_n.push_back(limb_n[li]);
      for (int k = 0; k < limb_n[li]; ++k) {
        dof_limb[limb_d0[li] + k] = L;
        dof_row[limb_d0[li] + k] = k;
      }
      mylimbs.push_back(L);
      ++li;
      ++nl;
    }
    T.gs_nlimb.push_back(nl);
    // element entries of this system: (row DOF, col DOF, source)
    std::vector<std::tuple<int32_t, int32_t, uint32_t>> ent;
    auto fixed = [&](int32_t g) { return T.dof_fixed[g] != 0; };
    auto add = [&](int32_t g1, int32_t g2, uint32_t src) {
      if (fixed(g1) || fixed(g2)) return;
      ent.emplace_back(g1, g2, src);
    };
    for (int64_t k = T.sys_st0[s]; k < T.sys_st0[s] + T.sys_nst[s]; ++k) {
      int32_t slots[11];
      for (int n = 0; n < 3; ++n)
        for (int c = 0; c < 3; ++c) slots[4 * n + c] = T.node_dof[T.st_node[n][k]] + c;
      slots[3] = T.edge_thdof[T.st_edge[0][k]];
      slots[7] = T.edge_thdof[T.st_edge[1][k]];
      for (int a = 0; a < 11; ++a)
        for (int b = 0; b < 11; ++b) {
          const int lo = a < b ? a : b, hi = a < b ? b : a;
          const int up = lo * 11 - lo * (lo - 1) / 2 + (hi - lo);
          add(slots[a], slots[b], src_code(SRC_STENCIL, (uint32_t)(up * T.n_stencils + k), false));
        }
    }
    for (int64_t e = T.sys_edge0[s]; e < T.sys_edge0[s] + T.sys_nedge[s]; ++e) {
      const int32_t ba = T.node_dof[T.edge_a[e]], bb = T.node_dof[T.edge_b[e]];
      for (int sa = 0; sa < 2; ++sa)
        for (int sb = 0; sb < 2; ++sb)
          for (int ca = 0; ca < 3; ++ca)
            for (int cb = 0; cb < 3; ++cb) {
              const int i = ca < cb ? ca : cb, j = ca < cb ? cb : ca;
              const int ks = 3 + (i == 0 ? j : (i == 1 ? 2 + j : 5));
              add((sa ? bb : ba) + ca, (sb ? bb : ba) + cb,
                  src_code(SRC_EDGE, (uint32_t)(ks * ne + e), sa != sb));
            }
    }
    for (int32_t g = T.sys_dof0[s]; g < T.sys_dof0[s] + T.sys_ndof[s]; ++g) {
      if (T.ground && T.dof_comp[g] < 3) {
        const int32_t v = T.dof_node[g], c = T.dof_comp[g];
        if (c == 0)
          for (int ca = 0; ca < 3; ++ca)
            for (int cb = 0; cb < 3; ++cb)
              add(g + ca, g + cb, src_code(SRC_NODE, (uint32_t)((3 + 3 * ca + cb) * nn + v), false));
      }
      ent.emplace_back(g, g, src_code(SRC_DIAG, (uint32_t)g, false));
    }
    // coupled rows (limb-local, natural order) and coupled border columns
    std::vector<std::vector<int32_t>> crow(nl), bcl(nl);
    for (auto &t : ent) {
      const int32_t g1 = std::get<0>(t), g2 = std::get<1>(t);
      if (dof_limb[g1] >= 0 && dof_bidx[g2] >= 0) {
        crow[dof_limb[g1] - mylimbs[0]].push_back(dof_row[g1]);
        bcl[dof_limb[g1] - mylimbs[0]].push_back(dof_bidx[g2]);
      }
      if (dof_bidx[g1] >= 0 && dof_limb[g2] >= 0) {
        crow[dof_limb[g2] - mylimbs[0]].push_back(dof_row[g2]);
        bcl[dof_limb[g2] - mylimbs[0]].push_back(dof_bidx[g1]);
      }
    }
    // Condensation path: every limb couples to the border only through its
    // first or its last kFastMaxM rows (a rod attached at one end).  The
    // limb is then eliminated from its free end, leaving an m x m block.
    bool fast = nB <= kFastMaxBorder;
    std::vector<int32_t> ldir(nl, 0), lm(nl, 0);
    for (int l = 0; l < nl; ++l) {
      auto &c = crow[l];
      std::sort(c.begin(), c.end());
      c.erase(std::unique(c.begin(), c.end()), c.end());
      auto &b = bcl[l];
      std::sort(b.begin(), b.end());
      b.erase(std::unique(b.begin(), b.end()), b.end());
      const int n = T.lb_n[mylimbs[l]];
      if (n > kFastMaxRows) fast = false;
      if (c.empty()) continue;
      if (c.back() < kFastMaxM) {
        ldir[l] = 1;
        lm[l] = c.back() + 1;
      } else if (c.front() >= n - kFastMaxM) {
        lm[l] = n - c.front();
      } else {
        fast = false;
      }
      if ((int)b.size() > kFastMaxBC) fast = false;
    }
    T.gs_fast.push_back(fast ? 1 : 0);
    std::vector<std::vector<int32_t>> crmap(nl), bcmap(nl);
    for (int l = 0; l < nl; ++l) {
      const int L = mylimbs[l];
      T.lb_gsys.push_back(gid);
      T.lb_ncr.push_back((int32_t)crow[l].size());
      T.lb_cr0.push_back((int32_t)T.coupled_rows.size());
      crmap[l].assign(T.lb_n[L], -1);
      for (size_t k = 0; k < crow[l].size(); ++k) {
        T.coupled_rows.push_back(crow[l][k]);
        crmap[l][crow[l][k]] = (int32_t)k;
      }
      const int64_t n = T.lb_n[L], ncr = (int64_t)crow[l].size();
      const int64_t nbc = (int64_t)bcl[l].size(), m = lm[l];
      T.lb_dir.push_back(fast ? ldir[l] : 0);
      T.lb_m.push_back(fast ? (int32_t)m : 0);
      T.lb_nbc.push_back(fast ? (int32_t)nbc : 0);
      T.lb_bc0.push_back((int32_t)T.lb_bcols.size());
      bcmap[l].assign(nB, -1);
      if (fast)
        for (int64_t k = 0; k < nbc; ++k) {
          T.lb_bcols.push_back(bcl[l][k]);
          bcmap[l][bcl[l][k]] = (int32_t)k;
        }
      if (fast) {
        T.lb_band.push_back(off); off += 21 * n;   // row-major [n][21]
        T.lb_piv.push_back(off); off += n;         // reciprocal pivots
        T.lb_C.push_back(off); off += m * nbc;
        T.lb_R.push_back(off); off += nbc * m;
        T.lb_Y.push_back(off); off += m * (nbc + 1);
        // [n][12]: U row (10 entries), eliminated right-hand side and
        // reciprocal pivot of each eliminated row (the band stays assembled)
        T.lb_y.push_back(off); off += 12 * n;
      } else {
        T.lb_band.push_back(off); off += 31 * n;   // kl = 10, ku + fill = 20
        T.lb_piv.push_back(off); off += n;
        T.lb_C.push_back(off); off += ncr * nB;
        T.lb_R.push_back(off); off += ncr * nB;
        T.lb_Y.push_back(off); off += n * nB;
        T.lb_y.push_back(off); off += n;
      }
    }
    T.gs_JBB.push_back(off); off += (int64_t)nB * nB;
    T.gs_rB.push_back(off); off += nB;
    T.gs_S.push_back(off); off += (int64_t)nB * nB;
    T.gs_xB.push_back(off); off += nB;
    T.gs_mat0.push_back(T.lb_band.empty() || nl == 0 ? T.gs_JBB.back() : T.lb_band[mylimbs[0]]);
    T.gs_mat1.push_back(off);
    for (auto &t : ent) {
      const int32_t g1 = std::get<0>(t), g2 = std::get<1>(t);
      const uint32_t src = std::get<2>(t);
      int64_t tgt = -1;
      const int L1 = dof_limb[g1], L2 = dof_limb[g2];
      // row of limb L in the elimination order of the condensation path
      auto mapped = [&](int L, int r) { return T.lb_dir[L] ? T.lb_n[L] - 1 - r : r; };
      if (L1 >= 0 && L2 >= 0) {
        const int r1 = dof_row[g1], r2 = dof_row[g2];
        if (L1 != L2 || r2 - r1 > 10 || r1 - r2 > 10) {
          set_error("internal: element couples DOFs outside a limb band");
          return false;
        }
        if (fast) {
          const int p1 = mapped(L1, r1), p2 = mapped(L1, r2);
          tgt = T.lb_band[L1] + (int64_t)p1 * 21 + (p2 - p1 + 10);
        } else {
          tgt = T.lb_band[L1] + (int64_t)(r2 - r1 + 10) * T.lb_n[L1] + r1;
        }
      } else if (L1 >= 0) {
        if (fast) {
          const int a = mapped(L1, dof_row[g1]) - (T.lb_n[L1] - T.lb_m[L1]);
          tgt = T.lb_C[L1] + (int64_t)a * T.lb_nbc[L1] + bcmap[L1 - mylimbs[0]][dof_bidx[g2]];
        } else {
          tgt = T.lb_C[L1] + (int64_t)crmap[L1 - mylimbs[0]][dof_row[g1]] * nB + dof_bidx[g2];
        }
      } else if (L2 >= 0) {
        if (fast) {
          const int a = mapped(L2, dof_row[g2]) - (T.lb_n[L2] - T.lb_m[L2]);
          tgt = T.lb_R[L2] + (int64_t)bcmap[L2 - mylimbs[0]][dof_bidx[g1]] * T.lb_m[L2] + a;
        } else {
          tgt = T.lb_R[L2] + (int64_t)dof_bidx[g1] * T.lb_ncr[L2] + crmap[L2 - mylimbs[0]][dof_row[g2]];
        }
      } else {
        tgt = T.gs_JBB[gid] + (int64_t)dof_bidx[g1] * nB + dof_bidx[g2];
      }
      pairs.emplace_back(tgt, src);
    }
  }
  T.gen_doubles = off;
  std::stable_sort(pairs.begin(), pairs.end(),
                   [](const std::pair<int64_t, uint32_t> &a, const std::pair<int64_t, uint32_t> &b) {
                     return a.first < b.first;
                   });
  T.asm_ptr.push_back(0);
  for (size_t k = 0; k < pairs.size(); ++k) {
    if (k == 0 || pairs[k].first != pairs[k - 1].first) {
      if (k > 0) T.asm_ptr.push_back((int32_t)k);
      T.asm_target.push_back(pairs[k].first);
    }
    T.asm_src.push_back(pairs[k].second);
  }
  if (!pairs.empty()) T.asm_ptr.push_back((int32_t)pairs.size());
  // system of each target (storage regions are contiguous and ascending)
  T.asm_sys.resize(T.asm_target.size());
  for (size_t k = 0; k < T.asm_target.size(); ++k) {
    const int64_t o = T.asm_target[k];
    const size_t w = std::upper_bound(T.gs_mat0.begin(), T.gs_mat0.end(), o) - T.gs_mat0.begin() - 1;
    T.asm_sys[k] = T.gen_sys[w];
  }
  // first target of each system's storage region
  T.asm_t0.resize(T.gen_sys.size() + 1);
  for (size_t w = 0; w < T.gen_sys.size(); ++w)
    T.asm_t0[w] = (int32_t)(std::lower_bound(T.asm_target.begin(), T.asm_target.end(),
                                             T.gs_mat0[w]) - T.asm_target.begin());
  T.asm_t0[T.gen_sys.size()] = (int32_t)T.asm_target.size();
  return true;
}

}  // namespace dm
