"""Sharding a batch of rod systems over ranks (one process per GPU).

Systems (a rod, or rods connected by joints or declared a contact group)
are independent: a step of one never reads another, so a batch splits into
contiguous ranges of systems, one per rank, with no exchange inside a step.
The ranges are balanced greedily by DOF count (4 N - 1 per rod of N nodes,
the size of the Newton system each rank factors) and never cut a system.
Each rank builds its own ``System`` from its sub-descriptor; the per-rank
states, in the per-rod layout of Eq. 1, concatenate in rank order into the
layout of the whole batch.  Host logic only: the arrays are numpy.
"""
import numpy as np

_ROD_KEYS = ("E", "nu", "rho", "radius", "ground_mu", "ground_kc")


def rod_systems(desc):
    """System index of every rod (connected components of the rods under the
    joints and the contact groups), systems numbered by their lowest rod."""
    R = len(desc["nodes_per_rod"])
    parent = list(range(R))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    def unite(a, b):
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)

    for grp in desc.get("joints") or []:
        for (r, _) in grp[1:]:
            unite(grp[0][0], r)
    for grp in desc.get("contact_groups") or []:
        for r in grp[1:]:
            unite(grp[0], r)
    roots = [find(r) for r in range(R)]
    ids = {}
    return np.array([ids.setdefault(x, len(ids)) for x in roots], np.int64)


def partition(desc, nranks):
    """Contiguous rod ranges [(begin, end)] for ranks 0..nranks-1, cut only
    between systems, each rank's DOF count as close to total / nranks as the
    cuts allow (greedy: the cut nearest to each rank's cumulative target).
    Ranks beyond the number of systems get empty ranges."""
    npr = np.asarray(desc["nodes_per_rod"], np.int64)
    R = len(npr)
    if nranks < 1:
        raise ValueError("nranks must be positive")
    sysid = rod_systems(desc)
    # a cut before rod r is allowed when no system spans it
    last = {}
    for r in range(R):
        last[sysid[r]] = r
    reach = np.maximum.accumulate(np.array([last[sysid[r]] for r in range(R)]))
    cuts = [r for r in range(1, R) if reach[r - 1] < r]
    dofs = np.concatenate([[0], np.cumsum(4 * npr - 1)])
    total = float(dofs[-1])
    bounds = [0]
    for k in range(1, nranks):
        target = total * k / nranks
        cand = [c for c in cuts if c > bounds[-1]]
        if not cand:
            bounds.append(bounds[-1])
            continue
        # leave at least one cut for each later rank where possible
        spare = nranks - k - 1
        if len(cand) > spare:
            cand = cand[:len(cand) - spare] if spare else cand
        best = min(cand, key=lambda c: (abs(dofs[c] - target), c))
        bounds.append(best)
    bounds.append(R)
    return [(bounds[k], max(bounds[k], bounds[k + 1])) for k in range(nranks)]


def sub_descriptor(desc, begin, end):
    """Descriptor of rods [begin, end) of a batch (whole systems), rods,
    joints and contact groups renumbered from 0."""
    npr = np.asarray(desc["nodes_per_rod"], np.int64)
    noff = np.concatenate([[0], np.cumsum(npr)])
    eoff = np.concatenate([[0], np.cumsum(npr - 1)])
    foff = np.concatenate([[0], np.cumsum(4 * npr - 1)])
    out = {"nodes_per_rod": npr[begin:end].astype(np.int32)}
    x0 = np.asarray(desc["x0"], np.float64).reshape(-1, 3)
    out["x0"] = x0[noff[begin]:noff[end]].copy()
    if desc.get("v0") is not None:
        out["v0"] = np.asarray(desc["v0"], np.float64).reshape(-1, 3)[noff[begin]:noff[end]].copy()
    for k in ("theta0", "theta_dot0"):
        if desc.get(k) is not None:
            out[k] = np.asarray(desc[k], np.float64)[eoff[begin]:eoff[end]].copy()
    for k in _ROD_KEYS:
        if desc.get(k) is not None:
            out[k] = np.asarray(desc[k])[begin:end].copy()
    if desc.get("fixed") is not None:
        out["fixed"] = np.asarray(desc["fixed"])[foff[begin]:foff[end]].copy()
    inside = lambda r: begin <= r < end
    joints = []
    for grp in desc.get("joints") or []:
        if inside(grp[0][0]):
            joints.append([(r - begin, i) for (r, i) in grp])
    if joints:
        out["joints"] = joints
    groups = [[r - begin for r in g] for g in (desc.get("contact_groups") or []) if inside(g[0])]
    if groups:
        out["contact_groups"] = groups
    return out


def layout_ranges(desc, parts):
    """(offset, length) of each rank's rods in the state layout of the batch
    (per rod of N nodes 4 N - 1 entries, Eq. 1, rods concatenated)."""
    npr = np.asarray(desc["nodes_per_rod"], np.int64)
    foff = np.concatenate([[0], np.cumsum(4 * npr - 1)])
    return [(int(foff[b]), int(foff[e] - foff[b])) for (b, e) in parts]


def kbar_ranges(desc, parts):
    """Row ranges of each rank in per-interior-node arrays (the natural
    curvature layout: N - 2 rows per rod)."""
    npr = np.asarray(desc["nodes_per_rod"], np.int64)
    koff = np.concatenate([[0], np.cumsum(npr - 2)])
    return [(int(koff[b]), int(koff[e])) for (b, e) in parts]


def initial_state(desc):
    """q of the descriptor in the per-rod layout of Eq. 1 (node positions
    and twist angles, rods concatenated): the state a System starts from."""
    npr = np.asarray(desc["nodes_per_rod"], np.int64)
    x0 = np.asarray(desc["x0"], np.float64).reshape(-1, 3)
    ne = int(np.sum(npr - 1))
    th = np.asarray(desc.get("theta0") if desc.get("theta0") is not None else np.zeros(ne))
    out, n0, e0 = [], 0, 0
    for N in npr:
        q = np.zeros(4 * N - 1)
        q[4 * np.arange(N)[:, None] + np.arange(3)] = x0[n0:n0 + N]
        q[4 * np.arange(N - 1) + 3] = th[e0:e0 + N - 1]
        out.append(q)
        n0 += N
        e0 += N - 1
    return np.concatenate(out) if out else np.zeros(0)


def gather_states(local, desc, parts, group=None):
    """Per-rank state arrays (this rank's rods, Eq. 1 layout) gathered on
    rank 0 into the layout of the whole batch; other ranks get None.  With
    no process group (one rank) the local array is returned as it is."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return np.asarray(local)
    rank = dist.get_rank(group)
    ws = dist.get_world_size(group)
    objs = [None] * ws if rank == 0 else None
    dist.gather_object(np.asarray(local), objs, dst=0, group=group)
    if rank != 0:
        return None
    ranges = layout_ranges(desc, parts)
    full = np.empty(sum(n for _, n in ranges))
    for (off, n), arr in zip(ranges, objs):
        if len(arr) != n:
            raise ValueError("rank state of %d entries, expected %d" % (len(arr), n))
        full[off:off + n] = arr
    return full
