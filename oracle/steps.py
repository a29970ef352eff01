"""Step oracles for the Borůvka round and Filter-Borůvka -- TEST INFRASTRUCTURE ONLY.

Plain numpy restatements of each step of the paper's method, one function per
step, in the paper's order, with no blocking, fusion or reordering.  Used by
the tests to check the GPU path step by step; never imported by it.

Edge lists are four equal-length arrays (u, v, w, id): current endpoint labels,
uint32 weight and the original input-edge id.  The key of an edge is the uint64
(w << 32) | id, a strict total order on edges (Section 2.3: ties broken
consistently, so the MST is unique).  INF = 2^64 - 1 means "no edge".
"""
from __future__ import annotations

import numpy as np

INF = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def keys(w, ids) -> np.ndarray:
    """uint64 key (w << 32) | id."""
    return (np.asarray(w, dtype=np.uint64) << np.uint64(32)) | np.asarray(ids, dtype=np.uint64)


def as_edges(src, dst, w, ids=None):
    src = np.asarray(src, dtype=np.uint32)
    ids = np.arange(src.shape[0], dtype=np.uint32) if ids is None else np.asarray(ids, dtype=np.uint32)
    return src, np.asarray(dst, dtype=np.uint32), np.asarray(w, dtype=np.uint32), ids


# ----------------------------------------------------------------- one round

def min_edges(n: int, u, v, w, ids) -> np.ndarray:
    """minEdges (Alg. 1; Section 2.3, first step of a round): for every vertex c,
    the minimum key over the non-self-loop edges incident to c; INF if none.
    Pinned by: every selected edge lies in the Kruskal MSF (min-cut property),
    and rounds composed from these steps reproduce Kruskal exactly."""
    best = np.full(n, INF, dtype=np.uint64)
    u, v, w, ids = as_edges(u, v, w, ids)
    live = u != v
    k = keys(w[live], ids[live])
    np.minimum.at(best, u[live], k)
    np.minimum.at(best, v[live], k)
    return best


def hook(n: int, u, v, w, ids, best):
    """Hooking (Section 2.3; Section 4.2 contractComponents): every vertex c with
    best[c] != INF points to the other endpoint of its minimum edge.  These
    pointers form pseudo-trees whose only cycles are 2-cycles, in which both
    ends chose the same edge; the smaller label of the two becomes the root (the
    paper leaves this tie-breaking rule open).  Returns (parent, chosen ids):
    parent[x] = x for roots and for vertices without an edge; every chosen edge
    is reported once.  Pinned by: chosen edges are MSF edges; 2-cycle cases."""
    u, v, w, ids = as_edges(u, v, w, ids)
    best = np.asarray(best, dtype=np.uint64)
    parent = np.arange(n, dtype=np.uint32)
    c = np.nonzero(best != INF)[0].astype(np.uint32)
    if c.size == 0:
        return parent, np.zeros(0, dtype=np.uint32)
    chosen = (best[c] & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    order = np.argsort(ids, kind="stable")
    j = order[np.searchsorted(ids[order], chosen)]
    assert np.array_equal(ids[j], chosen)
    other = np.where(u[j] == c, v[j], u[j])
    root = (best[other] == best[c]) & (c < other)
    parent[c] = np.where(root, c, other)
    return parent, np.unique(chosen[~root])


def roots(parent, max_iter: int | None = None) -> np.ndarray:
    """Pointer doubling to rooted stars (Section 4.2): repeat parent =
    parent[parent] until nothing changes; returns the root of every vertex."""
    p = np.asarray(parent, dtype=np.uint32).copy()
    limit = max_iter if max_iter is not None else 2 + int(np.ceil(np.log2(max(p.size, 2))))
    for _ in range(limit + 1):
        q = p[p]
        if np.array_equal(q, p):
            return p
        p = q
    raise RuntimeError("pointer doubling did not converge: the parent array has a cycle")


def relabel(label, u, v, w, ids):
    """Relabel (Section 4.3): edge (u,v) becomes (label[u], label[v]); edges with
    equal labels are self-loops and are dropped.  Survivors keep their order."""
    u, v, w, ids = as_edges(u, v, w, ids)
    label = np.asarray(label, dtype=np.uint32)
    nu, nv = label[u], label[v]
    keep = nu != nv
    return nu[keep], nv[keep], w[keep], ids[keep]


def dedupe(u, v, w, ids):
    """Parallel-edge removal (Section 2.3, "optionally"; Section 4.3 Redistribute):
    of the edges joining the same unordered pair {u,v} keep only the one with
    the smallest key.  Survivors keep their relative order and orientation."""
    u, v, w, ids = as_edges(u, v, w, ids)
    if u.size == 0:
        return u, v, w, ids
    a, b = np.minimum(u, v), np.maximum(u, v)
    order = np.lexsort((keys(w, ids), b, a))
    sa, sb = a[order], b[order]
    first = np.ones(order.size, dtype=bool)
    first[1:] = (sa[1:] != sa[:-1]) | (sb[1:] != sb[:-1])
    keep = np.zeros(u.size, dtype=bool)
    keep[order[first]] = True
    return u[keep], v[keep], w[keep], ids[keep]


def boruvka_round(n: int, u, v, w, ids, do_dedupe: bool = True):
    """One Borůvka round (Section 2.3): minEdges, hook, contract to roots,
    relabel + drop self-loops, optionally drop parallel edges.
    Returns (root label per vertex, chosen ids, next edge list)."""
    best = min_edges(n, u, v, w, ids)
    parent, chosen = hook(n, u, v, w, ids, best)
    r = roots(parent)
    nxt = relabel(r, u, v, w, ids)
    if do_dedupe:
        nxt = dedupe(*nxt)
    return r, chosen, nxt


def boruvka_msf(n: int, src, dst, w, do_dedupe: bool = True):
    """Plain Borůvka (Section 2.3) composed from the steps above until no edge
    is left.  Returns (ascending MSF ids, uint64 total, number of rounds)."""
    u, v, ww, ids = as_edges(src, dst, w)
    w_in = ww
    chosen_all = []
    rounds = 0
    u, v, ww, ids = relabel(np.arange(n, dtype=np.uint32), u, v, ww, ids)  # drop input self-loops
    while u.size:
        _, chosen, (u, v, ww, ids) = boruvka_round(n, u, v, ww, ids, do_dedupe)
        chosen_all.append(chosen)
        rounds += 1
    out = np.sort(np.concatenate(chosen_all)) if chosen_all else np.zeros(0, dtype=np.uint32)
    return out.astype(np.uint32), int(w_in[out].astype(np.uint64).sum()), rounds


# ----------------------------------------------------------- Filter-Borůvka

def splitmix64(state, i) -> np.ndarray:
    """Output #i of the splitmix64 sequence whose state starts at ``state``
    (Steele, Lea, Flood, OOPSLA 2014): mix(state + (i+1) * 0x9e3779b97f4a7c15)."""
    with np.errstate(over="ignore"):
        z = np.uint64(state) + (np.asarray(i, dtype=np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def mulhi_bounded(r, m: int) -> np.ndarray:
    """floor(r * m / 2^64) for uint64 r and m < 2^32 (multiply-shift range map)."""
    r = np.asarray(r, dtype=np.uint64)
    mm = np.uint64(m)
    hi = (r >> np.uint64(32)) * mm
    lo = ((r & np.uint64(0xFFFFFFFF)) * mm) >> np.uint64(32)
    return (hi + lo) >> np.uint64(32)


def pivot_state(seed: int, t: int) -> int:
    """Sampling state of the t-th pivot selection of one solve (pre-order of the
    recursion): output #t of splitmix64 started at the solver's seed."""
    return int(splitmix64(seed, t))


def pivot(w, ids, state: int, sample: int) -> np.uint64:
    """PivotSelection (Alg. 2; Section 5): the median of a random sample of edge
    keys.  Sample k (0 <= k < sample) is the edge at position
    floor(splitmix64(state, k) * m / 2^64) of the list (drawn with
    replacement); the pivot is the sorted sample's element of rank sample // 2.
    The paper splits on the weight; the key (w,id) is used here so that the
    split stays balanced when weights repeat."""
    w, ids = np.asarray(w, dtype=np.uint32), np.asarray(ids, dtype=np.uint32)
    m = int(w.shape[0])
    if m == 0:
        return INF
    idx = mulhi_bounded(splitmix64(state, np.arange(sample, dtype=np.uint64)), m).astype(np.int64)
    sk = np.sort(keys(w[idx], ids[idx]))
    return sk[sample // 2]


def partition_light(u, v, w, ids, pv):
    """Light part E<= of Alg. 2 (Section 5): edges with key <= pivot, minus
    self-loops, in their original order."""
    u, v, w, ids = as_edges(u, v, w, ids)
    keep = (keys(w, ids) <= np.uint64(pv)) & (u != v)
    return u[keep], v[keep], w[keep], ids[keep]


def filter_heavy(u, v, w, ids, pv, P):
    """Filter (Alg. 2; Section 5): the heavy edges (key > pivot) are relabelled
    with the component representatives held in P (after pointer doubling P to
    its roots); edges whose endpoints share a representative lie inside one
    component of the light MSF and are dropped.  Order is kept."""
    u, v, w, ids = as_edges(u, v, w, ids)
    heavy = keys(w, ids) > np.uint64(pv)
    return relabel(roots(P), u[heavy], v[heavy], w[heavy], ids[heavy])


def is_sparse(m: int, n: int, max_avg_degree: float = 4.0, min_edges: int = 1 << 16) -> bool:
    """isSparse (Alg. 2; Section 6.3): stop partitioning once the average degree
    2m/n is at most 4, or once the list is small."""
    return m < min_edges or 2.0 * m <= max_avg_degree * n


def filter_boruvka_msf(n: int, src, dst, w, seed: int = 0x2302121990, sample: int = 1 << 16,
                       max_avg_degree: float = 4.0, min_edges: int = 1 << 16, trace: list | None = None):
    """Filter-Borůvka (Alg. 2): Rec-Filter-MST on the whole edge list with a
    representative array P.  A sparse list is solved by Borůvka rounds that
    record each merged vertex's new representative in P; otherwise a pivot
    splits the list, the light part is solved recursively, the heavy part is
    filtered by P and then solved recursively.  ``trace`` (if given) receives
    (depth, m, pivot) for every pivot selection.
    Returns (ascending MSF ids, uint64 total)."""
    u, v, ww, ids = as_edges(src, dst, w)
    w_in = ww
    P = np.arange(n, dtype=np.uint32)
    chosen_all: list[np.ndarray] = []
    counter = [0]

    def base(u, v, ww, ids):
        u, v, ww, ids = relabel(np.arange(n, dtype=np.uint32), u, v, ww, ids)
        while u.size:
            r, chosen, (u, v, ww, ids) = boruvka_round(n, u, v, ww, ids, do_dedupe=True)
            chosen_all.append(chosen)
            moved = r != np.arange(n, dtype=np.uint32)
            P[moved] = r[moved]

    def rec(u, v, ww, ids, depth):
        if is_sparse(int(u.size), n, max_avg_degree, min_edges):
            base(u, v, ww, ids)
            return
        pv = pivot(ww, ids, pivot_state(seed, counter[0]), sample)
        counter[0] += 1
        if trace is not None:
            trace.append((depth, int(u.size), int(pv)))
        rec(*partition_light(u, v, ww, ids, pv), depth + 1)
        rec(*dedupe(*filter_heavy(u, v, ww, ids, pv, P)), depth + 1)

    rec(u, v, ww, ids, 0)
    out = np.sort(np.concatenate(chosen_all)) if chosen_all else np.zeros(0, dtype=np.uint32)
    return out.astype(np.uint32), int(w_in[out].astype(np.uint64).sum())


# ------------------------------------------------- local (tile) contraction

def local_contract(n: int, src, dst, w, tile: int):
    """Local preprocessing (Section 4.1) with vertex-range tiles standing in for
    PEs: vertex x belongs to tile x // tile; an edge is local when both ends are
    in one tile, a cut edge otherwise.  Borůvka rounds run on local edges only,
    and a component is hooked along its lightest local edge only if no cut
    edge incident to it is lighter (then that local edge is the component's
    overall minimum, hence an MSF edge).  Rounds repeat until no component
    hooks.  Returns (label per vertex, ascending contracted edge ids)."""
    u, v, ww, ids = as_edges(src, dst, w)
    tile_of = np.arange(n, dtype=np.int64) // int(tile)
    local = (tile_of[u] == tile_of[v]) & (u != v)
    cut = tile_of[u] != tile_of[v]
    k = keys(ww, ids)
    cutmin = np.full(n, INF, dtype=np.uint64)
    np.minimum.at(cutmin, u[cut], k[cut])
    np.minimum.at(cutmin, v[cut], k[cut])
    label = np.arange(n, dtype=np.uint32)
    lu, lv, lw, lid = u[local], v[local], ww[local], ids[local]
    contracted: list[np.ndarray] = []
    for _ in range(n + 2):  # every round with a hook removes at least one component
        comp_cut = np.full(n, INF, dtype=np.uint64)
        np.minimum.at(comp_cut, label, cutmin)
        best = min_edges(n, lu, lv, lw, lid)
        best = np.where(best < comp_cut, best, INF)
        if not np.any(best != INF):
            break
        parent, chosen = hook(n, lu, lv, lw, lid, best)
        contracted.append(chosen)
        r = roots(parent)
        label = r[label]
        lu, lv, lw, lid = relabel(r, lu, lv, lw, lid)
    else:
        raise RuntimeError("local contraction did not reach a fixed point")
    out = np.sort(np.concatenate(contracted)) if contracted else np.zeros(0, dtype=np.uint32)
    return label, out.astype(np.uint32)
