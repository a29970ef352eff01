"""Pins for the CPU oracle: each check ties the oracle to something other than
itself (brute force, an independent algorithm, closed forms, the MST cut and
cycle properties, published generator vectors, hand-derived fixtures)."""
import math

import numpy as np
import pytest

import oracle
from oracle import steps as S
from paper_2302_12199_gb300 import workloads as W
from tests.golden import fixtures


def rand_multigraph(rng, n, m, wmax):
    src = rng.integers(0, n, m, dtype=np.uint32)
    dst = rng.integers(0, n, m, dtype=np.uint32)
    w = rng.integers(1, wmax + 1, m, dtype=np.uint32)
    return src, dst, w


# ------------------------------------------------------------- fixtures

@pytest.mark.parametrize("path", fixtures.all_fixtures())
def test_hand_derived_fixtures(path):
    n, src, dst, w, msf, total = fixtures.load(path)
    for fn in (oracle.kruskal, oracle.prim):
        ids, tot = fn(n, src, dst, w)
        assert np.array_equal(ids, msf) and tot == total, fn.__name__
    ids, tot, _ = S.boruvka_msf(n, src, dst, w)
    assert np.array_equal(ids, msf) and tot == total
    assert oracle.check_msf(n, src, dst, w, msf) == 0


# --------------------------------------------------- published RNG vectors

def test_splitmix64_published_vector():
    # splitmix64 seeded with 1234567: the first five outputs of the published
    # reference sequence (Steele, Lea, Flood 2014 reference implementation).
    expect = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
              16408922859458223821]
    got = [int(x) for x in S.splitmix64(1234567, np.arange(5, dtype=np.uint64))]
    assert got == expect
    assert [W.splitmix64_at(1234567, i) for i in range(5)] == expect


def test_mulhi_bounded_matches_exact_integer_arithmetic():
    rng = np.random.default_rng(1)
    r = rng.integers(0, 2**63, 1000, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    for m in (1, 7, 1000, 2**31 + 11, 2**32 - 1):
        got = S.mulhi_bounded(r, m)
        want = [(int(x) * m) >> 64 for x in r]
        assert [int(x) for x in got] == want


# ----------------------------------------------------------- brute force

def test_kruskal_equals_brute_force_on_tiny_multigraphs():
    rng = np.random.default_rng(2302)
    for trial in range(300):
        n = int(rng.integers(1, 9))
        m = int(rng.integers(0, 15))
        src, dst, w = rand_multigraph(rng, n, m, wmax=int(rng.choice([1, 2, 3, 10])))
        kid, ktot = oracle.kruskal(n, src, dst, w)
        bid, btot, any_min = oracle.brute(n, src, dst, w)
        assert np.array_equal(kid, bid), (trial, n, src, dst, w)
        assert ktot == btot == any_min


# ---------------------------------------------- independent cross-checks

@pytest.mark.parametrize("family", ["gnm", "rmat", "rgg2", "rgg3", "sparse_forest", "grid2d", "rhg"])
def test_kruskal_equals_prim(family):
    if family == "grid2d":
        g = W.grid2d(60, 70, 16)
    elif family == "rhg":
        g = W.rhg(4000, 10.0, 17)
    elif family == "gnm":
        g = W.gnm(3000, 30000, 11)
    elif family == "rmat":
        g = W.rmat(12, 40000, 12)
    elif family == "rgg2":
        g = W.rgg(2, 4000, 8.0, 13)
    elif family == "rgg3":
        g = W.rgg(3, 4000, 8.0, 14)
    else:
        g = W.gnm(5000, 1500, 15)  # many components and isolated vertices
    kid, ktot = oracle.kruskal(g.n, g.src, g.dst, g.w)
    pid, ptot = oracle.prim(g.n, g.src, g.dst, g.w)
    assert np.array_equal(kid, pid) and ktot == ptot


@pytest.mark.parametrize("threads", [1, 3, 8, 64])
def test_parallel_sort_kruskal_equals_kruskal(threads):
    """The CPU-baseline Kruskal whose sort runs on several threads returns the
    same forest as the plain one: heavy weight ties (w in [1, 255], where the
    id order inside a weight must survive the threaded scatter), 32-bit weights
    (all four radix passes), self-loops, parallel edges, more threads than
    edges, and the empty graph."""
    cases = [W.rmat(14, 200000, 31), W.gnm(20000, 100000, 32, wmin=1, wmax=0xFFFFFFFF), W.rgg(2, 5000, 8.0, 33),
             W.Graph(5, np.array([0, 1, 1, 2, 4], np.uint32), np.array([1, 1, 0, 2, 3], np.uint32),
                     np.array([7, 1, 7, 3, 2], np.uint32)),
             W.Graph(3, np.empty(0, np.uint32), np.empty(0, np.uint32), np.empty(0, np.uint32))]
    for g in cases:
        kid, ktot = oracle.kruskal(g.n, g.src, g.dst, g.w)
        pid, ptot = oracle.kruskal_par(g.n, g.src, g.dst, g.w, threads)
        assert np.array_equal(kid, pid) and ktot == ptot


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_kruskal_satisfies_cut_and_cycle_properties(seed):
    rng = np.random.default_rng(seed)
    n = 300
    src, dst, w = rand_multigraph(rng, n, 1200, wmax=20)
    ids, _ = oracle.kruskal(n, src, dst, w)
    assert oracle.check_msf(n, src, dst, w, ids) == 0


def test_checker_rejects_planted_mistakes():
    rng = np.random.default_rng(7)
    n = 200
    src, dst, w = rand_multigraph(rng, n, 900, wmax=8)
    ids, _ = oracle.kruskal(n, src, dst, w)
    assert oracle.check_msf(n, src, dst, w, ids) == 0
    # dropped edge: no longer spanning
    assert oracle.check_msf(n, src, dst, w, ids[1:]) & 4
    # extra non-forest, non-self-loop edge: a cycle
    extra = next(e for e in range(len(src)) if e not in set(ids.tolist()) and src[e] != dst[e])
    assert oracle.check_msf(n, src, dst, w, np.sort(np.append(ids, extra))) & 2
    # swap a forest edge for the next-heavier edge that reconnects its cut
    in_f = set(ids.tolist())
    swapped = False
    for e in ids:
        rest = [x for x in ids if x != e]
        # label the side of src[e] in F minus e
        adj = {}
        for x in rest:
            adj.setdefault(int(src[x]), []).append(int(dst[x]))
            adj.setdefault(int(dst[x]), []).append(int(src[x]))
        side, stack = {int(src[e])}, [int(src[e])]
        while stack:
            a = stack.pop()
            for b in adj.get(a, []):
                if b not in side:
                    side.add(b)
                    stack.append(b)
        cross = [f for f in range(len(src)) if f != e and f not in in_f and (int(src[f]) in side) != (int(dst[f]) in side)]
        if cross:
            f = cross[0]
            bad = np.sort(np.array(rest + [f], dtype=np.uint32))
            mask = oracle.check_msf(n, src, dst, w, bad)
            assert mask & (8 | 16), mask
            swapped = True
            break
    assert swapped


def test_tie_order_is_by_id():
    # two parallel edges with equal weight: the smaller id must win; the checker
    # must reject the other one.
    src = np.array([0, 0], np.uint32)
    dst = np.array([1, 1], np.uint32)
    w = np.array([4, 4], np.uint32)
    assert oracle.kruskal(2, src, dst, w)[0].tolist() == [0]
    assert oracle.check_msf(2, src, dst, w, np.array([1], np.uint32)) != 0


# ------------------------------------------------------------ closed forms

def test_forest_input_returns_every_edge():
    rng = np.random.default_rng(3)
    n = 500
    perm = rng.permutation(n).astype(np.uint32)
    parent = np.array([rng.integers(0, i) for i in range(1, n)], dtype=np.uint32)  # a random tree
    src, dst = perm[1:], perm[parent]
    keep = rng.random(n - 1) < 0.7  # a forest
    src, dst = src[keep], dst[keep]
    w = rng.integers(1, 1000, src.size, dtype=np.uint32)
    ids, tot = oracle.kruskal(n, src, dst, w)
    assert ids.tolist() == list(range(src.size)) and tot == int(w.astype(np.uint64).sum())


def test_path_with_increasing_weights_and_cycle():
    n = 1000
    src = np.arange(n - 1, dtype=np.uint32)
    dst = src + 1
    w = np.arange(1, n, dtype=np.uint32)
    ids, tot = oracle.kruskal(n, src, dst, w)
    assert ids.size == n - 1 and tot == (n - 1) * n // 2
    # close the cycle with the heaviest edge: it is the one left out
    src2, dst2 = np.append(src, n - 1), np.append(dst, 0)
    for wc, out in ((n, n - 1), (0, n - 2)):
        w2 = np.append(w, wc).astype(np.uint32)
        ids2, _ = oracle.kruskal(n, src2, dst2, w2)
        assert out not in set(ids2.tolist()) and ids2.size == n - 1


def test_star_keeps_every_lightest_spoke():
    n = 300
    leaves = np.arange(1, n, dtype=np.uint32)
    src = np.concatenate([np.zeros(n - 1, np.uint32), leaves])  # two spokes per leaf
    dst = np.concatenate([leaves, np.zeros(n - 1, np.uint32)])
    w = np.concatenate([np.full(n - 1, 7, np.uint32), (leaves % 11 + 1).astype(np.uint32)])
    ids, tot = oracle.kruskal(n, src, dst, w)
    # leaf l keeps spoke (n-1)+(l-1) when (l % 11 + 1) < 7, else the first (equal weight 7 -> smaller id)
    expect = sorted((n - 2 + int(l)) if (l % 11 + 1) < 7 else int(l) - 1 for l in leaves)
    assert ids.tolist() == expect
    assert tot == int(sum(min(7, int(l) % 11 + 1) for l in leaves))


def test_complete_graph_with_distance_weights():
    # K_n with w(i,j) = |i-j|: the only weight-1 edges form the path 0-1-...-(n-1),
    # which is therefore the MST, of total n-1.
    n = 60
    i, j = np.triu_indices(n, 1)
    src, dst = i.astype(np.uint32), j.astype(np.uint32)
    w = (j - i).astype(np.uint32)
    ids, tot = oracle.kruskal(n, src, dst, w)
    assert tot == n - 1 and np.all(w[ids] == 1)


def test_equal_weights_give_the_id_order_forest():
    # With one weight the order is the id order: e is a forest edge iff its
    # endpoints are not joined by edges of smaller id (checked here by BFS).
    rng = np.random.default_rng(9)
    n = 80
    src, dst, _ = rand_multigraph(rng, n, 300, 1)
    w = np.full(src.size, 5, np.uint32)
    ids, _ = oracle.kruskal(n, src, dst, w)
    expect = []
    for e in range(src.size):
        if src[e] == dst[e]:
            continue
        adj = {}
        for f in range(e):
            adj.setdefault(int(src[f]), []).append(int(dst[f]))
            adj.setdefault(int(dst[f]), []).append(int(src[f]))
        seen, stack = {int(src[e])}, [int(src[e])]
        while stack:
            a = stack.pop()
            for b in adj.get(a, []):
                if b not in seen:
                    seen.add(b)
                    stack.append(b)
        if int(dst[e]) not in seen:
            expect.append(e)
    assert ids.tolist() == expect


def test_disconnected_union_is_union_of_parts():
    parts = [W.gnm(300, 2000, s) for s in range(4)] + [W.rgg(2, 500, 8.0, 9)]
    off_v, off_e = 0, 0
    src, dst, w, expect, total = [], [], [], [], 0
    for g in parts:
        ids, tot = oracle.kruskal(g.n, g.src, g.dst, g.w)
        src.append(g.src + off_v)
        dst.append(g.dst + off_v)
        w.append(g.w)
        expect.append(ids.astype(np.int64) + off_e)
        total += tot
        off_v += g.n
        off_e += g.m
    ids, tot = oracle.kruskal(off_v, np.concatenate(src), np.concatenate(dst), np.concatenate(w))
    assert np.array_equal(ids, np.concatenate(expect)) and tot == total


def test_degenerate_inputs():
    e = np.zeros(0, np.uint32)
    assert oracle.kruskal(0, e, e, e)[0].size == 0
    assert oracle.kruskal(10, e, e, e) [1] == 0
    loops = np.array([3, 3, 4], np.uint32)
    assert oracle.kruskal(5, loops, loops, np.array([1, 2, 3], np.uint32))[0].size == 0
    with pytest.raises(oracle.OracleError):
        oracle.kruskal(3, np.array([0], np.uint32), np.array([3], np.uint32), np.array([1], np.uint32))


# --------------------------------------------------------------- steps

def test_min_edges_pick_forest_edges_and_rounds_halve():
    rng = np.random.default_rng(4)
    n = 400
    src, dst, w = rand_multigraph(rng, n, 2000, wmax=5)
    ids, _ = oracle.kruskal(n, src, dst, w)
    best = S.min_edges(n, src, dst, w, np.arange(src.size, dtype=np.uint32))
    chosen = (best[best != S.INF] & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    assert np.isin(chosen, ids).all()  # min-cut property (Section 2.3)
    # each non-isolated vertex's choice is the lightest incident edge: no
    # incident non-self-loop edge has a smaller key
    k = S.keys(w, np.arange(src.size))
    for e in range(src.size):
        if src[e] != dst[e]:
            assert best[src[e]] <= k[e] and best[dst[e]] <= k[e]
    parent, chosen2 = S.hook(n, src, dst, w, np.arange(src.size, dtype=np.uint32), best)
    r = S.roots(parent)
    nonisolated = np.unique(np.concatenate([src[src != dst], dst[src != dst]]))
    assert np.unique(r[nonisolated]).size <= nonisolated.size // 2  # |V'| <= |V|/2
    assert np.isin(chosen2, ids).all()
    # hook roots are exactly the vertices that point to themselves
    assert np.all(parent[r] == r)


def test_hook_two_cycles_and_chains():
    """Hooking (Section 2.3): both ends of a mutually chosen edge form a 2-cycle
    whose smaller vertex stays root; every other active vertex points to the
    far end of its own choice, and each chosen edge is reported once."""
    def run(n, edges):
        u = np.array([e[0] for e in edges], np.uint32)
        v = np.array([e[1] for e in edges], np.uint32)
        w = np.array([e[2] for e in edges], np.uint32)
        ids = np.arange(len(edges), dtype=np.uint32)
        best = S.min_edges(n, u, v, w, ids)
        return S.hook(n, u, v, w, ids, best)

    parent, chosen = run(2, [(1, 0, 7)])  # one edge: a 2-cycle, vertex 0 is the root
    assert parent.tolist() == [0, 0] and chosen.tolist() == [0]
    # path 0-1 (w 1), 1-2 (w 2): 0 and 1 both choose edge 0 (2-cycle, root 0); 2 chooses edge 1
    parent, chosen = run(3, [(0, 1, 1), (1, 2, 2)])
    assert parent.tolist() == [0, 0, 1] and chosen.tolist() == [0, 1]
    # 2-cycle between 1 and 2 (edge 1, the lightest); 0 hangs off 1; 3 isolated
    parent, chosen = run(4, [(0, 1, 5), (2, 1, 3), (0, 2, 9)])
    assert parent.tolist() == [1, 1, 1, 3] and chosen.tolist() == [0, 1]
    # random multigraphs: one chosen edge per non-root active vertex, roots only in 2-cycles
    rng = np.random.default_rng(5)
    for _ in range(20):
        n = int(rng.integers(2, 60))
        src, dst, w = rand_multigraph(rng, n, int(rng.integers(1, 200)), wmax=4)
        ids = np.arange(src.size, dtype=np.uint32)
        best = S.min_edges(n, src, dst, w, ids)
        parent, chosen = S.hook(n, src, dst, w, ids, best)
        active = np.nonzero(best != S.INF)[0]
        nonroot = active[parent[active] != active]
        assert chosen.size == nonroot.size
        for c in active[parent[active] == active]:  # an active root has a partner choosing the same edge
            partners = np.nonzero((best == best[c]) & (np.arange(n) != c))[0]
            assert partners.size == 1 and parent[partners[0]] == c and c < partners[0]


@pytest.mark.parametrize("dd", [True, False])
def test_boruvka_composition_equals_kruskal(dd):
    for g in (W.gnm(2000, 16000, 21), W.rmat(11, 20000, 22), W.rgg(2, 3000, 8.0, 23), W.gnm(4000, 1000, 24)):
        kid, ktot = oracle.kruskal(g.n, g.src, g.dst, g.w)
        bid, btot, rounds = S.boruvka_msf(g.n, g.src, g.dst, g.w, do_dedupe=dd)
        assert np.array_equal(kid, bid) and ktot == btot
        assert rounds <= math.ceil(math.log2(g.n))  # Section 2.3: at most log|V| rounds


def test_dedupe_keeps_lightest_per_pair_in_order():
    rng = np.random.default_rng(5)
    u, v, w = rand_multigraph(rng, 30, 2000, wmax=4)
    keep = u != v
    u, v, w = u[keep], v[keep], w[keep]
    ids = np.arange(u.size, dtype=np.uint32) * 3 + 1
    du, dv, dw, did = S.dedupe(u, v, w, ids)
    pairs = list(zip(np.minimum(du, dv).tolist(), np.maximum(du, dv).tolist()))
    assert len(set(pairs)) == len(pairs)
    assert np.all(np.diff(did.astype(np.int64)) > 0)  # order kept
    kmin = {}
    for a, b, kk in zip(np.minimum(u, v), np.maximum(u, v), S.keys(w, ids)):
        kmin[(int(a), int(b))] = min(kmin.get((int(a), int(b)), 2**64), int(kk))
    assert sorted(int(x) for x in S.keys(dw, did)) == sorted(kmin.values())


def test_relabel_drops_self_loops_and_keeps_order():
    rng = np.random.default_rng(6)
    u, v, w = rand_multigraph(rng, 50, 500, wmax=9)
    label = rng.integers(0, 10, 50, dtype=np.uint32)
    ids = np.arange(500, dtype=np.uint32)
    nu, nv, nw, nid = S.relabel(label, u, v, w, ids)
    assert np.all(nu != nv) and np.all(np.diff(nid.astype(np.int64)) > 0)
    assert np.array_equal(nu, label[u[nid]]) and np.array_equal(nw, w[nid])
    assert nid.size == int(np.sum(label[u] != label[v]))


def test_pivot_is_sample_median():
    g = W.gnm(1 << 12, 1 << 16, 31)
    ids = np.arange(g.m, dtype=np.uint32)
    for sample in (1, 2, 1001, 1 << 12):
        st = S.pivot_state(0x1234, 3)
        pv = S.pivot(g.w, ids, st, sample)
        idx = [(int(x) * g.m) >> 64 for x in S.splitmix64(st, np.arange(sample, dtype=np.uint64))]
        sk = S.keys(g.w[idx], ids[idx])
        assert pv == np.partition(sk, sample // 2)[sample // 2]
    # balance: a 2^16 sample splits a list with heavily tied weights near 1/2
    pv = S.pivot(g.w, ids, S.pivot_state(7, 0), 1 << 16)
    frac = float(np.mean(S.keys(g.w, ids) <= pv))
    assert abs(frac - 0.5) < 0.02


def test_partition_and_filter_cover_the_list():
    rng = np.random.default_rng(8)
    n = 500
    u, v, w = rand_multigraph(rng, n, 6000, wmax=255)
    ids = np.arange(u.size, dtype=np.uint32)
    pv = S.pivot(w, ids, 99, 4096)
    lu, lv, lw, lid = S.partition_light(u, v, w, ids, pv)
    assert np.all(S.keys(lw, lid) <= pv) and np.all(lu != lv)
    P = np.arange(n, dtype=np.uint32)  # no components yet: filter = heavy minus self-loops
    hu, hv, hw, hid = S.filter_heavy(u, v, w, ids, pv, P)
    assert np.all(S.keys(hw, hid) > pv)
    assert lid.size + hid.size == int(np.sum(u != v))
    assert np.intersect1d(lid, hid).size == 0


@pytest.mark.parametrize("seed", [11, 12, 13, 14])
def test_filter_keeps_exactly_the_heavy_edges_between_light_components(seed):
    """Filter (Alg. 2): with P holding the components of the light part, the
    survivors are exactly the heavy edges whose ends lie in different
    components.  The components come from Kruskal's forest of the light edges
    and a plain union-find here, not from the step oracles; the Borůvka
    rounds' P must give the same partition."""
    rng = np.random.default_rng(seed)
    n = 800  # sparse enough that the light part falls into ~150 components
    u, v, w = rand_multigraph(rng, n, 1500, wmax=20)  # many equal weights
    ids = np.arange(u.size, dtype=np.uint32)
    pv = S.pivot(w, ids, seed, 1024)
    light = S.keys(w, ids) <= np.uint64(pv)
    lid = ids[light]
    forest = oracle.kruskal(n, u[light], v[light], w[light])[0]  # positions in the light sublist
    comp = list(range(n))

    def find(x):
        while comp[x] != x:
            comp[x] = comp[comp[x]]
            x = comp[x]
        return x

    for j in forest:
        e = int(lid[j])
        a, b = find(int(u[e])), find(int(v[e]))
        if a != b:
            comp[a] = b
    rep_of = np.array([find(x) for x in range(n)], dtype=np.uint32)
    expect = sorted(int(e) for e in ids[~light] if rep_of[u[e]] != rep_of[v[e]])
    assert 0 < len(expect) < int(np.sum(~light))  # some heavy edges survive, some are filtered
    hu, hv, hw, hid = S.filter_heavy(u, v, w, ids, pv, rep_of)
    assert sorted(hid.tolist()) == expect
    assert np.all(hu == rep_of[u[hid]]) and np.all(hv == rep_of[v[hid]])
    # the representative array that the Borůvka rounds build gives the same components
    P = np.arange(n, dtype=np.uint32)
    uu, vv, ww_, ii = S.partition_light(u, v, w, ids, pv)
    while uu.size:
        r, _, (uu, vv, ww_, ii) = S.boruvka_round(n, uu, vv, ww_, ii)
        moved = r != np.arange(n, dtype=np.uint32)
        P[moved] = r[moved]
    roots = S.roots(P)
    for x in range(n):
        for y in (0, 1, 2, x // 2, (x * 7) % n):
            assert (roots[x] == roots[y]) == (rep_of[x] == rep_of[y])


def test_filter_survivors_are_linear_in_n():
    # Theorem 1 / KKT sampling: heavy edges surviving the filter by the light
    # MSF number about n/p - n for a split fraction p = 1/2, i.e. O(n).
    g = W.gnm(1 << 13, 1 << 17, 41)
    ids = np.arange(g.m, dtype=np.uint32)
    pv = S.pivot(g.w, ids, S.pivot_state(41, 0), 1 << 16)
    lu, lv, lw, lid = S.partition_light(g.src, g.dst, g.w, ids, pv)
    # representatives of the light forest
    P = np.arange(g.n, dtype=np.uint32)
    uu, vv, ww_, ii = lu, lv, lw, lid
    while uu.size:
        r, _, (uu, vv, ww_, ii) = S.boruvka_round(g.n, uu, vv, ww_, ii)
        moved = r != np.arange(g.n, dtype=np.uint32)
        P[moved] = r[moved]
    surv = S.filter_heavy(g.src, g.dst, g.w, ids, pv, P)[0].size
    assert surv < 3 * g.n, surv


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_filter_boruvka_equals_kruskal(seed):
    for g in (W.gnm(3000, 48000, seed), W.rmat(12, 60000, seed), W.rgg(2, 4000, 8.0, seed)):
        kid, ktot = oracle.kruskal(g.n, g.src, g.dst, g.w)
        trace = []
        fid, ftot = S.filter_boruvka_msf(g.n, g.src, g.dst, g.w, seed=seed, sample=1024, min_edges=512, trace=trace)
        assert np.array_equal(kid, fid) and ktot == ftot
        assert len(trace) >= 1  # the recursion really partitioned


def test_local_contraction_is_safe_and_reaches_fixed_point():
    for g, tile in ((W.rgg(2, 4096, 8.0, 51), 256), (W.rgg(3, 4096, 8.0, 52), 512), (W.gnm(2000, 9000, 53), 100)):
        kid, ktot = oracle.kruskal(g.n, g.src, g.dst, g.w)
        label, con = S.local_contract(g.n, g.src, g.dst, g.w, tile)
        assert np.isin(con, kid).all()
        # labels stay inside their tile and are roots of themselves
        assert np.all(label // tile == np.arange(g.n) // tile) and np.all(label[label] == label)
        # fixed point: no component's overall lightest edge is a local edge
        u, v, ww, ids = S.relabel(label, g.src, g.dst, g.w, np.arange(g.m, dtype=np.uint32))
        best = S.min_edges(g.n, u, v, ww, ids)
        c = np.nonzero(best != S.INF)[0]
        e = (best[c] & np.uint64(0xFFFFFFFF)).astype(np.int64)
        local = (g.src[e] // tile) == (g.dst[e] // tile)
        assert not np.any(local)
        # contraction followed by plain Borůvka reproduces Kruskal
        rest = []
        while u.size:
            _, ch, (u, v, ww, ids) = S.boruvka_round(g.n, u, v, ww, ids)
            rest.append(ch)
        allids = np.sort(np.concatenate([con] + rest))
        assert np.array_equal(allids, kid)


def test_local_contraction_with_one_tile_is_the_whole_forest():
    g = W.gnm(500, 3000, 61)
    kid, _ = oracle.kruskal(g.n, g.src, g.dst, g.w)
    label, con = S.local_contract(g.n, g.src, g.dst, g.w, g.n)
    assert np.array_equal(con, kid)
