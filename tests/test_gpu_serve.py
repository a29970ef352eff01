"""GPU: batched and served solves give every graph exactly its own MSF.

The batched call solves the disjoint union of many graphs; the server batches
requests of different sizes as they arrive and keeps several batches in
flight.  Each response must equal the oracle's forest of that graph (ids and
uint64 weight), and the same whether the graph is solved alone or in a mix."""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_12199_gb300 import workloads as W
from paper_2302_12199_gb300.mst import Solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "a CUDA GPU is required for the gpu tests"
    return torch.device("cuda", 0)


def to_dev(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).to(dev)


def oracle_answers(b):
    out = []
    for g in range(b.num_graphs):
        gr = b.graph(g)
        out.append(oracle.kruskal(gr.n, gr.src, gr.dst, gr.w))
    return out


@pytest.mark.parametrize("cfg", [dict(variant="boruvka", dedupe="none"), dict(variant="filter"),
                                 dict(variant="boruvka", dedupe="hash", tile_contract=1, tile_vertices=256)])
def test_batched_mix_matches_oracle(dev, cfg):
    b = W.mix(60, 91, log_lo=6, log_hi=13)
    exp = oracle_answers(b)
    s = Solver(0, **cfg)
    try:
        ids, moff, tot = s.solve_batched(b.n, b.edge_off, to_dev(b.src, dev), to_dev(b.dst, dev), to_dev(b.w, dev))
        ids = ids.cpu().numpy().view(np.uint32)
        moff = moff.cpu().numpy().astype(np.int64)
        tot = tot.cpu().numpy().view(np.uint64)
        for g, (kid, ktot) in enumerate(exp):
            assert np.array_equal(ids[moff[g]:moff[g + 1]], kid), g
            assert int(tot[g]) == ktot, g
    finally:
        s.close()


def test_batched_device_tables_and_errors(dev):
    """The size tables of mst_solve_batched live in device memory: given as
    device tensors they give each graph its Kruskal forest; an offset table that
    does not start at 0, or that decreases, is MST_ERR_INVALID_ARG, reported by
    the call and by mst_get_error on the stream; the handle then solves again."""
    from paper_2302_12199_gb300.mst import MstError
    b = W.mix(30, 94, log_lo=5, log_hi=11)
    exp = oracle_answers(b)
    src, dst, w = to_dev(b.src, dev), to_dev(b.dst, dev), to_dev(b.w, dev)
    d_n = to_dev(b.n, dev)
    d_off = torch.from_numpy(np.asarray(b.edge_off, dtype=np.uint64).view(np.int64)).to(dev)
    s = Solver(0)
    try:
        stream = torch.cuda.Stream(dev)
        ids, moff, tot = s.solve_batched(d_n, d_off, src, dst, w, stream=stream)
        assert s.get_error(stream) == 0
        ids = ids.cpu().numpy().view(np.uint32)
        moff = moff.cpu().numpy().astype(np.int64)
        tot = tot.cpu().numpy().view(np.uint64)
        for g, (kid, ktot) in enumerate(exp):
            assert np.array_equal(ids[moff[g]:moff[g + 1]], kid) and int(tot[g]) == ktot, g
        for bad in ("first", "decreasing"):
            off_bad = np.asarray(b.edge_off, dtype=np.uint64).copy()
            if bad == "first":
                off_bad[0] = 1
            else:  # graph k's end lies before its start
                k = len(off_bad) // 2
                off_bad[k] = off_bad[k + 1] + 1
            with pytest.raises(MstError) as e:
                s.solve_batched(b.n, off_bad, src, dst, w)
            assert e.value.status == 1, bad
            assert s.get_error() == 1
        ids2, moff2, tot2 = s.solve_batched(b.n, b.edge_off, src, dst, w)
        assert s.get_error() == 0
        assert torch.equal(moff2.cpu(), torch.from_numpy(moff)) and np.array_equal(
            tot2.cpu().numpy().view(np.uint64), tot)
    finally:
        s.close()


def test_full_size_batch_matches_oracle(dev):
    """The batched benchmark's batch at its full size (4096 graphs, n
    log-uniform in [2^8, 2^16], about 335 M edges), under the configurations
    its autotuner chooses between for the solve: every graph's forest and
    total equal its own Kruskal forest."""
    b = W.mix(4096, W.DEFAULT_SEED, log_hi=16)
    exp = oracle_answers(b)
    src, dst, w = to_dev(b.src, dev), to_dev(b.dst, dev), to_dev(b.w, dev)
    for cfg in (dict(variant="filter"), dict(variant="boruvka")):
        s = Solver(0, **cfg)
        try:
            ids, moff, tot = s.solve_batched(b.n, b.edge_off, src, dst, w)
            ids = ids.cpu().numpy().view(np.uint32)
            moff = moff.cpu().numpy().astype(np.int64)
            tot = tot.cpu().numpy().view(np.uint64)
            bad = [g for g, (kid, ktot) in enumerate(exp)
                   if not (np.array_equal(ids[moff[g]:moff[g + 1]], kid) and int(tot[g]) == ktot)]
            assert not bad, (cfg, bad[:5])
        finally:
            s.close()
    del src, dst, w
    torch.cuda.empty_cache()


def test_full_size_served_pool_matches_oracle(dev):
    """The served benchmark's request pool at its full size (256 graphs, n
    log-uniform in [2^8, 2^20]): each graph solved alone through the server
    equals its Kruskal forest, and a stream of requests drawn from the pool
    (several batches in flight on three slots) returns exactly those answers."""
    from paper_2302_12199_gb300.serve import PoolGraph, Response, Server, poisson_arrivals
    b = W.mix(256, W.DEFAULT_SEED + 5, log_lo=8, log_hi=20)
    exp = oracle_answers(b)
    pool = []
    for g in range(b.num_graphs):
        gr = b.graph(g)
        pool.append(PoolGraph(gr.n, to_dev(gr.src, dev), to_dev(gr.dst, dev), to_dev(gr.w, dev)))
    expected = {g: Response(kid, ktot) for g, (kid, ktot) in enumerate(exp)}
    server = Server(0, slots=3, budget_bytes=6 << 30, stall_seconds=60.0)
    try:
        for g in range(len(pool)):
            r = server.solve_alone(pool[g])
            assert np.array_equal(r.ids, expected[g].ids) and r.total == expected[g].total, g
        arr = poisson_arrivals(4096.0, 0.25, seed=11)
        picks = np.random.default_rng(12).integers(0, len(pool), arr.size)
        st = server.run(pool, picks, arr, expected=expected, rate=4096.0, seconds=0.25)
        assert st.requests == arr.size and st.mismatches == 0 and st.batches >= 2
    finally:
        server.close()
        del pool
        torch.cuda.empty_cache()


def test_batched_with_empty_and_tiny_graphs(dev):
    n = np.array([1, 5, 3, 1, 4], dtype=np.uint32)
    src = np.array([0, 1, 2, 3, 0, 1, 2, 0, 0, 1], dtype=np.uint32)
    dst = np.array([1, 2, 3, 4, 4, 2, 0, 0, 1, 0], dtype=np.uint32)
    w = np.array([5, 1, 2, 3, 4, 7, 7, 9, 2, 2], dtype=np.uint32)
    off = np.array([0, 0, 5, 7, 8, 10], dtype=np.uint64)
    s = Solver(0)
    try:
        ids, moff, tot = s.solve_batched(n, off, to_dev(src, dev), to_dev(dst, dev), to_dev(w, dev))
        ids = ids.cpu().numpy().view(np.uint32)
        moff = moff.cpu().numpy().astype(np.int64)
        tot = tot.cpu().numpy().view(np.uint64)
        for g in range(5):
            lo, hi = int(off[g]), int(off[g + 1])
            kid, ktot = oracle.kruskal(int(n[g]), src[lo:hi], dst[lo:hi], w[lo:hi])
            assert np.array_equal(ids[moff[g]:moff[g + 1]], kid) and int(tot[g]) == ktot, g
    finally:
        s.close()


def test_served_responses_alone_and_in_the_mix(dev):
    from paper_2302_12199_gb300.serve import PoolGraph, Response, Server, poisson_arrivals
    b = W.mix(24, 92, log_lo=6, log_hi=12)
    exp = oracle_answers(b)
    pool = []
    for g in range(b.num_graphs):
        gr = b.graph(g)
        pool.append(PoolGraph(gr.n, to_dev(gr.src, dev), to_dev(gr.dst, dev), to_dev(gr.w, dev)))
    expected = {g: Response(kid, ktot) for g, (kid, ktot) in enumerate(exp)}
    # a small budget forces several batches; two slots keep batches in flight together
    server = Server(0, slots=2, budget_bytes=4 << 20, max_batch=16, stall_seconds=20.0)
    try:
        for g in range(len(pool)):  # alone
            r = server.solve_alone(pool[g])
            assert np.array_equal(r.ids, expected[g].ids) and r.total == expected[g].total, g
        arr = poisson_arrivals(20000.0, 0.02, seed=5)
        picks = np.random.default_rng(6).integers(0, len(pool), arr.size)
        st = server.run(pool, picks, arr, expected=expected, rate=20000.0, seconds=0.02)  # in the mix
        assert st.requests == arr.size and st.mismatches == 0
        assert st.batches >= 2 and sum(st.batch_sizes) == arr.size
        assert max(st.batch_sizes) <= 16
        assert np.all(st.latency > 0)
        # a burst of requests all waiting at once: both slots take a batch, so
        # two batches are on the device together, and every response is still
        # the graph's own forest
        burst = np.zeros(64)
        picks_b = np.random.default_rng(11).integers(0, len(pool), burst.size)
        stb = server.run(pool, picks_b, burst, expected=expected)
        assert stb.requests == burst.size and stb.mismatches == 0
        assert stb.max_in_flight >= 2 and stb.batches >= 2
        # the same server serves a second stream
        arr2 = poisson_arrivals(5000.0, 0.02, seed=7)
        picks2 = np.random.default_rng(8).integers(0, len(pool), arr2.size)
        st2 = server.run(pool, picks2, arr2, expected=expected, rate=5000.0, seconds=0.02)
        assert st2.requests == arr2.size and st2.mismatches == 0
        # one request larger than the whole budget is still admitted, alone
        tiny = Server(0, slots=1, budget_bytes=1, max_batch=8, stall_seconds=20.0)
        try:
            st1 = tiny.run(pool, np.arange(6) % len(pool), np.linspace(0, 1e-3, 6), expected=expected)
            assert st1.mismatches == 0 and st1.batch_sizes == [1] * 6
        finally:
            tiny.close()
    finally:
        server.close()


def test_served_host_payloads(dev):
    """Payloads in page-locked host memory (copied in per batch, empty graphs
    included) give the same responses as the oracle."""
    from paper_2302_12199_gb300.serve import PoolGraph, Response, Server, poisson_arrivals
    b = W.mix(20, 93, log_lo=6, log_hi=12)
    exp = oracle_answers(b)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).pin_memory()
    pool = []
    for g in range(b.num_graphs):
        gr = b.graph(g)
        pool.append(PoolGraph(gr.n, pin(gr.src), pin(gr.dst), pin(gr.w)))
    empty = np.empty(0, np.uint32)
    pool.append(PoolGraph(7, pin(empty), pin(empty), pin(empty)))
    exp.append((empty, 0))
    expected = {g: Response(kid, ktot) for g, (kid, ktot) in enumerate(exp)}
    server = Server(0, slots=2, budget_bytes=4 << 20, max_batch=16, stall_seconds=20.0)
    try:
        arr = poisson_arrivals(20000.0, 0.02, seed=9)
        picks = np.random.default_rng(10).integers(0, len(pool), arr.size)
        st = server.run(pool, picks, arr, expected=expected, rate=20000.0, seconds=0.02)
        assert st.requests == arr.size and st.mismatches == 0 and st.batches >= 2
    finally:
        server.close()


def test_batched_forest_capacity_residues(dev):
    """The forest count and weight follow the id array in one allocation: every
    residue of its capacity modulo 64 ids must keep them inside it."""
    s = Solver(0)
    try:
        for total_n in range(60, 70):
            n = np.array([total_n // 2, total_n - total_n // 2], dtype=np.uint32)
            parts = [W.gnm(int(k), 3 * int(k), 100 + total_n + i) for i, k in enumerate(n)]
            src = np.concatenate([p.src for p in parts])
            dst = np.concatenate([p.dst for p in parts])
            w = np.concatenate([p.w for p in parts])
            off = np.array([0, parts[0].m, parts[0].m + parts[1].m], dtype=np.uint64)
            ids, moff, tot = s.solve_batched(n, off, to_dev(src, dev), to_dev(dst, dev), to_dev(w, dev))
            ids = ids.cpu().numpy().view(np.uint32)
            moff = moff.cpu().numpy().astype(np.int64)
            tot = tot.cpu().numpy().view(np.uint64)
            for g, p in enumerate(parts):
                kid, ktot = oracle.kruskal(p.n, p.src, p.dst, p.w)
                assert np.array_equal(ids[moff[g]:moff[g + 1]], kid) and int(tot[g]) == ktot, (total_n, g)
    finally:
        s.close()


def test_concurrent_handles_grow_their_buffers(dev):
    """Three host threads, each with its own handle and stream, solve batches
    that grow from call to call, so every call regrows the handle's round lists
    and scan status words and captures new round graphs while the other
    threads launch and capture theirs (the server's pattern).  Every forest
    equals Kruskal's."""
    import threading
    sizes = [(1 << 10, 1 << 13), (1 << 12, 1 << 15), (1 << 14, 1 << 17), (1 << 15, 1 << 19), (1 << 16, 1 << 20)]
    cases = []
    for k, (n, m) in enumerate(sizes):
        a, b = W.gnm(n, m, 300 + k), W.rmat(max(10, n.bit_length() - 1), m // 2, 400 + k)
        cases.append((a, b, oracle.kruskal(a.n, a.src, a.dst, a.w), oracle.kruskal(b.n, b.src, b.dst, b.w)))
    errors = []

    # handles are made (and closed) while no other thread is at work: mst_create
    # and mst_destroy wait for the device
    solvers = [Solver(0, variant="filter" if t != 1 else "boruvka", filter_min_edges=1 << 12, pivot_sample=4096)
               for t in range(3)]

    def worker(t):
        torch.cuda.set_device(dev)
        stream = torch.cuda.Stream(device=dev)
        s = solvers[t]
        try:
            for rep in range(2):
                for a, b, ea, eb in cases:
                    with torch.cuda.stream(stream):
                        src = to_dev(np.concatenate([a.src, b.src]), dev)
                        dst = to_dev(np.concatenate([a.dst, b.dst]), dev)
                        w = to_dev(np.concatenate([a.w, b.w]), dev)
                        ids, moff, tot = s.solve_batched(np.array([a.n, b.n], np.uint32),
                                                         np.array([0, a.m, a.m + b.m], np.uint64), src, dst, w,
                                                         stream=stream)
                        ids = ids.cpu().numpy().view(np.uint32)
                        moff = moff.cpu().numpy().astype(np.int64)
                        tot = tot.cpu().numpy().view(np.uint64)
                    for g, (kid, ktot) in enumerate((ea, eb)):
                        got = np.sort(ids[moff[g]:moff[g + 1]])
                        if not (np.array_equal(got, kid) and int(tot[g]) == ktot):
                            errors.append((t, rep, g))
        except Exception as e:  # reported below
            errors.append((t, repr(e)))
        stream.synchronize()

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(3)]
    try:
        for th in threads:
            th.start()
        for th in threads:
            th.join()
    finally:
        for s in solvers:
            s.close()
    assert not errors, errors
