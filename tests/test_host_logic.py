"""Host-side logic that needs no GPU: the serving loop's arrival process and
the configuration autotuner."""
import numpy as np
import pytest

from paper_2302_12199_gb300.autotune import autotune, label


def test_poisson_arrivals_window_rate_and_order():
    pytest.importorskip("torch")
    from paper_2302_12199_gb300.serve import poisson_arrivals
    for rate, secs in ((4096.0, 2.0), (65536.0, 0.25), (10.0, 30.0)):
        t = poisson_arrivals(rate, secs, seed=3)
        assert t.size > 0 and np.all(np.diff(t) > 0) and t[0] >= 0 and t[-1] < secs
        # count of a Poisson process: mean rate*secs, sd sqrt(rate*secs)
        assert abs(t.size - rate * secs) < 6 * np.sqrt(rate * secs)
        # exponential gaps: mean 1/rate
        gaps = np.diff(np.concatenate([[0.0], t]))
        assert abs(gaps.mean() * rate - 1.0) < 6 / np.sqrt(t.size)
    assert np.array_equal(poisson_arrivals(100.0, 1.0, 9), poisson_arrivals(100.0, 1.0, 9))


def test_autotune_picks_the_fastest_and_caches():
    cost = {"a": 3.0, "b": 1.0, "c": 2.0}
    calls = []

    def trial(cfg):
        calls.append(cfg["k"])
        return cost[cfg["k"]]
    cands = [dict(k="a"), dict(k="b"), dict(k="c")]
    best, res = autotune(trial, cands, reps=2, key="t1", shapes=None)
    assert best == dict(k="b")
    assert [r[0] for r in res] == [label(c) for c in cands] and [r[1] for r in res] == [3.0, 1.0, 2.0]
    assert len(calls) == 9  # one untimed + two timed runs each
    best2, res2 = autotune(trial, cands, key="t1")
    assert best2 == best and res2 == [] and len(calls) == 9
    with pytest.raises(ValueError):
        autotune(trial, [], key=None)


def test_autotune_tunes_the_kernel_shape_on_the_best_configuration():
    """The shape stage runs every tile shape except the default one on top of
    the best configuration of the first stage, and keeps a faster shape."""
    from paper_2302_12199_gb300.autotune import SHAPE_CANDIDATES
    seen = []

    def trial(cfg):
        seen.append(dict(cfg))
        t = {"a": 3.0, "b": 2.0}[cfg["k"]]
        if cfg.get("block_threads") == 512 and cfg.get("items_per_thread") == 4:
            t -= 0.5
        return t
    best, res = autotune(trial, [dict(k="a"), dict(k="b")], reps=1, shapes=SHAPE_CANDIDATES)
    assert best == dict(k="b", block_threads=512, items_per_thread=4)
    shaped = [c for c in seen if "block_threads" in c]
    assert all(c["k"] == "b" for c in shaped)  # shapes only on the first stage's winner
    assert len({(c["block_threads"], c["items_per_thread"]) for c in shaped}) == 8  # 256 x 8 is the default
    assert len(res) == 2 + 8


def test_autotune_quantile_stage_only_for_the_filter_variant():
    """Pivot quantiles are tried on top of the best configuration only when it
    is Filter-Borůvka (the plain variant has no pivot), skipping the library's
    default quantile, and a faster quantile is kept."""
    from paper_2302_12199_gb300.autotune import QUANTILE_CANDIDATES
    seen = []

    def trial(cfg):
        seen.append(dict(cfg))
        t = {"boruvka": 3.0, "filter": 2.0}[cfg["variant"]]
        return t - (0.5 if cfg.get("pivot_quantile") == 0.25 else 0.0)
    best, res = autotune(trial, [dict(variant="boruvka"), dict(variant="filter")], reps=1, shapes=None)
    assert best == dict(variant="filter", pivot_quantile=0.25)
    tried = [c["pivot_quantile"] for c in seen if "pivot_quantile" in c]
    assert set(tried) == {q["pivot_quantile"] for q in QUANTILE_CANDIDATES} - {0.125}
    assert all(c["variant"] == "filter" for c in seen if "pivot_quantile" in c)
    seen.clear()
    best, _ = autotune(lambda cfg: seen.append(dict(cfg)) or 1.0, [dict(variant="boruvka")], reps=1, shapes=None)
    assert best == dict(variant="boruvka") and not any("pivot_quantile" in c for c in seen)


def test_autotune_relabel_shape_stage_runs_on_the_best_shape():
    """The relabel compaction's shapes are tried last, on top of the best
    configuration and kernel shape, skipping the default 128 x 4."""
    from paper_2302_12199_gb300.autotune import RELABEL_SHAPE_CANDIDATES, SHAPE_CANDIDATES
    seen = []

    def trial(cfg):
        seen.append(dict(cfg))
        t = 2.0
        if cfg.get("block_threads") == 128 and cfg.get("items_per_thread") == 16:
            t -= 0.5
        if cfg.get("relabel_block_threads") == 256 and cfg.get("relabel_items_per_thread") == 8:
            t -= 0.25
        return t
    best, res = autotune(trial, [dict(k="a")], reps=1, shapes=SHAPE_CANDIDATES,
                         relabel_shapes=RELABEL_SHAPE_CANDIDATES)
    assert best == dict(k="a", block_threads=128, items_per_thread=16, relabel_block_threads=256,
                        relabel_items_per_thread=8)
    relabel = [c for c in seen if "relabel_block_threads" in c]
    assert all(c["block_threads"] == 128 and c["items_per_thread"] == 16 for c in relabel)
    assert len({(c["relabel_block_threads"], c["relabel_items_per_thread"]) for c in relabel}) == 8
    assert len(res) == 1 + 8 + 8


class _FakeSlot:
    """Stands in for a GPU solver slot: 'solves' a batch after a short sleep and
    returns per-graph answers that encode the graph, so routing is checked."""

    def __init__(self, delay=0.002):
        import threading
        self.busy, self.job, self.stop = False, None, False
        self.cv = threading.Condition()
        self.delay = delay
        self.calls = []

    def workspace_bytes(self, n, m):
        return 100 * m + 10 * n

    def solve(self, graphs):
        import time
        self.calls.append(len(graphs))
        time.sleep(self.delay)
        ids = np.concatenate([np.array([g.n, g.m], dtype=np.uint32) for g in graphs])
        moff = np.arange(0, 2 * len(graphs) + 1, 2, dtype=np.int64)
        tot = np.array([g.n * 1000 + g.m for g in graphs], dtype=np.uint64)
        return ids, moff, tot

    def close(self):
        pass


class _G:
    def __init__(self, n, m):
        self.n, self.m = n, m


def test_server_scheduling_with_fake_slots():
    pytest.importorskip("torch")
    from paper_2302_12199_gb300.serve import Response, Server, poisson_arrivals
    pool = [_G(10 + i, 100 * (i + 1)) for i in range(8)]
    expected = {i: Response(np.array([g.n, g.m], dtype=np.uint32), g.n * 1000 + g.m) for i, g in enumerate(pool)}
    slots = []

    def factory():
        slots.append(_FakeSlot())
        return slots[-1]
    # budget fits about three requests per batch
    srv = Server(slots=2, budget_bytes=3 * 100 * 800, max_batch=5, slot_factory=factory, stall_seconds=5.0)
    for rep in range(3):  # one server, several request streams in turn
        arr = poisson_arrivals(4000.0, 0.05, seed=rep)
        picks = np.random.default_rng(rep).integers(0, len(pool), arr.size)
        st = srv.run(pool, picks, arr, expected=expected, rate=4000.0, seconds=0.05)
        assert st.requests == arr.size and st.mismatches == 0
        assert sum(st.batch_sizes) == arr.size and max(st.batch_sizes) <= 5
        assert np.all(st.latency > 0)
        assert st.max_in_flight >= 1
    assert all(sum(s.calls) > 0 for s in slots)  # both slots took batches
    # admission: a request over the whole budget goes alone; wrong answers are counted
    bad = {i: Response(np.array([0], dtype=np.uint32), 0) for i in range(len(pool))}
    srv1 = Server(slots=1, budget_bytes=1, max_batch=8, slot_factory=factory, stall_seconds=5.0)
    st = srv1.run(pool, np.arange(6), np.linspace(0, 1e-3, 6), expected=bad)
    assert st.batch_sizes == [1] * 6 and st.mismatches == 6
