"""Autotuner for the solver configuration of a workload.

The fastest way through a workload depends on its graphs: the Filter-Borůvka
variant (Alg. 2) pays off on dense, heavy-tailed graphs, parallel-edge removal
(Section 2.3, optional; by hashing or by sorting) on graphs whose contracted
rounds keep many parallel edges, and tile-local contraction (Section 4.1) only where vertex numbering
gives locality.  Rather than guess, the autotuner times each candidate
configuration on the caller's own input and keeps the fastest.  Every
candidate computes the same forest (the MSF under the (w, id) order is
unique), so the choice affects time only.

Host logic only: each trial is one call into the CUDA library.
"""
from __future__ import annotations

from typing import Callable, Dict, Iterable, List, Tuple

# Candidate configurations (keyword arguments of mst.Solver).
DEFAULT_CANDIDATES: Tuple[dict, ...] = (
    dict(variant="boruvka", dedupe="none", tile_contract=0),
    dict(variant="boruvka", dedupe="hash", tile_contract=0),
    dict(variant="boruvka", dedupe="sort", tile_contract=0),
    dict(variant="filter", dedupe="none", tile_contract=0),
    dict(variant="boruvka", dedupe="none", tile_contract=1),
    dict(variant="boruvka", dedupe="none", tile_contract=0, min_edges_sort=1),
)

# The Filter-Borůvka pivot's rank in its sample (the light share of each
# list; Alg. 2 takes the median, 1/2).  Tuned on the best configuration when
# that is the filter variant.
QUANTILE_CANDIDATES: Tuple[dict, ...] = tuple(dict(pivot_quantile=q) for q in (0.5, 0.25, 0.125, 0.0625))

# Tile shapes of the compaction and hook kernels: threads per block x items
# per thread.  Tuned on top of the best configuration above (every shape
# computes the same forest).
SHAPE_CANDIDATES: Tuple[dict, ...] = tuple(dict(block_threads=b, items_per_thread=i)
                                           for b in (128, 256, 512) for i in (4, 8, 16))

# The relabel compaction's own tile shape (it runs in every Borůvka round),
# tuned last, on top of the best configuration and shape.
RELABEL_SHAPE_CANDIDATES: Tuple[dict, ...] = tuple(dict(relabel_block_threads=b, relabel_items_per_thread=i)
                                                   for b in (128, 256, 512) for i in (4, 8, 16))

# The values a configuration gets for keys it does not set.
_DEFAULTS = dict(block_threads=256, items_per_thread=8, relabel_block_threads=128, relabel_items_per_thread=4,
                 pivot_quantile=0.125)

_cache: Dict[str, dict] = {}


def label(cfg: dict) -> str:
    return ",".join(f"{k}={cfg[k]}" for k in sorted(cfg))


def autotune(trial: Callable[[dict], float], candidates: Iterable[dict] = DEFAULT_CANDIDATES, reps: int = 2,
             key: str | None = None,
             shapes: Iterable[dict] | None = SHAPE_CANDIDATES,
             relabel_shapes: Iterable[dict] | None = None,
             quantiles: Iterable[dict] | None = QUANTILE_CANDIDATES) -> Tuple[dict, List[Tuple[str, float]]]:
    """Returns (best configuration, [(label, best seconds)] for every trial).

    trial(cfg) runs one solve of the workload with configuration cfg and
    returns its duration in seconds (the caller times it on the device).  Each
    candidate gets one untimed run and `reps` timed runs; its score is the
    fastest timed run.  The candidates are tried first; then, if the best of
    them is the filter variant, each of `quantiles` (pivot ranks; None or
    empty: none) on top of it; then each of `shapes` (kernel tile shapes) on
    top of the best so far; then each of `relabel_shapes` (e.g.
    RELABEL_SHAPE_CANDIDATES).  Settings equal to what the configuration
    already runs are skipped.  With `key`, the choice is remembered for the
    process and later calls with the same key return it without trials."""
    if key is not None and key in _cache:
        return dict(_cache[key]), []
    results: List[Tuple[str, float]] = []
    best, best_t = None, float("inf")

    def run(cfg):
        nonlocal best, best_t
        trial(cfg)
        t = min(trial(cfg) for _ in range(max(1, reps)))
        results.append((label(cfg), t))
        if t < best_t:
            best, best_t = dict(cfg), t

    for cfg in candidates:
        run(cfg)
    if best is None:
        raise ValueError("autotune needs at least one candidate")
    for stage in (quantiles, shapes, relabel_shapes):
        base = dict(best)
        if stage is quantiles and base.get("variant") != "filter":
            continue
        for shape in stage or ():
            if all(base.get(k, _DEFAULTS.get(k)) == v for k, v in shape.items()):
                continue  # already timed
            run({**base, **shape})
    if key is not None:
        _cache[key] = dict(best)
    return best, results
