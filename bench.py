"""Benchmark: device-timed input edges/s of one minimum-spanning-forest solve.

Default workload: RMAT, n = 2^24, m = 2^28 undirected edges, (a,b,c,d) =
(0.57,0.19,0.19,0.05), permuted ids, weights uniform in [1,255], solved with
Filter-Borůvka (pivot sample 2^16).  One step = one full mst_solve of that graph
(every step of the method: partitions, Borůvka rounds, filters, output), with
the input resident in HBM.  The input (3.2 GB) is larger than L2, so no flush
is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference] [--workload NAME]

With N > 1 (torchrun, one rank per GPU) every rank solves its own replica of
the graph: a single graph does not shard, so the GPUs run independent
replicas and `value` counts the edges of all replicas.

`--impl reference` times the CPU oracle (Kruskal) on a bounded sample of the
same workload on the host cores, for the same metric.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "input edges/s per MSF solve (device-timed)"
UNIT = "edges/s"

WORKLOADS = {
    # name: (description, generator, solver config)
    "rmat_filter": ("RMAT n=2^24 m=2^28 (0.57,0.19,0.19,0.05) permuted, w in [1,255], Filter-Boruvka",
                    lambda W: W.rmat_large(), dict(variant="filter")),
    "rmat_boruvka": ("RMAT n=2^24 m=2^28 (0.57,0.19,0.19,0.05) permuted, w in [1,255], plain Boruvka",
                     lambda W: W.rmat_large(), dict(variant="boruvka")),
    "rmat20_filter": ("RMAT n=2^20 m=2^24 (0.57,0.19,0.19,0.05) permuted, w in [1,255], Filter-Boruvka (profiling size)",
                      lambda W: W.rmat_large(scale=20, m=1 << 24), dict(variant="filter")),
    "rmat22_filter": ("RMAT n=2^22 m=2^26 (0.57,0.19,0.19,0.05) permuted, w in [1,255], Filter-Boruvka (profiling size)",
                      lambda W: W.rmat_large(scale=22, m=1 << 26), dict(variant="filter")),
    "gnm": ("GNM n=2^16 m=2^20, w in [1,255], plain Boruvka", lambda W: W.gnm_small(), dict(variant="boruvka")),
    "rgg2d": ("RGG2D n=2^22 degree 8, w in [1,2^32-1], plain Boruvka", lambda W: W.rgg2d_large(),
              dict(variant="boruvka")),
    "rgg3d": ("RGG3D n=2^21 degree 8, w in [1,2^32-1], plain Boruvka", lambda W: W.rgg3d_large(),
              dict(variant="boruvka")),
    "grid2d": ("2D grid 2048x2048 (n=2^22, m=8,384,512), w in [1,255], plain Boruvka", lambda W: W.grid2d_large(),
               dict(variant="boruvka")),
    "rhg": ("random hyperbolic graph n=2^22, gamma=3, average degree ~16, w in [1,255], plain Boruvka",
            lambda W: W.rhg_large(), dict(variant="boruvka")),
    "rgg2d_small": ("RGG2D n=2^20 degree 8, w in [1,2^32-1], plain Boruvka (profiling size)",
                    lambda W: W.rgg(2, 1 << 20, 8.0), dict(variant="boruvka")),
}


# DRAM traffic of the dominant kernel, from one ncu capture of the
# filter launches of a timed solve at RMAT scale 22 (n=2^22, m=2^26; the
# full-size workload holds tens of GB on the device, too much for a capture
# of many passes): dram__bytes_read.sum + dram__bytes_write.sum over those
# launches divided by the algorithmic bytes the library's profiler counted for
# them.  A full-size launch's traffic is taken as that ratio times its
# algorithmic bytes (at scale 24 the 64 MB label array shares the L2 with a
# longer stream, so the true ratio there is somewhat higher).  The ratio holds
# only for the kernel source it was measured on and for the pivot quantile
# that set the levels' mix: when the source regions below hash differently, or
# the quantile differs, traffic is reported as null until it is captured again.
TRAFFIC = {
    "class": "filter",
    "kernel": "stream_warp_kernel<CM_FILTER>",
    "dram_per_algorithmic_byte": 1.352,
    "measured_on": "RMAT n=2^22 m=2^26, both filter launches of one timed solve (pivot quantile 1/8)",
    "pivot_quantile": 0.125,
    "source_sha256": "a90ad8de4d5004aeb0ae6e62c8b2c6004d9762fb0085350b95469a5fbad917b5",
}
TRAFFIC_SOURCE = (
    ("paper_2302_12199_gb300/csrc/kernels.cu", "__device__ __forceinline__ uint32_t keep_flags",
     "// Writes the kept items of a tile"),
    ("paper_2302_12199_gb300/csrc/kernels.cu", "// ------------------------------------------------- warp-streamed passes",
     "// --------------------------------------------------------------- min edges"),
)


def traffic_source_digest():
    import hashlib
    h = hashlib.sha256()
    for path, start, end in TRAFFIC_SOURCE:
        try:
            with open(os.path.join(ROOT, path)) as f:
                text = f.read()
            i, j = text.index(start), text.index(end)
        except (OSError, ValueError):
            return None
        h.update(text[i:j].encode())
    return h.hexdigest()


def reduce_scalar(x: float, op: str, dist, device) -> float:
    """x combined over all ranks by "max" or "sum" (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units_per_rank: float, seconds: float, world: int, dist, device):
    """Whole-job rate of `world` replicas that each processed units_per_rank in
    `seconds`: all units over the slowest rank's time.  Returns (rate, slowest)."""
    slowest = reduce_scalar(seconds, "max", dist, device)
    return units_per_rank * world / slowest, slowest


def nvtx_mark(torch, what: str) -> None:
    """Opens or closes the NVTX range "timed" (no-op where NVTX is missing)."""
    try:
        if what == "push":
            torch.cuda.nvtx.range_push("timed")
        else:
            torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            if self.uuid and parts[0] != self.uuid:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- reference

def cpu_oracle_rate(g, sample_edges: int, repeats: int = 1, threads: int = 1) -> tuple[float, float]:
    """Kruskal (the CPU oracle; single-threaded, or with its sort on `threads`
    host threads) on the first `sample_edges` edges of the graph; returns
    (edges/s, seconds per run)."""
    import oracle
    k = min(sample_edges, g.m)
    src, dst, w = g.src[:k], g.dst[:k], g.w[:k]
    best = None
    for _ in range(repeats):
        t0 = time.perf_counter()
        if threads > 1:
            oracle.kruskal_par(g.n, src, dst, w, threads)
        else:
            oracle.kruskal(g.n, src, dst, w)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    return k / best, best


def reference_batched(args):
    """The oracle (Kruskal, one thread) on the first graphs of the batched mix
    (or of the served pool), as many as fit in about two seconds per step;
    reported in graphs/s."""
    import numpy as np
    import oracle
    from paper_2302_12199_gb300 import workloads as W
    if args.workload == "served":
        args.graphs = args.pool
        b = W.mix(args.pool, W.DEFAULT_SEED + 5, log_lo=8, log_hi=20)
    else:
        b = W.mix(args.graphs, W.DEFAULT_SEED)
    off = np.asarray(b.edge_off, dtype=np.int64)

    def step(limit_s=2.0):
        t0 = time.perf_counter()
        g = 0
        while g < args.graphs and time.perf_counter() - t0 < limit_s:
            lo, hi = off[g], off[g + 1]
            oracle.kruskal(int(b.n[g]), b.src[lo:hi], b.dst[lo:hi], b.w[lo:hi])
            g += 1
        return g, time.perf_counter() - t0
    for _ in range(args.warmup):
        step()
    done, secs = 0, 0.0
    for _ in range(args.steps):
        k, dt = step()
        done += k
        secs += dt
    value = done / secs
    line = {
        "impl": "reference", "value": value,
        "metric": ("served graphs/s (Poisson arrivals, continuous batching)" if args.workload == "served"
                   else "batched graphs/s (one mst_solve_batched call per step)"),
        "unit": "graphs/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic", "config": {"workload": args.workload, "graphs": args.graphs},
        "cpu_baseline": {"value": value, "unit": "graphs/s", "cores": 1, "kind": "oracle",
                         "sample": f"the first graphs of the {args.graphs}-graph {args.workload} mix, "
                                                   "~2 s of Kruskal per step"},
        "e2e": {"value": value, "unit": "graphs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


REF_BUDGET_S = 100.0  # wall time of a --impl reference run (steps + warm-up)


def reference_main(args, rank: int):
    if rank != 0:
        return 0
    from paper_2302_12199_gb300 import workloads as W
    if args.workload in ("batched", "served"):
        return reference_batched(args)
    desc, gen, cfg = WORKLOADS[args.workload]
    g = gen(W)
    sample = min(g.m, args.cpu_sample_edges)
    # the first warm-up step sizes the sample so that the whole run (steps and
    # warm-up) takes about REF_BUDGET_S; the rate is per edge, so a smaller
    # sample of the same list only shortens the run
    _, dt0 = cpu_oracle_rate(g, sample)
    per_step = REF_BUDGET_S / max(1, args.steps + args.warmup - 1)
    if dt0 > per_step:
        sample = max(min(sample, 1 << 20), int(sample * per_step / dt0))
    for _ in range(max(0, args.warmup - 1)):
        cpu_oracle_rate(g, sample)
    times = []
    for _ in range(args.steps):
        _, dt = cpu_oracle_rate(g, sample)
        times.append(dt)
    total = sum(times)
    value = sample * args.steps / total
    sample_desc = f"first {sample} of the {g.m} edges (n={g.n}), Kruskal, single thread"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "n": g.n, "m": g.m, **cfg},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample_desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------- gpu

def link_gbps(torch, dev, pin):
    """Host-to-device rate right now: one copy of the pinned input arrays
    (CUDA events on a side stream)."""
    side = torch.cuda.Stream(dev)
    bufs = [torch.empty(p.numel(), dtype=p.dtype, device=dev) for p in pin]
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(side):
        a.record(side)
        for d, h in zip(bufs, pin):
            d.copy_(h, non_blocking=True)
        b.record(side)
    torch.cuda.synchronize(dev)
    nbytes = sum(p.numel() * p.element_size() for p in pin)
    del bufs
    return nbytes / (a.elapsed_time(b) / 1e3) / 1e9


def e2e_breakdown(torch, solver, dev, stream, n, m, pin, d_in, out, ids_h, cnt, reps=3):
    """Parts of one end-to-end step, each timed with CUDA events (medians of
    `reps`): the input copy from pinned host memory alone, the solve alone,
    the solve while the next step's input copy runs on another stream (what
    the overlapped entry point does), and the read-back of the forest."""
    side = torch.cuda.Stream(dev)
    bufs = [torch.empty(m, dtype=torch.int32, device=dev) for _ in range(3)]

    def copy_in():
        with torch.cuda.stream(side):
            for d, h in zip(bufs, pin):
                d.copy_(h, non_blocking=True)

    def ev_pair():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    h2d, solo, during, d2h = [], [], [], []
    for _ in range(reps):
        torch.cuda.synchronize(dev)
        a, b = ev_pair()
        a.record(side)
        copy_in()
        b.record(side)
        torch.cuda.synchronize(dev)
        h2d.append(a.elapsed_time(b))
        a, b = ev_pair()
        a.record(stream)
        solver.solve(n, *d_in, out=out)
        b.record(stream)
        torch.cuda.synchronize(dev)
        solo.append(a.elapsed_time(b))
        copy_in()
        a, b = ev_pair()
        a.record(stream)
        solver.solve(n, *d_in, out=out)
        b.record(stream)
        torch.cuda.synchronize(dev)
        during.append(a.elapsed_time(b))
        a, b = ev_pair()
        a.record(stream)
        ids_h[:cnt].copy_(out.ids[:cnt], non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize(dev)
        d2h.append(a.elapsed_time(b))
    del bufs
    med = statistics.median
    return {"h2d": med(h2d), "solve": med(solo), "solve_during_h2d": med(during), "d2h": med(d2h),
            "h2d_GBps": 12 * m / med(h2d) / 1e6}


def gpu_main(args, rank: int, world: int, local_rank: int):
    import numpy as np
    import torch

    from paper_2302_12199_gb300 import workloads as W
    from paper_2302_12199_gb300.mst import Solver

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    desc, gen, cfg = WORKLOADS[args.workload]
    cfg = dict(cfg)
    if args.variant:
        cfg["variant"] = args.variant
    if args.dedupe:
        cfg["dedupe"] = args.dedupe
    if args.filter_max_avg_degree is not None:
        cfg["filter_max_avg_degree"] = args.filter_max_avg_degree
    if args.filter_min_edges is not None:
        cfg["filter_min_edges"] = args.filter_min_edges
    if args.tile_contract is not None:
        cfg["tile_contract"] = args.tile_contract
    if args.tile_vertices is not None:
        cfg["tile_vertices"] = args.tile_vertices
    if args.base_case is not None:
        cfg["base_case"] = args.base_case
    if args.graph_rounds is not None:
        cfg["graph_rounds"] = args.graph_rounds
    if args.filter_carry is not None:
        cfg["filter_carry"] = args.filter_carry
    if args.filter_split is not None:
        cfg["filter_split"] = args.filter_split
    if args.min_edges_sort is not None:
        cfg["min_edges_sort"] = args.min_edges_sort
    if args.tile_filter is not None:
        cfg["tile_filter"] = args.tile_filter
    if args.filter_plan is not None:
        cfg["filter_plan"] = args.filter_plan
    if args.pivot_quantile is not None:
        cfg["pivot_quantile"] = args.pivot_quantile
    g = gen(W)
    n, m = g.n, g.m
    src = torch.from_numpy(g.src.view(np.int32)).to(dev)
    dst = torch.from_numpy(g.dst.view(np.int32)).to(dev)
    w = torch.from_numpy(g.w.view(np.int32)).to(dev)
    solver = Solver(local_rank, **cfg)
    out = solver.alloc_forest(n, m)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        solver.solve(n, src, dst, w, out=out)
    torch.cuda.synchronize(dev)
    ref_ids, ref_total = out.to_host()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    # a profiled pass outside the timed region: every kernel class timed with
    # CUDA events (per-class table; picks the dominant class)
    prof_steps = max(1, min(args.steps, 5))
    solver.profile(True)
    for _ in range(prof_steps):
        solver.solve(n, src, dst, w, out=out)
    torch.cuda.synchronize(dev)
    solver.profile(False)
    stats_all = solver.profile_stats()
    # the dominant class among those whose bytes are counted (the graph
    # class's are not: its kernels are counted in no class)
    dom = max((k for k in stats_all if stats_all[k][2] > 0), key=lambda k: stats_all[k][1])
    sampler = ClockSampler(uuid)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    time.sleep(0.3)
    # the timed region: events around the dominant class's launches only (the
    # roofline's measured durations); every class still counts its launches
    # and algorithmic bytes, which costs the host almost nothing per launch
    solver.profile(True, classes=[dom])
    hc0 = solver.host_counters()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nvtx_mark(torch, "push")  # lets a profiler capture the timed solves only
    e0.record(stream)
    for _ in range(args.steps):
        solver.solve(n, src, dst, w, out=out)
    e1.record(stream)
    nvtx_mark(torch, "pop")
    hc1 = solver.host_counters()
    host = {"readbacks_per_step": (hc1["readbacks"] - hc0["readbacks"]) / args.steps,
            "planned_steps": hc1["planned"] - hc0["planned"],
            "plan_fallbacks": hc1["plan_fallbacks"] - hc0["plan_fallbacks"],
            "note": "host waits for device counts per solve; planned: Filter-Borůvka recursion laid out "
                    "from the top-level light count, lengths kept on the device"}
    torch.cuda.synchronize(dev)
    solver.profile(False)
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    stats = solver.profile_stats(with_min=True)
    ids, total = out.to_host()
    if not (np.array_equal(ids, ref_ids) and total == ref_total):
        raise RuntimeError("timed solves returned a different forest than the warm-up solve")

    value, slowest_s = job_rate(m * args.steps, ms / 1e3, world, dist, dev)
    ms_max = slowest_s * 1e3

    # end to end through the public API with host buffers: H2D of the inputs
    # from pinned memory and D2H of the forest inside the timed region
    pin = [torch.from_numpy(a.view(np.int32)).pin_memory() for a in (g.src, g.dst, g.w)]
    ids_h = torch.empty(max(1, min(m, n - 1)), dtype=torch.int32).pin_memory()
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    step_spec = (n, m, pin[0].data_ptr(), pin[1].data_ptr(), pin[2].data_ptr(), ids_h.data_ptr())
    # (a) one mst_solve_host call per step: copy in, solve, copy out
    solver.solve_host_ptr(n, m, *step_spec[2:])
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solver.solve_host_ptr(n, m, *step_spec[2:])
    torch.cuda.synchronize(dev)
    seq_value, _ = job_rate(m * e2e_steps, time.perf_counter() - t0, world, dist, dev)
    # (b) the steps as one mst_solve_host_many call: each step's inputs are
    # still copied from pinned host memory and its forest read back, but the
    # copy of step k+1 runs while step k is solved
    # Five such calls, the median reported: the host link and the host itself
    # are shared with the machine's other GPUs and their jobs, and single steps
    # of a call have been seen to stall for tens of milliseconds (the GPU idle
    # between two launches of a solve), so the link alone is timed right before
    # and right after as well.
    solver.solve_host_many_ptr([step_spec] * 2)
    link_before = link_gbps(torch, dev, pin)
    runs = []
    for _ in range(5):
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        res = solver.solve_host_many_ptr([step_spec] * e2e_steps)
        torch.cuda.synchronize(dev)
        runs.append(job_rate(m * e2e_steps, time.perf_counter() - t0, world, dist, dev)[0])
    link_after = link_gbps(torch, dev, pin)
    e2e_value = statistics.median(runs)
    cnt = res[-1][0]
    if any(r != (len(ref_ids), ref_total) for r in res) or \
            not np.array_equal(ids_h[:cnt].numpy().view(np.uint32), np.asarray(ref_ids, dtype=np.uint32)):
        raise RuntimeError("an end-to-end step returned a different forest")
    e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 12 * m,
           "d2h_bytes_per_step": 4 * cnt + 12, "steps": e2e_steps,
           "api": "mst_solve_host_many: step k+1's input copy overlaps step k's solve",
           "runs": runs, "note": f"median of {len(runs)} calls of {e2e_steps} steps",
           "link_GBps_before_after": [link_before, link_after],
           "one_call_per_step": {"value": seq_value, "api": "mst_solve_host"},
           "breakdown_ms": e2e_breakdown(torch, solver, dev, stream, n, m, pin, (src, dst, w), out, ids_h, cnt)}

    peaks = measured_peaks()
    kernels = {}
    all_bytes = 0.0
    launches = 0
    for name, (nl, kms, kbytes, _) in stats.items():  # timed region: launches and bytes of every class
        launches += nl
        all_bytes += kbytes
    for name, (nl, kms, kbytes) in stats_all.items():  # profiled pass: every class timed
        if nl:
            kernels[name] = {"launches_per_step": nl / prof_steps, "ms_per_step": kms / prof_steps,
                             "bytes_per_step": kbytes / prof_steps,
                             "GBps": (kbytes / (kms / 1e3) / 1e9) if kms > 0 else None}
    nl, kms, kbytes, kmin = stats[dom]
    achieved = kbytes / (kms / 1e3) / 1e9
    achieved_min = kmin / (kms / 1e3) / 1e9
    traffic = None
    if (dom == TRAFFIC["class"] and TRAFFIC["dram_per_algorithmic_byte"] and nl
            and abs(float(solver.cfg.pivot_quantile) - TRAFFIC["pivot_quantile"]) < 1e-6
            and traffic_source_digest() == TRAFFIC["source_sha256"]):
        traffic = TRAFFIC["dram_per_algorithmic_byte"] * kbytes / nl
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "peak_source": peaks["source"],
                "bytes_per_launch": kbytes / nl if nl else None,
                # the method's own bytes: for the filter only the heavy edges
                # read (the pass re-reads the light ones too) and the survivors
                "min_bytes_per_launch": kmin / nl if nl else None,
                "achieved_min": achieved_min, "frac_min": achieved_min / peaks["hbm_gbs"],
                "traffic": traffic,
                "traffic_source": (f"ncu DRAM bytes / algorithmic bytes of {TRAFFIC['kernel']} on "
                                   f"{TRAFFIC['measured_on']} ({TRAFFIC['dram_per_algorithmic_byte']}), times this "
                                   f"launch's algorithmic bytes (kernel source sha256 "
                                   f"{TRAFFIC['source_sha256'][:12]})") if traffic is not None else None,
                "time_share": kms / ms if ms > 0 else None}
    effective = all_bytes / args.steps / (ms / args.steps / 1e3) / 1e9

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "n": n, "m": m, **cfg,
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "inputs (12 B/edge) larger than L2, no flush"},
        "roofline": roofline,
        "effective_bw": {"GBps": effective, "frac": effective / peaks["hbm_gbs"],
                         "note": "sum of algorithmic bytes of all kernels / solve time"},
        "kernels": kernels,
        "kernels_note": f"per-class CUDA-event times of {prof_steps} profiled solves outside the timed region; "
                        "inside it only the dominant class is timed",
        "gpu_launches": launches,
        "host": host,
        "e2e": e2e,
        "clocks": clocks,
        "msf": {"edges": int(ids.size), "weight": int(total)},
    }
    if rank == 0 and not args.no_cpu_baseline:
        rate, dt = cpu_oracle_rate(g, args.cpu_sample_edges)
        sample = f"first {min(g.m, args.cpu_sample_edges)} of the {g.m} edges (n={n})"
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{sample}, Kruskal, single thread, {dt:.1f} s"}
        cores = host_cores()
        prate, pdt = cpu_oracle_rate(g, args.cpu_sample_edges, threads=cores)
        line["cpu_baseline_parallel_sort"] = {
            "value": prate, "unit": UNIT, "cores": cores, "kind": "oracle, sort on all host cores",
            "sample": f"{sample}, Kruskal with its radix sort on {cores} threads (union-find sequential), {pdt:.1f} s"}
    solver.close()
    del src, dst, w, pin
    torch.cuda.empty_cache()
    if not args.no_batched and args.workload == "rmat_filter":
        # the batched workload (4096 mixed graphs), compact: graphs/s, batch
        # latency and the one-solve-per-graph baseline on the same GPU
        import types
        bargs = types.SimpleNamespace(graphs=args.graphs, log_hi=args.log_hi, no_autotune=args.no_autotune,
                                      base_case=args.base_case, graph_rounds=args.graph_rounds,
                                      steps=args.batched_steps, warmup=3, e2e_steps=1)
        line["batched"] = measure_batched(bargs, rank, world, local_rank, dev, dist, compact=True)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def percentiles(xs, qs=(50, 99, 99.9)):
    import numpy as np
    a = np.asarray(xs, dtype=np.float64)
    return {f"p{q:g}": float(np.percentile(a, q)) for q in qs} if a.size else {}


def batched_main(args, rank: int, world: int, local_rank: int):
    """The batched configuration as its own bench line (see measure_batched)."""
    import torch
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    line = measure_batched(args, rank, world, local_rank, dev, dist)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def measure_batched(args, rank: int, world: int, local_rank: int, dev, dist, compact: bool = False) -> dict:
    """The batched configuration: G mixed graphs (n log-uniform in [2^8, 2^16];
    1/3 GNM with average degree in [4,32], 1/3 RGG2D degree 8, 1/3 RMAT degree
    16; w in [1,255]) solved by one mst_solve_batched call per step (the
    configuration chosen by the autotuner), against one mst_solve call per
    graph (plain Borůvka) on the same GPU; every batched forest is compared
    with the graph's own solve.  compact: only the throughput, the batch
    latencies and the per-graph baseline (no per-class profile, no clocks, no
    end-to-end leg)."""
    import numpy as np
    import torch

    from paper_2302_12199_gb300 import workloads as W
    from paper_2302_12199_gb300.autotune import RELABEL_SHAPE_CANDIDATES, autotune, label
    from paper_2302_12199_gb300.mst import Solver

    G = args.graphs
    b = W.mix(G, W.DEFAULT_SEED + rank, log_hi=args.log_hi)
    n_per = np.asarray(b.n, dtype=np.uint32)
    off = np.asarray(b.edge_off, dtype=np.uint64)
    m_tot = int(off[-1])
    n_tot = int(n_per.astype(np.int64).sum())
    to_dev = lambda a: torch.from_numpy(a.view(np.int32)).to(dev)
    src, dst, w = to_dev(b.src), to_dev(b.dst), to_dev(b.w)
    d_n = to_dev(n_per)  # the size tables stay on the device, like the edges
    d_off = torch.from_numpy(off.view(np.int64)).to(dev)
    stream = torch.cuda.current_stream(dev)

    def timed_batch(solver):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = solver.solve_batched(d_n, d_off, src, dst, w, capacity=n_tot)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / 1e3, res

    # autotuned configuration (variant, dedupe strategy, tile contraction,
    # then the kernels' tile shape); each candidate keeps one handle across its
    # runs, so the timed runs see the steady state (pool grown, round graphs
    # built), not a handle's first solves
    trial_solver = {}

    def trial(cfg):
        key = label(cfg)
        if key not in trial_solver:
            for k in list(trial_solver):
                trial_solver.pop(k).close()
            trial_solver[key] = Solver(local_rank, **cfg)
        return timed_batch(trial_solver[key])[0]
    if args.no_autotune:
        best, tuning = dict(variant="boruvka", dedupe="none", tile_contract=0), []
    else:
        best, tuning = autotune(trial, reps=3, relabel_shapes=RELABEL_SHAPE_CANDIDATES)
    for k in list(trial_solver):
        trial_solver.pop(k).close()
    if args.base_case is not None:
        best["base_case"] = args.base_case
    if args.graph_rounds is not None:
        best["graph_rounds"] = args.graph_rounds
    solver = Solver(local_rank, **best)
    for _ in range(args.warmup):
        timed_batch(solver)
    ref_ids, ref_off, ref_tot = [t.cpu() for t in solver.solve_batched(n_per, off, src, dst, w)]
    torch.cuda.synchronize(dev)
    # profiled batches outside the timed region (every class timed), as for
    # the single-graph workloads; inside it only the dominant class is timed
    prof_steps = max(1, min(args.steps, 3))
    dom = None
    if not compact:
        solver.profile(True)
        for _ in range(prof_steps):
            timed_batch(solver)
        solver.profile(False)
        stats_all = solver.profile_stats()
        # the dominant class among those whose bytes are counted
        dom = max((k for k in stats_all if stats_all[k][2] > 0), key=lambda k: stats_all[k][1])

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    if dist:
        dist.barrier()
    if not compact:
        sampler.start()
        time.sleep(0.3)
    solver.profile(True, classes=[dom] if dom else [])
    lat = []
    hc0 = solver.host_counters()
    nvtx_mark(torch, "push")
    for _ in range(args.steps):
        dt, res = timed_batch(solver)
        lat.append(dt)
    nvtx_mark(torch, "pop")
    hc1 = solver.host_counters()
    host = {"readbacks_per_step": (hc1["readbacks"] - hc0["readbacks"]) / args.steps,
            "planned_steps": hc1["planned"] - hc0["planned"],
            "plan_fallbacks": hc1["plan_fallbacks"] - hc0["plan_fallbacks"]}
    solver.profile(False)
    clocks = sampler.stop()
    stats = solver.profile_stats()
    ids, moff, tot = [t.cpu() for t in res]
    if not (torch.equal(ids, ref_ids) and torch.equal(moff, ref_off) and torch.equal(tot, ref_tot)):
        raise RuntimeError("timed batched solves returned different forests than the warm-up solve")
    value, total_s = job_rate(G * args.steps, sum(lat), world, dist, dev)

    # baseline: one mst_solve per graph, plain Borůvka, same GPU and stream
    base = Solver(local_rank, variant="boruvka", dedupe="none", tile_contract=0)
    outs = [base.alloc_forest(int(n_per[g]), int(off[g + 1] - off[g])) for g in range(G)]
    per = []
    for rep in range(2):  # the first pass warms the pool allocator
        per = []
        torch.cuda.synchronize(dev)
        t_all = time.perf_counter()
        for g in range(G):
            lo, hi = int(off[g]), int(off[g + 1])
            t0 = time.perf_counter()
            base.solve(int(n_per[g]), src[lo:hi], dst[lo:hi], w[lo:hi], out=outs[g])
            torch.cuda.synchronize(dev)
            per.append(time.perf_counter() - t0)
        t_all = time.perf_counter() - t_all
    base_value = G / t_all
    # the batched forests equal the per-graph ones
    mismatch = 0
    moff_np = moff.numpy().astype(np.int64)
    ids_np = ids.numpy().view(np.uint32)
    tot_np = tot.numpy().view(np.uint64)
    for g in range(G):
        gi, gt = outs[g].to_host()
        seg = ids_np[moff_np[g]:moff_np[g + 1]]
        if not (np.array_equal(np.sort(seg), gi) and int(tot_np[g]) == gt):
            mismatch += 1
    if mismatch:
        raise RuntimeError(f"{mismatch} graphs differ between the batched and the per-graph solves")
    base.close()
    launches = sum(v[0] for v in stats.values())
    if compact:
        solver.close()
        return {"metric": "batched graphs/s (one mst_solve_batched call per step)", "value": value,
                "unit": "graphs/s", "steps": args.steps, "ms_per_step": total_s * 1e3 / args.steps,
                "config": {"workload": "batched", "graphs": G, "n_total": n_tot, "m_total": m_tot,
                           "mix": f"n log-uniform [2^8,2^{args.log_hi}]; 1/3 GNM deg 4-32, 1/3 RGG2D deg 8, "
                                  "1/3 RMAT deg 16; w in [1,255]", "autotuned": best,
                           "autotune_trials_s": {k: v for k, v in tuning}},
                "latency_ms": {k: v * 1e3 for k, v in percentiles(lat).items()},
                "edges_per_s": m_tot * args.steps * world / total_s,
                "one_launch_per_graph": {"value": base_value, "unit": "graphs/s", "variant": "boruvka",
                                         "latency_ms": {k: v * 1e3 for k, v in percentiles(per).items()},
                                         "batched_over_per_graph": value / world / base_value},
                "gpu_launches": launches, "forests": "every batched forest equals the graph solved alone"}

    # end to end: pinned host batch -> device, solve, forests back to pinned
    # host memory.  Two device input sets: batch k+1 is copied on its own
    # stream while batch k is solved.
    pin = [torch.from_numpy(a.view(np.int32)).pin_memory() for a in (b.src, b.dst, b.w)]
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    copy_s, solve_s = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    sets = [[torch.empty(m_tot, dtype=torch.int32, device=dev) for _ in range(3)] for _ in range(2)]
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_free = [torch.cuda.Event() for _ in range(2)]
    ids_pin = torch.empty(max(1, int(ids.numel())), dtype=torch.int32).pin_memory()
    off_pin = torch.empty(G + 1, dtype=torch.int64).pin_memory()
    tot_pin = torch.empty(max(G, 1), dtype=torch.int64).pin_memory()

    def e2e_run(steps):
        torch.cuda.synchronize(dev)
        for e in ev_free:
            e.record(solve_s)

        def copy_in(k):
            with torch.cuda.stream(copy_s):
                copy_s.wait_event(ev_free[k % 2])
                for d_t, h_t in zip(sets[k % 2], pin):
                    d_t.copy_(h_t, non_blocking=True)
                ev_in[k % 2].record(copy_s)

        copy_in(0)
        nbytes = 0
        for k in range(steps):
            if k + 1 < steps:
                copy_in(k + 1)
            solve_s.wait_event(ev_in[k % 2])
            with torch.cuda.stream(solve_s):
                r_ids, r_off, r_tot = solver.solve_batched(d_n, d_off, *sets[k % 2], stream=solve_s, capacity=n_tot)
                ev_free[k % 2].record(solve_s)
                off_pin.copy_(r_off, non_blocking=True)
                tot_pin.copy_(r_tot[:G], non_blocking=True)
                solve_s.synchronize()
                used = int(off_pin[-1])
                ids_pin[:used].copy_(r_ids[:used], non_blocking=True)
                solve_s.synchronize()
            nbytes = used * 4 + (G + 1) * 8 + G * 8
        torch.cuda.synchronize(dev)
        return nbytes

    e2e_run(2)
    used_ids = int(moff[-1])
    if not (torch.equal(off_pin, moff) and torch.equal(tot_pin[:G], tot[:G])
            and torch.equal(ids_pin[:used_ids], ids[:used_ids])):
        raise RuntimeError("the end-to-end batches returned different forests")
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    d2h = e2e_run(e2e_steps)
    e2e_value, _ = job_rate(G * e2e_steps, time.perf_counter() - t0, world, dist, dev)
    e2e = {"value": e2e_value, "unit": "graphs/s", "h2d_bytes_per_step": 12 * m_tot,
           "d2h_bytes_per_step": d2h, "steps": e2e_steps,
           "api": "mst_solve_batched on device buffers; batch k+1's input copy overlaps batch k's solve"}

    peaks = measured_peaks()
    kernels, all_bytes = {}, 0.0
    for name, (nl, kms, kbytes) in stats.items():
        all_bytes += kbytes
    for name, (nl, kms, kbytes) in stats_all.items():
        if nl:
            kernels[name] = {"launches_per_step": nl / prof_steps, "ms_per_step": kms / prof_steps,
                             "bytes_per_step": kbytes / prof_steps,
                             "GBps": (kbytes / (kms / 1e3) / 1e9) if kms > 0 else None}
    nl, kms, kbytes = stats[dom]
    achieved = kbytes / (kms / 1e3) / 1e9
    ms = total_s * 1e3
    line = {
        "metric": "batched graphs/s (one mst_solve_batched call per step)", "value": value, "unit": "graphs/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "batched", "graphs": G, "n_total": n_tot, "m_total": m_tot,
                   "mix": f"n log-uniform [2^8,2^{args.log_hi}]; 1/3 GNM deg 4-32, 1/3 RGG2D deg 8, "
                          "1/3 RMAT deg 16; w in [1,255]",
                   "autotuned": best, "autotune_trials_s": {k: v for k, v in tuning},
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "inputs (12 B/edge) larger than L2, no flush"},
        "latency_ms": {k: v * 1e3 for k, v in percentiles(lat).items()},
        "edges_per_s": m_tot * args.steps * world / total_s,
        "one_launch_per_graph": {"value": base_value, "unit": "graphs/s", "variant": "boruvka",
                                 "latency_ms": {k: v * 1e3 for k, v in percentiles(per).items()},
                                 "batched_over_per_graph": value / world / base_value},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "peak_source": peaks["source"], "traffic": None,
                     "time_share": kms / ms if ms > 0 else None},
        "effective_bw": {"GBps": all_bytes / total_s / 1e9, "frac": all_bytes / total_s / 1e9 / peaks["hbm_gbs"]},
        "kernels": kernels,
        "kernels_note": f"per-class CUDA-event times of {prof_steps} profiled batches outside the timed region; "
                        "inside it only the dominant class is timed",
        "gpu_launches": launches,
        "host": host,
        "e2e": e2e,
        "clocks": clocks,
    }
    solver.close()
    return line


def served_main(args, rank: int, world: int, local_rank: int):
    """The served configuration: Poisson arrivals of mixed graphs (n log-uniform
    in [2^8, 2^20], families as in the batched mix) at each offered rate,
    served by the continuous-batching loop of paper_2302_12199_gb300.serve;
    graphs/s and latency percentiles per rate, every response compared with the
    same graph solved alone."""
    import numpy as np
    import torch

    from paper_2302_12199_gb300 import workloads as W
    from paper_2302_12199_gb300.serve import PoolGraph, Server, poisson_arrivals

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    b = W.mix(args.pool, W.DEFAULT_SEED + 5 + rank, log_lo=8, log_hi=20)
    off = np.asarray(b.edge_off, dtype=np.int64)
    to_dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev)
    pool = [PoolGraph(int(b.n[g]), to_dev(b.src[off[g]:off[g + 1]]), to_dev(b.dst[off[g]:off[g + 1]]),
                      to_dev(b.w[off[g]:off[g + 1]])) for g in range(args.pool)]
    scfg = dict(variant="filter", dedupe="none", tile_contract=0)
    if args.base_case is not None:
        scfg["base_case"] = args.base_case
    if args.graph_rounds is not None:
        scfg["graph_rounds"] = args.graph_rounds
    server = Server(local_rank, slots=args.slots, budget_bytes=int(args.slot_budget_gb * (1 << 30)), config=scfg)
    t_pre = time.perf_counter()
    expected = {g: server.solve_alone(pool[g]) for g in range(args.pool)}  # each graph solved alone
    t_pre = time.perf_counter() - t_pre
    verified = 0
    if args.verify_oracle:  # tie the pre-computed answers to the CPU oracle on a sample of the pool
        import oracle
        for g in range(min(args.verify_oracle, args.pool)):
            lo, hi = off[g], off[g + 1]
            kid, ktot = oracle.kruskal(int(b.n[g]), b.src[lo:hi], b.dst[lo:hi], b.w[lo:hi])
            if not (np.array_equal(kid, expected[g].ids) and ktot == expected[g].total):
                raise RuntimeError(f"pool graph {g}: the GPU's answer differs from Kruskal")
            verified += 1
    for s in server.slots:  # warm every slot
        s.solve(pool[:8])
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    sampler.start()
    time.sleep(0.3)
    rng = np.random.default_rng(77 + rank)
    per_rate = []
    for lg in args.rates:
        rate = float(1 << lg)
        seconds = min(args.serve_seconds, args.max_requests / rate)
        arr = poisson_arrivals(rate, seconds, seed=1000 + lg)
        picks = rng.integers(0, args.pool, arr.size)
        st = server.run(pool, picks, arr, expected=expected, rate=rate, seconds=seconds)
        if st.mismatches:
            raise RuntimeError(f"{st.mismatches} served responses differ from the graphs solved alone")
        per_rate.append(st.summary())
    # end to end: the same request stream at the best rate with the payloads
    # in page-locked host memory (every batch copies its graphs in), every
    # response compared with the graph solved alone
    best = max(per_rate, key=lambda r: r["graphs_per_s"])
    to_pin = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).pin_memory()
    e2e_pool = min(args.pool, args.e2e_pool) if args.e2e_pool else args.pool
    host_pool = [PoolGraph(int(b.n[g]), to_pin(b.src[off[g]:off[g + 1]]), to_pin(b.dst[off[g]:off[g + 1]]),
                           to_pin(b.w[off[g]:off[g + 1]])) for g in range(e2e_pool)]
    rate = best["rate"]
    seconds = min(args.serve_seconds, (args.e2e_max_requests or args.max_requests) / rate)
    arr = poisson_arrivals(rate, seconds, seed=2000)
    picks = rng.integers(0, e2e_pool, arr.size)
    st = server.run(host_pool, picks, arr, expected=expected, rate=rate, seconds=seconds)
    if st.mismatches:
        raise RuntimeError(f"{st.mismatches} end-to-end responses differ from the graphs solved alone")
    e2e_sum = st.summary()
    sizes = np.diff(off)
    e2e = {"value": e2e_sum["graphs_per_s"], "unit": "graphs/s",
           "h2d_bytes_per_step": float(12 * np.mean(sizes[picks])),
           "d2h_bytes_per_step": float(np.mean([4 * expected[int(p)].ids.size + 8 for p in picks])),
           "step": "one request", "rate": rate, "latency_ms": e2e_sum["latency_ms"],
           "payloads": f"page-locked host memory, copied in per batch (the first {e2e_pool} pool graphs)"}
    clocks = sampler.stop()
    server.close()
    line = {
        "metric": "served graphs/s (Poisson arrivals, continuous batching)", "value": best["graphs_per_s"],
        "unit": "graphs/s", "n_gpus": world, "steps": len(per_rate), "warmup": 1,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": "served", "pool_graphs": args.pool, "pool_mean_n": float(np.mean(b.n)),
                   "pool_mean_m": float(np.mean(sizes)),
                   "mix": "n log-uniform [2^8,2^20]; 1/3 GNM deg 4-32, 1/3 RGG2D deg 8, 1/3 RMAT deg 16; w in [1,255]",
                   "slots": args.slots, "slot_budget_gb": args.slot_budget_gb,
                   "payloads": "device-resident request pool, gathered per batch",
                   "pool_answers": f"every pool graph solved alone first ({t_pre:.1f} s); "
                                   f"{verified} of them checked against the CPU oracle (Kruskal)"},
        "rates": per_rate,
        "latency_ms_at_best": best["latency_ms"],
        "clocks": clocks,
        "e2e": e2e,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="rmat_filter", choices=sorted(WORKLOADS) + ["batched", "served"])
    ap.add_argument("--graphs", type=int, default=4096, help="graphs per batch (--workload batched)")
    ap.add_argument("--no-autotune", action="store_true", help="batched: skip the configuration autotuner")
    ap.add_argument("--log-hi", type=int, default=16, help="batched: graphs have n log-uniform in [2^8, 2^log_hi]")
    ap.add_argument("--pool", type=int, default=256, help="served: distinct request graphs")
    ap.add_argument("--slots", type=int, default=3, help="served: solver slots (batches in flight)")
    ap.add_argument("--slot-budget-gb", type=float, default=6.0, help="served: device memory per slot's batch")
    ap.add_argument("--rates", type=lambda t: [int(x) for x in t.split(",")], default=[12, 13, 14, 15, 16],
                    help="served: log2 of the offered arrival rates (requests/s)")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="served: arrival window per rate")
    ap.add_argument("--max-requests", type=int, default=20000, help="served: cap on requests per rate")
    ap.add_argument("--e2e-pool", type=int, default=0,
                    help="served: graphs of the pool copied to page-locked host memory for the e2e leg (0: all)")
    ap.add_argument("--e2e-max-requests", type=int, default=0,
                    help="served: cap on requests of the e2e leg (0: --max-requests)")
    ap.add_argument("--verify-oracle", type=int, default=0,
                    help="served: pool graphs whose pre-computed answer is checked against Kruskal")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-sample-edges", type=int, default=1 << 25)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="default workload: skip the batched sub-record (4096 mixed graphs)")
    ap.add_argument("--batched-steps", type=int, default=20, help="timed batches of the batched sub-record")
    ap.add_argument("--variant", default=None, choices=["boruvka", "filter", "auto"],
                    help="override the workload's solver variant")
    ap.add_argument("--dedupe", default=None, choices=["auto", "sort", "hash", "none"])
    ap.add_argument("--filter-max-avg-degree", type=float, default=None)
    ap.add_argument("--filter-min-edges", type=int, default=None)
    ap.add_argument("--tile-contract", type=int, default=None, choices=[-1, 0, 1])
    ap.add_argument("--tile-vertices", type=int, default=None)
    ap.add_argument("--base-case", type=int, default=None, choices=[0, 1])
    ap.add_argument("--graph-rounds", type=int, default=None, choices=[0, 1])
    ap.add_argument("--filter-carry", type=int, default=None, choices=[0, 1])
    ap.add_argument("--filter-split", type=int, default=None, choices=[0, 1])
    ap.add_argument("--min-edges-sort", type=int, default=None, choices=[0, 1])
    ap.add_argument("--tile-filter", type=int, default=None, choices=[0, 1])
    ap.add_argument("--filter-plan", type=int, default=None, choices=[0, 1])
    ap.add_argument("--pivot-quantile", type=float, default=None,
                    help="Filter-Borůvka: pivot rank in its sample as a fraction (0.5 = the sample median)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gpu":
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_main(args, rank)
    if args.workload == "batched":
        return batched_main(args, rank, world, local_rank)
    if args.workload == "served":
        return served_main(args, rank, world, local_rank)
    return gpu_main(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
