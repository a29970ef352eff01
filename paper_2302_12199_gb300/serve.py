"""A request loop that serves minimum-spanning-forest requests on one GPU.

Requests (independent graphs of different sizes) arrive over time.  The loop
batches them as they arrive: whenever a solver slot is free it takes the
waiting requests, oldest first, up to a device-memory budget per slot
(admission by footprint, from mst_workspace_bytes plus the batch's own
arrays), and solves them with one mst_solve_batched call, in which all graphs
of the batch share every round's launches (the disjoint union of the graphs;
its MSF is the union of their MSFs, each the unique one under the graphs' own
(w, id) order).  Several slots, each with its own solver handle, CUDA stream
and host thread, keep batches in flight at once, so requests that arrive while
others run on the GPU start as soon as a slot and memory free up, and their
work overlaps on the device.

Host logic only: every step of a solve runs in the CUDA library.  Request
payloads are either resident in device memory (a pool of graphs standing in
for uploaded requests; a batch gathers its graphs' edges into the slot's
contiguous buffers with device-to-device copies) or in page-locked host
memory (a batch copies each graph's edges to the device on the slot's stream).
"""
from __future__ import annotations

import threading
import time
from collections import deque
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from .mst import Solver


@dataclass
class PoolGraph:
    """One request payload: an undirected multigraph on the device or in
    page-locked host memory."""
    n: int
    src: torch.Tensor  # int32 (uint32 bits), device or pinned host
    dst: torch.Tensor
    w: torch.Tensor

    @property
    def m(self) -> int:
        return int(self.src.numel())


@dataclass
class Response:
    ids: np.ndarray  # ascending graph-local MSF edge ids (uint32)
    total: int       # uint64 MSF weight


@dataclass
class ServeStats:
    rate: float                 # offered arrivals per second
    seconds: float              # arrival window
    requests: int               # requests served
    wall: float                 # first arrival to last completion, seconds
    latency: np.ndarray         # per request, seconds (completion - arrival)
    batches: int
    batch_sizes: List[int] = field(default_factory=list)
    max_in_flight: int = 0      # most batches on the device at once
    mismatches: int = 0         # responses that differ from the expected ones
    phases_ms: dict = field(default_factory=dict)  # mean host time per batch by phase
    done_in_window: int = 0     # requests answered before the arrival window (seconds) ended

    def summary(self) -> dict:
        lat = self.latency * 1e3
        pct = {f"p{q:g}": float(np.percentile(lat, q)) for q in (50, 99, 99.9)} if lat.size else {}
        return {"rate": self.rate, "seconds": self.seconds, "requests": self.requests,
                "graphs_per_s": self.requests / self.wall if self.wall > 0 else 0.0,
                "latency_ms": pct, "batches": self.batches,
                "mean_batch": float(np.mean(self.batch_sizes)) if self.batch_sizes else 0.0,
                "max_batches_in_flight": self.max_in_flight, "mismatches": self.mismatches,
                "batch_phases_ms": self.phases_ms,
                # past saturation the queue grows through the window and drains after it
                "answered_in_window": self.done_in_window,
                "drain_s": max(0.0, self.wall - self.seconds) if self.seconds > 0 else 0.0}


def poisson_arrivals(rate: float, seconds: float, seed: int) -> np.ndarray:
    """Arrival times (seconds from the start) of a Poisson process."""
    rng = np.random.default_rng(seed)
    n_exp = int(rate * seconds * 1.2) + 16
    t = np.cumsum(rng.exponential(1.0 / rate, n_exp))
    while t[-1] < seconds:
        t = np.concatenate([t, t[-1] + np.cumsum(rng.exponential(1.0 / rate, n_exp))])
    return t[t < seconds]


class _Slot:
    def __init__(self, device: int, config: dict):
        self.solver = Solver(device, **config)
        self.dev = self.solver.device
        self.stream = torch.cuda.Stream(device=self.dev)
        self.cap = 0
        self.bufs = None
        self.pinned = None
        self.phases = []  # (gather, solve, copy back) host seconds per batch
        self.busy = False
        self.job = None
        self.cv = threading.Condition()
        self.stop = False

    def ensure(self, m: int):
        if m > self.cap:
            cap = max(m, int(self.cap * 1.5), 1 << 16)
            with torch.cuda.stream(self.stream):
                self.bufs = [torch.empty(cap, dtype=torch.int32, device=self.dev) for _ in range(3)]
            self.cap = cap

    def solve(self, graphs: Sequence[PoolGraph]):
        m = sum(g.m for g in graphs)
        self.ensure(max(m, 1))
        n_per = np.array([g.n for g in graphs], dtype=np.uint32)
        off = np.zeros(len(graphs) + 1, dtype=np.uint64)
        np.cumsum([g.m for g in graphs], out=off[1:])
        src, dst, w = (b[:m] for b in self.bufs)
        t0 = time.perf_counter()
        with torch.cuda.stream(self.stream):
            if m and graphs[0].src.is_cuda:  # gather the batch: one concatenation per array
                torch.cat([g.src for g in graphs], out=src)
                torch.cat([g.dst for g in graphs], out=dst)
                torch.cat([g.w for g in graphs], out=w)
            elif m:  # host payloads: copy each graph's arrays in
                o = 0
                for g in graphs:
                    k = g.m
                    if k:
                        src[o:o + k].copy_(g.src, non_blocking=True)
                        dst[o:o + k].copy_(g.dst, non_blocking=True)
                        w[o:o + k].copy_(g.w, non_blocking=True)
                    o += k
            t1 = time.perf_counter()
            ids, moff, tot = self.solver.solve_batched(n_per, off, src, dst, w, stream=self.stream)
            t2 = time.perf_counter()
            moff_h = moff.cpu().numpy().astype(np.int64)
            k = int(moff_h[-1])  # copy back only the forests, through pinned memory
            if self.pinned is None or self.pinned.numel() < k:
                self.pinned = torch.empty(max(k, 1 << 16), dtype=torch.int32, pin_memory=True)
            self.pinned[:k].copy_(ids[:k], non_blocking=True)
            tot_h = tot.cpu().numpy().view(np.uint64)
        self.stream.synchronize()
        t3 = time.perf_counter()
        self.phases.append((t1 - t0, t2 - t1, t3 - t2))
        # the ids view stays valid until this slot's next solve
        return self.pinned[:k].numpy().view(np.uint32), moff_h, tot_h

    def workspace_bytes(self, n: int, m: int) -> int:
        return self.solver.workspace_bytes(n, m)

    def close(self):
        self.solver.close()


class Server:
    """Continuous-batching MSF server over `slots` solver slots.

    budget_bytes: device memory one slot's batch may occupy (scratch from
    mst_workspace_bytes plus the batch's input, union and output arrays).
    max_batch: most requests in one batch."""

    def __init__(self, device: int = 0, slots: int = 2, budget_bytes: int = 8 << 30, max_batch: int = 4096,
                 config: Optional[dict] = None, stall_seconds: float = 60.0, slot_factory=None):
        self.device = device
        self.stall_seconds = float(stall_seconds)
        self.config = dict(config or dict(variant="filter", dedupe="none", tile_contract=0))
        make = slot_factory or (lambda: _Slot(device, self.config))
        self.slots = [make() for _ in range(slots)]
        self.budget = int(budget_bytes)
        self.max_batch = int(max_batch)

    def footprint(self, g: PoolGraph) -> int:
        """Device bytes request g adds to a batch: solver scratch
        (mst_workspace_bytes) plus its input, union-id and output arrays."""
        scratch = self.slots[0].workspace_bytes(g.n, g.m)
        return scratch + 12 * g.m + 8 * g.m + 4 * max(g.n, 1) + 64

    def solve_alone(self, g: PoolGraph) -> Response:
        """One request by itself (a batch of one) on the first slot."""
        ids, moff, tot = self.slots[0].solve([g])
        return Response(np.sort(ids[moff[0]:moff[1]]), int(tot[0]))

    def run(self, pool: Sequence[PoolGraph], picks: np.ndarray, arrivals: np.ndarray,
            expected: Optional[Dict[int, Response]] = None, rate: float = 0.0,
            seconds: float = 0.0) -> ServeStats:
        """Serves request i = pool[picks[i]] arriving at arrivals[i] seconds after
        the start; returns latency and throughput statistics.  With `expected`
        (responses by pool index), every response is compared with it."""
        nreq = int(arrivals.size)
        foot = {int(p): self.footprint(pool[int(p)]) for p in np.unique(picks)}
        done_at = np.zeros(nreq)
        lock = threading.Lock()
        state = {"in_flight": 0, "max_in_flight": 0, "mismatches": 0, "batches": 0, "sizes": [], "error": None,
                 "verify": []}
        for slot in self.slots:
            if hasattr(slot, "phases"):
                slot.phases.clear()

        clock0 = [time.perf_counter()]

        def worker(slot: _Slot):
            if getattr(slot, "dev", None) is not None:
                torch.cuda.set_device(slot.dev)
            while True:
                with slot.cv:
                    while slot.job is None and not slot.stop:
                        slot.cv.wait()
                    if slot.stop and slot.job is None:
                        return
                    batch = slot.job
                try:
                    ids, moff, tot = slot.solve([pool[int(picks[i])] for i in batch])
                    t_done = time.perf_counter() - clock0[0]
                    tv = time.perf_counter()
                    bad = 0
                    if expected is not None:
                        for k, i in enumerate(batch):
                            e = expected[int(picks[i])]
                            got = ids[moff[k]:moff[k + 1]]  # segments come out ascending
                            if int(tot[k]) != e.total or not np.array_equal(got, e.ids):
                                bad += 1
                    with lock:
                        for i in batch:
                            done_at[i] = t_done
                        state["mismatches"] += bad
                        state["verify"].append(time.perf_counter() - tv)
                        state["in_flight"] -= 1
                except Exception as exc:  # surface the first failure to the scheduler
                    with lock:
                        state["error"] = exc
                        state["in_flight"] -= 1
                with slot.cv:
                    slot.job = None
                    slot.busy = False

        for slot in self.slots:  # a server runs many request streams in turn
            slot.stop, slot.job, slot.busy = False, None, False
        threads = [threading.Thread(target=worker, args=(s,), daemon=True) for s in self.slots]
        for t in threads:
            t.start()
        waiting: deque = deque()
        nxt = 0
        t0 = time.perf_counter()
        clock0[0] = t0
        last_progress, last_done = t0, 0
        try:
            while nxt < nreq or waiting or any(s.busy for s in self.slots):
                if state["error"] is not None:
                    raise state["error"]
                now = time.perf_counter() - t0
                done = state["batches"] - state["in_flight"]
                if done != last_done or nxt < nreq:
                    last_progress, last_done = time.perf_counter(), done
                elif time.perf_counter() - last_progress > self.stall_seconds:
                    raise RuntimeError(f"no batch finished for {self.stall_seconds} s")
                while nxt < nreq and arrivals[nxt] <= now:
                    waiting.append(nxt)
                    nxt += 1
                launched = False
                for slot in self.slots:
                    if not waiting:
                        break
                    if slot.busy:
                        continue
                    batch, used = [], 0
                    while waiting and len(batch) < self.max_batch:
                        f = foot[int(picks[waiting[0]])]
                        if batch and used + f > self.budget:
                            break
                        batch.append(waiting.popleft())
                        used += f
                    with lock:
                        state["in_flight"] += 1
                        state["max_in_flight"] = max(state["max_in_flight"], state["in_flight"])
                        state["batches"] += 1
                        state["sizes"].append(len(batch))
                    with slot.cv:
                        slot.busy = True
                        slot.job = batch
                        slot.cv.notify()
                    launched = True
                if not launched:
                    time.sleep(50e-6)
        finally:
            for slot in self.slots:
                with slot.cv:
                    slot.stop = True
                    slot.cv.notify()
            for t in threads:
                t.join(timeout=60)
        if state["error"] is not None:
            raise state["error"]
        latency = done_at - arrivals
        wall = float(done_at.max()) if nreq else 0.0
        ph = [p for slot in self.slots for p in getattr(slot, "phases", [])]
        phases_ms = {}
        if ph:
            a = np.asarray(ph) * 1e3
            phases_ms = {"gather": float(a[:, 0].mean()), "solve": float(a[:, 1].mean()),
                         "copy_back": float(a[:, 2].mean())}
        if state["verify"]:
            phases_ms["verify"] = float(np.mean(state["verify"]) * 1e3)
        return ServeStats(rate=rate, seconds=seconds, requests=nreq, wall=wall, latency=latency,
                          batches=state["batches"], batch_sizes=state["sizes"],
                          max_in_flight=state["max_in_flight"], mismatches=state["mismatches"],
                          phases_ms=phases_ms,
                          done_in_window=int((done_at <= seconds).sum()) if seconds > 0 else nreq)

    def close(self):
        for s in self.slots:
            s.close()
