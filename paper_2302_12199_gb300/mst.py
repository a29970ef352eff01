"""Python binding of libmstgpu (include/mst.h): argument marshalling only.

Every step of the solver runs in the CUDA library; this module only turns
torch tensors into device pointers and sizes, passes the current CUDA stream,
and maps status codes to exceptions.  There is no CPU fallback: if the library
is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import build as _build

_lib = None

MST_OK = 0
MST_ERR_CUDA = 5
STATUS_NAMES = {0: "MST_OK", 1: "MST_ERR_INVALID_ARG", 2: "MST_ERR_VERTEX_RANGE", 3: "MST_ERR_TOO_LARGE",
                4: "MST_ERR_OOM", 5: "MST_ERR_CUDA", 6: "MST_ERR_INTERNAL", 7: "MST_ERR_NOT_SUPPORTED"}
VARIANTS = {"boruvka": 0, "filter": 1, "auto": 2}
DEDUPE = {"auto": 0, "sort": 1, "hash": 2, "none": 3}
KEY_INF = 0xFFFFFFFFFFFFFFFF


class MstError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}")


KERNEL_CLASSES = ["min_edges", "relabel_min", "hook", "jump", "dedupe", "pivot", "partition", "filter", "finalize",
                  "tile", "base", "graph"]


class HostGraph(ctypes.Structure):
    """mst_host_graph: one graph in host memory for mst_solve_host_many."""
    _fields_ = [("n", ctypes.c_uint32), ("m", ctypes.c_uint64), ("src", ctypes.c_void_p), ("dst", ctypes.c_void_p),
                ("w", ctypes.c_void_p), ("msf_ids", ctypes.c_void_p), ("msf_count", ctypes.c_uint32),
                ("total_weight", ctypes.c_uint64), ("status", ctypes.c_int)]


class KernelStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("ms", ctypes.c_double), ("bytes", ctypes.c_double),
                ("min_bytes", ctypes.c_double)]


class HostCounters(ctypes.Structure):
    _fields_ = [("solves", ctypes.c_uint64), ("readbacks", ctypes.c_uint64), ("planned", ctypes.c_uint64),
                ("plan_fallbacks", ctypes.c_uint64)]


class MstConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("variant", ctypes.c_int), ("dedupe", ctypes.c_int),
                ("tile_contract", ctypes.c_int), ("tile_vertices", ctypes.c_uint32),
                ("pivot_sample", ctypes.c_uint32), ("seed", ctypes.c_uint64), ("filter_min_edges", ctypes.c_uint64),
                ("filter_max_avg_degree", ctypes.c_float), ("base_case", ctypes.c_int),
                ("graph_rounds", ctypes.c_int), ("graph_jump_launches", ctypes.c_int),
                ("filter_carry", ctypes.c_int), ("filter_split", ctypes.c_int),
                ("min_edges_sort", ctypes.c_int), ("jump_steps", ctypes.c_uint32),
                ("tile_filter", ctypes.c_int), ("spin_limit", ctypes.c_uint32),
                ("block_threads", ctypes.c_uint32), ("items_per_thread", ctypes.c_uint32),
                ("filter_plan", ctypes.c_int), ("relabel_block_threads", ctypes.c_uint32),
                ("relabel_items_per_thread", ctypes.c_uint32), ("pivot_quantile", ctypes.c_float)]


_P = ctypes.c_void_p
_U32, _U64, _I = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int

_SIGNATURES = {
    "mst_config_default": (None, [ctypes.POINTER(MstConfig)]),
    "mst_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(MstConfig)]),
    "mst_destroy": (None, [_P]),
    "mst_set_config": (_I, [_P, ctypes.POINTER(MstConfig)]),
    "mst_status_string": (ctypes.c_char_p, [_I]),
    "mst_get_error": (_I, [_P, _P]),
    "mst_last_cuda_error": (_I, [_P, _P]),
    "mst_workspace_bytes": (_U64, [_U32, _U64, ctypes.POINTER(MstConfig)]),
    "mst_solve": (_I, [_P, _U32, _U64, _P, _P, _P, _P, _P, _P, _P]),
    "mst_solve_host": (_I, [_P, _U32, _U64, _P, _P, _P, _P, _P, _P, _P]),
    "mst_solve_batched": (_I, [_P, _U32, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "mst_solve_host_many": (_I, [_P, _U32, _P, _P]),
    "mst_step_min_edges": (_I, [_P, _U32, _U64, _P, _P, _P, _P, _P, _P]),
    "mst_step_contract": (_I, [_P, _U32, _U64, _P, _P, _P, _P, _P, _P, _P]),
    "mst_step_relabel": (_I, [_P, _U32, _U64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "mst_step_dedupe": (_I, [_P, _U64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "mst_step_pivot": (_I, [_P, _U64, _P, _P, _U64, _U32, _P, _P]),
    "mst_step_partition": (_I, [_P, _U64, _P, _P, _P, _P, _U64, _P, _P, _P, _P, _P, _P]),
    "mst_step_filter": (_I, [_P, _U32, _U64, _P, _P, _P, _P, _U64, _P, _P, _P, _P, _P, _P, _P]),
    "mst_step_finalize": (_I, [_P, _U64, _P, _P, _P, _P, _P, _P]),
    "mst_step_tile_contract": (_I, [_P, _U32, _U64, _P, _P, _P, _U32, _P, _P, _P]),
    "mst_profile_enable": (_I, [_P, _I]),
    "mst_profile_classes": (_I, [_P, _U32]),
    "mst_profile_get": (_I, [_P, _I, ctypes.POINTER(KernelStats)]),
    "mst_host_counters_get": (_I, [_P, ctypes.POINTER(HostCounters)]),
    "mst_pivot_noalloc": (_I, [_U64, _P, _P, _U64, _U32, _P, _P]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libmstgpu.so (building it with nvcc first if it is missing)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libmstgpu.so is not built ({path})")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _check(st: int, where: str, lib=None, h=None):
    if st != MST_OK:
        if st == MST_ERR_CUDA and lib is not None and h:
            line = ctypes.c_int(0)
            code = lib.mst_last_cuda_error(h, ctypes.byref(line))
            where = f"{where} (cudaError {code} at solver.cu:{line.value})"
        raise MstError(st, where)


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _u32(t: torch.Tensor, name: str, device: torch.device) -> torch.Tensor:
    if t.dtype not in (torch.int32, torch.uint32):
        raise TypeError(f"{name} must be int32/uint32, got {t.dtype}")
    if t.device != device:
        raise ValueError(f"{name} must be on {device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def default_config(**kw) -> MstConfig:
    cfg = MstConfig()
    load().mst_config_default(ctypes.byref(cfg))
    for k, v in kw.items():
        if k == "variant":
            v = VARIANTS[v] if isinstance(v, str) else v
        elif k == "dedupe":
            v = DEDUPE[v] if isinstance(v, str) else v
        setattr(cfg, k, v)
    return cfg


@dataclass
class Forest:
    ids: torch.Tensor  # int32 device tensor with capacity >= count (ids ascending)
    count: torch.Tensor  # int32[1] device
    total: torch.Tensor  # int64[1] device (uint64 bit pattern)

    def to_host(self):
        """(ascending ids as a numpy uint32 array, total weight as int)."""
        k = int(self.count.item())
        ids = self.ids[:k].cpu().numpy().view("uint32").copy()
        return ids, int(self.total.item()) & 0xFFFFFFFFFFFFFFFF


class Solver:
    """A handle on one GPU (mst_create / mst_destroy)."""

    def __init__(self, device: int = 0, **config):
        self.lib = load()
        self.device = torch.device("cuda", device)
        self.cfg = default_config(device=device, **config)
        h = ctypes.c_void_p()
        _check(self.lib.mst_create(ctypes.byref(h), ctypes.byref(self.cfg)), "mst_create")
        self.h = h

    def _check(self, st: int, where: str):
        _check(st, where, self.lib, self.h)

    def close(self):
        if getattr(self, "h", None):
            self.lib.mst_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def configure(self, **kw):
        for k, v in kw.items():
            if k == "variant":
                v = VARIANTS[v] if isinstance(v, str) else v
            elif k == "dedupe":
                v = DEDUPE[v] if isinstance(v, str) else v
            setattr(self.cfg, k, v)
        self._check(self.lib.mst_set_config(self.h, ctypes.byref(self.cfg)), "mst_set_config")

    def profile(self, enable: bool = True, classes=None):
        """Start (and clear) or stop per-kernel-class statistics.  `classes`
        (names from KERNEL_CLASSES; None = all) are timed with CUDA events; the
        others only count launches and algorithmic bytes."""
        mask = 0xFFFFFFFF if classes is None else sum(1 << KERNEL_CLASSES.index(c) for c in classes)
        self._check(self.lib.mst_profile_classes(self.h, mask), "mst_profile_classes")
        self._check(self.lib.mst_profile_enable(self.h, 1 if enable else 0), "mst_profile_enable")

    def profile_stats(self, with_min: bool = False) -> dict:
        """{class: (launches, ms, algorithmic bytes)} since profiling was enabled;
        with_min adds the method's own byte count as a fourth entry."""
        out = {}
        for k, name in enumerate(KERNEL_CLASSES):
            st = KernelStats()
            self._check(self.lib.mst_profile_get(self.h, k, ctypes.byref(st)), "mst_profile_get")
            out[name] = (int(st.launches), float(st.ms), float(st.bytes)) + ((float(st.min_bytes),) if with_min else ())
        return out

    def host_counters(self) -> dict:
        """mst_host_counters_get: solves, readbacks, planned, plan_fallbacks since the handle was made."""
        hc = HostCounters()
        self._check(self.lib.mst_host_counters_get(self.h, ctypes.byref(hc)), "mst_host_counters_get")
        return {k: int(getattr(hc, k)) for k, _ in HostCounters._fields_}

    def workspace_bytes(self, n: int, m: int) -> int:
        return int(self.lib.mst_workspace_bytes(n, m, ctypes.byref(self.cfg)))

    # ----------------------------------------------------------- solves
    def solve(self, n: int, src: torch.Tensor, dst: torch.Tensor, w: torch.Tensor, out: Forest | None = None,
              stream=None) -> Forest:
        """mst_solve on device tensors; returns device tensors."""
        m = src.numel()
        for t, name in ((src, "src"), (dst, "dst"), (w, "w")):
            _u32(t, name, self.device)
            if t.numel() != m:
                raise ValueError("src, dst and w must have equal length")
        if out is None:
            out = self.alloc_forest(n, m)
        self._check(self.lib.mst_solve(self.h, n, m, _ptr(src), _ptr(dst), _ptr(w), _ptr(out.ids), _ptr(out.count),
                                  _ptr(out.total), _stream(stream)), "mst_solve")
        return out

    def alloc_forest(self, n: int, m: int) -> Forest:
        cap = max(1, min(m, max(n - 1, 0)))
        return Forest(torch.empty(cap, dtype=torch.int32, device=self.device),
                      torch.zeros(1, dtype=torch.int32, device=self.device),
                      torch.zeros(1, dtype=torch.int64, device=self.device))

    def solve_host(self, n: int, src, dst, w, stream=None):
        """mst_solve_host on host (numpy or CPU tensor) arrays: returns (ids, total)."""
        import numpy as np
        src = np.ascontiguousarray(src, dtype=np.uint32)
        dst = np.ascontiguousarray(dst, dtype=np.uint32)
        w = np.ascontiguousarray(w, dtype=np.uint32)
        m = src.size
        cap = max(1, min(m, max(n - 1, 0)))
        ids = np.empty(cap, dtype=np.uint32)
        cnt = ctypes.c_uint32(0)
        tot = ctypes.c_uint64(0)
        self._check(self.lib.mst_solve_host(self.h, n, m, src.ctypes.data_as(_P), dst.ctypes.data_as(_P),
                                       w.ctypes.data_as(_P), ids.ctypes.data_as(_P), ctypes.byref(cnt),
                                       ctypes.byref(tot), _stream(stream)), "mst_solve_host")
        return ids[: cnt.value].copy(), int(tot.value)

    def solve_host_ptr(self, n: int, m: int, src_ptr: int, dst_ptr: int, w_ptr: int, ids_ptr: int, stream=None):
        """mst_solve_host on raw host pointers (e.g. pinned tensors): returns (count, total)."""
        cnt = ctypes.c_uint32(0)
        tot = ctypes.c_uint64(0)
        self._check(self.lib.mst_solve_host(self.h, n, m, _P(src_ptr), _P(dst_ptr), _P(w_ptr), _P(ids_ptr),
                                       ctypes.byref(cnt), ctypes.byref(tot), _stream(stream)), "mst_solve_host")
        return int(cnt.value), int(tot.value)

    def solve_host_many_ptr(self, graphs, stream=None):
        """mst_solve_host_many on raw host pointers: graphs is a sequence of
        (n, m, src_ptr, dst_ptr, w_ptr, ids_ptr); returns [(count, total)].
        Graph i+1's inputs are copied while graph i is solved."""
        arr = (HostGraph * max(1, len(graphs)))()
        for i, (n, m, s_p, d_p, w_p, i_p) in enumerate(graphs):
            arr[i] = HostGraph(n, m, s_p, d_p, w_p, i_p, 0, 0, 0)
        st = self.lib.mst_solve_host_many(self.h, len(graphs), ctypes.cast(arr, _P), _stream(stream))
        bad = [(i, arr[i].status) for i in range(len(graphs)) if arr[i].status != MST_OK]
        if st != MST_OK or bad:
            self._check(st if st != MST_OK else bad[0][1], f"mst_solve_host_many (graph {bad[0][0] if bad else '?'})")
        return [(int(arr[i].msf_count), int(arr[i].total_weight)) for i in range(len(graphs))]

    def solve_host_many(self, graphs, stream=None):
        """mst_solve_host_many on host arrays: graphs is a sequence of (n, src,
        dst, w); returns [(ids, total)] (ascending ids)."""
        import numpy as np
        keep, spec, outs = [], [], []
        for n, src, dst, w in graphs:
            arrs = [np.ascontiguousarray(a, dtype=np.uint32) for a in (src, dst, w)]
            m = arrs[0].size
            ids = np.empty(max(1, min(m, max(n - 1, 0))), dtype=np.uint32)
            keep.append(arrs)
            outs.append(ids)
            spec.append((n, m, *(a.ctypes.data for a in arrs), ids.ctypes.data))
        res = self.solve_host_many_ptr(spec, stream)
        return [(outs[i][:cnt].copy(), tot) for i, (cnt, tot) in enumerate(res)]

    def solve_batched(self, n_per_graph, edge_off, src: torch.Tensor, dst: torch.Tensor, w: torch.Tensor,
                      stream=None, capacity: int | None = None):
        """mst_solve_batched: returns (ids, msf_off, totals) device tensors; segment g of ids holds
        graph-local edge ids.  The size tables may be host arrays (copied to the device here) or
        device tensors (uint32/int32 vertex counts, uint64/int64 edge offsets).  `capacity`: the
        total vertex count when the caller knows it (otherwise it is summed from the table)."""
        import numpy as np
        m = src.numel()
        for t, name in ((src, "src"), (dst, "dst"), (w, "w")):
            _u32(t, name, self.device)
        if isinstance(n_per_graph, torch.Tensor) and n_per_graph.is_cuda:
            d_n = n_per_graph.contiguous()
            G = d_n.numel()
            n_total = int(capacity) if capacity is not None else int(d_n.to(torch.int64).sum().item())
        else:
            n_h = np.ascontiguousarray(n_per_graph, dtype=np.uint32)
            G = n_h.size
            n_total = int(capacity) if capacity is not None else int(n_h.astype(np.int64).sum())
            d_n = torch.from_numpy(n_h.view(np.int32)).to(self.device)
        if isinstance(edge_off, torch.Tensor) and edge_off.is_cuda:
            d_off = edge_off.contiguous()
        else:
            d_off = torch.from_numpy(np.ascontiguousarray(edge_off, dtype=np.uint64).view(np.int64)).to(self.device)
        if d_n.dtype not in (torch.int32, torch.uint32) or d_off.dtype not in (torch.int64, torch.uint64):
            raise TypeError("vertex counts must be 32-bit and edge offsets 64-bit integers")
        if d_off.numel() != G + 1:
            raise ValueError("edge_off needs num_graphs + 1 entries")
        cap = max(1, min(m, n_total))
        ids = torch.empty(cap, dtype=torch.int32, device=self.device)
        msf_off = torch.zeros(G + 1, dtype=torch.int64, device=self.device)
        totals = torch.zeros(max(G, 1), dtype=torch.int64, device=self.device)
        if stream is not None:  # the tables were copied on the current stream
            stream.wait_stream(torch.cuda.current_stream(self.device))
        self._check(self.lib.mst_solve_batched(self.h, G, _ptr(d_n), _ptr(d_off), _ptr(src), _ptr(dst), _ptr(w),
                                               _ptr(ids), _ptr(msf_off), _ptr(totals), _stream(stream)),
                    "mst_solve_batched")
        return ids, msf_off, totals

    def get_error(self, stream=None) -> int:
        """mst_get_error: waits for the stream and returns the handle's status code."""
        return int(self.lib.mst_get_error(self.h, _stream(stream)))

    # ----------------------------------------------------------- steps
    def _list(self, u, v, w, ids):
        m = u.numel()
        for t, name in ((u, "u"), (v, "v"), (w, "w")):
            _u32(t, name, self.device)
            if t.numel() != m:
                raise ValueError("edge arrays must have equal length")
        if ids is not None:
            _u32(ids, "id", self.device)
        return m

    def _outlist(self, m):
        return [torch.empty(max(m, 1), dtype=torch.int32, device=self.device) for _ in range(4)], \
            torch.zeros(1, dtype=torch.int64, device=self.device)

    def min_edges(self, n, u, v, w, ids=None, stream=None) -> torch.Tensor:
        m = self._list(u, v, w, ids)
        best = torch.empty(max(n, 1), dtype=torch.int64, device=self.device)
        self._check(self.lib.mst_step_min_edges(self.h, n, m, _ptr(u), _ptr(v), _ptr(w), _ptr(ids), _ptr(best),
                                           _stream(stream)), "mst_step_min_edges")
        return best[:n]

    def contract(self, n, u, v, w, ids=None, id_bound=None, stream=None):
        m = self._list(u, v, w, ids)
        parent = torch.empty(max(n, 1), dtype=torch.int32, device=self.device)
        nbits = (id_bound if id_bound is not None else m) + 1
        chosen = torch.zeros((nbits + 31) // 32, dtype=torch.int32, device=self.device)
        self._check(self.lib.mst_step_contract(self.h, n, m, _ptr(u), _ptr(v), _ptr(w), _ptr(ids), _ptr(parent),
                                          _ptr(chosen), _stream(stream)), "mst_step_contract")
        return parent[:n], chosen

    def relabel(self, n, u, v, w, ids, label, stream=None):
        m = self._list(u, v, w, ids)
        (ou, ov, ow, oi), cnt = self._outlist(m)
        self._check(self.lib.mst_step_relabel(self.h, n, m, _ptr(u), _ptr(v), _ptr(w), _ptr(ids), _ptr(label), _ptr(ou),
                                         _ptr(ov), _ptr(ow), _ptr(oi), _ptr(cnt), _stream(stream)),
               "mst_step_relabel")
        k = int(cnt.item())
        return ou[:k], ov[:k], ow[:k], oi[:k]

    def dedupe(self, u, v, w, ids, stream=None):
        m = self._list(u, v, w, ids)
        (ou, ov, ow, oi), cnt = self._outlist(m)
        self._check(self.lib.mst_step_dedupe(self.h, m, _ptr(u), _ptr(v), _ptr(w), _ptr(ids), _ptr(ou), _ptr(ov),
                                        _ptr(ow), _ptr(oi), _ptr(cnt), _stream(stream)), "mst_step_dedupe")
        k = int(cnt.item())
        return ou[:k], ov[:k], ow[:k], oi[:k]

    def pivot(self, w, ids, state: int, sample: int, stream=None) -> int:
        m = w.numel()
        out = torch.zeros(1, dtype=torch.int64, device=self.device)
        self._check(self.lib.mst_step_pivot(self.h, m, _ptr(w), _ptr(ids), state, sample, _ptr(out), _stream(stream)),
               "mst_step_pivot")
        return int(out.item()) & 0xFFFFFFFFFFFFFFFF

    def partition(self, u, v, w, ids, pivot: int, stream=None):
        m = self._list(u, v, w, ids)
        (ou, ov, ow, oi), cnt = self._outlist(m)
        self._check(self.lib.mst_step_partition(self.h, m, _ptr(u), _ptr(v), _ptr(w), _ptr(ids), pivot, _ptr(ou),
                                           _ptr(ov), _ptr(ow), _ptr(oi), _ptr(cnt), _stream(stream)),
               "mst_step_partition")
        k = int(cnt.item())
        return ou[:k], ov[:k], ow[:k], oi[:k]

    def filter(self, n, u, v, w, ids, pivot: int, P: torch.Tensor, stream=None):
        m = self._list(u, v, w, ids)
        (ou, ov, ow, oi), cnt = self._outlist(m)
        self._check(self.lib.mst_step_filter(self.h, n, m, _ptr(u), _ptr(v), _ptr(w), _ptr(ids), pivot, _ptr(P),
                                        _ptr(ou), _ptr(ov), _ptr(ow), _ptr(oi), _ptr(cnt), _stream(stream)),
               "mst_step_filter")
        k = int(cnt.item())
        return ou[:k], ov[:k], ow[:k], oi[:k]

    def tile_contract(self, n, src, dst, w, tile_vertices: int, stream=None):
        m = self._list(src, dst, w, None)
        parent = torch.empty(max(n, 1), dtype=torch.int32, device=self.device)
        chosen = torch.zeros((m + 32) // 32, dtype=torch.int32, device=self.device)
        self._check(self.lib.mst_step_tile_contract(self.h, n, m, _ptr(src), _ptr(dst), _ptr(w), tile_vertices,
                                               _ptr(parent), _ptr(chosen), _stream(stream)), "mst_step_tile_contract")
        return parent[:n], chosen

    def finalize(self, m, chosen, w, stream=None):
        ids = torch.empty(max(m, 1), dtype=torch.int32, device=self.device)
        cnt = torch.zeros(1, dtype=torch.int32, device=self.device)
        tot = torch.zeros(1, dtype=torch.int64, device=self.device)
        self._check(self.lib.mst_step_finalize(self.h, m, _ptr(chosen), _ptr(w), _ptr(ids), _ptr(cnt), _ptr(tot),
                                          _stream(stream)), "mst_step_finalize")
        return Forest(ids, cnt, tot)


def declared_symbols(header: str | None = None) -> list[str]:
    """Names of the functions declared in include/mst.h."""
    import re
    header = header or os.path.join(_build.INCLUDE, "mst.h")
    text = open(header).read()
    return sorted(set(re.findall(r"\b(mst_[a-z_]+)\s*\(", text)))
