"""CPU oracle for the minimum spanning forest -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU solver never imports, links or
calls it, and the two share no code: the oracle's C sources (``oracle.c``) and
numpy steps (``steps.py``) are written independently from the paper.

What it computes (paper Section 2.2): for an undirected weighted multigraph, a
minimum spanning tree of every connected component (a minimum spanning forest),
returned as ascending input-edge ids plus the uint64 total weight.  Ties are
broken by the strict total order (w, edge id) (Section 2.3: consistent tie
breaking makes the MST unique), so the forest is unique and every correct
method must return exactly this id set.

Parity status of each function is recorded in its docstring ("pinned by ...").
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import steps  # noqa: F401  (numpy step oracles)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into oracle/_build/liboracle.so."""
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp], check=True)
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        for name in ("oracle_kruskal", "oracle_prim"):
            f = getattr(lib, name)
            f.restype = ctypes.c_int
            f.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _u32p, _u32p, _u32p, _u32p, _u64p, _u64p]
        lib.oracle_kruskal_par.restype = ctypes.c_int
        lib.oracle_kruskal_par.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _u32p, _u32p, _u32p, ctypes.c_int,
                                           _u32p, _u64p, _u64p]
        lib.oracle_brute.restype = ctypes.c_int
        lib.oracle_brute.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _u32p, _u32p, _u32p, _u32p, _u64p, _u64p,
                                     _u64p]
        lib.oracle_check_msf.restype = ctypes.c_int
        lib.oracle_check_msf.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _u32p, _u32p, _u32p, _u32p,
                                         ctypes.c_uint64]
        _lib = lib
    return _lib


def _arr(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


def _p32(a: np.ndarray):
    return a.ctypes.data_as(_u32p)


_STATUS = {1: "vertex id out of range", 2: "graph too large for this routine", 3: "out of memory"}


def _run(fname: str, n: int, src, dst, w, cap: int):
    src, dst, w = _arr(src), _arr(dst), _arr(w)
    m = int(src.shape[0])
    out = np.empty(max(cap, 1), dtype=np.uint32)
    cnt = ctypes.c_uint64(0)
    tot = ctypes.c_uint64(0)
    rc = getattr(_load(), fname)(n, m, _p32(src), _p32(dst), _p32(w), _p32(out), ctypes.byref(cnt),
                                 ctypes.byref(tot))
    if rc != 0:
        raise OracleError(f"{fname}: {_STATUS.get(rc, rc)}")
    return out[: cnt.value].copy(), int(tot.value)


def kruskal(n: int, src, dst, w):
    """Kruskal's algorithm (edges in (w,id) order, union-find with path halving
    and union by size).  Returns (ascending MSF edge ids, uint64 total weight).
    Pinned by: brute force on tiny graphs, Prim, cut/cycle checks, closed forms."""
    m = len(src)
    return _run("oracle_kruskal", n, src, dst, w, min(m, max(n - 1, 0)) if n > 0 else 0)


def kruskal_par(n: int, src, dst, w, threads: int):
    """Kruskal with its radix sort spread over `threads` host threads (the
    union-find pass stays sequential).  Same output as kruskal(); for timing
    the CPU baseline on many cores.  Pinned by equality with kruskal()."""
    src, dst, w = _arr(src), _arr(dst), _arr(w)
    m = int(src.shape[0])
    out = np.empty(max(min(m, max(n - 1, 0)) if n > 0 else 0, 1), dtype=np.uint32)
    cnt = ctypes.c_uint64(0)
    tot = ctypes.c_uint64(0)
    rc = _load().oracle_kruskal_par(n, m, _p32(src), _p32(dst), _p32(w), int(threads), _p32(out),
                                    ctypes.byref(cnt), ctypes.byref(tot))
    if rc != 0:
        raise OracleError(f"oracle_kruskal_par: {_STATUS.get(rc, rc)}")
    return out[: cnt.value].copy(), int(tot.value)


def prim(n: int, src, dst, w):
    """Jarnik-Prim with a lazy binary heap keyed by (w,id), restarted from every
    unvisited vertex; an implementation independent of ``kruskal``."""
    m = len(src)
    return _run("oracle_prim", n, src, dst, w, min(m, max(n - 1, 0)) if n > 0 else 0)


def brute(n: int, src, dst, w):
    """Exhaustive search over edge subsets (n <= 16, m <= 22).  Returns
    (ids, total, min_total_over_all_spanning_forests)."""
    src, dst, w = _arr(src), _arr(dst), _arr(w)
    m = int(src.shape[0])
    out = np.empty(max(m, 1), dtype=np.uint32)
    cnt, tot, anyw = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
    rc = _load().oracle_brute(n, m, _p32(src), _p32(dst), _p32(w), _p32(out), ctypes.byref(cnt), ctypes.byref(tot),
                              ctypes.byref(anyw))
    if rc != 0:
        raise OracleError(f"oracle_brute: {_STATUS.get(rc, rc)}")
    return out[: cnt.value].copy(), int(tot.value), int(anyw.value)


CHECK_BITS = {1: "bad id list", 2: "cycle", 4: "not spanning", 8: "cut property", 16: "cycle property",
              64: "out of memory"}


def check_msf(n: int, src, dst, w, ids) -> int:
    """Returns 0 iff ``ids`` is the (w,id)-unique MSF (acyclic, spanning, cut
    and cycle properties); otherwise a bit mask naming the failed checks."""
    src, dst, w, ids = _arr(src), _arr(dst), _arr(w), _arr(ids)
    return int(_load().oracle_check_msf(n, int(src.shape[0]), _p32(src), _p32(dst), _p32(w), _p32(ids),
                                        int(ids.shape[0])))


def describe_check(mask: int) -> str:
    return ", ".join(v for k, v in CHECK_BITS.items() if mask & k) or "ok"
