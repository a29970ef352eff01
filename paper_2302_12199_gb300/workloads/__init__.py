"""Seeded synthetic graph workloads (GNM, 2D/3D RGG, RMAT, mixed batches).

These stand in for the graph families the paper evaluates on (Section 7,
"Instances and Methodology": KaGen GNM / RGG generators, an RMAT generator with
the Graph500 probabilities, weights drawn uniformly from [1,255)).  No real-world
graph is used.

The module only generates inputs; it contains no step of any MST method, so the
CPU oracle tests and the GPU path may both draw their inputs from it.  The work
is done by ``gen.c`` (compiled with gcc on first use, or by ``build()``), which
draws every random number from a counter-based splitmix64 stream, so the graphs
are identical on every host and for every thread count.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_OUT = os.path.join(_HERE, "_build", "libmstgen.so")
_lib = None

DEFAULT_SEED = 0x2302121990

_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile gen.c into a shared library (gcc, no vendor tools)."""
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-pthread", _SRC, "-o", tmp, "-lm"],
                       check=True)
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.gen_splitmix64_at.restype = ctypes.c_uint64
        lib.gen_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.gen_gnm.restype = None
        lib.gen_gnm.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                ctypes.c_int, _u32p, _u32p, _u32p]
        lib.gen_rmat.restype = None
        lib.gen_rmat.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                 ctypes.c_int, _u32p, _u32p, _u32p]
        lib.gen_rgg_count.restype = ctypes.c_uint64
        lib.gen_rgg_count.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_uint64]
        lib.gen_rgg_fill.restype = ctypes.c_uint64
        lib.gen_rgg_fill.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                                     ctypes.c_uint32, _u32p, _u32p, _u32p]
        lib.gen_grid2d.restype = ctypes.c_uint64
        lib.gen_grid2d.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                   _u32p, _u32p, _u32p]
        lib.gen_rhg_radius.restype = ctypes.c_double
        lib.gen_rhg_radius.argtypes = [ctypes.c_uint64, ctypes.c_double, ctypes.c_double]
        lib.gen_rhg.restype = ctypes.c_uint64
        lib.gen_rhg.argtypes = [ctypes.c_uint64, ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                                ctypes.c_uint32, ctypes.c_int, _u32p, _u32p, _u32p]
        lib.gen_mix_sizes.restype = None
        lib.gen_mix_sizes.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, _u32p, _u64p,
                                      _u32p]
        lib.gen_mix_graph.restype = None
        lib.gen_mix_graph.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      _u32p, _u32p, _u32p]
        _lib = lib
    return _lib


def _p32(a: np.ndarray):
    return a.ctypes.data_as(_u32p)


def _p64(a: np.ndarray):
    return a.ctypes.data_as(_u64p)


def _threads(nthreads: int | None) -> int:
    if nthreads:
        return int(nthreads)
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def splitmix64_at(state: int, i: int) -> int:
    """Output #i of the splitmix64 sequence whose state starts at ``state``."""
    return int(_load().gen_splitmix64_at(state, i))


@dataclass
class Graph:
    """An undirected multigraph as an edge list; edge id = index."""
    n: int
    src: np.ndarray  # uint32 [m]
    dst: np.ndarray  # uint32 [m]
    w: np.ndarray  # uint32 [m]
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.src.shape[0])


def _empty(m: int):
    return (np.empty(m, dtype=np.uint32), np.empty(m, dtype=np.uint32), np.empty(m, dtype=np.uint32))


def gnm(n: int, m: int, seed: int = DEFAULT_SEED, wmin: int = 1, wmax: int = 255, nthreads=None) -> Graph:
    """G(n, m): m uniform endpoint pairs, duplicates kept, self-loops redrawn."""
    src, dst, w = _empty(m)
    _load().gen_gnm(n, m, seed, wmin, wmax, _threads(nthreads), _p32(src), _p32(dst), _p32(w))
    return Graph(n, src, dst, w, f"gnm_n{n}_m{m}")


def rmat(scale: int, m: int, seed: int = DEFAULT_SEED, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         permute: bool = True, wmin: int = 1, wmax: int = 255, n: int | None = None, nthreads=None) -> Graph:
    """RMAT with quadrant probabilities (a, b, c, 1-a-b-c) (Graph500 defaults),
    vertex ids randomly permuted; self-loops and duplicates kept as drawn."""
    n = (1 << scale) if n is None else n
    src, dst, w = _empty(m)
    _load().gen_rmat(scale, n, m, a, b, c, int(permute), seed, wmin, wmax, _threads(nthreads), _p32(src), _p32(dst),
                     _p32(w))
    return Graph(n, src, dst, w, f"rmat_s{scale}_m{m}")


def rgg_radius(dim: int, n: int, deg: float) -> float:
    """Radius giving expected degree ``deg`` for n uniform points in the unit square/cube."""
    if dim == 2:
        return math.sqrt(deg / (math.pi * n))
    return (3.0 * deg / (4.0 * math.pi * n)) ** (1.0 / 3.0)


def rgg(dim: int, n: int, deg: float = 8.0, seed: int = DEFAULT_SEED, wmin: int = 1, wmax: int = 0xFFFFFFFF) -> Graph:
    """Random geometric graph in [0,1)^dim with vertices numbered in grid-cell order."""
    r = rgg_radius(dim, n, deg)
    lib = _load()
    m = int(lib.gen_rgg_count(dim, n, r, seed))
    src, dst, w = _empty(m)
    got = int(lib.gen_rgg_fill(dim, n, r, seed, wmin, wmax, _p32(src), _p32(dst), _p32(w)))
    assert got == m
    return Graph(n, src, dst, w, f"rgg{dim}d_n{n}")


def grid2d(rows: int, cols: int, seed: int = DEFAULT_SEED, wmin: int = 1, wmax: int = 255) -> Graph:
    """rows x cols 4-neighbour grid (vertex r*cols + c), weights uniform in [wmin, wmax]."""
    lib = _load()
    m = int(lib.gen_grid2d(rows, cols, seed, wmin, wmax, None, None, None))
    src, dst, w = _empty(m)
    got = int(lib.gen_grid2d(rows, cols, seed, wmin, wmax, _p32(src), _p32(dst), _p32(w)))
    assert got == m
    return Graph(rows * cols, src, dst, w, f"grid2d_{rows}x{cols}")


def rhg_radius(n: int, deg: float, gamma: float = 3.0) -> float:
    return float(_load().gen_rhg_radius(n, deg, (gamma - 1.0) / 2.0))


def rhg(n: int, deg: float = 16.0, seed: int = DEFAULT_SEED, gamma: float = 3.0, wmin: int = 1, wmax: int = 255,
        nthreads=None) -> Graph:
    """Threshold random hyperbolic graph: power-law degrees with exponent gamma,
    expected average degree about deg, vertices numbered by angle."""
    lib = _load()
    alpha = (gamma - 1.0) / 2.0
    R = rhg_radius(n, deg, gamma)
    nt = _threads(nthreads)
    m = int(lib.gen_rhg(n, alpha, R, seed, wmin, wmax, nt, None, None, None))
    src, dst, w = _empty(m)
    got = int(lib.gen_rhg(n, alpha, R, seed, wmin, wmax, nt, _p32(src), _p32(dst), _p32(w)))
    assert got == m
    return Graph(n, src, dst, w, f"rhg_n{n}_d{deg:g}_g{gamma:g}")


@dataclass
class Batch:
    """Many independent graphs, concatenated; vertex ids are graph-local."""
    n: np.ndarray  # uint32 [G]
    edge_off: np.ndarray  # uint64 [G+1]
    src: np.ndarray
    dst: np.ndarray
    w: np.ndarray
    kind: np.ndarray  # uint32 [G]: 0 GNM, 1 RGG2D, 2 RMAT

    @property
    def num_graphs(self) -> int:
        return int(self.n.shape[0])

    def graph(self, g: int) -> Graph:
        lo, hi = int(self.edge_off[g]), int(self.edge_off[g + 1])
        return Graph(int(self.n[g]), self.src[lo:hi], self.dst[lo:hi], self.w[lo:hi], f"batch_g{g}")


def mix(num_graphs: int, seed: int = DEFAULT_SEED, log_lo: int = 8, log_hi: int = 16, nthreads=None) -> Batch:
    """Mixed batch: n log-uniform in [2^log_lo, 2^log_hi]; graph g is GNM (avg
    degree uniform in [4,32]) when g%3==0, RGG2D (degree 8) when g%3==1 and
    RMAT (degree 16, ids folded mod n) when g%3==2; weights in [1,255]."""
    lib = _load()
    n = np.empty(num_graphs, dtype=np.uint32)
    m = np.empty(num_graphs, dtype=np.uint64)
    kind = np.empty(num_graphs, dtype=np.uint32)
    lib.gen_mix_sizes(seed, num_graphs, log_lo, log_hi, _p32(n), _p64(m), _p32(kind))
    off = np.zeros(num_graphs + 1, dtype=np.uint64)
    np.cumsum(m, out=off[1:])
    total = int(off[-1])
    src, dst, w = _empty(total)

    def fill(g):  # graphs are independent: one generator thread each (the C call releases the GIL)
        lo = int(off[g])
        lib.gen_mix_graph(seed, g, log_lo, log_hi, 1, _p32(src[lo:]), _p32(dst[lo:]), _p32(w[lo:]))
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=_threads(nthreads)) as ex:
        list(ex.map(fill, range(num_graphs)))
    return Batch(n, off, src, dst, w, kind)


# Named workloads with their sizes (the families of the paper's Section 7).
def gnm_small(seed: int = DEFAULT_SEED) -> Graph:
    """GNM, n = 2^16, m = 2^20, weights uniform in [1,255]."""
    return gnm(1 << 16, 1 << 20, seed)


def grid2d_large(seed: int = DEFAULT_SEED) -> Graph:
    """2D grid 2048 x 2048 (n = 2^22, m ~ 2^23), weights uniform in [1,255]."""
    return grid2d(2048, 2048, seed)


def rhg_large(seed: int = DEFAULT_SEED) -> Graph:
    """Random hyperbolic graph, n = 2^22, gamma = 3, average degree about 16, weights in [1,255]."""
    return rhg(1 << 22, 16.0, seed)


def rgg2d_large(seed: int = DEFAULT_SEED) -> Graph:
    """2D RGG, n = 2^22, expected degree 8, weights uniform in [1, 2^32-1]."""
    return rgg(2, 1 << 22, 8.0, seed)


def rgg3d_large(seed: int = DEFAULT_SEED) -> Graph:
    """3D RGG, n = 2^21, expected degree 8, weights uniform in [1, 2^32-1]."""
    return rgg(3, 1 << 21, 8.0, seed)


def rmat_large(seed: int = DEFAULT_SEED, scale: int = 24, m: int = 1 << 28) -> Graph:
    """RMAT scale 24 (n = 2^24), m = 2^28, permuted ids, weights in [1,255]."""
    return rmat(scale, m, seed)
