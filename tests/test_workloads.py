"""The seeded generators produce the families they claim (no MST arithmetic
here): 2D grids by their closed form, random hyperbolic graphs against an
all-pairs distance check, and determinism."""
import math

import numpy as np

from paper_2302_12199_gb300 import workloads as W

GOLDEN = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1


def mix(z):
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def sub_seed(seed, tag):
    return mix(seed ^ mix((tag + GOLDEN) & MASK))


def test_grid2d_closed_form():
    rows, cols = 7, 11
    g = W.grid2d(rows, cols, 3)
    assert g.n == rows * cols and g.m == rows * (cols - 1) + (rows - 1) * cols
    pairs = set(zip(g.src.tolist(), g.dst.tolist()))
    want = {(r * cols + c, r * cols + c + 1) for r in range(rows) for c in range(cols - 1)}
    want |= {(r * cols + c, (r + 1) * cols + c) for r in range(rows - 1) for c in range(cols)}
    assert pairs == want and len(pairs) == g.m
    assert g.w.min() >= 1 and g.w.max() <= 255
    g2 = W.grid2d(rows, cols, 3)
    assert np.array_equal(g.w, g2.w)
    assert W.grid2d(1, 1, 3).m == 0


def test_rhg_matches_all_pairs_distances():
    n, deg, seed = 1500, 10.0, 11
    g = W.rhg(n, deg, seed)
    alpha = 1.0
    R = W.rhg_radius(n, deg, 3.0)
    s1, s2 = sub_seed(seed, 5), sub_seed(seed, 6)
    th = np.array([2 * math.pi * ((W.splitmix64_at(s1, i) >> 11) / 2.0 ** 53) for i in range(n)])
    u2 = np.array([(W.splitmix64_at(s2, i) >> 11) / 2.0 ** 53 for i in range(n)])
    r = np.arccosh(1.0 + u2 * (math.cosh(alpha * R) - 1.0)) / alpha
    order = np.argsort(th, kind="stable")
    th, r = th[order], r[order]
    cd = np.cosh(r)[:, None] * np.cosh(r)[None, :] - np.sinh(r)[:, None] * np.sinh(r)[None, :] * np.cos(
        th[:, None] - th[None, :])
    iu = np.triu_indices(n, 1)
    close = cd[iu] < math.cosh(R)
    margin = np.abs(cd[iu] - math.cosh(R)) < 1e-9 * math.cosh(R)
    want = {(int(a), int(b)) for a, b, c, mg in zip(iu[0], iu[1], close, margin) if c and not mg}
    undecided = {(int(a), int(b)) for a, b, mg in zip(iu[0], iu[1], margin) if mg}
    got = set(zip(g.src.tolist(), g.dst.tolist()))
    assert len(got) == g.m  # each pair once, src < dst
    assert all(a < b for a, b in got)
    assert want <= got and got - want <= undecided


def test_rhg_degree_and_tail():
    g = W.rhg(1 << 16, 16.0, 12)
    deg = np.bincount(np.concatenate([g.src, g.dst]), minlength=g.n)
    assert abs(deg.mean() - 16.0) < 2.0
    assert deg.max() > 20 * deg.mean()  # power-law tail (gamma = 3)
    assert np.array_equal(W.rhg(1 << 12, 8.0, 13, nthreads=1).dst, W.rhg(1 << 12, 8.0, 13, nthreads=4).dst)
