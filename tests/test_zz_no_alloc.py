"""The allocation-free pivot selection (mst_pivot_noalloc) against the regular
step entry point (mst_step_pivot).

mst_pivot_noalloc serves callers that cannot allocate device memory (they may
not call cudaMalloc, or cannot create a handle because mst_create allocates):
its scratch is a fixed device array inside the library.  This file is named so
that pytest collects it last.  It must pass on its own in a fresh process (the
first call on the device looks the array's address up) and after every other
test, and it checks two calls in a row because the shared array keeps the
previous call's samples.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2302_12199_gb300 import mst
from paper_2302_12199_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MAX_SAMPLE = 65536


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def noalloc_pivot(lib, w, ids, state, sample):
    out = torch.zeros(1, dtype=torch.int64, device=w.device)
    st = lib.mst_pivot_noalloc(w.numel(), _ptr(w), _ptr(ids), state, sample, _ptr(out),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, int(out.item()) & 0xFFFFFFFFFFFFFFFF


def test_noalloc_pivot_matches_step_pivot_on_consecutive_calls():
    assert torch.cuda.is_available(), "a CUDA GPU is required"
    dev = torch.device("cuda", 0)
    lib = mst.load()
    g = W.gnm(1 << 14, 300_001, 4242)
    w = torch.from_numpy(g.w.view(np.int32)).to(dev)
    ids = torch.from_numpy((np.arange(g.m, dtype=np.uint32) * 2 + 1).view(np.int32)).to(dev)
    ref = mst.Solver(0)
    try:
        # a full-size sample, then a small one: the second call must not see the
        # first call's leftover samples in the shared array
        cases = [(ids, 0x1234567, MAX_SAMPLE), (ids, 0x89ABCDEF, 1000), (None, 77, 4097)]
        for i, (idv, state, sample) in enumerate(cases):
            st, got = noalloc_pivot(lib, w, idv, state, sample)
            assert st == 0, f"call {i}: status {st}"
            want = ref.pivot(w, idv, state=state, sample=sample)
            assert got == want, f"call {i}: {got:#x} != {want:#x}"
    finally:
        ref.close()


def test_noalloc_pivot_rejects_oversized_sample():
    dev = torch.device("cuda", 0)
    lib = mst.load()
    w = torch.ones(100, dtype=torch.int32, device=dev)
    st, _ = noalloc_pivot(lib, w, None, 1, MAX_SAMPLE + 1)
    assert st == 3  # MST_ERR_TOO_LARGE
    st, _ = noalloc_pivot(lib, w, None, 1, 0)
    assert st == 1  # MST_ERR_INVALID_ARG
