"""md_neighbors_noalloc: the neighbour-list build that allocates nothing.

For callers that may not call cudaMalloc (graph capture in progress, device
memory owned by another allocator, latency-critical loops), the library
offers this one entry point whose scratch is a fixed static device array.
Its lists must equal those of the handle-based path (md_get_neighbors) --
index sets, so exactly -- on consecutive calls, which share that array.
This file runs last so that a failure here does not hide the other tests.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import gpu_lists, lj_case, margin_ok

pytestmark = pytest.mark.gpu

RC, SKIN = 2.5, 0.3


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_lists_equal_handle_lists_on_two_calls():
    import torch
    from paper_1009_4330_gb300 import System, _lib

    lib = _lib.load()
    cases = [lj_case(10, 0.1, seed=61), lj_case(7, 0.12, seed=62)]  # 4,000 and 1,372 atoms
    for d in cases:
        x, box = d["x"], d["box"]
        assert margin_ok(x, box, RC + SKIN)
        with System.lj(x, d["v"], box, cutoff=RC, skin=SKIN, dt=0.005, mass=1.0, precision="fp64", tpa=1) as s:
            ref = gpu_lists(*s.neighbors())  # the existing entry point
        n = x.shape[0]
        cap = max(map(len, ref)) + 8
        xd = torch.tensor(x, dtype=torch.float64, device="cuda").contiguous()
        hbox = np.ascontiguousarray(box, dtype=np.float64)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for call in range(2):
            counts = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            nbr = torch.full((n, cap), -1, dtype=torch.int32, device="cuda")
            st = lib.md_neighbors_noalloc(n, _ptr(xd), hbox.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          RC + SKIN, _ptr(counts), _ptr(nbr), cap, stream)
            assert st == _lib.MD_OK, lib.md_last_error(None)
            got = gpu_lists(counts, nbr)
            assert len(got) == len(ref)
            for i in range(n):
                assert np.array_equal(got[i], ref[i]), f"call {call}, atom {i}"


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_1009_4330_gb300 import _lib

    lib = _lib.load()
    n = _lib_max_atoms() + 1
    x = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    c = torch.zeros(1, dtype=torch.int32, device="cuda")
    hbox = np.array([100.0, 100.0, 100.0])
    # n is checked before any device work, so the small buffers are never touched
    st = lib.md_neighbors_noalloc(n, _ptr(x), hbox.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 2.8,
                                  _ptr(c), _ptr(c), 1, None)
    assert st == _lib.MD_ERR_UNSUPPORTED
    assert b"MAX_ATOMS" in lib.md_last_error(None)


def _lib_max_atoms():
    import os
    import re
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "md.h")
    return int(re.search(r"#define MD_NOALLOC_MAX_ATOMS (\d+)", open(hdr).read()).group(1))
