"""md_neighbors_noalloc: the neighbour-list build that allocates nothing.

Some callers cannot call cudaMalloc -- their device memory belongs to another
allocator (a framework's caching pool, a fixed arena), or their loop cannot
afford an allocation -- so the library offers this one entry point whose
scratch is a fixed static device array.  Its lists must equal the FP64
definition (the oracle's brute-force sets) and those of the handle-based path
(md_get_neighbors), as index sets, exactly, on consecutive calls, which share
that array.  The cases reach every branch of its cell grid: the full 27-cell
stencil, a box only two cells wide on some axes (each neighbour cell visited
once), and a dilute box whose grid is coarsened to fit the scratch; and every
documented error return.  This file runs last so that a failure here does not
hide the other tests.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth
from gpu_util import gpu_lists, lj_case, margin_ok

pytestmark = pytest.mark.gpu

RC, SKIN = 2.5, 0.3
RL = RC + SKIN


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _header_int(name):
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "md.h")
    return int(re.search(rf"#define {name} (\d+)", open(hdr).read()).group(1))


def _call(lib, x, box, rl, cap, n=None, counts=None, nbr=None):
    """One call through the C ABI; returns (status, counts, nbr) as device tensors."""
    import torch
    xd = torch.as_tensor(x, dtype=torch.float64, device="cuda").contiguous()
    n = xd.shape[0] if n is None else n
    if counts is None:
        counts = torch.full((xd.shape[0],), -1, dtype=torch.int32, device="cuda")
    if nbr is None:
        nbr = torch.full((xd.shape[0], cap), -1, dtype=torch.int32, device="cuda")
    hbox = np.ascontiguousarray(np.broadcast_to(np.asarray(box, np.float64), (3,)))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.md_neighbors_noalloc(n, _ptr(xd), hbox.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), rl,
                                  _ptr(counts), _ptr(nbr), cap, stream)
    return st, counts, nbr


def _two_cells_case():
    # 4 x 4 x 8 fcc cells at rho 0.8442: edges 6.72, 6.72, 13.4 against rl 2.8
    # give a 2 x 2 x 4 cell grid (two cells per axis on x and y)
    a = synth.fcc_constant(0.8442)
    x, box = synth.fcc_lattice(4, 4, 8, a)
    return synth.displace(x, box, 0.08, 71), box


def _coarsened_case():
    # 20,000 atoms spread through a 100^3 box: 35^3 = 42,875 cells of edge
    # >= rl would exceed the scratch's cell table, so the grid is coarsened
    rng = np.random.default_rng(72)
    box = np.array([100.0, 100.0, 100.0])
    return rng.uniform(0.0, 100.0, size=(20000, 3)), box


CASES = {
    "liquid4000": lambda: (lambda d: (d["x"], d["box"]))(lj_case(10, 0.1, seed=61)),
    "liquid1372": lambda: (lambda d: (d["x"], d["box"]))(lj_case(7, 0.12, seed=62)),
    "two_cells": _two_cells_case,
    "coarsened": _coarsened_case,
}


def test_case_geometries_reach_their_branches():
    # host arithmetic of the grid, as the entry point does it
    max_bins = _header_int("MD_NOALLOC_MAX_BINS")
    x, box = _two_cells_case()
    assert [int(np.floor(b / RL)) for b in box] == [2, 2, 4]
    x, box = _coarsened_case()
    assert int(np.prod([np.floor(b / RL) for b in box])) > max_bins


@pytest.mark.parametrize("name", list(CASES))
def test_noalloc_lists_equal_oracle_and_handle_lists_on_two_calls(name):
    from paper_1009_4330_gb300 import System, _lib

    lib = _lib.load()
    x, box = CASES[name]()
    assert margin_ok(x, box, RL)
    ref = oracle.neighbors(x, box, RL)  # the FP64 definition, brute force
    handle = None
    if name != "coarsened":  # the handle path needs no dilute-box case
        v = np.zeros_like(x)
        with System.lj(x, v, box, cutoff=RC, skin=SKIN, dt=0.005, mass=1.0, precision="fp64", tpa=1) as s:
            handle = gpu_lists(*s.neighbors())  # the existing entry point
    n = x.shape[0]
    cap = max(map(len, ref)) + 8
    for call in range(2):
        st, counts, nbr = _call(lib, x, box, RL, cap)
        assert st == _lib.MD_OK, lib.md_last_error(None)
        got = gpu_lists(counts, nbr)
        assert len(got) == n
        for i in range(n):
            assert np.array_equal(got[i], ref[i]), f"call {call}, atom {i}: differs from the oracle"
            if handle is not None:
                assert np.array_equal(got[i], handle[i]), f"call {call}, atom {i}: differs from md_get_neighbors"


def test_noalloc_overflow_keeps_counts_and_valid_prefixes():
    from paper_1009_4330_gb300 import _lib

    lib = _lib.load()
    d = lj_case(7, 0.12, seed=62)
    x, box = d["x"], d["box"]
    ref = oracle.neighbors(x, box, RL)
    cap = max(map(len, ref)) - 1
    st, counts, nbr = _call(lib, x, box, RL, cap)
    assert st == _lib.MD_ERR_LIST_OVERFLOW
    assert b"cap" in lib.md_last_error(None)
    c = counts.cpu().numpy()
    nb = nbr.cpu().numpy()
    assert np.array_equal(c, np.array([len(r) for r in ref]))  # true lengths
    for i in range(x.shape[0]):
        row = nb[i, :min(c[i], cap)]
        assert len(set(row.tolist())) == len(row)  # no duplicates
        assert set(row.tolist()) <= set(ref[i].tolist())  # only true neighbours
    # the next call with room succeeds on the same (shared) scratch
    st, counts, nbr = _call(lib, x, box, RL, cap + 1)
    assert st == _lib.MD_OK
    assert all(np.array_equal(g, r) for g, r in zip(gpu_lists(counts, nbr), ref))


def test_noalloc_rejects_bad_arguments_on_the_host():
    import torch
    from paper_1009_4330_gb300 import _lib

    lib = _lib.load()
    x = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    c = torch.zeros(4, dtype=torch.int32, device="cuda")
    hbox = np.array([10.0, 10.0, 10.0])
    bp = hbox.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    # each is refused before any device work, so the small buffers are never touched
    assert lib.md_neighbors_noalloc(4, _ptr(x), bp, 2.8, _ptr(c), _ptr(c), 0, None) == _lib.MD_ERR_INVALID
    assert lib.md_neighbors_noalloc(0, _ptr(x), bp, 2.8, _ptr(c), _ptr(c), 1, None) == _lib.MD_ERR_INVALID
    assert lib.md_neighbors_noalloc(4, _ptr(x), bp, -1.0, _ptr(c), _ptr(c), 1, None) == _lib.MD_ERR_INVALID
    assert lib.md_neighbors_noalloc(4, None, bp, 2.8, _ptr(c), _ptr(c), 1, None) == _lib.MD_ERR_INVALID
    # a box edge below 2 rl
    small = np.array([10.0, 5.0, 10.0])
    st = lib.md_neighbors_noalloc(4, _ptr(x), small.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 2.8,
                                  _ptr(c), _ptr(c), 1, None)
    assert st == _lib.MD_ERR_BOX_TOO_SMALL
    assert b"2 rl" in lib.md_last_error(None)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_1009_4330_gb300 import _lib

    lib = _lib.load()
    n = _header_int("MD_NOALLOC_MAX_ATOMS") + 1
    x = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    c = torch.zeros(1, dtype=torch.int32, device="cuda")
    hbox = np.array([100.0, 100.0, 100.0])
    # n is checked before any device work, so the small buffers are never touched
    st = lib.md_neighbors_noalloc(n, _ptr(x), hbox.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 2.8,
                                  _ptr(c), _ptr(c), 1, None)
    assert st == _lib.MD_ERR_UNSUPPORTED
    assert b"MAX_ATOMS" in lib.md_last_error(None)
