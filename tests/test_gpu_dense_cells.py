"""GPU parity where the list build shares each cell over several warps: the LJ
liquid at rc 5.0 (r_l = 5.3) in boxes only two or three cells wide, so that a
cell holds ~170 atoms (six 32-atom home chunks, four-warp blocks) and, along
an axis two cells wide, the stencil reaches the other cell through two
periodic images (offsets -1 and +1), of which at most one can be within r_l
(the box edge is at least 2 r_l).  Lists must equal the oracle's exactly
(full and half), forces within 1e-12 (FP64) and 1e-5 (mixed), for one and
eight threads per atom."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TOL_FP64, TOL_MIXED, assert_lists_equal, gpu_lists, half_pairs, margin_ok, oracle_pairs, rel_maxnorm

pytestmark = pytest.mark.gpu

RC, SKIN = 5.0, 0.3


def dense_case(nx, ny, nz, seed):
    a = synth.fcc_constant(0.8442)
    x, box = synth.fcc_lattice(nx, ny, nz, a)
    x = synth.displace(x, box, 0.08, seed)
    v = synth.maxwell_boltzmann(x.shape[0], 1.44, 1.0, seed + 1)
    return {"x": x, "v": v, "box": box}


@pytest.fixture(scope="module")
def cases():
    out = {}
    # 7 x 7 x 7 cells: box 11.76, two bins per axis; 7 x 7 x 10: (2, 2, 3) bins
    for name, (nx, ny, nz, seed) in (("two_bins", (7, 7, 7, 91)), ("two_two_three", (7, 7, 10, 93))):
        d = dense_case(nx, ny, nz, seed)
        x, box = d["x"], d["box"]
        assert margin_ok(x, box, RC + SKIN)
        f, _, _ = oracle.lj(x, box, RC)
        out[name] = dict(d, f=f, nbr=oracle.neighbors(x, box, RC + SKIN))
    return out


def make(d, prec, tpa, lst):
    from paper_1009_4330_gb300 import System
    return System.lj(d["x"], d["v"], d["box"], cutoff=RC, skin=SKIN, dt=0.005, mass=1.0, precision=prec,
                     list=lst, tpa=tpa)


@pytest.mark.parametrize("name", ["two_bins", "two_two_three"])
def test_cells_are_shared_over_warps(cases, name):
    d = cases[name]
    with make(d, "mixed", 1, "full") as s:
        inf = s.info()
    nb = inf["bins"]
    assert min(nb) == 2 and max(nb) <= 3
    assert d["x"].shape[0] / np.prod(nb) > 96  # more than three 32-atom home chunks per cell


@pytest.mark.parametrize("name", ["two_bins", "two_two_three"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("tpa", [1, 8])
def test_full_lists_and_forces(cases, name, prec, tpa):
    d = cases[name]
    with make(d, prec, tpa, "full") as s:
        counts, nbr = s.neighbors()
        assert_lists_equal(gpu_lists(counts, nbr), d["nbr"])
        f = s.compute_forces().cpu().numpy()
    assert rel_maxnorm(f, d["f"]) < (TOL_FP64 if prec == "fp64" else TOL_MIXED)


@pytest.mark.parametrize("name", ["two_bins", "two_two_three"])
def test_half_lists_and_forces(cases, name):
    d = cases[name]
    with make(d, "fp64", 4, "half") as s:
        counts, nbr = s.neighbors()
        assert int(counts.sum()) == sum(map(len, d["nbr"])) // 2
        assert half_pairs(counts, nbr) == oracle_pairs(d["nbr"])
        f = s.compute_forces().cpu().numpy()
    assert rel_maxnorm(f, d["f"]) < TOL_FP64
