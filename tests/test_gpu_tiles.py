"""Block-local lists (md_set_staging: force blocks stage the records of the
cells around their atoms in shared memory): the tile set-up reported by
md_info, forces, lists and gradients identical to the oracle, also when some
tiles are too dense to stage and keep slot entries, and the same trajectory
with and without staging."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import RC_MARGIN_CELL_PASS, TOL_MIXED, assert_lists_equal, gpu_lists, lj_case, margin_ok, rel_maxnorm

pytestmark = pytest.mark.gpu

RC, SKIN = 2.5, 0.3


def dense_cluster_case(seed=42):
    """LJ liquid (16^3 fcc cells) with a 9^3 cube at density 4 in the middle: the cells there
    are too full for a tile to stage, the rest stage."""
    a_lo = synth.fcc_constant(0.8442)
    x_lo, box = synth.fcc_lattice(16, 16, 16, a_lo)
    inside = np.all((x_lo >= 8.5) & (x_lo < 18.5), axis=1)
    x_hi, _ = synth.fcc_lattice(9, 9, 9, 1.0)
    x = np.concatenate([x_lo[~inside], x_hi + 9.0])
    x = synth.displace(x, box, 0.03, seed)
    v = synth.maxwell_boltzmann(x.shape[0], 1.0, 1.0, seed + 1)
    return x, v, box


def test_info_reports_tiles():
    from paper_1009_4330_gb300 import System
    d = lj_case(15, 0.1, seed=1002)
    n = d["x"].shape[0]
    with System.lj(d["x"], d["v"], d["box"], cutoff=RC, skin=SKIN, dt=0.005, mass=1.0, precision="mixed",
                   tpa=1) as s:
        assert s.info()["tile_atoms"] == 0  # off by default
        s.set_staging(True)
        inf = s.info()
        assert inf["block"] == 128 and inf["tile_atoms"] == 128
        assert inf["n_tiles_force"] == (n + 127) // 128
        # a small box (9 cells per axis): tiles whose atoms straddle Morton-order
        # boundaries span wide boxes of cells and keep slot entries
        assert inf["tiles_staged"] >= 0.7 * inf["n_tiles_force"]
    with System.lj(d["x"], d["v"], d["box"], cutoff=RC, skin=SKIN, dt=0.005, mass=1.0, precision="fp64",
                   tpa=1) as s:
        s.set_staging(True)
        assert s.info()["tile_atoms"] == 0


@pytest.mark.parametrize("tpa", [1, 2, 4])
def test_dense_tiles_fall_back_and_match_oracle(tpa):
    from paper_1009_4330_gb300 import System
    x, v, box = dense_cluster_case()
    assert margin_ok(x, box, RC + SKIN)
    f_ref = oracle.lj(x, box, RC)[0]
    nbr_ref = oracle.neighbors(x, box, RC + SKIN)
    with System.lj(x, v, box, cutoff=RC, skin=SKIN, dt=0.005, mass=1.0, precision="mixed", tpa=tpa) as s:
        s.set_staging(True)
        inf = s.info()
        assert inf["tile_atoms"] == 128 // tpa
        assert 0 < inf["tiles_staged"] < inf["n_tiles_force"]
        f = s.compute_forces().cpu().numpy()
        counts, nbr = s.neighbors()
    assert rel_maxnorm(f, f_ref) < TOL_MIXED
    assert_lists_equal(gpu_lists(counts, nbr), nbr_ref)


def test_trajectory_same_with_and_without_staging():
    # the staged records are the same FP32 values and the pair terms are summed
    # in the same order: bitwise the same trajectory
    from paper_1009_4330_gb300 import System
    d = lj_case(15, 0.02, seed=1002)  # small jitter: no close pairs to blow up in 50 steps
    out = []
    for staged in (True, False):
        with System.lj(d["x"], d["v"], d["box"], cutoff=RC, skin=SKIN, dt=0.005, mass=1.0, precision="mixed",
                       tpa=1) as s:
            s.set_staging(staged)
            inf = s.info()
            assert (inf["tile_atoms"] > 0 and inf["tiles_staged"] > 0) == staged
            s.step(50)
            out.append([a.cpu().numpy() for a in s.state()])
    for a, b in zip(*out):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["mixed"])
def test_staged_eam_and_backward_match_oracle(prec):
    # EAM density and force passes and the two backward passes (which map
    # block-local entries back to slots) with staging on
    from paper_1009_4330_gb300 import System
    P = np.array(synth.EAM_PARAMS)
    x, box = synth.fcc_lattice(8, 8, 8, 3.615)
    x = synth.displace(x, box, 0.1, 7)
    assert margin_ok(x, box, P[0] + 0.5)
    f_ref = oracle.eam(x, box, P)[0]
    g = np.random.default_rng(8).standard_normal(x.shape)
    gx_ref, gp_ref = oracle.eam_vjp(x, box, P, g)
    with System.eam(x, np.zeros_like(x), box, eam_params=P, skin=0.5, dt=1.0, mass=63.55,
                    ftm2v=synth.FTM2V_METAL, precision=prec, tpa=1) as s:
        s.set_staging(True)
        inf = s.info()
        assert inf["tile_atoms"] == 128 and inf["tiles_staged"] > 0
        f = s.compute_forces().cpu().numpy()
        gx, gp = s.backward(g)
    assert rel_maxnorm(f, f_ref) < TOL_MIXED
    assert rel_maxnorm(gx.cpu().numpy(), gx_ref) < 1e-11
    assert np.allclose(gp.cpu().numpy()[1:], gp_ref[1:], rtol=1e-11, atol=1e-11 * np.abs(gp_ref).max())



@pytest.mark.parametrize("case", ["liquid", "dense_cluster"])
def test_cell_list_forces_match_oracle(case):
    # md_cell_forces: no Verlet list, every atom of the 27 cells tested; also
    # after some steps (atoms moved, cells as binned at the last rebuild)
    from paper_1009_4330_gb300 import System
    if case == "liquid":
        d = lj_case(15, 0.05, seed=1003)
        x, v, box = d["x"], d["v"], d["box"]
    else:
        x, v, box = dense_cluster_case()
    with System.lj(x, v, box, cutoff=RC, skin=SKIN, dt=0.002, mass=1.0, precision="mixed", tpa=1) as s:
        s.set_staging(True)
        # this pass decides cut-offs in FP32 (no FP64 band): inputs keep pairs off rc
        assert margin_ok(x, box, RC, margin=RC_MARGIN_CELL_PASS)
        f_ref = oracle.lj(x, box, RC)[0]
        f_cell, ms = s.cell_forces(reps=3)
        assert ms > 0.0
        assert rel_maxnorm(f_cell.cpu().numpy(), f_ref) < TOL_MIXED
        if case != "liquid":
            return  # the density-4 cluster is far from equilibrium: no stepping
        # after steps, on sampled atoms none of whose pairs lies near rc
        s.step(7)
        xs = s.state()[0].cpu().numpy()
        rng = np.random.default_rng(5)
        idx = [int(i) for i in rng.choice(xs.shape[0], 96, replace=False)
               if oracle.min_gap(xs, box, RC, [int(i)]) > RC_MARGIN_CELL_PASS]
        assert len(idx) > 48
        fr, _, _ = oracle.lj_at(xs, box, RC, idx)
        f_cell = s.cell_forces()[0].cpu().numpy()
        assert rel_maxnorm(f_cell[idx], fr) < TOL_MIXED


def test_cell_list_needs_staging():
    from paper_1009_4330_gb300 import MDError, System
    d = lj_case(15, 0.02, seed=1002)
    with System.lj(d["x"], d["v"], d["box"], cutoff=RC, skin=SKIN, dt=0.005, mass=1.0, precision="mixed",
                   tpa=1) as s:
        with pytest.raises(MDError):
            s.cell_forces()
