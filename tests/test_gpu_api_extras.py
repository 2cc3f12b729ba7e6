"""Contracts of the ABI's measurement, tuning and decomposition entry points on
the GPU: md_vv phases composed into velocity-Verlet steps follow md_step's
trajectory; halo pack/unpack round trips; the set-up benchmark's timing table
names the variant it chose; the ceiling probes return sane figures."""
import numpy as np
import pytest

import oracle
from gpu_util import lj_case, rel_maxnorm, wrap_diff

pytestmark = pytest.mark.gpu

RC, SKIN, DT = 2.5, 0.3, 0.005


def _lj(d, prec="fp64", tpa=4, lst="full"):
    from paper_1009_4330_gb300 import System
    return System.lj(d["x"], d["v"], d["box"], cutoff=RC, skin=SKIN, dt=DT, mass=1.0, precision=prec, tpa=tpa,
                     list=lst)


@pytest.mark.parametrize("lst", ["full", "half"])
def test_split_phases_follow_md_step(lst):
    # DRIFT, DISP (rebuild above skin/2), FORCE, KICK per step: textbook
    # velocity Verlet, the same positions as md_step's leapfrog form up to rounding
    from paper_1009_4330_gb300 import _lib as L
    d = lj_case(8, 0.05, seed=71)
    ref = oracle.nve(d["x"], d["v"], d["box"], 60, DT, RC, SKIN)
    with _lj(d, lst=lst) as a, _lj(d, lst=lst) as b:
        rebuilds = 0
        for _ in range(60):
            a.vv(L.MD_VV_DRIFT)
            if a.vv(L.MD_VV_DISP) > 0.5 * SKIN:
                a.build_neighbors()
                rebuilds += 1
            a.vv(L.MD_VV_FORCE)
            a.vv(L.MD_VV_KICK)
        b.step(60)
        xa, va, fa = (t.cpu().numpy() for t in a.state())
        xb, vb, fb = (t.cpu().numpy() for t in b.state())
    assert rebuilds >= 2
    assert np.abs(wrap_diff(xa, xb, d["box"])).max() < 1e-11
    assert np.abs(va - vb).max() < 1e-11
    assert np.abs(wrap_diff(xa, ref["x"], d["box"])).max() < 1e-9
    assert rel_maxnorm(fa, ref["f"]) < 1e-9


def test_halo_round_trips():
    import torch
    from paper_1009_4330_gb300 import _lib as L
    d = lj_case(6, 0.05, seed=72)
    n = d["x"].shape[0]
    with _lj(d, prec="mixed", tpa=1) as s:
        x0, v0, f0 = (t.clone() for t in s.state())
        idx = torch.arange(0, n, 7, dtype=torch.int32, device="cuda")
        rows = s.halo_pack(idx, L.MD_HALO_X | L.MD_HALO_V | L.MD_HALO_F)
        assert rows.shape == (idx.numel(), 9)
        assert torch.allclose(rows[:, 0:3], x0[idx.long()], rtol=0, atol=1e-12)
        assert torch.equal(rows[:, 3:6], v0[idx.long()]) and torch.equal(rows[:, 6:9], f0[idx.long()])
        # positions and velocities written back unchanged; forces accumulated twice
        s.halo_unpack(idx, L.MD_HALO_X | L.MD_HALO_V, rows[:, 0:6].contiguous())
        s.halo_unpack(idx, L.MD_HALO_F, rows[:, 6:9].contiguous(), accumulate=True)
        x1, v1, f1 = s.state()
        assert torch.allclose(x1, x0, rtol=0, atol=1e-12) and torch.equal(v1, v0)
        assert torch.allclose(f1[idx.long()], 2 * f0[idx.long()], rtol=1e-15, atol=0)
        # a shift moves the packed positions only
        sh = np.array([0.0, 0.0, -1.5])
        rs = s.halo_pack(idx, L.MD_HALO_X, shift=sh)
        assert torch.allclose(rs, rows[:, 0:3] + torch.tensor(sh, device="cuda"), rtol=0, atol=1e-12)
        # displacement since the build: none moved
        assert s.vv(L.MD_VV_DISP) < 1e-6


def test_autotune_table_names_the_choice():
    d = lj_case(8, 0.1, seed=73)
    with _lj(d, prec="mixed", tpa=1, lst="auto") as s:
        s.autotune()
        rows = s.autotune_table()
        inf = s.info()
    assert len(rows) == 72 and all(r["ms"] > 0 for r in rows)
    best = min(rows, key=lambda r: r["ms"])
    assert (best["tpa"], best["list"], best["block"], best["vec"]) == (inf["tpa"], inf["list"], inf["block"], inf["vec"])


def test_ceiling_probes_are_sane():
    from paper_1009_4330_gb300 import probe_ceilings
    c = probe_ceilings()
    assert c["fp32_fma_tflops"] > 10 * c["fp64_fma_tflops"] > 0
    assert 1000 < c["hbm_copy_gbs"] < 20000
    assert c["l2_gather_gps"] > 10 and c["l2_gather_gbs"] == pytest.approx(16 * c["l2_gather_gps"])


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_reset_within_capacity_equals_a_new_handle(prec, tol):
    # one handle made with room for 1,000 more atoms, reset to a smaller, then a
    # larger system: forces, energies and lists as a fresh handle's (stale data in
    # slots that became padding must not leak into sums), and steps that follow
    from paper_1009_4330_gb300 import MDError, System
    from gpu_util import gpu_lists
    a = lj_case(7, 0.08, seed=74)   # 1,372 atoms
    c = lj_case(7, 0.10, seed=76)   # the same box
    n_cap = a["x"].shape[0] + 1000
    with System.lj(a["x"], a["v"], a["box"], cutoff=RC, skin=SKIN, dt=DT, mass=1.0, precision=prec, tpa=4,
                   capacity=n_cap, energy_shift=False) as s:
        assert s.capacity == n_cap
        # a system of the same box with fewer atoms: drop the last 400 of case c
        xs, vs = c["x"][:-400], c["v"][:-400]
        s.energy_virial()  # fill the per-atom terms of all 1,372 slots
        s.reset(xs, vs)
        f, e, w = oracle.lj(xs, c["box"], RC)
        assert rel_maxnorm(s.compute_forces().cpu().numpy(), f) < tol
        ev = s.energy_virial().cpu().numpy()[0]
        assert ev[0] == pytest.approx(e, rel=max(tol, 1e-7))
        assert ev[1] == pytest.approx(oracle.kinetic(vs, [1.0]), rel=1e-12)
        ref = oracle.neighbors(xs, c["box"], RC + SKIN)
        got = gpu_lists(*s.neighbors())
        assert all(np.array_equal(g, r) for g, r in zip(got, ref))
        # back up to the full case c (more atoms than the handle held), then step
        s.reset(c["x"], c["v"])
        s.step(30)
        x1 = s.state()[0].cpu().numpy()
        refn = oracle.nve(c["x"], c["v"], c["box"], 30, DT, RC, SKIN)
        assert np.abs(wrap_diff(x1, refn["x"], c["box"])).max() < (1e-9 if prec == "fp64" else 1e-5)
        with pytest.raises(MDError, match="capacity"):
            big = np.concatenate([c["x"]] * 2)
            s.reset(big, np.zeros_like(big))
