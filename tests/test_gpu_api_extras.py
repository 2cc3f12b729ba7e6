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
