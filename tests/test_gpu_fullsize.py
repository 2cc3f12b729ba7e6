"""Parity at the benchmark's full sizes, on sampled atoms the oracle computes
one by one (O(N) each): the 864,000-atom LJ liquid at rc 2.5 and 5.0 (mixed,
every threads-per-atom layout, plus FP64) and the 500,000-atom EAM metal.
Inputs are jittered lattices (the perfect lattice has zero net forces, which
would make a relative force error meaningless)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TOL_FP64, TOL_MIXED, TPAS, rel_maxnorm

pytestmark = pytest.mark.gpu

SKIN = 0.3


def sample(n, m=48, seed=0):
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(n, m, replace=False))
    return np.concatenate([[0, n - 1], idx])


@pytest.fixture(scope="module", params=[2.5, 5.0])
def lj864k(request):
    rc = request.param
    d = synth.config1(rc=rc, displacement=0.1)
    x, box = d["x"], d["box"]
    idx = sample(x.shape[0], 40 if rc == 2.5 else 24, seed=int(rc * 10))
    assert oracle.min_gap(x, box, rc + SKIN, idx) > 1e-9
    f, _, _ = oracle.lj_at(x, box, rc, idx)
    nbr = oracle.neighbors(x, box, rc + SKIN, idx)
    return dict(d, idx=idx, f=f, nbr=nbr)


def test_lj864k_mixed_all_layouts(lj864k):
    from paper_1009_4330_gb300 import System
    d = lj864k
    idx = d["idx"]
    with System.lj(d["x"], d["v"], d["box"], cutoff=d["rc"], skin=SKIN, dt=0.005, mass=1.0, precision="mixed",
                   tpa=1) as s:
        for k, tpa in enumerate(TPAS):
            for lst, vec in (("full", 1), ("full", 4), ("half", 4 if tpa <= 8 else 1)):
                s.set_kernel(tpa, lst, 256, vec)
                f = s.compute_forces().cpu().numpy()
                assert rel_maxnorm(f[idx], d["f"]) < TOL_MIXED, (tpa, lst)
                if lst == "full" and k in (0, 5):
                    counts, nbr = s.neighbors()
                    c = counts.cpu().numpy()[idx]
                    nb = nbr[idx].cpu().numpy()
                    for q in range(len(idx)):
                        assert np.array_equal(np.sort(nb[q, :c[q]]), d["nbr"][q])


def test_lj864k_fp64(lj864k):
    from paper_1009_4330_gb300 import System
    d = lj864k
    with System.lj(d["x"], d["v"], d["box"], cutoff=d["rc"], skin=SKIN, dt=0.005, mass=1.0, precision="fp64",
                   tpa=8) as s:
        f = s.compute_forces().cpu().numpy()
    assert rel_maxnorm(f[d["idx"]], d["f"]) < TOL_FP64


def test_lj864k_steps_keep_parity():
    # the benchmark input itself (fcc + Maxwell-Boltzmann at T = 1.44): after
    # the step loop with in-graph rebuilds, the forces the library holds are
    # those of its positions, checked on a sample
    from paper_1009_4330_gb300 import System
    d = synth.config1(rc=2.5)
    with System.lj(d["x"], d["v"], d["box"], cutoff=2.5, skin=SKIN, dt=0.005, mass=1.0, precision="mixed",
                   tpa=4) as s:
        s.step(60)
        x, _, f = (a.cpu().numpy() for a in s.state())
        assert s.info()["rebuilds"] >= 2
    idx = sample(x.shape[0], 32, seed=9)
    fr, _, _ = oracle.lj_at(x, d["box"], 2.5, idx)
    assert rel_maxnorm(f[idx], fr) < TOL_MIXED


def test_eam500k_mixed_and_fp64():
    from paper_1009_4330_gb300 import System
    d = synth.config2(displacement=0.1)
    x, box = d["x"], d["box"]
    idx = sample(x.shape[0], 12, seed=3)
    fr, rho = oracle.eam_at(x, box, d["eam"], idx)
    for prec, tol in (("mixed", TOL_MIXED), ("fp64", TOL_FP64)):
        with System.eam(x, d["v"], box, eam_params=d["eam"], skin=d["skin"], dt=d["dt"], mass=d["mass"],
                        ftm2v=d["ftm2v"], precision=prec, tpa=4) as s:
            f = s.compute_forces().cpu().numpy()
        assert rel_maxnorm(f[idx], fr) < tol, prec


def test_eam500k_backward_directional_fd():
    # property at full size: grad_x . delta and dL/dA, dL/dc0..c2 equal central
    # differences of L = sum g.F computed with the FP64 forward (which is
    # parity-checked above), to 1e-6.  F is linear in A and in each c_q, so
    # the two-point difference is exact up to rounding there; the position
    # direction uses the fourth-order difference.
    import torch
    from paper_1009_4330_gb300 import System
    d = synth.config2(displacement=0.1)
    x, box = d["x"], d["box"]
    rng = np.random.default_rng(17)
    g = rng.standard_normal(x.shape)
    # direction supported on sampled atoms none of whose pairs lies within 1e-4
    # of rc: the force derivatives jump there, and only the moved atoms' pairs move
    idx = [i for i in sample(x.shape[0], 300, seed=23) if oracle.min_gap(x, box, d["rc"], [i]) > 1e-4]
    assert len(idx) > 250
    delta = np.zeros_like(x)
    delta[idx] = rng.standard_normal((len(idx), 3))
    gt = torch.tensor(g, device="cuda")
    with System.eam(x, d["v"], box, eam_params=d["eam"], skin=d["skin"], dt=d["dt"], mass=d["mass"],
                    ftm2v=d["ftm2v"], precision="fp64", tpa=4) as s:
        gx, gp = s.backward(g)
        gdx = float((gx.cpu().numpy() * delta).sum())
        gp = gp.cpu().numpy()

        def l_at_x(h):
            s.set_state(x=torch.tensor(x + h * delta, device="cuda"))
            return float((s.compute_forces() * gt).sum())

        h = 1e-5
        fd_x = (8.0 * (l_at_x(h) - l_at_x(-h)) - (l_at_x(2 * h) - l_at_x(-2 * h))) / (12.0 * h)
        s.set_state(x=torch.tensor(x, device="cuda"))
        fd_p = {}
        for q in (1, 2, 3, 4):  # A, c0, c1, c2
            hq = 1e-4 * abs(d["eam"][q])
            lv = []
            for sgn in (1, -1):
                p = np.array(d["eam"], dtype=np.float64)
                p[q] += sgn * hq
                s.set_params(p)
                lv.append(float((s.compute_forces() * gt).sum()))
            fd_p[q] = (lv[0] - lv[1]) / (2 * hq)
        s.set_params(np.array(d["eam"], dtype=np.float64))
    assert gdx == pytest.approx(fd_x, rel=1e-6)
    for q, fdv in fd_p.items():
        assert gp[q] == pytest.approx(fdv, rel=1e-6), q
    assert gp[0] == 0.0  # the cut-off is not differentiated


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_lj864k_nve_drift_over_1000_steps(prec):
    # the benchmark workload itself (fcc start, Maxwell-Boltzmann at T = 1.44,
    # rc 2.5, skin 0.3, dt 0.005): total energy per atom (shifted LJ, continuous
    # at rc) sampled every 50 steps over 1,000 steps; the least-squares slope x
    # 1000 must stay below 1e-4 per atom per 1,000 steps
    from paper_1009_4330_gb300 import System
    d = synth.config1(rc=2.5)
    n = d["x"].shape[0]
    es = []
    with System.lj(d["x"], d["v"], d["box"], cutoff=2.5, skin=SKIN, dt=0.005, mass=1.0, precision=prec,
                   tpa=1 if prec == "mixed" else 4, energy_shift=True) as s:
        s.step(100)  # past the melting of the lattice start
        for k in range(21):
            ev = s.energy_virial().cpu().numpy()[0]
            es.append((ev[0] + ev[1]) / n)
            if k < 20:
                s.step(50)
        assert s.info()["rebuilds"] > 100
    es = np.array(es)
    slope = np.polyfit(np.arange(21) * 50, es, 1)[0]
    assert abs(slope) * 1000 < 1e-4, f"{prec}: drift {slope * 1000:.2e} per atom per 1000 steps"
    assert np.abs(es - es[0]).max() < 5e-3
