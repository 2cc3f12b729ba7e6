"""GPU parity of velocity-Verlet NVE (with in-graph list rebuilds), EAM,
the LJ backward pass, batched replicas, and the error paths."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import (TOL_FP64, TOL_MIXED, assert_lists_equal, gpu_lists, lj_case, margin_ok,
                      rel_maxnorm, wrap_diff)

pytestmark = pytest.mark.gpu

RC, SKIN, DT = 2.5, 0.3, 0.005


def lj_system(d, prec="fp64", tpa=4, lst="full", **kw):
    from paper_1009_4330_gb300 import System
    return System.lj(d["x"], d["v"], d["box"], cutoff=RC, skin=SKIN, dt=DT, mass=1.0, precision=prec, tpa=tpa,
                     list=lst, **kw)


# ------------------------------------------------------------------ NVE ----

@pytest.mark.parametrize("lst", ["full", "half"])
def test_config0_trajectory_matches_oracle(lst):
    d = synth.config0()  # 4,000 atoms, fcc + MB at T = 1.44, FP64, 100 steps
    ref = oracle.nve(d["x"], d["v"], d["box"], 100, DT, RC, SKIN)
    assert ref["rebuilds"] >= 1
    with lj_system(d, "fp64", 4, lst) as s:
        s.step(100)
        x, v, f = (a.cpu().numpy() for a in s.state())
        info = s.info()
    assert info["steps"] == 100 and info["rebuilds"] >= 2  # creation + at least one in-graph rebuild
    assert np.abs(wrap_diff(x, ref["x"], d["box"])).max() < 1e-9
    assert np.abs(v - ref["v"]).max() < 1e-9
    assert rel_maxnorm(f, ref["f"]) < 1e-9


def test_step_calls_compose():
    d = lj_case(6, 0.05, seed=12)
    with lj_system(d) as a, lj_system(d) as b:
        a.step(40)
        for _ in range(4):
            b.step(10)
        xa, va, _ = (t.cpu().numpy() for t in a.state())
        xb, vb, _ = (t.cpu().numpy() for t in b.state())
    assert np.abs(wrap_diff(xa, xb, d["box"])).max() < 1e-11
    assert np.abs(va - vb).max() < 1e-11


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_eager_step_equals_graph_step(prec):
    d = lj_case(7, 0.05, seed=14)
    with lj_system(d, prec, 2) as a, lj_system(d, prec, 2) as b:
        a.step(35)
        b.step(35, eager=True)
        ia, ib = a.info(), b.info()
        sa = [t.cpu().numpy() for t in a.state()]
        sb = [t.cpu().numpy() for t in b.state()]
    assert ia["steps"] == ib["steps"] == 35 and ia["rebuilds"] == ib["rebuilds"]
    for u, w in zip(sa, sb):
        assert np.array_equal(u, w)


def test_mixed_trajectory_tracks_oracle_short():
    d = lj_case(8, 0.05, seed=21)
    ref = oracle.nve(d["x"], d["v"], d["box"], 20, DT, RC, SKIN)
    with lj_system(d, "mixed", 4) as s:
        s.step(20)
        x, v, _ = (a.cpu().numpy() for a in s.state())
    assert np.abs(wrap_diff(x, ref["x"], d["box"])).max() < 1e-6
    assert np.abs(v - ref["v"]).max() < 1e-4


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_nve_drift_below_bound(prec):
    # least-squares slope of E_tot/N (shifted LJ energy) x 1000 steps < 1e-4
    d = synth.lj_liquid(12, seed=1001)  # 6,912 atoms at T = 1.44
    from paper_1009_4330_gb300 import System
    es = []
    with System.lj(d["x"], d["v"], d["box"], cutoff=RC, skin=SKIN, dt=DT, mass=1.0, precision=prec, tpa=4,
                   energy_shift=True) as s:
        for k in range(21):
            ev = s.energy_virial().cpu().numpy()[0]
            es.append((ev[0] + ev[1]) / d["x"].shape[0])
            if k < 20:
                s.step(50)
    steps = np.arange(21) * 50
    slope = np.polyfit(steps, np.array(es), 1)[0]
    assert abs(slope) * 1000 < 1e-4, f"drift {slope * 1000:.2e} per atom per 1000 steps"
    assert np.abs(np.array(es) - es[0]).max() < 5e-3


# ------------------------------------------------------------------ EAM ----

@pytest.fixture(scope="module")
def eam_case():
    d = synth.config2(cells=8, displacement=0.1)  # 2,048 atoms
    x, box = d["x"], d["box"]
    assert margin_ok(x, box, d["rc"] + d["skin"])
    f, e, w, rho, fp = oracle.eam(x, box, d["eam"])
    return dict(d, f=f, e=e, w=w, nbr=oracle.neighbors(x, box, d["rc"] + d["skin"]),
                ke=oracle.kinetic(d["v"], d["mass"], ftm2v=d["ftm2v"]))


def eam_system(d, prec, tpa):
    from paper_1009_4330_gb300 import System
    return System.eam(d["x"], d["v"], d["box"], eam_params=d["eam"], skin=d["skin"], dt=d["dt"], mass=d["mass"],
                      ftm2v=d["ftm2v"], precision=prec, tpa=tpa)


@pytest.mark.parametrize("prec,tol", [("fp64", TOL_FP64), ("mixed", TOL_MIXED)])
@pytest.mark.parametrize("tpa", [1, 2, 8, 32])
def test_eam_forces_energy_virial(eam_case, prec, tol, tpa):
    d = eam_case
    with eam_system(d, prec, tpa) as s:
        counts, nbr = s.neighbors()
        assert_lists_equal(gpu_lists(counts, nbr), d["nbr"])
        f = s.compute_forces().cpu().numpy()
        ev = s.energy_virial().cpu().numpy()[0]
    assert rel_maxnorm(f, d["f"]) < tol
    assert ev[0] == pytest.approx(d["e"], rel=max(tol, 1e-7))
    assert ev[1] == pytest.approx(d["ke"], rel=1e-13)
    assert np.abs(ev[2:] - d["w"]).max() / np.abs(d["w"]).max() < max(tol, 1e-6)


def test_eam_trajectory_matches_oracle(eam_case):
    d = eam_case
    ref = oracle.nve(d["x"], d["v"], d["box"], 30, d["dt"], d["rc"], d["skin"], pot="eam", eam_params=d["eam"],
                     mass=d["mass"], ftm2v=d["ftm2v"])
    with eam_system(d, "fp64", 4) as s:
        s.step(30)
        x, v, _ = (a.cpu().numpy() for a in s.state())
    assert np.abs(wrap_diff(x, ref["x"], d["box"])).max() < 1e-9
    assert np.abs(v - ref["v"]).max() < 1e-11


# ------------------------------------------------------------- backward ----

@pytest.fixture(scope="module")
def ka_case():
    a = synth.fcc_constant(1.2)
    x, box = synth.fcc_lattice(4, 4, 8, a)
    x = synth.displace(x, box, 0.05, 4)
    t = synth.binary_types(x.shape[0], int(round(0.2 * x.shape[0])), 5)
    et, st = synth.pair_matrix(synth.KA_EPS), synth.pair_matrix(synth.KA_SIG)
    ftrue = oracle.lj(x, box, RC, eps=et, sig=st, types=t, n_types=2)[0]
    e0 = synth.pair_matrix(np.array(synth.KA_EPS) * [1.05, 0.95, 1.07])
    s0 = synth.pair_matrix(np.array(synth.KA_SIG) * [0.98, 1.03, 1.01])
    f0 = oracle.lj(x, box, RC, eps=e0, sig=s0, types=t, n_types=2)[0]
    g = 2 * (f0 - ftrue)
    gx, ge, gs = oracle.lj_vjp(x, box, RC, g, e0, s0, types=t, n_types=2)
    return dict(x=x, box=box, t=t, e0=e0, s0=s0, ftrue=ftrue, g=g, gx=gx, ge=ge, gs=gs)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("tpa", [1, 4, 32])
def test_backward_matches_oracle_vjp(ka_case, prec, tpa):
    from paper_1009_4330_gb300 import System
    c = ka_case
    v = np.zeros_like(c["x"])
    with System.lj(c["x"], v, c["box"], eps=c["e0"], sig=c["s0"], types=c["t"], n_types=2, cutoff=RC, skin=SKIN,
                   dt=DT, mass=[1.0, 1.0], precision=prec, tpa=tpa) as s:
        gx, gp = s.backward(c["g"])
    gx = gx.cpu().numpy()
    gp = gp.cpu().numpy()
    assert rel_maxnorm(gx, c["gx"]) < 1e-10
    assert np.allclose(gp[:4].reshape(2, 2), c["ge"], rtol=1e-10, atol=1e-10 * np.abs(c["ge"]).max())
    assert np.allclose(gp[4:].reshape(2, 2), c["gs"], rtol=1e-10, atol=1e-10 * np.abs(c["gs"]).max())


def test_autograd_function_against_central_fd(ka_case):
    import torch
    from paper_1009_4330_gb300 import LJForces, System
    c = ka_case
    v = np.zeros_like(c["x"])
    ep = torch.tensor([c["e0"][0, 0], c["e0"][0, 1], c["e0"][1, 1]], dtype=torch.float32, requires_grad=True)
    sp = torch.tensor([c["s0"][0, 0], c["s0"][0, 1], c["s0"][1, 1]], dtype=torch.float32, requires_grad=True)
    x = torch.tensor(c["x"], dtype=torch.float64, device="cuda", requires_grad=True)
    ft = torch.tensor(c["ftrue"], device="cuda")
    with System.lj(c["x"], v, c["box"], eps=c["e0"], sig=c["s0"], types=c["t"], n_types=2, cutoff=RC, skin=SKIN,
                   dt=DT, mass=[1.0, 1.0], precision="fp64", tpa=4) as s:
        f = LJForces.apply(s, x, ep, sp)
        loss = ((f - ft) ** 2).sum()
        loss.backward()
    # the oracle's loss, differenced centrally in each parameter (FP64)
    h = 1e-6
    t = c["t"]

    def L(e, sg):
        return float(((oracle.lj(c["x"], c["box"], RC, eps=e, sig=sg, types=t, n_types=2)[0] - c["ftrue"]) ** 2).sum())

    e0 = np.array([ep.detach().double().numpy()[k] for k in range(3)])
    s0 = np.array([sp.detach().double().numpy()[k] for k in range(3)])
    for k in range(3):
        for which, grad in (("eps", ep.grad), ("sig", sp.grad)):
            a = e0.copy(); b = s0.copy()
            ap = a.copy(); bp = b.copy(); am = a.copy(); bm = b.copy()
            if which == "eps":
                ap[k] += h; am[k] -= h
            else:
                bp[k] += h; bm[k] -= h
            fd = (L(synth.pair_matrix(ap), synth.pair_matrix(bp)) - L(synth.pair_matrix(am), synth.pair_matrix(bm))) / (2 * h)
            assert float(grad[k]) == pytest.approx(fd, rel=1e-5, abs=1e-6 * abs(fd) + 1e-6)
    # position gradient against the oracle's analytic VJP at the float32-rounded parameters
    e32 = synth.pair_matrix(e0)
    s32 = synth.pair_matrix(s0)
    f0 = oracle.lj(c["x"], c["box"], RC, eps=e32, sig=s32, types=t, n_types=2)[0]
    gx_ref = oracle.lj_vjp(c["x"], c["box"], RC, 2 * (f0 - c["ftrue"]), e32, s32, types=t, n_types=2)[0]
    assert rel_maxnorm(x.grad.cpu().numpy(), gx_ref) < 1e-9


# ---------------------------------------------------------------- batch ----

@pytest.fixture(scope="module")
def batch_case():
    sizes = [500, 777, 1234, 2048, 613, 3001]
    reps = []
    for r, n in enumerate(sizes):
        x, box = synth.fcc_subset(n, 0.8442, 900 + r)
        x = synth.displace(x, box, 0.05, 950 + r)
        v = synth.maxwell_boltzmann(n, 1.44, 1.0, 980 + r)
        reps.append({"x": x, "v": v, "box": box})
    return reps


@pytest.mark.parametrize("prec,tol", [("fp64", TOL_FP64), ("mixed", TOL_MIXED)])
def test_batch_forces_and_lists_per_replica(batch_case, prec, tol):
    from paper_1009_4330_gb300 import System, lj_params
    with System.batch(batch_case, params=lj_params(1.0, 1.0, 1), cutoff=RC, skin=SKIN, dt=DT, mass=1.0,
                      precision=prec, tpa=2) as s:
        f = s.compute_forces().cpu().numpy()
        counts, nbr = s.neighbors()
        lists = gpu_lists(counts, nbr)
        ev = s.energy_virial().cpu().numpy()
    o = 0
    for r, rep in enumerate(batch_case):
        n = rep["x"].shape[0]
        fr, er, wr = oracle.lj(rep["x"], rep["box"], RC)
        assert rel_maxnorm(f[o:o + n], fr) < tol
        ref = oracle.neighbors(rep["x"], rep["box"], RC + SKIN)
        assert_lists_equal(lists[o:o + n], ref)
        assert ev[r, 0] == pytest.approx(er, rel=max(tol, 1e-7))
        o += n


def test_batch_replica_equals_solo_run(batch_case):
    from paper_1009_4330_gb300 import System, lj_params
    with System.batch(batch_case, params=lj_params(1.0, 1.0, 1), cutoff=RC, skin=SKIN, dt=DT, mass=1.0,
                      precision="fp64", tpa=4) as b:
        b.step(60)
        xb, vb, _ = (a.cpu().numpy() for a in b.state())
    o = 0
    for rep in batch_case:
        n = rep["x"].shape[0]
        with lj_system(rep, "fp64", 4) as s:
            s.step(60)
            xs, vs, _ = (a.cpu().numpy() for a in s.state())
        # same replica, same kernels, same per-replica rebuild decisions: bitwise
        assert np.array_equal(xb[o:o + n], xs) and np.array_equal(vb[o:o + n], vs)
        o += n


def test_batch_trajectory_matches_oracle(batch_case):
    from paper_1009_4330_gb300 import System, lj_params
    with System.batch(batch_case[:3], params=lj_params(1.0, 1.0, 1), cutoff=RC, skin=SKIN, dt=DT, mass=1.0,
                      precision="fp64", tpa=1) as b:
        b.step(40)
        xb, vb, _ = (a.cpu().numpy() for a in b.state())
    o = 0
    for rep in batch_case[:3]:
        n = rep["x"].shape[0]
        ref = oracle.nve(rep["x"], rep["v"], rep["box"], 40, DT, RC, SKIN)
        assert np.abs(wrap_diff(xb[o:o + n], ref["x"], rep["box"])).max() < 1e-9
        o += n


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_partial_batch_rebuild_gives_exact_lists(batch_case, prec):
    """Step a batch until a step rebuilds some replicas but not all (the
    work-list build and sort passes): every replica rebuilt in that step has
    exactly the oracle's Verlet sets at the current positions, and every list is
    still valid (all pairs within rc present, none beyond rc + 2 skin)."""
    from paper_1009_4330_gb300 import System, lj_params
    n_rep = len(batch_case)
    with System.batch(batch_case, params=lj_params(1.0, 1.0, 1), cutoff=RC, skin=SKIN, dt=DT, mass=1.0,
                      precision=prec, tpa=1) as s:
        for _ in range(400):
            before = s.info()["rebuilds"]
            s.step(1)
            k = s.info()["rebuilds"] - before
            if 0 < k < n_rep:
                break
        else:
            pytest.fail("no step rebuilt a strict subset of the replicas")
        x = s.state()[0].cpu().numpy()
        counts, nbr = s.neighbors()
        lists = gpu_lists(counts, nbr)
    o = 0
    exact = 0
    for rep in batch_case:
        n = rep["x"].shape[0]
        xr, box = x[o:o + n], rep["box"]
        got = lists[o:o + n]
        ref = oracle.neighbors(xr, box, RC + SKIN)
        if margin_ok(xr, box, RC + SKIN) and all(np.array_equal(g, r) for g, r in zip(got, ref)):
            exact += 1
        inner = oracle.neighbors(xr, box, RC)
        outer = oracle.neighbors(xr, box, RC + 2 * SKIN)
        for i in range(n):
            assert set(inner[i].tolist()) <= set(got[i].tolist()) <= set(outer[i].tolist())
        o += n
    assert exact >= k


# --------------------------------------------------------------- errors ----

def test_list_overflow_grows_capacity():
    # a dense slab in a mostly empty box: the density-based first guess of the
    # list capacity is far too small, so the first build overflows and grows
    from paper_1009_4330_gb300 import System
    a = synth.fcc_constant(0.8442)
    x, _ = synth.fcc_lattice(6, 6, 6, a)
    box = np.array([6 * a, 6 * a, 60 * a])
    x = synth.displace(x, box, 0.05, 3)
    v = synth.maxwell_boltzmann(x.shape[0], 1.44, 1.0, 4)
    f_ref = oracle.lj(x, box, RC)[0]
    ref = oracle.neighbors(x, box, RC + SKIN)
    with System.lj(x, v, box, cutoff=RC, skin=SKIN, dt=DT, mass=1.0, precision="fp64", tpa=8) as s:
        inf = s.info()
        assert inf["maxneigh"] >= inf["max_count"] == max(map(len, ref))
        assert_lists_equal(gpu_lists(*s.neighbors()), ref)
        assert rel_maxnorm(s.compute_forces().cpu().numpy(), f_ref) < TOL_FP64
        s.step(20)
        s.sync_status()


def test_nonfinite_state_is_reported_and_recoverable():
    from paper_1009_4330_gb300 import MDError
    d = lj_case(6, 0.05, seed=8)
    with lj_system(d, "mixed", 4) as s:
        v = d["v"].copy()
        v[5, 1] = np.nan
        s.set_state(v=v)
        with pytest.raises(MDError) as ei:
            s.step(5)
        assert "NONFINITE" in str(ei.value)
        with pytest.raises(MDError):
            s.sync_status()  # latched word cleared by this call
        s.set_state(x=d["x"], v=d["v"])
        s.sync_status()
        s.step(5)


def test_box_too_small_rejected():
    from paper_1009_4330_gb300 import MDError, System
    x, box = synth.fcc_lattice(3, 3, 3, synth.fcc_constant(0.8442))
    with pytest.raises(MDError) as ei:
        System.lj(x, np.zeros_like(x), box, cutoff=RC, skin=SKIN, dt=DT, mass=1.0)
    assert "BOX_TOO_SMALL" in str(ei.value)


def test_set_state_and_params_roundtrip():
    d = lj_case(6, 0.08, seed=41)
    d2 = lj_case(6, 0.08, seed=42)
    with lj_system(d, "fp64", 2) as s:
        s.set_state(x=d2["x"], v=d2["v"])
        f = s.compute_forces().cpu().numpy()
        assert rel_maxnorm(f, oracle.lj(d2["x"], d2["box"], RC)[0]) < TOL_FP64
        from paper_1009_4330_gb300 import lj_params
        s.set_params(lj_params(1.3, 0.95, 1))
        f = s.compute_forces().cpu().numpy()
        assert rel_maxnorm(f, oracle.lj(d2["x"], d2["box"], RC, eps=1.3, sig=0.95)[0]) < TOL_FP64


def test_autotune_picks_a_valid_layout_and_keeps_parity(tmp_path):
    d = lj_case(8, 0.1, seed=51)
    f_ref = oracle.lj(d["x"], d["box"], RC)[0]
    cache = str(tmp_path / "tune.txt")
    with lj_system(d, "mixed", 1, lst="auto") as s:
        s.autotune(cache)
        inf = s.info()
        assert inf["tpa"] in (1, 2, 4, 8, 16, 32) and inf["list"] in ("full", "half")
        assert rel_maxnorm(s.compute_forces().cpu().numpy(), f_ref) < TOL_MIXED
    with lj_system(d, "mixed", 1, lst="auto") as s:
        s.autotune(cache)  # cache hit
        assert s.info()["tpa"] == inf["tpa"]


def test_backward_of_a_stale_forward_is_refused(ka_case):
    # the backward kernels differentiate at the system's current state: after a
    # step (or new parameters) the recorded forward no longer matches, and the
    # autograd functions refuse instead of returning wrong gradients
    import torch
    from paper_1009_4330_gb300 import LJForces, MDError, System
    c = ka_case
    v = np.zeros_like(c["x"])
    ep = torch.tensor([1.0, 1.5, 0.5], dtype=torch.float64, requires_grad=True)
    sp = torch.tensor([1.0, 0.8, 0.88], dtype=torch.float64, requires_grad=True)
    with System.lj(c["x"], v, c["box"], eps=c["e0"], sig=c["s0"], types=c["t"], n_types=2, cutoff=RC, skin=SKIN,
                   dt=DT, mass=[1.0, 1.0], precision="fp64", tpa=4) as s:
        f = LJForces.apply(s, None, ep, sp)
        s.step(1)
        with pytest.raises(MDError, match="stale"):
            f.sum().backward()
        f = LJForces.apply(s, None, ep, sp)
        f2 = LJForces.apply(s, None, ep * 1.01, sp)  # a second forward re-parameterises the system
        with pytest.raises(MDError, match="stale"):
            f.sum().backward()
        f2.sum().backward()  # the latest forward is still current
        assert ep.grad is not None and torch.isfinite(ep.grad).all()
