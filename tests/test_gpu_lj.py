"""GPU parity of the LJ path against the oracle: neighbour lists (exact),
forces (FP64 1e-12, mixed 1e-5 relative max-norm), energy, kinetic energy
and virial, for every threads-per-atom layout and both list kinds."""
import numpy as np
import pytest

import oracle
from gpu_util import (TOL_FP64, TOL_MIXED, TPAS, assert_lists_equal, gpu_lists, half_pairs,
                      lj_case, margin_ok, oracle_pairs, ragged_case, rel_maxnorm)

pytestmark = pytest.mark.gpu

RC, SKIN = 2.5, 0.3


@pytest.fixture(scope="module")
def cases():
    out = {}
    for name, d in (("lj4000", lj_case(10, 0.1, seed=1000)), ("lj500", lj_case(5, 0.12, seed=5)),
                    ("ragged777", ragged_case())):
        x, box = d["x"], d["box"]
        assert margin_ok(x, box, RC + SKIN)
        f, e, w = oracle.lj(x, box, RC)
        ref = oracle.neighbors(x, box, RC + SKIN)
        out[name] = dict(d, f=f, e=e, w=w, nbr=ref, ke=oracle.kinetic(d["v"], [1.0]))
    return out


def make(d, prec, tpa, lst):
    from paper_1009_4330_gb300 import System
    return System.lj(d["x"], d["v"], d["box"], cutoff=RC, skin=SKIN, dt=0.005, mass=1.0, precision=prec,
                     list=lst, tpa=tpa)


@pytest.mark.parametrize("name", ["lj4000", "lj500", "ragged777"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("tpa", [1, 4, 32])
def test_full_list_equals_oracle(cases, name, prec, tpa):
    d = cases[name]
    with make(d, prec, tpa, "full") as s:
        counts, nbr = s.neighbors()
        assert_lists_equal(gpu_lists(counts, nbr), d["nbr"])


@pytest.mark.parametrize("name", ["lj4000", "ragged777"])
@pytest.mark.parametrize("tpa", [1, 8])
def test_half_list_holds_each_pair_once(cases, name, tpa):
    d = cases[name]
    with make(d, "mixed", tpa, "half") as s:
        counts, nbr = s.neighbors()
        assert int(counts.sum()) == sum(map(len, d["nbr"])) // 2
        assert half_pairs(counts, nbr) == oracle_pairs(d["nbr"])


@pytest.mark.parametrize("name", ["lj4000", "ragged777"])
@pytest.mark.parametrize("prec,tol", [("fp64", TOL_FP64), ("mixed", TOL_MIXED)])
@pytest.mark.parametrize("tpa", TPAS)
@pytest.mark.parametrize("lst", ["full", "half"])
def test_forces_match_oracle(cases, name, prec, tol, tpa, lst):
    d = cases[name]
    with make(d, prec, tpa, lst) as s:
        f = s.compute_forces().cpu().numpy()
    err = rel_maxnorm(f, d["f"])
    assert err < tol, f"{prec} tpa={tpa} {lst}: {err:.3e}"


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
@pytest.mark.parametrize("lst", ["full", "half"])
def test_energy_kinetic_virial(cases, prec, tol, lst):
    d = cases["lj4000"]
    with make(d, prec, 4, lst) as s:
        ev = s.energy_virial().cpu().numpy()[0]
    assert ev[0] == pytest.approx(d["e"], rel=tol)
    assert ev[1] == pytest.approx(d["ke"], rel=1e-13)
    w = d["w"]
    scale = np.abs(w).max()
    assert np.abs(ev[2:] - w).max() / scale < tol


def test_energy_shift_and_multitype():
    import synth
    from paper_1009_4330_gb300 import System
    d = lj_case(6, 0.1, seed=31)
    x, box = d["x"], d["box"]
    t = synth.binary_types(x.shape[0], 170, 3)
    eps, sig = synth.pair_matrix(synth.KA_EPS), synth.pair_matrix(synth.KA_SIG)
    f, e, w = oracle.lj(x, box, RC, eps=eps, sig=sig, types=t, n_types=2, shift=True)
    for prec, tol in (("fp64", 1e-12), ("mixed", 1e-5)):
        for tpa in (1, 8):
            with System.lj(x, d["v"], box, eps=eps, sig=sig, types=t, n_types=2, cutoff=RC, skin=SKIN, dt=0.005,
                           mass=[1.0, 1.0], energy_shift=True, precision=prec, tpa=tpa) as s:
                assert rel_maxnorm(s.compute_forces().cpu().numpy(), f) < tol
                ev = s.energy_virial().cpu().numpy()[0]
                assert ev[0] == pytest.approx(e, rel=10 * tol)


def test_state_roundtrip_in_original_order(cases):
    d = cases["ragged777"]
    with make(d, "fp64", 2, "full") as s:
        x, v, f = s.state()
        x = x.cpu().numpy()
        assert np.abs(x - d["x"]).max() < 1e-12  # inputs already inside the box
        assert np.array_equal(v.cpu().numpy(), d["v"])
        assert rel_maxnorm(f.cpu().numpy(), d["f"]) < TOL_FP64


def test_repeat_runs_are_bitwise_identical(cases):
    d = cases["lj4000"]
    outs = []
    for _ in range(2):
        with make(d, "fp64", 4, "full") as s:
            s.step(30)
            outs.append([a.cpu().numpy() for a in s.state()])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
