"""Pins of the oracle's Lennard-Jones forces, energy and virial.

Each check fixes the oracle to something other than itself: textbook values
of the 12-6 dimer, fcc lattice sums from an independent lattice enumeration,
and invariants (Newton's third law, F = -grad E, virial = -dE/dlambda).
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dimer(r, box=20.0, axis=0):
    x = np.zeros((2, 3)) + box / 2
    x[1, axis] += r
    return x, np.array([box, box, box])


# ---------------------------------------------------------------- dimer ----

def test_dimer_textbook_values():
    # sigma = eps = 1: U(1) = 0, |F(1)| = 24 and repulsive; minimum at 2^(1/6) with U = -1, F = 0
    x, box = dimer(1.0)
    f, e, _ = oracle.lj(x, box, 2.5)
    assert abs(e) < 1e-14
    assert f[0, 0] == pytest.approx(-24.0, abs=1e-12)  # atom 0 pushed away from atom 1 (at +x)
    assert f[1, 0] == pytest.approx(24.0, abs=1e-12)
    rm = 2.0 ** (1.0 / 6.0)
    assert rm == pytest.approx(1.122462048309373, abs=1e-15)
    x, box = dimer(rm)
    f, e, _ = oracle.lj(x, box, 2.5)
    assert e == pytest.approx(-1.0, abs=1e-14)
    assert np.abs(f).max() < 1e-13


def test_dimer_scales_with_eps_sigma():
    # U_{eps,sig}(r) = eps U_{1,1}(r/sig): minimum -eps at sig 2^(1/6); |F(sig)| = 24 eps/sig
    eps, sig = 1.5, 0.8
    x, box = dimer(sig * 2.0 ** (1.0 / 6.0))
    f, e, _ = oracle.lj(x, box, 2.5, eps=eps, sig=sig)
    assert e == pytest.approx(-1.5, abs=1e-13)
    assert np.abs(f).max() < 1e-12
    x, box = dimer(sig)
    f, e, _ = oracle.lj(x, box, 2.5, eps=eps, sig=sig)
    assert abs(e) < 1e-13
    assert f[1, 0] == pytest.approx(24.0 * eps / sig, rel=1e-14)


def test_dimer_cutoff_is_strict_and_periodic():
    # beyond rc nothing; across a periodic face the minimum image is used
    x, box = dimer(2.6)
    f, e, _ = oracle.lj(x, box, 2.5)
    assert e == 0.0 and np.all(f == 0.0)
    x = np.array([[0.1, 5.0, 5.0], [9.9 - 2.0 ** (1.0 / 6.0) + 0.2, 5.0, 5.0]])
    box = np.array([10.0, 10.0, 10.0])
    # separation across the face: 0.1 + (10 - x1) = 2^(1/6)
    x[1, 0] = 10.0 - (2.0 ** (1.0 / 6.0) - 0.1)
    f, e, _ = oracle.lj(x, box, 2.5)
    assert e == pytest.approx(-1.0, abs=1e-13)


def test_shift_subtracts_u_at_cutoff_per_pair():
    rng = np.random.default_rng(3)
    d = synth.lj_liquid(4, displacement=0.1)
    _, e0, _ = oracle.lj(d["x"], d["box"], 2.5)
    _, e1, _ = oracle.lj(d["x"], d["box"], 2.5, shift=True)
    # number of interacting pairs from the neighbour sets at r = rc
    npairs = sum(len(s) for s in oracle.neighbors(d["x"], d["box"], 2.5)) // 2
    uc = 4.0 * (2.5 ** -12 - 2.5 ** -6)
    assert e1 - e0 == pytest.approx(-npairs * uc, rel=1e-12)
    del rng


# -------------------------------------------------------- lattice sums ----

def fcc_shells(a, rmax):
    """Independent enumeration of fcc lattice vectors: {r^2 (units a^2/2): count}."""
    kmax = int(math.ceil(rmax / a)) + 1
    r = np.arange(-kmax, kmax + 1)
    cx, cy, cz = np.meshgrid(r, r, r, indexing="ij")
    cells = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], 1).astype(float)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    pts = (cells[:, None, :] + basis[None]).reshape(-1, 3)
    k = np.rint((pts ** 2).sum(1) * 2).astype(int)  # r^2 in units of a^2/2
    k = k[(k > 0) & (k * a * a / 2 < rmax * rmax)]
    vals, counts = np.unique(k, return_counts=True)
    return dict(zip(vals.tolist(), counts.tolist()))


def test_fcc_shell_enumeration_matches_textbook():
    table = {}
    with open(os.path.join(GOLDEN, "fcc_shells.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, c = line.split()
                table[int(k)] = int(c)
    shells = fcc_shells(1.0, 1.8)
    for k, c in table.items():
        assert shells[k] == c


@pytest.mark.parametrize("rc", [2.5, 5.0])
def test_fcc_lattice_energy_equals_shell_sum(rc):
    rho = 0.8442
    a = synth.fcc_constant(rho)
    cells = 10 if rc == 5.0 else 5
    x, box = synth.fcc_lattice(cells, cells, cells, a)
    f, e, w = oracle.lj(x, box, rc)
    fe, fs = oracle.lj(x, box, rc, shift=True)[1], None
    n = x.shape[0]
    shells = fcc_shells(a, rc)
    e_ref = 0.0
    w_ref = 0.0
    uc = 4.0 * (rc ** -12 - rc ** -6)
    nn = 0
    for k, c in shells.items():
        r = math.sqrt(k / 2.0) * a
        e_ref += 0.5 * c * 4.0 * (r ** -12 - r ** -6)
        w_ref += 0.5 * c * 24.0 * (2.0 * r ** -12 - r ** -6)  # r . f(r) per pair
        nn += c
    assert e / n == pytest.approx(e_ref, rel=1e-12)
    assert fe / n == pytest.approx(e_ref - 0.5 * nn * uc, rel=1e-12)
    assert (w[0] + w[1] + w[2]) / n == pytest.approx(w_ref, rel=1e-11)
    assert np.abs(f).max() < 1e-10  # perfect lattice: zero net force by symmetry
    assert nn == (54 if rc == 2.5 else 428)
    del fs


# ----------------------------------------------------------- invariants ---

def liquidish(cells=4, jitter=0.12, seed=5, rho=0.8442):
    a = synth.fcc_constant(rho)
    x, box = synth.fcc_lattice(cells, cells, cells, a)
    return synth.displace(x, box, jitter, seed), box


def test_newton_third_law_net_force_zero():
    x, box = liquidish(5)
    f, _, _ = oracle.lj(x, box, 2.5)
    assert np.abs(f.sum(0)).max() <= 1e-12 * np.abs(f).max() * math.sqrt(x.shape[0])


def test_force_is_minus_energy_gradient():
    x, box = liquidish(4, jitter=0.1, seed=9)
    f, _, _ = oracle.lj(x, box, 2.5, shift=True)
    rng = np.random.default_rng(1)
    h = 1e-5
    e0 = abs(oracle.lj(x, box, 2.5, shift=True)[1])
    # central difference: truncation O(h^2 |E'''|), rounding ~ 2 eps |E| / (2h)
    tol = 1e-6 * np.abs(f).max() * 1e-2 + 20 * np.finfo(float).eps * e0 / h
    assert oracle.min_gap(x, box, 2.5) > 2 * h  # no pair crosses the cut-off within +-h
    for i in rng.choice(x.shape[0], 6, replace=False):
        for a in range(3):
            xp = x.copy(); xp[i, a] += h
            xm = x.copy(); xm[i, a] -= h
            ep = oracle.lj(xp, box, 2.5, shift=True)[1]
            em = oracle.lj(xm, box, 2.5, shift=True)[1]
            assert -(ep - em) / (2 * h) == pytest.approx(f[i, a], abs=tol)


@pytest.mark.parametrize("axis", [None, 0, 2])
def test_virial_is_minus_dE_dlambda(axis):
    # E(lambda) under x -> lambda x, L -> lambda L (whole box, or one axis):
    # dE/dlambda at 1 = -sum_pairs d.f  (trace, or the axis' diagonal entry)
    x, box = liquidish(4, jitter=0.1, seed=11)
    rc = 2.5
    _, _, w = oracle.lj(x, box, rc, shift=True)
    h = 1e-6
    s = np.ones(3)

    def e_at(lam):
        sc = s.copy()
        if axis is None:
            sc[:] = lam
        else:
            sc[axis] = lam
        return oracle.lj(x * sc, box * sc, rc, shift=True)[1]

    dedl = (e_at(1 + h) - e_at(1 - h)) / (2 * h)
    ref = (w[0] + w[1] + w[2]) if axis is None else w[axis]
    assert -dedl == pytest.approx(ref, rel=1e-6)


def test_two_identical_types_equal_one_type():
    x, box = liquidish(4, seed=2)
    t = synth.binary_types(x.shape[0], 50, 4)
    f1, e1, w1 = oracle.lj(x, box, 2.5)
    f2, e2, w2 = oracle.lj(x, box, 2.5, eps=np.ones((2, 2)), sig=np.ones((2, 2)), types=t, n_types=2)
    assert np.array_equal(f1, f2) and e1 == e2 and np.array_equal(w1, w2)


def test_type_relabelling_is_symmetric():
    x, box = liquidish(4, seed=3)
    t = synth.binary_types(x.shape[0], 60, 7)
    eps = synth.pair_matrix(synth.KA_EPS)
    sig = synth.pair_matrix(synth.KA_SIG)
    f1, e1, _ = oracle.lj(x, box, 2.5, eps=eps, sig=sig, types=t, n_types=2)
    perm = np.array([1, 0])
    f2, e2, _ = oracle.lj(x, box, 2.5, eps=eps[perm][:, perm], sig=sig[perm][:, perm], types=1 - t, n_types=2)
    assert np.array_equal(f1, f2) and e1 == pytest.approx(e2, rel=1e-15)


def test_lj_at_matches_full():
    x, box = liquidish(4, seed=8)
    f, e, _ = oracle.lj(x, box, 2.5)
    idx = np.array([0, 17, 100, x.shape[0] - 1])
    fa, ea, ca = oracle.lj_at(x, box, 2.5, idx)
    assert np.array_equal(fa, f[idx])
    _, e_all, _ = oracle.lj_at(x, box, 2.5, np.arange(x.shape[0]))
    assert e_all.sum() == pytest.approx(e, rel=1e-13)
    nb = oracle.neighbors(x, box, 2.5, idx)
    assert [len(s) for s in nb] == ca.tolist()


def test_box_precondition_rejected():
    x, box = dimer(1.0, box=4.0)
    with pytest.raises(ValueError):
        oracle.lj(x, box, 2.5)


def test_virial_components_of_a_skew_dimer():
    # for one pair, W = d (x) f with f parallel to d, so every entry is
    # W_aa * d_b / d_a: fixes the order xx, yy, zz, xy, xz, yz
    u = np.array([1.0, 2.0, 3.0]) / math.sqrt(14.0)
    x = np.array([[6.0, 6.0, 6.0], [6.0, 6.0, 6.0]]) + 0.0
    x[0] += 1.1 * u  # d = x0 - x1 = 1.1 u
    box = np.array([12.0, 12.0, 12.0])
    _, _, w = oracle.lj(x, box, 2.5)
    wxx, wyy, wzz, wxy, wxz, wyz = w
    assert wyy == pytest.approx(4 * wxx, rel=1e-13) and wzz == pytest.approx(9 * wxx, rel=1e-13)
    assert wxy == pytest.approx(2 * wxx, rel=1e-13)
    assert wxz == pytest.approx(3 * wxx, rel=1e-13)
    assert wyz == pytest.approx(6 * wxx, rel=1e-13)
    # the trace is d.f = r |f| along the pair (repulsive at 1.1 < 2^(1/6))
    assert wxx + wyy + wzz > 0
