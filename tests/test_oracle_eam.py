"""Pins of the oracle's Finnis-Sinclair EAM (the paper's App. A EAM benchmark;
analytic form rho = (rc-r)^2, F = -A sqrt(rho), phi = (rc-r)^2 (c0+c1 r+c2 r^2)).
"""
import math

import numpy as np
import pytest

import oracle
import synth

P = np.array(synth.EAM_PARAMS)


def fcc_shells(a, rmax):
    kmax = int(math.ceil(rmax / a)) + 1
    r = np.arange(-kmax, kmax + 1)
    cx, cy, cz = np.meshgrid(r, r, r, indexing="ij")
    cells = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], 1).astype(float)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    pts = (cells[:, None, :] + basis[None]).reshape(-1, 3)
    k = np.rint((pts ** 2).sum(1) * 2).astype(int)
    k = k[(k > 0) & (k * a * a / 2 < rmax * rmax)]
    vals, counts = np.unique(k, return_counts=True)
    return [(math.sqrt(v / 2.0) * a, c) for v, c in zip(vals.tolist(), counts.tolist())]


def test_fcc_lattice_energy_from_shells():
    a = 3.615
    x, box = synth.fcc_lattice(4, 4, 4, a)
    f, e, w, rho, fp = oracle.eam(x, box, P)
    rc, A, c0, c1, c2 = P
    shells = fcc_shells(a, rc)
    assert [c for _, c in shells] == [12, 6, 24]
    rho_ref = sum(c * (rc - r) ** 2 for r, c in shells)
    pair_ref = 0.5 * sum(c * (rc - r) ** 2 * (c0 + c1 * r + c2 * r * r) for r, c in shells)
    assert np.allclose(rho, rho_ref, rtol=1e-13)
    assert fp[0] == pytest.approx(-0.5 * A / math.sqrt(rho_ref), rel=1e-13)
    assert e / x.shape[0] == pytest.approx(-A * math.sqrt(rho_ref) + pair_ref, rel=1e-13)
    assert np.abs(f).max() < 1e-11


def dimer(r, box=20.0):
    x = np.zeros((2, 3)) + box / 2
    x[1, 0] += r
    return x, np.array([box, box, box])


def test_pure_embedding_dimer_closed_form():
    # c = 0: E = 2 F(rho) with rho = (rc - r)^2 on both atoms = -2 A (rc - r);
    # dE/dr = 2 A, so atom 0 (at smaller x) is pulled toward atom 1 with |F| = 2A
    p = np.array([4.95, 1.3, 0.0, 0.0, 0.0])
    x, box = dimer(3.0)
    f, e, _, rho, _ = oracle.eam(x, box, p)
    assert e == pytest.approx(-2 * 1.3 * 1.95, rel=1e-14)
    assert rho == pytest.approx([1.95 ** 2] * 2, rel=1e-14)
    assert f[0, 0] == pytest.approx(2 * 1.3, rel=1e-14)
    assert f[1, 0] == pytest.approx(-2 * 1.3, rel=1e-14)


def test_isolated_atom_has_zero_density_and_energy():
    x, box = dimer(6.0)
    f, e, _, rho, fp = oracle.eam(x, box, P)
    assert e == 0.0 and np.all(rho == 0) and np.all(fp == 0) and np.all(f == 0)


def jittered(cells=4, s=0.08, seed=3):
    x, box = synth.fcc_lattice(cells, cells, cells, 3.615)
    return synth.displace(x, box, s, seed), box


def test_newton_third_law():
    x, box = jittered(4)
    f = oracle.eam(x, box, P)[0]
    assert np.abs(f.sum(0)).max() <= 1e-12 * np.abs(f).max() * math.sqrt(x.shape[0])


def test_force_is_minus_energy_gradient():
    x, box = jittered(4, 0.1, 5)
    f = oracle.eam(x, box, P)[0]
    rng = np.random.default_rng(2)
    h = 1e-5
    e0 = abs(oracle.eam(x, box, P)[1])
    # central difference: truncation O(h^2 |E'''|), rounding ~ 2 eps |E| / (2h)
    tol = 1e-8 + 20 * np.finfo(float).eps * e0 / h
    for i in rng.choice(x.shape[0], 5, replace=False):
        for a in range(3):
            xp = x.copy(); xp[i, a] += h
            xm = x.copy(); xm[i, a] -= h
            d = -(oracle.eam(xp, box, P)[1] - oracle.eam(xm, box, P)[1]) / (2 * h)
            assert d == pytest.approx(f[i, a], abs=tol)


@pytest.mark.parametrize("axis", [None, 1])
def test_virial_is_minus_dE_dlambda(axis):
    x, box = jittered(4, 0.1, 6)
    w = oracle.eam(x, box, P)[2]
    h = 1e-6

    def e_at(lam):
        s = np.ones(3)
        if axis is None:
            s[:] = lam
        else:
            s[axis] = lam
        return oracle.eam(x * s, box * s, P)[1]

    dedl = (e_at(1 + h) - e_at(1 - h)) / (2 * h)
    ref = (w[0] + w[1] + w[2]) if axis is None else w[axis]
    assert -dedl == pytest.approx(ref, rel=1e-6)


def test_eam_at_matches_full():
    x, box = jittered(4, 0.1, 7)
    f, _, _, rho, _ = oracle.eam(x, box, P)
    idx = np.array([0, 5, 200])
    fa, ra = oracle.eam_at(x, box, P, idx)
    assert np.allclose(fa, f[idx], rtol=0, atol=1e-13 * np.abs(f).max())
    assert np.allclose(ra, rho[idx], rtol=1e-14)


def test_virial_components_of_a_skew_dimer():
    u = np.array([3.0, 1.0, 2.0]) / math.sqrt(14.0)
    x = np.array([[10.0, 10.0, 10.0], [10.0, 10.0, 10.0]])
    x[0] += 2.9 * u
    box = np.array([20.0, 20.0, 20.0])
    w = oracle.eam(x, box, P)[2]
    wxx, wyy, wzz, wxy, wxz, wyz = w
    assert wyy == pytest.approx(wxx / 9, rel=1e-13) and wzz == pytest.approx(4 * wxx / 9, rel=1e-13)
    assert wxy == pytest.approx(wxx / 3, rel=1e-13)
    assert wxz == pytest.approx(2 * wxx / 3, rel=1e-13)
    assert wyz == pytest.approx(2 * wxx / 9, rel=1e-13)
