"""Pins of the oracle's EAM force backward pass (L = sum_i g_i.F_i for the
Finnis-Sinclair form of App. A): the dimer in closed form (where the embedding
terms of the chain rule must cancel, the dimer's embedding energy being linear
in r), central finite differences of the loss in every parameter and in
positions, and zero gradients beyond the cut-off."""
import numpy as np
import pytest
from numpy.polynomial import Polynomial

import oracle
import synth

P = synth.EAM_PARAMS  # rc, A, c0, c1, c2


def metal(cells=3, jitter=0.1, seed=3):
    x, box = synth.fcc_lattice(cells, cells, cells, 3.615)
    return synth.displace(x, box, jitter, seed), box


def linear_loss(x, box, p, g):
    return float((oracle.eam(x, box, p)[0] * g).sum())


def test_dimer_closed_form():
    rc, A, c0, c1, c2 = P
    x = np.array([[5.0, 5.0, 5.0], [7.2, 5.9, 4.6]])
    box = np.array([12.0, 12.0, 12.0])
    g = np.array([[0.3, -0.2, 0.5], [0.1, 0.4, -0.6]])
    gx, gp = oracle.eam_vjp(x, box, P, g)
    d = x[0] - x[1]
    r = np.linalg.norm(d)
    u = d / r
    assert r < rc
    # dimer energy: phi(r) + 2 F(rho) with rho = (rc - r)^2, i.e. phi(r) - 2 A (rc - r)
    t = Polynomial([rc, -1.0])
    phi = t**2 * Polynomial([c0, c1, c2])
    e1 = phi.deriv()(r) + 2 * A
    e2 = phi.deriv(2)(r)
    w = (g[0] - g[1]) @ u
    assert gp[0] == 0.0
    assert gp[1] == pytest.approx(-2 * w, rel=1e-13)
    for q in range(3):
        dphi_dc = (t**2 * Polynomial([0.0] * q + [1.0])).deriv()(r)
        assert gp[2 + q] == pytest.approx(-w * dphi_dc, rel=1e-12)
    m = -(e2 * np.outer(u, u) + (e1 / r) * (np.eye(3) - np.outer(u, u)))
    assert np.allclose(gx[0], m @ (g[0] - g[1]), rtol=1e-12, atol=1e-14)
    assert np.allclose(gx[1], -gx[0], rtol=1e-12, atol=1e-14)


def test_beyond_cutoff_is_zero():
    x = np.array([[1.0, 1.0, 1.0], [6.5, 1.0, 1.0]])
    gx, gp = oracle.eam_vjp(x, np.array([12.0, 12.0, 12.0]), P, np.ones((2, 3)))
    assert not gx.any() and not gp.any()


def test_parameter_gradient_matches_central_fd():
    x, box = metal()
    g = np.random.default_rng(11).standard_normal(x.shape)
    _, gp = oracle.eam_vjp(x, box, P, g)
    for q in range(1, 5):
        h = 1e-6 * max(1.0, abs(P[q]))
        pp, pm = list(P), list(P)
        pp[q] += h
        pm[q] -= h
        fd = (linear_loss(x, box, pp, g) - linear_loss(x, box, pm, g)) / (2 * h)
        assert gp[q] == pytest.approx(fd, rel=2e-6, abs=1e-8 * np.abs(gp).max())


def test_position_gradient_matches_central_fd():
    x, box = metal(seed=8)
    g = np.random.default_rng(12).standard_normal(x.shape)
    gx, _ = oracle.eam_vjp(x, box, P, g)
    rng = np.random.default_rng(1)
    idx = rng.choice(x.shape[0], 4, replace=False)
    h = 1e-6
    # the force derivatives jump where a pair crosses rc: keep those away from +-h
    assert oracle.min_gap(x, box, P[0], idx) > 1e-4
    for i in idx:
        for a in range(3):
            xp = x.copy(); xp[i, a] += h
            xm = x.copy(); xm[i, a] -= h
            fd = (linear_loss(xp, box, P, g) - linear_loss(xm, box, P, g)) / (2 * h)
            assert gx[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(gx).max())


def test_force_matching_loss_gradient():
    # L = sum |F(theta) - F*|^2, g = 2 (F - F*): FD of the full quadratic loss in A
    x, box = metal(seed=5)
    ftrue = oracle.eam(x, box, P)[0]
    p0 = list(P)
    p0[1] *= 1.07
    f0 = oracle.eam(x, box, p0)[0]
    _, gp = oracle.eam_vjp(x, box, p0, 2 * (f0 - ftrue))
    h = 1e-6

    def loss(pa):
        p = list(p0)
        p[1] = pa
        return float(((oracle.eam(x, box, p)[0] - ftrue) ** 2).sum())
    fd = (loss(p0[1] + h) - loss(p0[1] - h)) / (2 * h)
    assert gp[1] == pytest.approx(fd, rel=1e-6)
