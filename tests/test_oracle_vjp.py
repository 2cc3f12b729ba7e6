"""Pins of the oracle's LJ force backward pass (force matching, the
differentiable extension of the pair-force step): central finite differences
of the loss, the zero gradient at the true parameters and the dimer Jacobian.
"""
import numpy as np
import pytest

import oracle
import synth


def binary_system(shape=(4, 4, 8), seed=5):
    a = synth.fcc_constant(1.2)
    x, box = synth.fcc_lattice(*shape, a)
    x = synth.displace(x, box, 0.05, seed)
    t = synth.binary_types(x.shape[0], int(round(0.2 * x.shape[0])), seed + 1)
    return x, box, t


def loss(x, box, t, eps, sig, ftarget, rc=2.5):
    f = oracle.lj(x, box, rc, eps=eps, sig=sig, types=t, n_types=2)[0]
    return float(((f - ftarget) ** 2).sum()), f


def test_parameter_gradient_matches_central_fd():
    x, box, t = binary_system()
    et, st = synth.pair_matrix(synth.KA_EPS), synth.pair_matrix(synth.KA_SIG)
    ftrue = oracle.lj(x, box, 2.5, eps=et, sig=st, types=t, n_types=2)[0]
    e0 = synth.pair_matrix(np.array(synth.KA_EPS) * [1.05, 0.93, 1.08])
    s0 = synth.pair_matrix(np.array(synth.KA_SIG) * [0.97, 1.04, 1.02])
    _, f = loss(x, box, t, e0, s0, ftrue)
    g = 2 * (f - ftrue)
    _, ge, gs = oracle.lj_vjp(x, box, 2.5, g, e0, s0, types=t, n_types=2)
    assert np.array_equal(ge, ge.T) and np.array_equal(gs, gs.T)
    h = 1e-6
    for (a, b) in [(0, 0), (0, 1), (1, 1)]:
        for which, grad in (("eps", ge), ("sig", gs)):
            def perturbed(delta):
                e, s = e0.copy(), s0.copy()
                m = e if which == "eps" else s
                m[a, b] += delta
                if a != b:
                    m[b, a] += delta
                return loss(x, box, t, e, s, ftrue)[0]
            fd = (perturbed(h) - perturbed(-h)) / (2 * h)
            assert grad[a, b] == pytest.approx(fd, rel=1e-6, abs=1e-6 * abs(fd) + 1e-9)


def test_position_gradient_matches_central_fd():
    x, box, t = binary_system(seed=9)
    et, st = synth.pair_matrix(synth.KA_EPS), synth.pair_matrix(synth.KA_SIG)
    ftrue = oracle.lj(x, box, 2.5, eps=et, sig=st, types=t, n_types=2)[0]
    e0 = et * 1.02
    _, f = loss(x, box, t, e0, st, ftrue)
    gx, _, _ = oracle.lj_vjp(x, box, 2.5, 2 * (f - ftrue), e0, st, types=t, n_types=2)
    # FD needs no pair to cross rc within +-h: check the sampled atoms' margins
    rng = np.random.default_rng(0)
    h = 1e-6
    idx = rng.choice(x.shape[0], 4, replace=False)
    assert oracle.min_gap(x, box, 2.5, idx) > 1e-4
    for i in idx:
        for a in range(3):
            xp = x.copy(); xp[i, a] += h
            xm = x.copy(); xm[i, a] -= h
            fd = (loss(xp, box, t, e0, st, ftrue)[0] - loss(xm, box, t, e0, st, ftrue)[0]) / (2 * h)
            assert gx[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(gx).max())


def test_gradient_vanishes_at_truth():
    x, box, t = binary_system(seed=2)
    et, st = synth.pair_matrix(synth.KA_EPS), synth.pair_matrix(synth.KA_SIG)
    f = oracle.lj(x, box, 2.5, eps=et, sig=st, types=t, n_types=2)[0]
    gx, ge, gs = oracle.lj_vjp(x, box, 2.5, 2 * (f - f), et, st, types=t, n_types=2)
    assert not gx.any() and not ge.any() and not gs.any()


def test_dimer_jacobian_by_fd():
    # for a dimer, grad_x of atom 0 with g = e_k on atom 0 is column k of dF_0/dx_0
    x = np.array([[5.0, 5.0, 5.0], [6.0, 5.3, 4.8]])
    box = np.array([12.0, 12.0, 12.0])
    h = 1e-6
    for k in range(3):
        g = np.zeros((2, 3)); g[0, k] = 1.0
        gx, _, _ = oracle.lj_vjp(x, box, 2.5, g, 1.0, 1.0)
        for a in range(3):
            xp = x.copy(); xp[0, a] += h
            xm = x.copy(); xm[0, a] -= h
            dfa = (oracle.lj(xp, box, 2.5)[0][0, k] - oracle.lj(xm, box, 2.5)[0][0, k]) / (2 * h)
            assert gx[0, a] == pytest.approx(dfa, rel=1e-7, abs=1e-7)
