"""Gradients of the force-matching workload at its full size: the binary LJ
mixture of 32,768 atoms (16 x 16 x 32 fcc cells at density 1.2, 6,554 type-B
atoms, start parameters a seeded +-10 % away from the true ones), loss
L = sum_i |F_i(theta) - F*_i|^2 with F* the forces at the true parameters.

* The backward kernel (md_forces_backward), given the oracle's dL/dF, equals
  the oracle's FP64 vector-Jacobian product element by element to 1e-10
  (relative max-norm) for dL/dx and for all six (eps, sigma) entries, in both
  precision modes (the backward pass is FP64 in both).
* LJForces (FP64 forward) gives dL/dtheta and dL/dx within 1e-6 (relative)
  of central finite differences of the ORACLE's loss, for all six parameters
  and for sampled positions.  eps enters F linearly, so L is quadratic in
  eps and the two-point difference is exact up to rounding; sigma and
  positions use the fourth-order difference (8 [L(h) - L(-h)] - [L(2h) -
  L(-2h)]) / 12h.  Sampled positions keep every pair at least 1e-3 from rc
  (the force jumps at rc, so a difference across it measures the jump).
  The parameters are FP32 learnable tensors, so the differences are taken
  at their FP32 values.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import rel_maxnorm

pytestmark = pytest.mark.gpu

RC, SKIN, DT = 2.5, 0.3, 0.005
PAIRS = ((0, 0), (0, 1), (1, 1))  # AA, AB, BB


@pytest.fixture(scope="module")
def fm():
    c = synth.config3()
    x, box, t = c["x"], c["box"], c["types"]
    assert x.shape[0] == 32768 and int((t == 1).sum()) == 6554
    # the learnable start values as FP32 tensors hold them
    e0 = np.array(c["eps0"], np.float32).astype(np.float64)
    s0 = np.array(c["sig0"], np.float32).astype(np.float64)
    et, st = synth.pair_matrix(c["eps_true"]), synth.pair_matrix(c["sig_true"])
    ftrue = oracle.lj(x, box, RC, eps=et, sig=st, types=t, n_types=2)[0]
    f0 = oracle.lj(x, box, RC, eps=synth.pair_matrix(e0), sig=synth.pair_matrix(s0), types=t, n_types=2)[0]
    g = 2.0 * (f0 - ftrue)
    gx, ge, gs = oracle.lj_vjp(x, box, RC, g, synth.pair_matrix(e0), synth.pair_matrix(s0), types=t, n_types=2)
    return dict(x=x, box=box, t=t, e0=e0, s0=s0, ftrue=ftrue, f0=f0, g=g, gx=gx, ge=ge, gs=gs)


def _system(c, prec, tpa):
    from paper_1009_4330_gb300 import System
    v = np.zeros_like(c["x"])
    return System.lj(c["x"], v, c["box"], eps=synth.pair_matrix(c["e0"]), sig=synth.pair_matrix(c["s0"]),
                     types=c["t"], n_types=2, cutoff=RC, skin=SKIN, dt=DT, mass=[1.0, 1.0], precision=prec, tpa=tpa)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("tpa", [1, 8])
def test_backward_equals_oracle_vjp_at_full_size(fm, prec, tpa):
    c = fm
    with _system(c, prec, tpa) as s:
        gx, gp = s.backward(c["g"])
    gx, gp = gx.cpu().numpy(), gp.cpu().numpy()
    assert rel_maxnorm(gx, c["gx"]) < 1e-10
    for a, b in PAIRS:
        for got, ref in ((gp[a * 2 + b], c["ge"][a, b]), (gp[4 + a * 2 + b], c["gs"][a, b])):
            assert abs(got - ref) <= 1e-10 * abs(ref), (prec, tpa, a, b, got, ref)


def _loss(c, e, s, x=None, idx=None):
    """The oracle's loss; with idx, only the terms of atoms idx (the others do
    not change when only atoms whose neighbours are all in idx move)."""
    x = c["x"] if x is None else x
    kw = dict(eps=synth.pair_matrix(e), sig=synth.pair_matrix(s), types=c["t"], n_types=2)
    if idx is None:
        f = oracle.lj(x, c["box"], RC, **kw)[0]
        return float(((f - c["ftrue"]) ** 2).sum())
    f = oracle.lj_at(x, c["box"], RC, idx, **kw)[0]
    return float(((f - c["ftrue"][idx]) ** 2).sum())


def _fd4(fun, h):
    return (8.0 * (fun(h) - fun(-h)) - (fun(2 * h) - fun(-2 * h))) / (12.0 * h)


def test_ljforces_gradients_match_central_fd_of_oracle_loss(fm):
    import torch
    from paper_1009_4330_gb300 import LJForces
    c = fm
    ep = torch.tensor([c["e0"][k] for k in range(3)], dtype=torch.float32, requires_grad=True)
    sp = torch.tensor([c["s0"][k] for k in range(3)], dtype=torch.float32, requires_grad=True)
    x = torch.tensor(c["x"], dtype=torch.float64, device="cuda", requires_grad=True)
    ft = torch.tensor(c["ftrue"], device="cuda")
    with _system(c, "fp64", 4) as s:
        f = LJForces.apply(s, x, ep, sp)
        loss = ((f - ft) ** 2).sum()
        loss.backward()
    # the forward at the FP32 parameters is the oracle's (FP64 parity)
    assert rel_maxnorm(f.detach().cpu().numpy(), c["f0"]) < 1e-12
    # parameters: six central differences of the oracle's loss
    for k in range(3):
        def along_eps(h, k=k):
            e = c["e0"].copy()
            e[k] += h
            return _loss(c, e, c["s0"])

        def along_sig(h, k=k):
            sg = c["s0"].copy()
            sg[k] += h
            return _loss(c, c["e0"], sg)

        fd_e = (along_eps(1e-3 * c["e0"][k]) - along_eps(-1e-3 * c["e0"][k])) / (2e-3 * c["e0"][k])
        fd_s = _fd4(along_sig, 1e-4 * c["s0"][k])
        assert float(ep.grad[k]) == pytest.approx(fd_e, rel=1e-6), ("eps", k)
        assert float(sp.grad[k]) == pytest.approx(fd_s, rel=1e-6), ("sigma", k)
    # positions: sampled atoms away from the cut-off discontinuity
    gx = x.grad.cpu().numpy()
    rng = np.random.default_rng(33)
    cand = rng.choice(c["x"].shape[0], 64, replace=False)
    idx = [int(i) for i in cand if oracle.min_gap(c["x"], c["box"], RC, [int(i)]) > 1e-3][:12]
    assert len(idx) >= 8
    fd, an = [], []
    for i in idx:
        near = oracle.neighbors(c["x"], c["box"], RC + SKIN, [i])[0]
        terms = np.concatenate([[i], near]).astype(np.int64)  # the atoms whose forces x_i moves
        for a in range(3):
            def along(h, i=i, a=a):
                xx = c["x"].copy()
                xx[i, a] += h
                return _loss(c, c["e0"], c["s0"], x=xx, idx=terms)
            fd.append(_fd4(along, 1e-5))
            an.append(gx[i, a])
    fd, an = np.array(fd), np.array(an)
    assert np.abs(an - fd).max() <= 1e-6 * np.abs(fd).max(), (np.abs(an - fd).max(), np.abs(fd).max())
