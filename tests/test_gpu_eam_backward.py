"""GPU parity of the EAM force backward (two list passes, chain rule through
F'(rho)) against the oracle's vector-Jacobian product, for both precision
modes and several thread-group sizes, plus the autograd wrapper against
central differences of a force-matching loss."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import margin_ok, rel_maxnorm

pytestmark = pytest.mark.gpu

P = np.array(synth.EAM_PARAMS)
SKIN = 0.5


def metal_case(cells, jitter, seed, n=None):
    x, box = synth.fcc_lattice(cells, cells, cells, 3.615)
    if n is not None:  # ragged: a random subset of the sites
        keep = np.sort(np.random.default_rng(seed + 7).choice(x.shape[0], n, replace=False))
        x = x[keep]
    x = synth.displace(x, box, jitter, seed)
    assert margin_ok(x, box, P[0] + SKIN) and margin_ok(x, box, P[0], margin=1e-9)
    g = np.random.default_rng(seed + 1).standard_normal(x.shape)
    gx, gp = oracle.eam_vjp(x, box, P, g)
    return dict(x=x, box=box, g=g, gx=gx, gp=gp)


@pytest.fixture(scope="module")
def cases():
    return {"eam256": metal_case(4, 0.1, 21), "eam_ragged601": metal_case(6, 0.12, 33, n=601)}


def make(c, prec, tpa):
    from paper_1009_4330_gb300 import System
    v = np.zeros_like(c["x"])
    return System.eam(c["x"], v, c["box"], eam_params=P, skin=SKIN, dt=1.0, mass=63.55, ftm2v=synth.FTM2V_METAL,
                      precision=prec, tpa=tpa)


@pytest.mark.parametrize("name", ["eam256", "eam_ragged601"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("tpa", [1, 4, 32])
def test_backward_matches_oracle_vjp(cases, name, prec, tpa):
    c = cases[name]
    with make(c, prec, tpa) as s:
        gx, gp = s.backward(c["g"])
    gx, gp = gx.cpu().numpy(), gp.cpu().numpy()
    assert rel_maxnorm(gx, c["gx"]) < 1e-11
    assert gp[0] == 0.0
    assert np.allclose(gp[1:], c["gp"][1:], rtol=1e-11, atol=1e-11 * np.abs(c["gp"]).max())


def test_autograd_against_central_fd(cases):
    import torch
    from paper_1009_4330_gb300 import EAMForces
    c = cases["eam256"]
    ftrue = oracle.eam(c["x"], c["box"], P)[0]
    p0 = P.copy()
    p0[1:] *= [1.06, 0.95, 1.04, 0.97]
    pt = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    x = torch.tensor(c["x"], dtype=torch.float64, device="cuda", requires_grad=True)
    with make(c, "fp64", 4) as s:
        f = EAMForces.apply(s, x, pt)
        loss = ((f - torch.tensor(ftrue, device="cuda")) ** 2).sum()
        loss.backward()
    assert pt.grad[0].item() == 0.0

    def L(p, xx=c["x"]):
        return float(((oracle.eam(xx, c["box"], p)[0] - ftrue) ** 2).sum())
    for q in range(1, 5):
        h = 1e-6 * max(1.0, abs(p0[q]))
        pp, pm = p0.copy(), p0.copy()
        pp[q] += h
        pm[q] -= h
        fd = (L(pp) - L(pm)) / (2 * h)
        assert pt.grad[q].item() == pytest.approx(fd, rel=2e-6)
    gx = x.grad.cpu().numpy()
    h = 1e-6
    for i in (3, 100, 201):
        assert oracle.min_gap(c["x"], c["box"], P[0], [i]) > 1e-4
        for a in range(3):
            xp = c["x"].copy(); xp[i, a] += h
            xm = c["x"].copy(); xm[i, a] -= h
            fd = (L(p0, xp) - L(p0, xm)) / (2 * h)
            assert gx[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(gx).max())


def test_half_list_is_rejected_for_eam(cases):
    from paper_1009_4330_gb300 import MDError
    c = cases["eam256"]
    with make(c, "mixed", 1) as s:
        with pytest.raises(MDError):
            s.set_kernel(1, "half")
