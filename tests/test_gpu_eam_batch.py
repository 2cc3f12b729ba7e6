"""EAM in a batch of uneven replicas: per-replica forces and energies equal
the oracle's, a replica stepped inside the batch equals the same replica
stepped alone (FP64: bitwise), and the batch backward equals the sum over
replicas (shared parameters) and the concatenation (positions)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import margin_ok, rel_maxnorm

pytestmark = pytest.mark.gpu

P = np.array(synth.EAM_PARAMS)
SKIN, DT, MASS = 0.5, 1.0, 63.55


def replicas():
    out = []
    for k, cells in enumerate((4, 5, 6)):
        x, box = synth.fcc_lattice(cells, cells, cells, 3.615)
        x = synth.displace(x, box, 0.08, 50 + k)
        v = synth.maxwell_boltzmann(x.shape[0], 300.0, MASS, 60 + k, kb=synth.KB_METAL, ftm2v=synth.FTM2V_METAL)
        assert margin_ok(x, box, P[0] + SKIN)
        out.append({"x": x, "v": v, "box": box})
    return out


def make(reps, prec):
    from paper_1009_4330_gb300 import System
    return System.batch(reps, potential="eam", params=P, cutoff=float(P[0]), skin=SKIN, dt=DT, mass=MASS,
                        ftm2v=synth.FTM2V_METAL, precision=prec, tpa=1)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_batch_forces_and_energies(prec, tol):
    reps = replicas()
    with make(reps, prec) as s:
        f = s.compute_forces().cpu().numpy()
        ev = s.energy_virial().cpu().numpy()
    o = 0
    for r, rep in enumerate(reps):
        n = rep["x"].shape[0]
        fr, er, wr, _, _ = oracle.eam(rep["x"], rep["box"], P)
        assert rel_maxnorm(f[o:o + n], fr) < tol
        assert ev[r, 0] == pytest.approx(er, rel=10 * tol)
        o += n


def test_batch_replica_steps_like_solo_fp64():
    from paper_1009_4330_gb300 import System
    reps = replicas()
    with make(reps, "fp64") as s:
        s.step(25)
        xb = s.state()[0].cpu().numpy()
    rep = reps[1]
    with System.eam(rep["x"], rep["v"], rep["box"], eam_params=P, skin=SKIN, dt=DT, mass=MASS,
                    ftm2v=synth.FTM2V_METAL, precision="fp64", tpa=1) as s1:
        s1.step(25)
        x1 = s1.state()[0].cpu().numpy()
    o = reps[0]["x"].shape[0]
    assert np.array_equal(xb[o:o + x1.shape[0]], x1)


def test_batch_backward_is_the_sum_over_replicas():
    reps = replicas()
    rng = np.random.default_rng(9)
    gs = [rng.standard_normal(r["x"].shape) for r in reps]
    with make(reps, "fp64") as s:
        gx, gp = s.backward(np.concatenate(gs))
    gx, gp = gx.cpu().numpy(), gp.cpu().numpy()
    gp_sum = np.zeros(5)
    o = 0
    for rep, g in zip(reps, gs):
        n = rep["x"].shape[0]
        gxr, gpr = oracle.eam_vjp(rep["x"], rep["box"], P, g)
        assert rel_maxnorm(gx[o:o + n], gxr) < 1e-11
        gp_sum += gpr
        o += n
    assert np.allclose(gp[1:], gp_sum[1:], rtol=1e-11, atol=1e-11 * np.abs(gp_sum).max())
