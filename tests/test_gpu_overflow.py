"""A list overflow in the middle of md_step: two liquid slabs driven into
each other compress the contact region until the longest list outgrows the
capacity chosen at creation.  The step loop must grow the list, rebuild and
carry on without losing or repeating a step: the FP64 trajectory equals the
oracle's and md_info counts every step."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

RC, SKIN, DT = 2.5, 0.3, 0.0005


def colliding_slabs(vz=16.0):
    a = synth.fcc_constant(0.8442)
    x1, _ = synth.fcc_lattice(6, 6, 4, a)
    box = np.array([6 * a, 6 * a, 30.0])
    xa = x1.copy(); xa[:, 2] += 2.0
    xb = x1.copy(); xb[:, 2] += 2.0 + 4 * a + 1.5
    x = synth.displace(np.concatenate([xa, xb]), box, 0.03, 11)
    v = synth.maxwell_boltzmann(x.shape[0], 0.5, 1.0, 12)
    v[:len(xa), 2] += vz
    v[len(xa):, 2] -= vz
    return x, v, box


@pytest.mark.parametrize("prec,tpa", [("fp64", 1), ("fp64", 8), ("mixed", 1)])
def test_overflow_inside_md_step(prec, tpa):
    from paper_1009_4330_gb300 import System
    x, v, box = colliding_slabs()
    nsteps = 300
    ref = oracle.nve(x, v, box, nsteps, DT, RC, SKIN)
    with System.lj(x, v, box, cutoff=RC, skin=SKIN, dt=DT, mass=1.0, precision=prec, tpa=tpa) as s:
        cap0 = s.info()["maxneigh"]
        s.step(nsteps)
        inf = s.info()
        xs, vs, _ = [a.cpu().numpy() for a in s.state()]
    assert inf["steps"] == nsteps
    assert inf["maxneigh"] > cap0 and inf["max_count"] > cap0  # the capacity grew during the run
    d = xs - ref["x"]
    d -= box * np.round(d / box)
    tol = 1e-7 if prec == "fp64" else 1e-3  # one lost step would shift atoms by ~dt * 16 = 8e-3
    assert np.abs(d).max() < tol
