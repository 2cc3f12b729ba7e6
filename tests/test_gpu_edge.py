"""Degenerate inputs on the GPU: a single atom (no neighbours), a dimer
across the periodic boundary (closed-form LJ force and energy), and a dilute
gas whose lists are all empty; both precisions and several layouts."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

RC, SKIN, DT = 2.5, 0.3, 0.005


def make(x, v, box, prec, tpa=1, lst="full"):
    from paper_1009_4330_gb300 import System
    return System.lj(x, v, box, cutoff=RC, skin=SKIN, dt=DT, mass=1.0, precision=prec, tpa=tpa, list=lst)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_single_atom_moves_in_a_straight_line(prec):
    box = np.array([12.0, 12.0, 12.0])
    x = np.array([[3.0, 4.0, 5.0]])
    v = np.array([[1.3, -0.7, 0.2]])
    with make(x, v, box, prec) as s:
        counts, _ = s.neighbors(cap=1)
        assert int(counts.sum()) == 0
        assert not s.compute_forces().cpu().numpy().any()
        ev = s.energy_virial().cpu().numpy()[0]
        assert ev[0] == 0.0 and not ev[2:].any()
        s.step(40)  # moves 0.26 in 40 steps: more than skin/2, so the lists are rebuilt on the way
        xs, vs, _ = [a.cpu().numpy() for a in s.state()]
    want = (x + 40 * DT * v) % box
    assert np.abs(xs - want).max() < 1e-12
    assert np.array_equal(vs, v)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
@pytest.mark.parametrize("tpa,lst", [(1, "full"), (4, "full"), (1, "half")])
def test_dimer_across_the_boundary(prec, tol, tpa, lst):
    box = np.array([10.0, 11.0, 12.0])
    x = np.array([[0.3, 5.0, 6.0], [9.2, 5.4, 5.8]])  # image distance (1.1, -0.4, 0.2)
    v = np.zeros_like(x)
    d = x[0] - x[1] - box * np.round((x[0] - x[1]) / box)
    r = np.linalg.norm(d)
    f0 = 24.0 * (2.0 * r ** -14 - r ** -8) * d
    with make(x, v, box, prec, tpa, lst) as s:
        counts, nbr = s.neighbors(cap=2)
        f = s.compute_forces().cpu().numpy()
        ev = s.energy_virial().cpu().numpy()[0]
    c = counts.cpu().numpy()
    assert c.sum() == (1 if lst == "half" else 2)
    assert np.abs(f[0] - f0).max() < tol * np.abs(f0).max()
    assert np.abs(f[1] + f0).max() < tol * np.abs(f0).max()
    assert ev[0] == pytest.approx(4.0 * (r ** -12 - r ** -6), rel=tol)
    assert np.allclose(f, oracle.lj(x, box, RC)[0], rtol=0, atol=tol * np.abs(f0).max())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_dilute_gas_has_empty_lists(prec):
    g = np.arange(4) * 3.2 + 0.5  # spacing 3.2 > rc + skin
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    box = np.array([12.8, 12.8, 12.8])
    v = np.random.default_rng(3).standard_normal(x.shape) * 0.1
    with make(x, v, box, prec) as s:
        counts, _ = s.neighbors(cap=1)
        assert int(counts.sum()) == 0
        assert not s.compute_forces().cpu().numpy().any()
        s.step(5)
        assert not s.state()[2].cpu().numpy().any()
