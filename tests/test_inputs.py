"""The seeded synthetic workloads follow their stated recipes: sizes, boxes
and densities of the LJ and EAM benchmark systems (App. A), Maxwell-Boltzmann
velocities with zero net momentum at exactly the target temperature (3N - 3
degrees of freedom), the binary force-matching box and its type-B count, and
the log-uniform replica sizes of the batch; every generator is reproducible
from its seed."""
import math

import numpy as np
import pytest

import synth


def kinetic_temperature(v, m, kb=1.0, ftm2v=1.0):
    m = np.broadcast_to(np.asarray(m, dtype=np.float64), (v.shape[0],))
    ke = 0.5 * float((m[:, None] * v * v).sum()) / ftm2v
    return 2.0 * ke / ((3 * v.shape[0] - 3) * kb)


def test_lj_4000_recipe():
    d = synth.config0()
    x, box = d["x"], d["box"]
    assert x.shape == (4000, 3)
    assert np.allclose(box, 16.795961913825074)  # 10 fcc cells of a = (4/0.8442)^(1/3)
    assert 4000 / np.prod(box) == pytest.approx(0.8442, rel=1e-12)
    assert np.all((x >= 0) & (x < box))
    assert (d["rc"], d["skin"], d["dt"]) == (2.5, 0.3, 0.005)
    assert np.abs(d["v"].sum(axis=0)).max() < 1e-12
    assert kinetic_temperature(d["v"], 1.0) == pytest.approx(1.44, rel=1e-12)


def test_lj_864000_recipe_small_cells():
    # same recipe as the 60^3-cell bench system, at 8^3 cells (the generator is
    # the same function; the full size only multiplies the work)
    d = synth.config1(cells=8)
    assert d["x"].shape == (4 * 8 ** 3, 3)
    assert d["x"].shape[0] / np.prod(d["box"]) == pytest.approx(0.8442, rel=1e-12)
    assert kinetic_temperature(d["v"], 1.0) == pytest.approx(1.44, rel=1e-12)
    assert synth.config1(rc=5.0, cells=8)["rc"] == 5.0


def test_eam_recipe_small_cells():
    d = synth.config2(cells=6)
    assert d["x"].shape == (4 * 6 ** 3, 3)
    assert np.allclose(d["box"], 6 * 3.615)
    assert tuple(d["eam"]) == (4.95, 1.0, 0.5, -0.2, 0.02)
    assert (d["skin"], d["dt"]) == (0.5, 1.0)
    t = kinetic_temperature(d["v"], 63.55, kb=synth.KB_METAL, ftm2v=synth.FTM2V_METAL)
    assert t == pytest.approx(300.0, rel=1e-12)
    assert np.abs((63.55 * d["v"]).sum(axis=0)).max() < 1e-9


def test_force_matching_recipe():
    d = synth.config3()
    n = d["x"].shape[0]
    assert n == 32768  # 16 x 16 x 32 fcc cells
    assert n / np.prod(d["box"]) == pytest.approx(1.2, rel=1e-12)
    assert int(d["types"].sum()) == 6554  # round(0.2 N) type-B atoms
    assert set(np.unique(d["types"]).tolist()) == {0, 1}
    for start, true in ((d["eps0"], d["eps_true"]), (d["sig0"], d["sig_true"])):
        rel = start / true - 1.0
        assert np.all(np.abs(rel) <= 0.1) and np.any(rel != 0)


def test_replica_sizes_and_boxes():
    sizes = synth.replica_sizes(512, 500, 20000, synth.SEED_BASE + 4)
    assert sizes.shape == (512,)
    assert sizes.min() >= 500 and sizes.max() <= 20000
    # log-uniform: the median near the geometric mean sqrt(500 * 20000)
    assert abs(math.log(np.median(sizes)) - 0.5 * math.log(500 * 20000)) < 0.3
    for r, n in enumerate((500, 777, 20000)):
        x, box = synth.fcc_subset(n, 0.8442, 7 + r)
        assert x.shape == (n, 3)
        assert n / np.prod(box) == pytest.approx(0.8442, rel=1e-12)
        assert np.all((x >= 0) & (x < box))
        assert len({tuple(p) for p in np.round(x, 9)}) == n  # distinct lattice sites


def test_generators_are_reproducible():
    a, b = synth.config0(displacement=0.05), synth.config0(displacement=0.05)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["v"], b["v"])
    c = synth.config0()
    assert not np.array_equal(a["x"], c["x"])  # the jitter moves the atoms
    assert np.array_equal(synth.binary_types(1000, 200, 5), synth.binary_types(1000, 200, 5))
