"""Pins of the oracle's velocity-Verlet NVE integrator (the paper's GPU NVE
integration, Sec. II): time reversibility, second-order energy error, momentum
conservation and the small-amplitude dimer period.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def small_liquid(cells=4, seed=1000):
    d = synth.lj_liquid(cells, seed=seed, displacement=0.05)
    return d


def test_time_reversibility():
    d = small_liquid()
    x0, v0 = d["x"].copy(), d["v"].copy()
    a = oracle.nve(x0, v0, d["box"], 50, 0.005, 2.5, 0.3)
    b = oracle.nve(a["x"], -a["v"], d["box"], 50, 0.005, 2.5, 0.3)
    assert np.abs(b["x"] - x0).max() < 1e-10
    assert np.abs(-b["v"] - v0).max() < 1e-10


def test_momentum_conserved():
    d = small_liquid()
    r = oracle.nve(d["x"], d["v"], d["box"], 40, 0.005, 2.5, 0.3)
    assert np.abs(r["v"].sum(0)).max() < 1e-12


def test_energy_error_is_second_order():
    d = small_liquid(seed=1003)
    errs = []
    for dt, n in [(0.004, 50), (0.002, 100)]:
        r = oracle.nve(d["x"], d["v"], d["box"], n, dt, 2.5, 0.3, shift=True)
        etot = r["epot"] + r["ekin"]
        errs.append(np.abs(etot - etot[0]).max())
    ratio = errs[0] / errs[1]
    assert 3.0 < ratio < 5.0  # halving dt divides the energy error by ~4


def test_dimer_small_amplitude_period():
    # LJ dimer near r_m = 2^(1/6): U''(r_m) = 144 * 2^(-4/3); reduced mass m/2
    # period T = 2 pi sqrt(mu / U'');  with m = 2 (mass scaling pinned too) mu = 1
    rm = 2.0 ** (1.0 / 6.0)
    k = 144.0 * 2.0 ** (-4.0 / 3.0)
    for m in (1.0, 2.0):
        T = 2 * math.pi * math.sqrt((m / 2) / k)
        x = np.array([[5.0, 5.0, 5.0], [5.0 + rm + 1e-4, 5.0, 5.0]])
        v = np.zeros((2, 3))
        dt = T / 2000
        nsteps = 4000
        # record r(t) by running one step at a time
        rs = []
        xc, vc = x, v
        for _ in range(nsteps):
            res = oracle.nve(xc, vc, np.array([10.0, 10.0, 10.0]), 1, dt, 2.5, 10.0, mass=(m,))
            xc, vc = res["x"], res["v"]
            rs.append(xc[1, 0] - xc[0, 0] - rm)
        rs = np.array(rs)
        # upward zero crossings of r - r_m
        cross = [i for i in range(1, len(rs)) if rs[i - 1] < 0 <= rs[i]]
        per = (cross[-1] - cross[0]) * dt / (len(cross) - 1)
        assert per == pytest.approx(T, rel=2e-3)


def test_rebuild_policy_counts():
    d = small_liquid()
    r_big = oracle.nve(d["x"], d["v"], d["box"], 30, 0.005, 2.5, 3.0)
    assert r_big["rebuilds"] == 0
    r = oracle.nve(d["x"], d["v"], d["box"], 30, 0.005, 2.5, 0.3)
    assert r["rebuilds"] >= 1
    # the trajectory does not depend on the skin (forces never use the list)
    assert np.array_equal(r["x"], r_big["x"])


def test_eam_nve_units_conserve_energy():
    d = synth.config2(cells=4, displacement=0.05)
    r = oracle.nve(d["x"], d["v"], d["box"], 40, 1.0, d["rc"], 0.5, pot="eam", eam_params=d["eam"],
                   mass=d["mass"], ftm2v=d["ftm2v"])
    etot = r["epot"] + r["ekin"]
    assert np.abs(etot - etot[0]).max() / d["x"].shape[0] < 1e-4
    # temperature near 300 K at the start (dof 3N - 3)
    n = d["x"].shape[0]
    t0 = 2 * r["ekin"][0] / ((3 * n - 3) * synth.KB_METAL)
    assert t0 == pytest.approx(300.0, rel=1e-12)
