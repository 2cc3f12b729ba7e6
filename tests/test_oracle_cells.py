"""Pins of the O(N) cell-list CPU baseline against the O(N^2) definition:
the same forces (to rounding of the summation order) and the same
velocity-Verlet trajectory."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import lj_case, ragged_case


@pytest.mark.parametrize("maker", [lambda: lj_case(6, 0.1, seed=3), lambda: ragged_case(777, 8)])
def test_cell_list_forces_equal_definition(maker):
    d = maker()
    f_ref = oracle.lj(d["x"], d["box"], 2.5)[0]
    f = oracle.lj_cells(d["x"], d["box"], 2.5)
    assert np.abs(f - f_ref).max() <= 1e-12 * np.abs(f_ref).max()


def test_cell_list_handles_unwrapped_positions():
    d = lj_case(6, 0.1, seed=4)
    shifted = d["x"] + d["box"] * np.array([1.0, -2.0, 3.0])  # outside the box: same periodic system
    assert np.abs(oracle.lj_cells(shifted, d["box"], 2.5) - oracle.lj_cells(d["x"], d["box"], 2.5)).max() < 1e-9


def test_cell_list_needs_three_cells():
    x, box = synth.fcc_lattice(3, 3, 3, synth.fcc_constant(0.8442))  # box 5.04 < 3 rc
    with pytest.raises(ValueError):
        oracle.lj_cells(x, box, 2.5)


def test_cell_list_trajectory_equals_definition():
    d = lj_case(6, 0.05, seed=6)
    ref = oracle.nve(d["x"], d["v"], d["box"], 20, 0.005, 2.5, 0.3)
    x, v, f = oracle.nve_cells(d["x"], d["v"], d["box"], 2.5, 0.005, 1.0, 20)
    assert np.abs(x - ref["x"]).max() < 1e-11
    assert np.abs(v - ref["v"]).max() < 1e-10
    assert np.abs(f - ref["f"]).max() < 1e-9 * np.abs(ref["f"]).max()
