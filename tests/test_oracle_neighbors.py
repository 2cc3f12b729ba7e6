"""Pins of the oracle's neighbour sets (the Verlet list, paper Sec. III.B).

Hand-built cases with known answers, fcc coordination numbers, symmetry of
the relation and periodic images.
"""
import numpy as np
import pytest

import oracle
import synth


def test_hand_built_line():
    # atoms on the x axis of a 10^3 box at 0.5, 1.5, 3.4, 9.0 (9.0 is 1.5 from 0.5 across the face)
    x = np.array([[0.5, 5, 5], [1.5, 5, 5], [3.4, 5, 5], [9.0, 5, 5]], dtype=float)
    box = np.array([10.0, 10.0, 10.0])
    nb = oracle.neighbors(x, box, 2.0)
    assert [s.tolist() for s in nb] == [[1, 3], [0, 2], [1], [0]]
    nb = oracle.neighbors(x, box, 1.95)  # 1.5 -> 3.4 is 1.9 apart, 0.5 -> 9.0 is 1.5 apart
    assert [s.tolist() for s in nb] == [[1, 3], [0, 2], [1], [0]]
    nb = oracle.neighbors(x, box, 1.5)  # strict: exactly-1.5 pair excluded, 1.0 pair kept
    assert [s.tolist() for s in nb] == [[1], [0], [], []]


@pytest.mark.parametrize("a,rl,count", [(synth.fcc_constant(0.8442), 2.8, 78),
                                        (synth.fcc_constant(0.8442), 5.3, 530),
                                        (3.615, 5.45, 54)])
def test_fcc_coordination(a, rl, count):
    cells = max(4, int(np.ceil(2 * rl / a)) + 1)
    x, box = synth.fcc_lattice(cells, cells, cells, a)
    idx = np.arange(0, x.shape[0], 37)
    nb = oracle.neighbors(x, box, rl, idx)
    assert all(len(s) == count for s in nb)


def test_relation_is_symmetric_and_irreflexive():
    a = synth.fcc_constant(0.8442)
    x, box = synth.fcc_lattice(4, 4, 4, a)
    x = synth.displace(x, box, 0.15, 3)
    nb = oracle.neighbors(x, box, 2.8)
    pairs = {(i, int(j)) for i, s in enumerate(nb) for j in s}
    assert all((j, i) in pairs for i, j in pairs)
    assert all(i != j for i, j in pairs)


def test_sampled_equals_full_and_gap():
    a = synth.fcc_constant(0.8442)
    x, box = synth.fcc_lattice(5, 5, 5, a)
    x = synth.displace(x, box, 0.1, 4)
    full = oracle.neighbors(x, box, 2.8)
    idx = np.array([3, 99, 250, 499])
    part = oracle.neighbors(x, box, 2.8, idx)
    for k, i in enumerate(idx):
        assert np.array_equal(part[k], full[i])
    # the gap is the distance of the nearest pair to the list radius: moving the
    # radius by less than the gap leaves every set unchanged
    g = oracle.min_gap(x, box, 2.8)
    assert g > 0
    shifted = oracle.neighbors(x, box, 2.8 + 0.5 * g)
    assert all(np.array_equal(s, t) for s, t in zip(full, shifted))
    grown = oracle.neighbors(x, box, 2.8 + 1.5 * g)
    assert sum(map(len, grown)) > sum(map(len, full))
