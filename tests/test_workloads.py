"""The seeded synthetic workloads: sizes as stated, clusters that fit the box, reproducible draws.

The atom counts are those of the workload table (diamond: 8 atoms per cubic cell, fcc: 4, less
the vacancies); every cluster radius stays below half the box edge (the minimum-image cluster
definition needs it); the same seed gives the same positions, and the displacements have the
stated standard deviation.
"""
import numpy as np
import pytest

from synth import WORKLOADS, lattice_positions, workload_positions

EXPECTED = {"diamond512": 512, "diamond1m": 1_000_000, "diamond10m": 10_077_696, "diamond262k": 262_144}


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_workload_sizes_and_radius(name):
    w = WORKLOADS[name]
    pos, box = workload_positions(w)
    if name in EXPECTED:
        assert pos.shape == (EXPECTED[name], 3)
    else:                                     # fcc with vacancies: within 1 % of the expected 5 %
        full = 4 * w.ncell ** 3
        assert abs(1 - pos.shape[0] / full - w.vacancy) < 0.01
    assert np.all(w.R < box / 2) and np.all(w.sk.rc < box / 2)
    assert np.all((pos >= 0) & (pos < box))


def test_draws_are_reproducible_and_have_the_stated_spread():
    a, box = lattice_positions("diamond", 3.567, 6, 0.1, 0.0, 7)
    b, _ = lattice_positions("diamond", 3.567, 6, 0.1, 0.0, 7)
    c, _ = lattice_positions("diamond", 3.567, 6, 0.1, 0.0, 8)
    ideal, _ = lattice_positions("diamond", 3.567, 6, 0.0, 0.0, 7)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)
    d = a - ideal
    d -= box * np.rint(d / box)               # undo the wrap into the box
    assert abs(d.std() - 0.1) < 0.005 and abs(d.mean()) < 0.005
