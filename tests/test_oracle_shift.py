"""Pins of the oracle's on-site shift (a charge-self-consistent potential added to the diagonal of every
atom's on-site H block, Sec. 2): the GPU's CSC reuse test compares against it, so it is fixed here by
facts that do not use it:

* with S = I (overlap parameters zero), a uniform shift delta moves every level of every column by
  exactly delta and leaves the weights: the Krylov spaces of H and H + delta I are the same;
* a shift on an atom outside a column's cluster changes nothing (the column sees P H P only);
* a shift on the column's own atom does change its levels (the shift reaches the matrices).
"""
from dataclasses import replace

import numpy as np

from oracle import sk as skmod
from oracle import system as osys
from synth import SK_CARBON_LIKE, lattice_positions

R = 4.0


def test_uniform_shift_with_identity_overlap_moves_levels_by_delta():
    sk0 = replace(SK_CARBON_LIKE, Sv=(0.0, 0.0, 0.0, 0.0))
    pos, box = lattice_positions("diamond", 3.567, 2, 0.05, 0.0, 7)
    delta = 0.37
    for a in (0, 9, 33):
        r0 = osys.solve_atom(pos, box, sk0, R, a, 6, 4)
        r1 = osys.solve_atom(pos, box, sk0, R, a, 6, 4, onsite_shift=np.full(len(pos), delta))
        for c0, c1 in zip(r0.data, r1.data):
            assert c0.nu_eff == c1.nu_eff
            np.testing.assert_allclose(c1.eps, c0.eps + delta, rtol=0, atol=1e-12)
            np.testing.assert_allclose(c1.w, c0.w, rtol=0, atol=1e-12)


def test_shift_reaches_only_the_cluster():
    pos, box = lattice_positions("diamond", 3.567, 2, 0.05, 0.0, 7)
    a = 9
    cl = set(skmod.cluster_atoms(pos, box, a, R).tolist())
    far = next(b for b in range(len(pos)) if b not in cl)
    r0 = osys.solve_atom(pos, box, SK_CARBON_LIKE, R, a, 6, 4)
    shift = np.zeros(len(pos))
    shift[far] = 1.0
    r1 = osys.solve_atom(pos, box, SK_CARBON_LIKE, R, a, 6, 4, onsite_shift=shift)
    for c0, c1 in zip(r0.data, r1.data):
        np.testing.assert_array_equal(c1.eps, c0.eps)
        np.testing.assert_array_equal(c1.w, c0.w)
    shift[:] = 0.0
    shift[a] = 0.5
    r2 = osys.solve_atom(pos, box, SK_CARBON_LIKE, R, a, 6, 4, onsite_shift=shift)
    assert max(np.abs(c2.eps - c0.eps).max() for c0, c2 in zip(r0.data, r2.data)) > 1e-3
