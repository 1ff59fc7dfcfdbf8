"""The density of states on the GPU (mka_dos) against the oracle's (Sec. 3):
D(E) = -(1/pi) Im sum_j (G(E + i eta) S)_jj from the columns' levels and weights, FP64 (relative 1e-10),
for subspaces of nu = 30 and nu = 300 (the size the paper takes for an energy-resolved DOS; the large
instance of the reduced kernel), the levels themselves against the oracle's at 1e-10."""
import numpy as np
import pytest

from oracle import mka as omka, system as osys
from oracle.parallel import solve_atoms_parallel
from synth import WORKLOADS, workload_positions

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1202_0098_gb300 import build, mka
    build.build()
    mka.load()
    return mka


@pytest.mark.parametrize("half", [15, 150])
def test_dos_matches_oracle(lib, half):
    mka = lib
    w = WORKLOADS["diamond512"]
    pos, box = workload_positions(w)
    atoms = np.array([5, 99, 200, 333, 500], dtype=np.int64)
    ores = solve_atoms_parallel(pos, box, w.sk, w.R, atoms, half, half)
    oe, ow = osys.stack_eps_w(ores)
    grid = np.linspace(-20.0, 30.0, 301)
    eta = 0.1
    ref = omka.dos(oe, ow, grid, eta)
    s = mka.mka_build_system(pos, box, w.sk, "fp64", cluster_radius=w.R)
    try:
        res = mka.mka_solve_columns(s, atoms, mka.solve_params(half, half, cg_tol=1e-13, keep_vectors=False))
        lv = mka.mka_result_copy_levels(res)
        np.testing.assert_allclose(lv["eps"], oe, rtol=0, atol=1e-10)
        np.testing.assert_allclose(lv["w"], ow, rtol=0, atol=1e-10)
        e_ptr, w_ptr = mka.mka_result_device_levels(res)
        got = mka.mka_dos(e_ptr, w_ptr, lv["eps"].size, grid, eta)
        np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12 * ref.max())
        # sum rule: every column's weights add to one, so the integral is the number of columns
        integral = np.trapezoid(got, grid)
        assert abs(integral - 4 * len(atoms)) < 0.02 * 4 * len(atoms)
        mka.mka_result_destroy(res)
    finally:
        mka.mka_system_destroy(s)
