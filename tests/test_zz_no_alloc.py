"""The allocation-free entry point mka_solve_columns_static against mka_solve_columns.

Some callers cannot allocate device memory: their GPU memory belongs to a
framework's caching allocator that has already reserved it, or they run in a
loop where cudaMalloc's implicit synchronisation is not acceptable. For them
the library solves columns with a fixed device scratch array and the caller's
own output buffers. This test calls it through the C ABI twice in a row, on two
different atom selections, and checks each call against the allocating entry
point on the same atoms, with the tolerance of the other GPU parity tests.
It lives in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

from synth import SK_CARBON_LIKE, lattice_positions

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def lib():
    from paper_1202_0098_gb300 import build, mka
    build.build()
    mka.load()
    return mka


def reference_levels(mka, s, atoms, p, q):
    res = mka.mka_solve_columns(s, atoms, mka.solve_params(p, q, arith="fp64", cg_tol=1e-13, keep_vectors=False))
    try:
        return mka.mka_result_copy_levels(res)
    finally:
        mka.mka_result_destroy(res)


def static_levels(mka, s, atoms, p, q, max_cl):
    n, nu = 4 * len(atoms), p + q
    eps = torch.full((n, nu), float("nan"), dtype=torch.float64, device="cuda")
    w = torch.full((n, nu), float("nan"), dtype=torch.float64, device="cuda")
    nu_eff = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    it = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    mka.mka_solve_columns_static(s, atoms, p, q, 1e-13, 500, max_cl, eps.data_ptr(), w.data_ptr(), nu_eff.data_ptr(),
                                 it.data_ptr(), st.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return {"eps": eps.cpu().numpy(), "w": w.cpu().numpy(), "nu_eff": nu_eff.cpu().numpy(),
            "cg_iters": it.cpu().numpy(), "status": st.cpu().numpy()}


def test_static_scratch_matches_allocating_solve_twice(lib):
    mka = lib
    pos, box = lattice_positions("diamond", 3.567, 3, 0.08, 0.0, 13)
    p, q, R = 10, 10, 5.0
    s = mka.mka_build_system(pos, box, SK_CARBON_LIKE, "fp64", cluster_radius=R)
    try:
        max_cl = int(mka.mka_cluster_sizes(s).max())
        selections = [np.array([0, 9, 31, 64, 150, 215], dtype=np.int64),
                      np.array([2, 3, 100, 101, 199], dtype=np.int64)]
        for atoms in selections:          # two calls in a row on the shared scratch array
            ref = reference_levels(mka, s, atoms, p, q)
            got = static_levels(mka, s, atoms, p, q, max_cl)
            np.testing.assert_array_equal(got["status"], ref["status"])
            np.testing.assert_array_equal(got["nu_eff"], ref["nu_eff"])
            np.testing.assert_array_equal(got["cg_iters"], ref["cg_iters"])
            np.testing.assert_allclose(got["eps"], ref["eps"], rtol=0, atol=TOL)
            np.testing.assert_allclose(got["w"], ref["w"], rtol=0, atol=TOL)
    finally:
        mka.mka_system_destroy(s)


def test_static_scratch_in_chunks(lib):
    """nu = 64 leaves room for only about 120 atoms' reduced problems per pass: 216 atoms take two."""
    mka = lib
    pos, box = lattice_positions("diamond", 3.567, 3, 0.08, 0.0, 13)
    p, q, R = 32, 32, 5.0
    s = mka.mka_build_system(pos, box, SK_CARBON_LIKE, "fp64", cluster_radius=R)
    try:
        max_cl = int(mka.mka_cluster_sizes(s).max())
        atoms = np.arange(pos.shape[0], dtype=np.int64)
        ref = reference_levels(mka, s, atoms, p, q)
        got = static_levels(mka, s, atoms, p, q, max_cl)
        np.testing.assert_array_equal(got["status"], ref["status"])
        np.testing.assert_array_equal(got["nu_eff"], ref["nu_eff"])
        np.testing.assert_allclose(got["eps"], ref["eps"], rtol=0, atol=TOL)
        np.testing.assert_allclose(got["w"], ref["w"], rtol=0, atol=TOL)
    finally:
        mka.mka_system_destroy(s)


def test_static_scratch_on_bf16_storage(lib):
    """BF16-stored values decoded to FP64 (the allocation-free call always runs the FP64 form): the
    same as the allocating call in FP64 arithmetic on the same stored system, twice in a row."""
    mka = lib
    pos, box = lattice_positions("diamond", 3.567, 3, 0.08, 0.0, 14)
    p, q, R = 8, 8, 5.0
    s = mka.mka_build_system(pos, box, SK_CARBON_LIKE, "bf16", cluster_radius=R)
    try:
        max_cl = int(mka.mka_cluster_sizes(s).max())
        for atoms in (np.array([1, 40, 77, 180], dtype=np.int64), np.array([5, 6, 7], dtype=np.int64)):
            ref = reference_levels(mka, s, atoms, p, q)
            got = static_levels(mka, s, atoms, p, q, max_cl)
            np.testing.assert_array_equal(got["status"], ref["status"])
            np.testing.assert_array_equal(got["nu_eff"], ref["nu_eff"])
            np.testing.assert_allclose(got["eps"], ref["eps"], rtol=0, atol=TOL)
            np.testing.assert_allclose(got["w"], ref["w"], rtol=0, atol=TOL)
    finally:
        mka.mka_system_destroy(s)


def test_static_scratch_cluster_cap(lib):
    """max_cluster_atoms below some atoms' clusters: those atoms' columns report
    MKA_ERR_CLUSTER_TOO_LARGE with zero levels, weights and nu_eff; the others match the
    allocating call."""
    mka = lib
    pos, box = lattice_positions("fcc", 4.0, 4, 0.08, 0.08, 15)
    from synth import SK_FCC_METAL
    p, q, R = 6, 6, 5.5
    s = mka.mka_build_system(pos, box, SK_FCC_METAL, "fp64", cluster_radius=R)
    try:
        sizes = mka.mka_cluster_sizes(s)
        cap = int(np.median(sizes))
        atoms = np.arange(0, pos.shape[0], 5, dtype=np.int64)
        big = np.repeat(sizes[atoms] > cap, 4)
        assert big.any() and (~big).any()
        ref = reference_levels(mka, s, atoms, p, q)
        got = static_levels(mka, s, atoms, p, q, cap)
        assert np.all(got["status"][big] == mka.MKA_ERR_CLUSTER_TOO_LARGE)
        assert np.all(got["nu_eff"][big] == 0)
        assert np.all(got["eps"][big] == 0) and np.all(got["w"][big] == 0)
        np.testing.assert_array_equal(got["status"][~big], ref["status"][~big])
        np.testing.assert_array_equal(got["nu_eff"][~big], ref["nu_eff"][~big])
        np.testing.assert_allclose(got["eps"][~big], ref["eps"][~big], rtol=0, atol=TOL)
        np.testing.assert_allclose(got["w"][~big], ref["w"][~big], rtol=0, atol=TOL)
    finally:
        mka.mka_system_destroy(s)


def test_static_scratch_rejects_bad_requests_on_the_host(lib):
    """Rejected requests fail validation before any device work (the buffers are sized for the
    request all the same, so a request that were not rejected would still stay in bounds)."""
    mka = lib
    pos, box = lattice_positions("diamond", 3.567, 3, 0.08, 0.0, 13)
    s = mka.mka_build_system(pos, box, SK_CARBON_LIKE, "fp64", cluster_radius=5.0)
    try:
        atoms = np.array([0], dtype=np.int64)
        for p, q, max_cl in ((200, mka.MKA_MAX_NU - 199, 64), (8, 8, mka.MKA_MAX_CLUSTER_ATOMS + 1), (0, 8, 64)):
            n, nu = 4 * len(atoms), max(1, p + q)
            buf = torch.empty(n * nu, dtype=torch.float64, device="cuda")
            buf2 = torch.empty(n * nu, dtype=torch.float64, device="cuda")
            ib = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(3)]
            with pytest.raises(mka.MkaError) as e:
                mka.mka_solve_columns_static(s, atoms, p, q, 1e-12, 500, max_cl, buf.data_ptr(), buf2.data_ptr(),
                                             ib[0].data_ptr(), ib[1].data_ptr(), ib[2].data_ptr())
            assert e.value.status == mka.MKA_ERR_INVALID_ARG
    finally:
        mka.mka_system_destroy(s)
