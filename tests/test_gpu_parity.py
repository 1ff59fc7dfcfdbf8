"""GPU parity: the CUDA path, called through the C ABI, against the FP64 oracle.

Bars (FP64 form): |d rho_ij| <= 1e-10, |d E| <= 1e-10 eV/atom, |d mu| <= 1e-9 eV,
eps_alpha and w_alpha within 1e-10, integer outputs (pattern, cluster sizes,
nu_eff) bit-exact. rho is compared at the oracle's mu; mu separately.
"""
import numpy as np
import pytest

from oracle import sk as osk, system as osys
from oracle.rounding import round_storage
from synth import SK_CARBON_LIKE, WORKLOADS, lattice_positions, workload_positions, sample_atoms
from oracle.parallel import solve_atoms_parallel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def lib():
    from paper_1202_0098_gb300 import build, mka
    build.build()
    mka.load()
    return mka


def gpu_solve(mka, sysh, atoms, p, q, cg_tol=1e-13, arith="fp64"):
    prm = mka.solve_params(p, q, arith=arith, cg_tol=cg_tol, keep_vectors=True)
    res = mka.mka_solve_columns(sysh, atoms, prm)
    lv = mka.mka_result_copy_levels(res)
    return res, lv


def gpu_density(mka, sysh, res, mu, kT):
    nb = mka.mka_result_info(res)["n_blocks"]
    rho = torch.empty(nb * 16, dtype=torch.float64, device="cuda")
    e, n = mka.mka_density_energy(sysh, res, mu, kT, rho.data_ptr())
    return rho.cpu().numpy().reshape(nb, 4, 4), e, n


def gpu_greens(mka, sysh, res, z):
    nb = mka.mka_result_info(res)["n_blocks"]
    g = torch.empty(nb * 32, dtype=torch.float64, device="cuda")
    mka.mka_greens(sysh, res, z, g.data_ptr())
    g = g.cpu().numpy().reshape(nb, 4, 4, 2)
    return g[..., 0] + 1j * g[..., 1]


def compare_levels(lv, ores, tol=TOL):
    oe, ow = osys.stack_eps_w(ores)
    nu_eff = np.array([c.nu_eff for r in ores for c in r.data])
    np.testing.assert_array_equal(lv["nu_eff"], nu_eff)
    np.testing.assert_allclose(lv["eps"], oe, rtol=0, atol=tol)
    np.testing.assert_allclose(lv["w"], ow, rtol=0, atol=tol)


def test_native_build_matches_oracle(lib):
    mka = lib
    for lat, n, sig, vac in (("diamond", 2, 0.1, 0.0), ("fcc", 3, 0.08, 0.05)):
        pos, box = lattice_positions(lat, 3.567 if lat == "diamond" else 4.0, n, sig, vac, 7)
        skp = SK_CARBON_LIKE
        g = osk.global_bsr(pos, box, skp)
        for storage in ("fp64", "fp32", "bf16"):
            s = mka.mka_build_system(pos, box, skp, storage, cluster_radius=min(box) / 2 - 0.01)
            try:
                b = mka.mka_system_copy_bsr(s)
                np.testing.assert_array_equal(b["row_ptr"], g["row_ptr"])
                np.testing.assert_array_equal(b["col"], g["col"])
                if storage == "fp64":
                    np.testing.assert_allclose(b["H"], g["H"], rtol=0, atol=1e-14)
                    np.testing.assert_allclose(b["S"], g["S"], rtol=0, atol=1e-15)
                else:
                    np.testing.assert_allclose(b["H"], round_storage(g["H"], storage), rtol=0, atol=1e-14)
                    np.testing.assert_allclose(b["S"], round_storage(g["S"], storage), rtol=0, atol=1e-15)
            finally:
                mka.mka_system_destroy(s)


def test_cluster_sizes_match_oracle(lib):
    mka = lib
    for name, nsamp in (("diamond512", None), ("fcc32k", 300)):
        w = WORKLOADS[name]
        pos, box = workload_positions(w)
        s = mka.mka_build_system(pos, box, w.sk, "fp64", cluster_radius=w.R)
        try:
            atoms = np.arange(pos.shape[0]) if nsamp is None else sample_atoms(pos.shape[0], nsamp, 11)
            got = mka.mka_cluster_sizes(s, atoms)
            ref = np.array([len(osk.cluster_atoms(pos, box, int(a), w.R)) for a in atoms])
            np.testing.assert_array_equal(got, ref)
        finally:
            mka.mka_system_destroy(s)


@pytest.fixture(scope="module")
def diamond_sample(lib):
    mka = lib
    w = WORKLOADS["diamond512"]
    pos, box = workload_positions(w)
    atoms = np.array([0, 3, 77, 128, 255, 256, 300, 401, 466, 510, 511, 9], dtype=np.int64)
    ores = solve_atoms_parallel(pos, box, w.sk, w.R, atoms, w.p, w.q)
    s = mka.mka_build_system(pos, box, w.sk, "fp64", cluster_radius=w.R)
    res, lv = gpu_solve(mka, s, atoms, w.p, w.q)
    yield mka, w, pos, box, atoms, ores, s, res, lv
    mka.mka_result_destroy(res)
    mka.mka_system_destroy(s)


def test_levels_and_weights(diamond_sample):
    mka, w, pos, box, atoms, ores, s, res, lv = diamond_sample
    compare_levels(lv, ores)
    assert np.all(lv["status"] == 0)
    # iteration counts of the inner CG agree within one step (different rounding order)
    ocg = np.array([c.cg_iters for r in ores for c in r.data])
    assert np.all(np.abs(lv["cg_iters"] - ocg) <= 1)
    # sum_alpha w_alpha = 1 for every column (e_j lies in the subspace)
    np.testing.assert_allclose(lv["w"].sum(1), 1.0, atol=1e-12)


def test_density_energy_greens(diamond_sample):
    mka, w, pos, box, atoms, ores, s, res, lv = diamond_sample
    mu = 0.4
    rho, e, n = gpu_density(mka, s, res, mu, w.kT)
    orho, oe, on = osys.density(ores, mu, w.kT)
    np.testing.assert_allclose(rho, np.concatenate(orho), rtol=0, atol=TOL)
    assert abs(e - oe) / len(atoms) < TOL
    assert abs(n - on) < 1e-9
    z = 0.3 + 0.2j
    g = gpu_greens(mka, s, res, z)
    np.testing.assert_allclose(g, np.concatenate(osys.greens(ores, z)), rtol=0, atol=1e-9)


def test_mu_bisection_on_sample(diamond_sample):
    mka, w, pos, box, atoms, ores, s, res, lv = diamond_sample
    n_e = w.electrons_per_atom * len(atoms)
    mu_gpu = mka.mka_find_mu(res, n_e, w.kT)
    mu_ref = osys.find_mu(ores, n_e, w.kT)
    assert abs(mu_gpu - mu_ref) < 1e-9


def test_full_system_diamond512(lib):
    """Every column of the 512-atom system: mu, band energy, rho at the oracle's mu."""
    mka = lib
    w = WORKLOADS["diamond512"]
    pos, box = workload_positions(w)
    atoms = np.arange(pos.shape[0], dtype=np.int64)
    ores = solve_atoms_parallel(pos, box, w.sk, w.R, atoms, w.p, w.q)
    s = mka.mka_build_system(pos, box, w.sk, "fp64", cluster_radius=w.R)
    try:
        res, lv = gpu_solve(mka, s, None, w.p, w.q)
        compare_levels(lv, ores)
        n_e = w.electrons_per_atom * len(atoms)
        mu_ref = osys.find_mu(ores, n_e, w.kT)
        mu_gpu = mka.mka_find_mu(res, n_e, w.kT)
        assert abs(mu_gpu - mu_ref) < 1e-9
        rho, e, n = gpu_density(mka, s, res, mu_ref, w.kT)
        orho, oe, on = osys.density(ores, mu_ref, w.kT)
        np.testing.assert_allclose(rho, np.concatenate(orho), rtol=0, atol=TOL)
        assert abs(e - oe) / len(atoms) < TOL
        assert abs(n - n_e) < 1e-9 * n_e
        # band energy two ways (Tr[rho H] = Tr[pi S], exact for p >= 1)
        assert abs(oe - osys.band_energy_from_levels(ores, mu_ref, w.kT)) / len(atoms) < 1e-11
        mka.mka_result_destroy(res)
    finally:
        mka.mka_system_destroy(s)


@pytest.mark.parametrize("case", ["identity_overlap", "q0", "small_cluster", "p1q1"])
def test_edge_cases(lib, case):
    mka = lib
    w = WORKLOADS["diamond512"]
    pos, box = lattice_positions("diamond", 3.567, 3, 0.07, 0.0, 21)
    skp, R, p, q = w.sk, 5.0, 8, 8
    if case == "identity_overlap":
        from dataclasses import replace
        skp = replace(w.sk, Sv=(0.0, 0.0, 0.0, 0.0))   # S = I: the seam vector s_j = e_j drops out
    elif case == "q0":
        p, q = 12, 0
    elif case == "small_cluster":
        R, p, q = 2.0, 15, 15                            # 5 atoms, m_c = 20 < nu; pattern reaches beyond R
    elif case == "p1q1":
        p, q = 1, 1
    atoms = np.array([0, 5, 17, 100, 215], dtype=np.int64)
    ores = solve_atoms_parallel(pos, box, skp, R, atoms, p, q)
    s = mka.mka_build_system(pos, box, skp, "fp64", cluster_radius=R)
    try:
        res, lv = gpu_solve(mka, s, atoms, p, q)
        compare_levels(lv, ores)
        mu = 0.2
        rho, e, n = gpu_density(mka, s, res, mu, 0.1)
        orho, oe, on = osys.density(ores, mu, 0.1)
        np.testing.assert_allclose(rho, np.concatenate(orho), rtol=0, atol=TOL)
        assert abs(e - oe) / len(atoms) < TOL
        if case == "small_cluster":
            assert np.all(lv["nu_eff"] <= 20) and np.all(lv["status"] == mka.MKA_ERR_BREAKDOWN)
        mka.mka_result_destroy(res)
    finally:
        mka.mka_system_destroy(s)


def test_uneven_clusters_fcc(lib):
    mka = lib
    w = WORKLOADS["fcc32k"]
    pos, box = workload_positions(w)
    atoms = sample_atoms(pos.shape[0], 24, 5)
    ores = solve_atoms_parallel(pos, box, w.sk, w.R, atoms, w.p, w.q)
    s = mka.mka_build_system(pos, box, w.sk, "fp64", cluster_radius=w.R)
    try:
        res, lv = gpu_solve(mka, s, atoms, w.p, w.q)
        compare_levels(lv, ores)
        rho, e, _ = gpu_density(mka, s, res, 0.9, w.kT)
        orho, oe, _ = osys.density(ores, 0.9, w.kT)
        np.testing.assert_allclose(rho, np.concatenate(orho), rtol=0, atol=TOL)
        mka.mka_result_destroy(res)
    finally:
        mka.mka_system_destroy(s)


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_fp64_arithmetic_on_rounded_storage(lib, storage):
    """Values stored in FP32/BF16, FP64 arithmetic: equals the oracle run on the same rounded values."""
    mka = lib
    w = WORKLOADS["diamond512"]
    pos, box = workload_positions(w)
    atoms = np.array([1, 222, 444], dtype=np.int64)
    ores = solve_atoms_parallel(pos, box, w.sk, w.R, atoms, w.p, w.q, storage=storage)
    s = mka.mka_build_system(pos, box, w.sk, storage, cluster_radius=w.R)
    try:
        res, lv = gpu_solve(mka, s, atoms, w.p, w.q)
        compare_levels(lv, ores)
        mka.mka_result_destroy(res)
    finally:
        mka.mka_system_destroy(s)


def test_global_spmv(lib):
    mka = lib
    pos, box = lattice_positions("diamond", 3.567, 3, 0.1, 0.0, 3)
    g = osk.global_bsr(pos, box, SK_CARBON_LIKE)
    H = osk.bsr_to_dense(g["row_ptr"], g["col"], g["H"])
    S = osk.bsr_to_dense(g["row_ptr"], g["col"], g["S"])
    M = H.shape[0]
    rng = np.random.default_rng(4)
    for storage in ("fp64", "fp32", "bf16"):
        s = mka.mka_build_system(pos, box, SK_CARBON_LIKE, storage, cluster_radius=4.0)
        try:
            for k in (1, 2, 4):
                x = rng.normal(size=(M, k))
                for which, A in ((0, H), (1, S)):
                    A = round_storage(A, storage)
                    xd = torch.from_numpy(x).cuda()
                    yd = torch.empty_like(xd)
                    mka.mka_spmv(s, which, mka.MKA_FP64, xd.data_ptr(), yd.data_ptr(), k)
                    np.testing.assert_allclose(yd.cpu().numpy(), A @ x, rtol=0, atol=1e-12)
                    xf = xd.float().contiguous()
                    yf = torch.empty_like(xf)
                    mka.mka_spmv(s, which, mka.MKA_MIXED_FP32, xf.data_ptr(), yf.data_ptr(), k)
                    # FP32 products and sums of FP32-rounded x: the n-term dot-product bound
                    # |fl(a.x) - a.x| <= gamma_n |a|.|x| (gamma_n = n u / (1 - n u), u = 2^-24), plus x's
                    # own rounding |a|.|x| u, with n the longest row's entry count
                    xr = xf.double().cpu().numpy()
                    n = 4 * int(np.diff(g["row_ptr"]).max())
                    u = 2.0 ** -24
                    bound = (n * u / (1 - n * u) + u) * (np.abs(A) @ np.abs(x)) + 1e-30
                    err = np.abs(yf.double().cpu().numpy() - A @ xr)
                    assert np.all(err <= bound), float((err / bound).max())
        finally:
            mka.mka_system_destroy(s)


@pytest.mark.parametrize("storage", ["bf16", "fp32"])
def test_mixed_form_against_oracle_on_stored_values(lib, storage):
    """Mixed form (FP32 products, CG and basis; FP64 cross-thread sums, reduced solve and mu):
    |d rho| <= 1e-6 and |d E| <= 1e-5 eV/atom against the oracle run on the same stored values."""
    mka = lib
    w = WORKLOADS["diamond512"]
    pos, box = workload_positions(w)
    atoms = np.array([0, 1, 50, 99, 222, 301, 444, 511], dtype=np.int64)
    ores = solve_atoms_parallel(pos, box, w.sk, w.R, atoms, w.p, w.q, storage=storage)
    s = mka.mka_build_system(pos, box, w.sk, storage, cluster_radius=w.R)
    try:
        res, lv = gpu_solve(mka, s, atoms, w.p, w.q, cg_tol=1e-7, arith="mixed")
        assert np.all(lv["status"] == 0)
        oe, ow = osys.stack_eps_w(ores)
        print(f"mixed {storage}: max|d eps| {np.abs(lv['eps'] - oe).max():.2e}  max|d w| {np.abs(lv['w'] - ow).max():.2e}")
        # the mixed form's subspace differs from the FP64 form's by about 1e-7 (FP32 pairs, s_j to 1e-7 and
        # refined); a Ritz value moves by at most about ||H|| times that (||H|| ~ 30 eV here) and a weight
        # by a modest multiple of it: eps within 1e-5 eV and w within 5e-6 (observed 2e-6 and 5e-7)
        assert np.abs(lv["eps"] - oe).max() < 1e-5 and np.abs(lv["w"] - ow).max() < 5e-6
        for mu in (0.3, 1.9):
            rho, e, n = gpu_density(mka, s, res, mu, w.kT)
            orho, oe_band, on = osys.density(ores, mu, w.kT)
            drho = np.abs(rho - np.concatenate(orho)).max()
            de = abs(e - oe_band) / len(atoms)
            print(f"mixed {storage} mu={mu}: max|d rho| {drho:.2e}  |d E| {de:.2e} eV/atom")
            assert drho <= 1e-6 and de <= 1e-5
        n_e = w.electrons_per_atom * len(atoms)
        dmu = abs(mka.mka_find_mu(res, n_e, w.kT) - osys.find_mu(ores, n_e, w.kT))
        print(f"mixed {storage}: |d mu| {dmu:.2e} eV")
        assert dmu < 1e-4
        mka.mka_result_destroy(res)
    finally:
        mka.mka_system_destroy(s)
