"""The whole-system work flow on the GPU: every column's levels, one mu, then rho (Eq. EQ-WORK-FLOW).

Bars as in the other parity tests: FP64 form against the oracle |d rho| <= 1e-10, |d E| <= 1e-10
eV/atom, |d mu| <= 1e-9 eV; the mixed form against the FP64 form on the same stored values
|d rho| <= 1e-6, |d E| <= 1e-5 eV/atom. The device bisection, the host driver over the library's
chunk sums, and the driver over two chunk-aligned range sweeps (two processes' worth of data on
one GPU, exchanged by concatenation) must agree bit for bit.
"""
import numpy as np
import pytest

from oracle import system as osys
from oracle.parallel import solve_atoms_parallel
from synth import WORKLOADS, workload_positions

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def lib():
    from paper_1202_0098_gb300 import build, mka
    build.build()
    mka.load()
    return mka


@pytest.fixture(scope="module")
def d512(lib):
    """The 512-atom diamond system: the oracle over every atom, its mu and rho at that mu."""
    w = WORKLOADS["diamond512"]
    pos, box = workload_positions(w)
    atoms = np.arange(pos.shape[0], dtype=np.int64)
    ores = solve_atoms_parallel(pos, box, w.sk, w.R, atoms, w.p, w.q)
    n_e = w.electrons_per_atom * len(atoms)
    mu = osys.find_mu(ores, n_e, w.kT)
    orho, oe, on = osys.density(ores, mu, w.kT)
    return w, pos, box, ores, mu, np.concatenate(orho), oe


def sweep_system(mka, s, w, n_atoms, arith, kp, win, batch, ranges=None, chunk=64, stream=0):
    """Sweeps over `ranges` (default: the whole system) fed by one plan; returns (plan, sweeps)."""
    cg_tol = 1e-13 if arith == "fp64" else 1e-7
    prm = mka.solve_params(w.p, w.q, arith=arith, cg_tol=cg_tol, keep_vectors=True)
    plan = mka.mka_plan_create(s, batch, prm, None, stream)
    sweeps = []
    for a0, a1 in ranges or [(0, n_atoms)]:
        sw = mka.mka_sweep_create(s, a0, a1, w.nu, win[0], win[1], kp, chunk, stream)
        for b in range(a0, a1, batch):
            mka.mka_plan_run_sweep(plan, sw, np.arange(b, min(a1, b + batch), dtype=np.int64))
        sweeps.append(sw)
    return plan, sweeps


def rho_of(mka, sw, plan, mu, kT):
    nb = mka.mka_sweep_info(sw)["n_blocks"]
    rho = torch.full((nb * 16,), float("nan"), dtype=torch.float64, device="cuda")
    n_again = mka.mka_sweep_density(sw, plan, mu, kT, rho.data_ptr())
    torch.cuda.synchronize()
    return rho.cpu().numpy().reshape(nb, 4, 4), n_again


def test_sweep_matches_oracle_and_driver(lib, d512):
    mka = lib
    from paper_1202_0098_gb300 import distributed as D
    w, pos, box, ores, mu_ref, orho, oe = d512
    N = pos.shape[0]
    s = mka.mka_build_system(pos, box, w.sk, "fp64", cluster_radius=w.R)
    try:
        win = (mu_ref - 2.0 - 40 * w.kT, mu_ref + 2.0 + 40 * w.kT)
        plan, (sw,) = sweep_system(mka, s, w, N, "fp64", 12, win, 100)
        assert mka.mka_sweep_status(sw) == (N, 0)
        n_e = w.electrons_per_atom * N
        mu = mka.mka_sweep_find_mu(sw, n_e, w.kT)
        assert abs(mu - mu_ref) < 1e-9
        # the host driver over the library's chunk sums: the same mu, bit for bit
        nch = mka.mka_sweep_info(sw)["n_chunks"]
        mu_d, _ = D.find_mu([D.SweepPart(mka, sw)], nch, n_e, w.kT)
        assert mu_d == mu
        # rho at the oracle's mu from the stored pieces, and the band energy three ways
        rho, n_again = rho_of(mka, sw, plan, mu_ref, w.kT)
        assert n_again == 0
        np.testing.assert_allclose(rho, orho, rtol=0, atol=TOL)
        tot = D.totals([D.SweepPart(mka, sw)], nch, mu_ref, w.kT)
        assert abs(tot["e_band"] - oe) / N < TOL
        assert abs(tot["e_band_levels"] - tot["e_band"]) / N < 1e-11
        assert abs(tot["n_electrons"] - osys.density(ores, mu_ref, w.kT)[2]) < 1e-9
        # two chunk-aligned range sweeps, exchanged by concatenation: the same mu and totals, bit for bit
        plan2, parts = sweep_system(mka, s, w, N, "fp64", 12, win, 100, ranges=D.atom_ranges(N, 2, 64))
        P = [D.SweepPart(mka, x) for x in parts]
        mu2, _ = D.find_mu(P, nch, n_e, w.kT)
        assert mu2 == mu
        for x in parts:
            rho_of(mka, x, plan2, mu, w.kT)
        t2 = D.totals(P, nch, mu, w.kT)
        rho_of(mka, sw, plan, mu, w.kT)
        t1 = D.totals([D.SweepPart(mka, sw)], nch, mu, w.kT)
        assert t1 == t2
        for x in parts:
            mka.mka_sweep_destroy(x)
        mka.mka_plan_destroy(plan2)
        mka.mka_sweep_destroy(sw)
        mka.mka_plan_destroy(plan)
    finally:
        mka.mka_system_destroy(s)


def test_sweep_resolves_overflow_and_outside_window(lib, d512):
    """kp below some atoms' count of window levels: those atoms are solved again at mu; a window far
    from mu forces every atom to be solved again. rho and E still match the oracle."""
    mka = lib
    from paper_1202_0098_gb300 import distributed as D
    w, pos, box, ores, mu_ref, orho, oe = d512
    N = pos.shape[0]
    win = (mu_ref - 0.5 - 40 * w.kT, mu_ref + 0.5 + 40 * w.kT)
    oeps, ow = osys.stack_eps_w(ores)
    nu_eff = np.array([c.nu_eff for r in ores for c in r.data])
    inwin = ((oeps >= win[0]) & (oeps <= win[1]) & (np.arange(w.nu)[None, :] < nu_eff[:, None])).sum(1)
    atom_max = inwin.reshape(N, 4).max(1)
    kp = max(1, int(np.median(atom_max)))
    if kp >= atom_max.max():
        kp = max(1, atom_max.max() - 1)
    expect_over = int((atom_max > kp).sum())
    assert 0 < expect_over < N
    s = mka.mka_build_system(pos, box, w.sk, "fp64", cluster_radius=w.R)
    try:
        for kp_, win_, expect in ((kp, win, "some"), (4, (40.0, 60.0), "all")):
            plan, (sw,) = sweep_system(mka, s, w, N, "fp64", kp_, win_, 128)
            stored, over = mka.mka_sweep_status(sw)
            assert stored == N
            rho, n_again = rho_of(mka, sw, plan, mu_ref, w.kT)
            if expect == "some":
                assert abs(over - expect_over) <= 2 and n_again == over
            else:
                assert n_again == N
            np.testing.assert_allclose(rho, orho, rtol=0, atol=TOL)
            nch = mka.mka_sweep_info(sw)["n_chunks"]
            tot = D.totals([D.SweepPart(mka, sw)], nch, mu_ref, w.kT)
            assert abs(tot["e_band"] - oe) / N < TOL
            mka.mka_sweep_destroy(sw)
            mka.mka_plan_destroy(plan)
        with pytest.raises(mka.MkaError):       # atoms missing: no mu, no rho
            sw = mka.mka_sweep_create(s, 0, N, w.nu, -1.0, 1.0, 4, 64)
            try:
                mka.mka_sweep_find_mu(sw, 4.0 * N, w.kT)
            finally:
                mka.mka_sweep_destroy(sw)
    finally:
        mka.mka_system_destroy(s)


def test_sweep_mixed_form_against_fp64_form(lib, d512):
    """BF16-stored values, the mixed form against the FP64 form over the whole system: the global
    mu, rho on every pattern entry and the band energy."""
    mka = lib
    from paper_1202_0098_gb300 import distributed as D
    w, pos, box, ores, mu_ref, orho, oe = d512
    N = pos.shape[0]
    s = mka.mka_build_system(pos, box, w.sk, "bf16", cluster_radius=w.R)
    try:
        win = (mu_ref - 2.0 - 40 * w.kT, mu_ref + 2.0 + 40 * w.kT)
        out = {}
        for arith in ("fp64", "mixed"):
            plan, (sw,) = sweep_system(mka, s, w, N, arith, 12, win, 128)
            mu = mka.mka_sweep_find_mu(sw, w.electrons_per_atom * N, w.kT)
            rho, _ = rho_of(mka, sw, plan, mu, w.kT)
            nch = mka.mka_sweep_info(sw)["n_chunks"]
            out[arith] = (mu, rho, D.totals([D.SweepPart(mka, sw)], nch, mu, w.kT)["e_band"])
            mka.mka_sweep_destroy(sw)
            mka.mka_plan_destroy(plan)
        dmu = abs(out["mixed"][0] - out["fp64"][0])
        drho = np.abs(out["mixed"][1] - out["fp64"][1]).max()
        de = abs(out["mixed"][2] - out["fp64"][2]) / N
        print(f"whole system, mixed vs fp64: |d mu| {dmu:.2e} eV, max|d rho| {drho:.2e}, |d E| {de:.2e} eV/atom")
        assert drho <= 1e-6 and de <= 1e-5 and dmu < 1e-4
    finally:
        mka.mka_system_destroy(s)
