"""The fcc workload in full: every column of the ~30,400-atom fcc system with vacancies through
graph-replayed plan batches into a sweep, one mu for the whole system, rho on the whole pattern,
and the oracle on every atom (FP64 form: |d rho| <= 1e-10, |d E| <= 1e-10 eV/atom, |d mu| <= 1e-9 eV).
The Fermi level lies inside a band here: the density of states at mu, (eta / pi) sum_j sum_alpha
w_alpha / ((mu - eps_alpha)^2 + eta^2) = -(1/pi) Im sum_j (G(mu + i eta) S)_jj, is far from zero.
"""
import numpy as np
import pytest

from oracle import system as osys
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


def oracle_dos(eps, w, E, eta):
    return float(eta / np.pi * np.sum(w / ((E - eps) ** 2 + eta ** 2)))


def test_fcc_whole_system_against_oracle(lib):
    mka = lib
    from paper_1202_0098_gb300 import distributed as D
    w = WORKLOADS["fcc32k"]
    pos, box = workload_positions(w)
    N = pos.shape[0]
    atoms = np.arange(N, dtype=np.int64)
    ores = solve_atoms_parallel(pos, box, w.sk, w.R, atoms, w.p, w.q)
    n_e = w.electrons_per_atom * N
    mu_o = osys.find_mu(ores, n_e, w.kT)
    orho, oe, _ = osys.density(ores, mu_o, w.kT)
    oeps, ow = osys.stack_eps_w(ores)
    dos_mu = oracle_dos(oeps, ow, mu_o, w.kT) / N
    print(f"fcc, {N} atoms: oracle mu {mu_o:.6f} eV, DOS at mu {dos_mu:.3f} states/eV/atom")
    assert dos_mu > 0.05
    s = mka.mka_build_system(pos, box, w.sk, "fp64", cluster_radius=w.R)
    try:
        B = 4096
        plan = mka.mka_plan_create(s, B, mka.solve_params(w.p, w.q, cg_tol=1e-13, keep_vectors=True))
        sw = mka.mka_sweep_create(s, 0, N, w.nu, mu_o - 3.0, mu_o + 3.0, w.nu, 1024)
        for b in range(0, N, B):
            mka.mka_plan_run_sweep(plan, sw, atoms[b:b + B])
        mu = mka.mka_sweep_find_mu(sw, n_e, w.kT)
        assert abs(mu - mu_o) < 1e-9
        nb = mka.mka_sweep_info(sw)["n_blocks"]
        rho = torch.empty(nb * 16, dtype=torch.float64, device="cuda")
        assert mka.mka_sweep_density(sw, plan, mu_o, w.kT, rho.data_ptr()) == 0
        torch.cuda.synchronize()
        np.testing.assert_allclose(rho.cpu().numpy().reshape(nb, 4, 4), np.concatenate(orho), rtol=0, atol=1e-10)
        tot = D.totals([D.SweepPart(mka, sw)], mka.mka_sweep_info(sw)["n_chunks"], mu_o, w.kT)
        assert abs(tot["e_band"] - oe) / N < 1e-10
        # the DOS of the whole system from the sweep's levels (mka_dos), around mu, against the oracle's
        e_ptr, w_ptr = mka.mka_sweep_device_levels(sw)
        grid = np.linspace(mu_o - 1.0, mu_o + 1.0, 41)
        got = mka.mka_dos(e_ptr, w_ptr, 4 * N * w.nu, grid, w.kT) / N
        ref = np.array([oracle_dos(oeps, ow, E, w.kT) for E in grid]) / N
        np.testing.assert_allclose(got, ref, rtol=1e-10)
        assert got[20] > 0.05
        mka.mka_sweep_destroy(sw)
        mka.mka_plan_destroy(plan)
    finally:
        mka.mka_system_destroy(s)
