"""Persistent graph-captured batches (plans) and the autotuner, through the C ABI.

A plan runs the whole batch (per-atom kernel, device bisection for mu, rho and the
band energy) as one CUDA graph. With the direct path's CTA size (256) a plan must
reproduce the direct entry points bit for bit, whatever the work order or CTA count
(the per-atom arithmetic does not depend on which CTA takes an atom); another CTA
size changes the order of in-CTA sums, so there the parity tolerances apply (FP64
1e-10; mixed rho 1e-6, E 1e-5 eV/atom). Graph replay with new atoms must match a
fresh direct solve.
"""
import json

import numpy as np
import pytest

from synth import WORKLOADS, workload_positions

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_1202_0098_gb300 import build, mka
    build.build()
    mka.load()
    w = WORKLOADS["diamond512"]
    pos, box = workload_positions(w)
    s = mka.mka_build_system(pos, box, w.sk, "fp64", cluster_radius=w.R)
    yield mka, w, s
    mka.mka_system_destroy(s)


def direct(mka, s, w, atoms, arith, tol):
    prm = mka.solve_params(w.p, w.q, arith=arith, cg_tol=tol, keep_vectors=True)
    res = mka.mka_solve_columns(s, atoms, prm)
    lv = mka.mka_result_copy_levels(res)
    n_e = w.electrons_per_atom * len(atoms)
    mu = mka.mka_find_mu(res, n_e, w.kT)
    nb = mka.mka_result_info(res)["n_blocks"]
    rho = torch.empty(nb * 16, dtype=torch.float64, device="cuda")
    e, n = mka.mka_density_energy(s, res, mu, w.kT, rho.data_ptr())
    mka.mka_result_destroy(res)
    return lv, mu, e, n, rho.cpu().numpy()


def via_plan(mka, plan, w, atoms, rho):
    mka.mka_plan_run(plan, atoms, w.electrons_per_atom * len(atoms), w.kT, rho.data_ptr())
    mu, e, n = mka.mka_plan_scalars(plan)
    lv = mka.mka_result_copy_levels(mka.mka_plan_result(plan))
    return lv, mu, e, n, rho.cpu().numpy()


@pytest.mark.parametrize("arith,tol", [("fp64", 1e-13), ("mixed", 1e-7)])
@pytest.mark.parametrize("threads,ctas,order", [(256, 0, False), (128, 1, True), (512, 0, True), (256, 2, False)])
def test_plan_matches_direct_path(setup, arith, tol, threads, ctas, order):
    mka, w, s = setup
    prm = mka.solve_params(w.p, w.q, arith=arith, cg_tol=tol, keep_vectors=True)
    plan = mka.mka_plan_create(s, 40, prm, mka.tuning(threads, ctas, order))
    try:
        info = mka.mka_plan_info(plan)
        assert info["threads"] == threads and info["grid"] >= 1
        mrb = mka.mka_system_info(s)["max_row_blocks"]
        rho = torch.empty(40 * mrb * 16, dtype=torch.float64, device="cuda")
        for atoms in (np.arange(0, 40, dtype=np.int64), np.arange(300, 340, dtype=np.int64)):   # capture, replay
            k0 = mka.mka_kernel_launches()
            lv, mu, e, n, rh = via_plan(mka, plan, w, atoms, rho)
            assert mka.mka_kernel_launches() > k0
            dlv, dmu, de, dn, drh = direct(mka, s, w, atoms, arith, tol)
            np.testing.assert_array_equal(lv["nu_eff"], dlv["nu_eff"])
            np.testing.assert_array_equal(lv["status"], dlv["status"])
            if threads == 256:
                for key in ("eps", "w", "cg_iters"):
                    np.testing.assert_array_equal(lv[key], dlv[key])
                assert mu == dmu and e == de and n == dn
                np.testing.assert_array_equal(rh[:drh.size], drh)
            elif arith == "fp64":
                np.testing.assert_allclose(lv["eps"], dlv["eps"], rtol=0, atol=1e-10)
                np.testing.assert_allclose(lv["w"], dlv["w"], rtol=0, atol=1e-10)
                np.testing.assert_allclose(rh[:drh.size], drh, rtol=0, atol=1e-10)
                assert abs(mu - dmu) < 1e-9 and abs(e - de) / len(atoms) < 1e-10
            else:
                np.testing.assert_allclose(rh[:drh.size], drh, rtol=0, atol=1e-6)
                assert abs(mu - dmu) < 1e-4 and abs(e - de) / len(atoms) < 1e-5
    finally:
        mka.mka_plan_destroy(plan)


def test_plan_rejects_oversized_batch(setup):
    mka, w, s = setup
    plan = mka.mka_plan_create(s, 8, mka.solve_params(w.p, w.q))
    try:
        with pytest.raises(mka.MkaError) as e:
            mka.mka_plan_run(plan, np.arange(9, dtype=np.int64), 36.0, w.kT)
        assert e.value.status == mka.MKA_ERR_INVALID_ARG
    finally:
        mka.mka_plan_destroy(plan)


def test_autotune_picks_a_shape_and_caches_it(setup, tmp_path):
    mka, w, s = setup
    prm = mka.solve_params(w.p, w.q, arith="mixed", cg_tol=1e-7, keep_vectors=True)
    cache = str(tmp_path / "tune.json")
    sample = np.arange(0, 64, dtype=np.int64)
    t1 = mka.mka_autotune(s, prm, sample, 4.0 * 64, w.kT, cache)
    assert t1.threads in (128, 256, 512) and t1.ctas_per_sm in (0, 1, 2) and t1.order_by_size in (0, 1)
    entries = json.load(open(cache))["entries"]
    assert len(entries) == 1 and entries[0]["threads"] == t1.threads and entries[0]["ms"] > 0
    t2 = mka.mka_autotune(s, prm, sample, 4.0 * 64, w.kT, cache)     # from the cache
    assert (t2.threads, t2.ctas_per_sm, t2.order_by_size) == (t1.threads, t1.ctas_per_sm, t1.order_by_size)


def test_autotune_batch_picks_a_candidate_and_caches_it(setup, tmp_path):
    mka, w, s = setup
    prm = mka.solve_params(w.p, w.q, arith="mixed", cg_tol=1e-7, keep_vectors=True)
    cache = str(tmp_path / "tune.json")
    cands = [32, 128, 512]
    b = mka.mka_autotune_batch(s, prm, mka.tuning(), cands, 0, w.electrons_per_atom, w.kT, cache)
    assert b in cands
    entry = [e for e in json.load(open(cache))["entries"] if "batch_of" in e["key"]]
    assert len(entry) == 1 and entry[0]["batch"] == b and entry[0]["columns_per_s"] > 0
    assert mka.mka_autotune_batch(s, prm, mka.tuning(), cands, 0, w.electrons_per_atom, w.kT, cache) == b
