"""The learned CG warm start on the GPU, against the FP64 oracle of the network and its inputs.

Inputs and patches against oracle.mlp.features; forward, loss gradient and one Adam step
against oracle.mlp on the same BF16-rounded parameters (FP32 products and sums on the
GPU, so relative agreement ~1e-4); CG targets against the oracle's CG solution; and the
gain: after training on CG solutions of other seeds, solves started from the network's
prediction take fewer inner-CG iterations for the same tolerance, with rho unchanged
within the mixed form's bar. The saving is bounded by the patch: s_j beyond the 17
nearest atoms (third shell, ~1e-2 per entry for this model) stays in the first residual
even for a perfect prediction, worth about two of the ~12 iterations.
"""
import numpy as np
import pytest

from oracle import mlp as omlp, mka as omka, sk as osk
from synth import WORKLOADS, lattice_positions, workload_positions

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1202_0098_gb300 import build, mka
    build.build()
    mka.load()
    return mka


def test_features_match_oracle(lib):
    mka = lib
    for lat, a, sig, vac, R in (("diamond", 3.567, 0.1, 0.0, 6.0), ("fcc", 4.0, 0.08, 0.05, 7.0),
                                ("diamond", 3.567, 0.0, 0.0, 6.0)):
        pos, box = lattice_positions(lat, a, 4, sig, vac, 3)
        s = mka.mka_build_system(pos, box, WORKLOADS["diamond512"].sk, "fp64", cluster_radius=R)
        try:
            atoms = np.array([0, 5, 17, 100, pos.shape[0] - 1], dtype=np.int64)
            X = torch.empty((4 * len(atoms), 132), dtype=torch.float32, device="cuda")
            P = torch.empty((len(atoms), 17), dtype=torch.int32, device="cuda")
            mka.mka_warm_start_features(s, atoms, X.data_ptr(), P.data_ptr())
            X, P = X.cpu().numpy(), P.cpu().numpy()
            for t, at in enumerate(atoms):
                ox, op = omlp.features(pos, box, int(at))
                np.testing.assert_array_equal(P[t], op)
                np.testing.assert_allclose(X[4 * t:4 * t + 4], ox, rtol=0, atol=1e-6)
        finally:
            mka.mka_system_destroy(s)


def test_forward_gradient_and_adam_match_oracle(lib):
    mka = lib
    rng = np.random.default_rng(3)
    B = 64
    net = mka.mka_mlp_create(7)
    try:
        X = rng.normal(size=(B, 132)).astype(np.float32)
        T = (rng.normal(size=(B, 68)) * 0.1).astype(np.float32)
        Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
        theta_b = mka.mka_mlp_get_params(net, bf16_rounded=True).astype(np.float64)
        Y = torch.empty((B, 68), dtype=torch.float32, device="cuda")
        mka.mka_mlp_forward(net, Xd.data_ptr(), Y.data_ptr(), B)
        Yo, _ = omlp.forward(theta_b, X.astype(np.float64))
        np.testing.assert_allclose(Y.cpu().numpy(), Yo, rtol=0, atol=1e-4 * (1 + np.abs(Yo).max()))
        g = torch.empty(mka.mka_mlp_num_params(), dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        mka.mka_mlp_gradients(net, Xd.data_ptr(), Td.data_ptr(), B, g.data_ptr(), loss.data_ptr())
        Lo, go = omlp.loss_and_grad(theta_b, X.astype(np.float64), T.astype(np.float64))
        assert abs(loss.item() - Lo) <= 1e-4 * Lo
        gg = g.cpu().numpy()
        # element by element: FP32 sums of FP32 activations against FP64 (parameters BF16-rounded on both
        # sides); the floor 1e-5 max|g| covers entries that are sums cancelling to near zero
        np.testing.assert_allclose(gg, go, rtol=1e-3, atol=1e-5 * np.abs(go).max())
        assert np.linalg.norm(gg - go) <= 1e-4 * np.linalg.norm(go)
        theta = mka.mka_mlp_get_params(net).astype(np.float64)
        mka.mka_mlp_train_step(net, Xd.data_ptr(), Td.data_ptr(), B, 1e-3)
        ref, _, _ = omlp.adam_step(theta, gg.astype(np.float64), np.zeros_like(theta), np.zeros_like(theta), 1)
        np.testing.assert_allclose(mka.mka_mlp_get_params(net), ref, rtol=0, atol=2e-7)
    finally:
        mka.mka_mlp_destroy(net)


def test_cg_targets_match_oracle(lib):
    mka = lib
    w = WORKLOADS["diamond512"]
    pos, box = workload_positions(w)
    s = mka.mka_build_system(pos, box, w.sk, "fp64", cluster_radius=w.R)
    try:
        atoms = np.array([3, 300], dtype=np.int64)
        X = torch.empty((8, 132), dtype=torch.float32, device="cuda")
        P = torch.empty((2, 17), dtype=torch.int32, device="cuda")
        Y = torch.empty((8, 68), dtype=torch.float32, device="cuda")
        mka.mka_warm_start_features(s, atoms, X.data_ptr(), P.data_ptr())
        mka.mka_cg_patch_targets(s, atoms, "fp64", 1e-13, P.data_ptr(), Y.data_ptr())
        Y, P = Y.cpu().numpy(), P.cpu().numpy()
        for t, a in enumerate(atoms):
            cl = osk.cluster_atoms(pos, box, int(a), w.R)
            _, Sc = osk.cluster_matrices(pos, box, cl, w.sk)
            loc = np.searchsorted(cl, P[t])
            rows = (4 * loc[:, None] + np.arange(4)).ravel()
            for o in range(4):
                e = np.zeros(Sc.shape[0])
                e[4 * int(np.searchsorted(cl, a)) + o] = 1.0
                s_ref = np.linalg.solve(Sc, e)
                np.testing.assert_allclose(Y[4 * t + o], s_ref[rows], rtol=0, atol=1e-6)
    finally:
        mka.mka_system_destroy(s)


def test_trained_network_saves_cg_iterations(lib):
    """Train on CG solutions of other seeds, then solve held-out atoms with and without the warm start."""
    mka = lib
    from paper_1202_0098_gb300 import warm_start
    w = WORKLOADS["diamond512"]
    Xs, Ys = [], []
    for seed in (101, 102, 103):
        pos, box = lattice_positions("diamond", 3.567, 6, 0.1, 0.0, seed)
        s = mka.mka_build_system(pos, box, w.sk, "bf16", cluster_radius=6.0)
        X, Y, _ = warm_start.collect(s, np.arange(0, pos.shape[0], 2, dtype=np.int64))
        Xs.append(X)
        Ys.append(Y)
        mka.mka_system_destroy(s)
    X, Y = torch.cat(Xs), torch.cat(Ys)
    net = mka.mka_mlp_create(1)
    try:
        before = warm_start.mse(net, X, Y)
        hist = warm_start.train(net, X, Y, epochs=30, batch=512, lr=2e-3)
        after = warm_start.mse(net, X, Y)
        assert after < 0.05 * before and hist[-1] < hist[0]
        pos, box = lattice_positions("diamond", 3.567, 6, 0.1, 0.0, 104)      # held-out seed
        s = mka.mka_build_system(pos, box, w.sk, "bf16", cluster_radius=6.0)
        mka.mka_system_set_warm_start(s, net)
        atoms = np.arange(0, 400, dtype=np.int64)
        out = {}
        for ws in (False, True):
            prm = mka.solve_params(15, 15, arith="mixed", cg_tol=1e-7, keep_vectors=True, use_warm_start=ws)
            res = mka.mka_solve_columns(s, atoms, prm)
            lv = mka.mka_result_copy_levels(res)
            nb = mka.mka_result_info(res)["n_blocks"]
            rho = torch.empty(nb * 16, dtype=torch.float64, device="cuda")
            e, _ = mka.mka_density_energy(s, res, 1.9, 0.1, rho.data_ptr())
            fb = mka.mka_result_copy_warm_start(res) if ws else None
            out[ws] = (lv, rho.cpu().numpy(), e, fb)
            mka.mka_result_destroy(res)
        it0, it1 = out[False][0]["cg_iters"].mean(), out[True][0]["cg_iters"].mean()
        print(f"train mse {before:.3e} -> {after:.3e}; CG iterations {it0:.2f} -> {it1:.2f}; "
              f"fallback rate {out[True][3].mean():.3f}")
        assert it1 < 0.97 * it0
        assert out[True][3].mean() < 0.05
        assert np.abs(out[True][1] - out[False][1]).max() < 1e-6
        assert abs(out[True][2] - out[False][2]) / len(atoms) < 1e-5
        mka.mka_system_destroy(s)
    finally:
        mka.mka_mlp_destroy(net)
