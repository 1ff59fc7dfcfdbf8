"""Pins for the oracle's energy density matrix and forces (Sec. 2, Eqs. EQ-FORCE, EQ-FORCE-PART).

* the analytic Slater-Koster block derivative against central differences of the block;
* in the complete limit (cluster = every atom, nu >= M) the force from the method's rho and pi
  equals minus the finite-difference derivative of the grand potential
  Omega = -2 kT sum_n ln(1 + exp(-(eps_n - mu)/kT)) of the dense generalized eigenvalues at fixed
  mu (a brute-force reference that shares nothing with the force code); the sign the paper prints
  for the pi term fails that check;
* pi_{.j} at full occupation with weights f eps: sum_i pi_ij S_ji = sum_alpha eps_alpha w_alpha;
* Newton's third law: the forces of any set of columns sum to zero.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import forces as ofo, mka as omka, sk as osk, system as osys
from synth import SK_CARBON_LIKE, WORKLOADS, workload_positions


def small_molecule(seed=0, n=6):
    """n atoms in a 30 A box, pair distances kept clear of the cutoff by more than 0.05 A."""
    rng = np.random.default_rng(seed)
    box = np.array([30.0, 30.0, 30.0])
    while True:
        pos = 12.0 + rng.uniform(0, 3.2, size=(n, 3))
        d = np.linalg.norm(pos[:, None] - pos[None, :], axis=2)[np.triu_indices(n, 1)]
        if d.min() > 1.2 and np.all(np.abs(d - SK_CARBON_LIKE.rc) > 0.05):
            return pos, box


def dense_pencil(pos, box, sk):
    g = osk.global_bsr(pos, box, sk)
    return osk.bsr_to_dense(g["row_ptr"], g["col"], g["H"]), osk.bsr_to_dense(g["row_ptr"], g["col"], g["S"])


def test_sk_block_grad_matches_finite_differences():
    rng = np.random.default_rng(2)
    for V in (SK_CARBON_LIKE.V, SK_CARBON_LIKE.Sv):
        for _ in range(6):
            d = rng.normal(size=3) * 1.3
            G = ofo.sk_block_grad(d, V, SK_CARBON_LIKE.d0)
            h = 1e-6
            for l in range(3):
                e = np.zeros(3)
                e[l] = h
                fd = (osk.sk_block(d + e, V, SK_CARBON_LIKE.d0) - osk.sk_block(d - e, V, SK_CARBON_LIKE.d0)) / (2 * h)
                np.testing.assert_allclose(G[l], fd, rtol=0, atol=1e-8)


@pytest.mark.parametrize("seed,mu,kT", [(0, 0.5, 0.3), (1, -1.0, 0.2), (3, 1.5, 0.5)])
def test_complete_limit_force_is_minus_grad_of_grand_potential(seed, mu, kT):
    sk = SK_CARBON_LIKE
    pos, box = small_molecule(seed)
    N = pos.shape[0]
    atoms = np.arange(N)
    res = osys.solve_atoms(pos, box, sk, 14.0, atoms, 2 * N, 2 * N, keep_full=False)
    rho, _, _ = osys.density(res, mu, kT)
    pi = ofo.energy_density(res, mu, kT)
    F = ofo.forces(pos, box, sk, res, rho, pi)

    def omega(p):
        H, S = dense_pencil(p, box, sk)
        return ofo.grand_potential(scipy.linalg.eigh(H, S, eigvals_only=True), mu, kT)

    h = 1e-5
    Ffd = np.zeros_like(F)
    for K in range(N):
        for l in range(3):
            e = np.zeros_like(pos)
            e[K, l] = h
            Ffd[K, l] = -(omega(pos + e) - omega(pos - e)) / (2 * h)
    np.testing.assert_allclose(F, Ffd, rtol=0, atol=2e-6)
    assert np.abs(F).max() > 1.0                              # a real test: the forces are not small
    # the sign printed in the paper (+ pi dS inside the braces) is not the derivative
    Fp = ofo.forces(pos, box, sk, res, rho, [-p for p in pi])
    assert np.abs(Fp - Ffd).max() > 1e-2


def test_forces_sum_to_zero_and_pi_sum_rule():
    w = WORKLOADS["diamond512"]
    pos, box = workload_positions(w)
    res = osys.solve_atoms(pos, box, w.sk, w.R, [3, 100, 377], w.p, w.q, keep_full=True)
    mu, kT = 1.9, w.kT
    rho, _, _ = osys.density(res, mu, kT)
    pi = ofo.energy_density(res, mu, kT)
    F = ofo.forces(pos, box, w.sk, res, rho, pi)
    np.testing.assert_allclose(F.sum(0), 0.0, atol=1e-11)
    assert np.abs(F).max() > 0.1
    # full occupation: pi_{.j} = sum_alpha eps v_alpha v_alpha,j, so sum_i pi_ij S_ji = sum eps w
    for r in res:
        Hc, Sc = osk.cluster_matrices(pos, box, r.cluster, w.sk)
        for c in r.cols:
            full = c.V @ (c.eps * c.V[c.j, :])
            assert abs(full @ Sc[c.j, :] - np.sum(c.eps * c.w)) < 1e-11
