"""Pins for the oracle's method layer (Sec. 2 and 3 of the paper).

The references here are independent of the oracle's own code path:
* a dense generalized eigensolve (LAPACK sygvd through scipy) and a dense
  complex solve of (zS - H) x = e_j, which the method must reproduce when the
  subspace is the complete space (Sec. 2: exact as nu -> M);
* numpy's dense linear solve for s_j = S^{-1} e_j;
* a textbook three-term Lanczos recurrence (S = I) for the reductions to the
  earlier Krylov-subspace diagonalisation (Sec. 1, Sec. 2 q = 0 remark);
* an explicit Krylov matrix, QR-orthonormalised, with a generalized Galerkin
  solve, for q = 0 and q = 1, where the subspace has a closed form;
* the identities the paper proves: full occupation gives rho_{.j} = s_j
  (Eq. EQ-PHYS-FULL-OCC with the projection theorem of the NOTE-PROOF note),
  sum_alpha w_alpha = 1, and Tr[rho H] = Tr[pi S] per column (Sec. 3).
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.optimize

from oracle import mka, sk as osk, system
from synth import WORKLOADS, lattice_positions, random_symmetric_pair, workload_positions


def dense_reference(H, S, f_of_eps):
    """rho = Phi f(E) Phi^T from the dense generalized eigensolution (Phi^T S Phi = I)."""
    E, Phi = scipy.linalg.eigh(H, S)
    return E, Phi, (Phi * f_of_eps(E)) @ Phi.T


@pytest.mark.parametrize("m,seed", [(8, 0), (13, 1), (24, 2)])
def test_complete_subspace_equals_dense_solution(m, seed):
    """P1: nu >= M on a tiny system, cluster = everything: rho, G, E match the dense problem."""
    H, S = random_symmetric_pair(m, seed)
    mu, kT, z = 0.1, 0.3, 0.2 + 0.5j
    f = lambda e: mka.fermi(e, mu, kT)
    E, Phi, rho_ref = dense_reference(H, S, f)
    G_ref = np.linalg.solve(z * S - H, np.eye(m).astype(complex))
    p = q = m
    for j in range(m):
        col = mka.solve_column(H, S, j, p, q)
        assert col.basis.nu_eff == m
        fj = mka.fermi(col.eps, mu, kT)
        rows = np.arange(m)
        np.testing.assert_allclose(mka.rho_column(col, fj, rows), rho_ref[:, j], atol=1e-11)
        np.testing.assert_allclose(mka.greens_column(col, z, rows), G_ref[:, j], atol=1e-11)
        np.testing.assert_allclose(np.sort(col.eps), E, atol=1e-11)
        e_j = float(mka.rho_column(col, fj, rows) @ H[j, :])
        np.testing.assert_allclose(e_j, (rho_ref @ H)[j, j], atol=1e-11)
    # G is symmetric in the complete limit (P10)
    np.testing.assert_allclose(G_ref, G_ref.T, atol=1e-12)


def test_complete_subspace_electron_count_and_mu():
    """P1/P9: in the complete limit sum_j sum_alpha f w = sum_k f(E_k); bisection finds that mu."""
    m = 16
    H, S = random_symmetric_pair(m, 5)
    kT = 0.2
    E = scipy.linalg.eigh(H, S, eigvals_only=True)
    eps, w = [], []
    for j in range(m):
        c = mka.solve_column(H, S, j, m, m)
        eps.append(c.eps)
        w.append(c.w)
    eps, w = np.concatenate(eps), np.concatenate(w)
    n_e = 10.0
    mu = mka.find_mu(eps, w, n_e, kT)
    dense_count = lambda x: 2.0 * np.sum(mka.fermi(E, x, kT)) - n_e
    mu_ref = scipy.optimize.brentq(dense_count, E.min() - 5, E.max() + 5, xtol=1e-14)
    assert abs(mu - mu_ref) < 1e-10
    assert abs(mka.electron_count(eps, w, mu, kT) - n_e) < 1e-9 * n_e


def test_cluster_subspace_complete_equals_dense_cluster_solve():
    """P2: nu = m_c on one cluster: rho_{.j} equals the dense solve of (P H P, P S P)."""
    pos, box = lattice_positions("diamond", 3.567, 2, 0.05, 0.0, 3)
    skp = WORKLOADS["diamond512"].sk
    cl = osk.cluster_atoms(pos, box, 0, 2.6)
    Hc, Sc = osk.cluster_matrices(pos, box, cl, skp)
    m = Hc.shape[0]
    mu, kT = 0.5, 0.1
    _, _, rho_ref = dense_reference(Hc, Sc, lambda e: mka.fermi(e, mu, kT))
    for j in range(4):
        col = mka.solve_column(Hc, Sc, j, m // 2, m - m // 2)
        np.testing.assert_allclose(mka.rho_column(col, mka.fermi(col.eps, mu, kT), np.arange(m)),
                                   rho_ref[:, j], atol=1e-10)


@pytest.fixture(scope="module")
def diamond_atoms():
    w = WORKLOADS["diamond512"]
    pos, box = workload_positions(w)
    res = system.solve_atoms(pos, box, w.sk, w.R, [0, 201], w.p, w.q)
    return w, pos, box, res


def test_full_occupation_gives_s_and_duality(diamond_atoms):
    """P3: f = 1 gives rho_{.j} = s_j = S^{-1} e_j and sum_i rho_ij S_ji = 1 (q >= 1)."""
    w, pos, box, res = diamond_atoms
    for r in res:
        Hc, Sc = osk.cluster_matrices(pos, box, r.cluster, w.sk)
        for c in r.cols:
            e = np.zeros(Hc.shape[0])
            e[c.j] = 1.0
            s_ref = np.linalg.solve(Sc, e)
            rho1 = mka.rho_column(c, np.ones_like(c.eps), np.arange(Hc.shape[0]))
            np.testing.assert_allclose(rho1, s_ref, atol=1e-12)
            assert abs(rho1 @ Sc[c.j, :] - 1.0) < 1e-12


def test_weights_sum_to_one_and_energy_identity(diamond_atoms):
    """P4: sum_alpha w_alpha = 1 (e_j in L). P5: sum_i rho_ij H_ji = sum_alpha f eps w (p >= 1)."""
    w, pos, box, res = diamond_atoms
    mu, kT = 0.3, w.kT
    for r in res:
        Hc, _ = osk.cluster_matrices(pos, box, r.cluster, w.sk)
        for c in r.cols:
            assert abs(c.w.sum() - 1.0) < 1e-12
            f = mka.fermi(c.eps, mu, kT)
            lhs = mka.rho_column(c, f, np.arange(Hc.shape[0])) @ Hc[c.j, :]
            assert abs(lhs - np.sum(f * c.eps * c.w)) < 1e-11


def test_pattern_rows_hold_the_whole_energy(diamond_atoms):
    """The pattern rows (H_ji != 0) carry all of E^(j): restricting the sum changes nothing."""
    w, pos, box, res = diamond_atoms
    for r in res:
        Hc, _ = osk.cluster_matrices(pos, box, r.cluster, w.sk)
        nz = np.nonzero(Hc[r.cols[0].j, :])[0]
        assert set(nz.tolist()) <= set(r.rows.tolist())


def test_basis_is_s_orthonormal_and_projection_symmetric(diamond_atoms):
    """P8: U^T S U = I and H_r = U^T H U symmetric before symmetrisation."""
    _, _, _, res = diamond_atoms
    for r in res:
        for c in r.cols:
            B = c.basis
            np.testing.assert_allclose(B.U.T @ B.SU, np.eye(B.nu_eff), atol=1e-12)
            Hr = B.U.T @ B.K
            np.testing.assert_allclose(Hr, Hr.T, atol=1e-10)


def lanczos(H, j, nu):
    """Textbook Lanczos on K_nu(H; e_j) with full re-orthogonalisation: returns Q, alpha, beta."""
    m = H.shape[0]
    Q = np.zeros((m, nu))
    a, b = np.zeros(nu), np.zeros(nu - 1)
    Q[j, 0] = 1.0
    for n in range(nu):
        v = H @ Q[:, n]
        a[n] = Q[:, n] @ v
        v -= a[n] * Q[:, n]
        if n > 0:
            v -= b[n - 1] * Q[:, n - 1]
        v -= Q[:, :n + 1] @ (Q[:, :n + 1].T @ v)
        if n < nu - 1:
            b[n] = np.linalg.norm(v)
            Q[:, n + 1] = v / b[n]
    return Q, a, b


def test_q0_identity_overlap_is_lanczos():
    """P6: S = I, q = 0: H_r is tridiagonal with the Lanczos coefficients."""
    H, S = random_symmetric_pair(30, 11, identity_s=True)
    nu = 10
    col = mka.solve_column(H, S, 3, nu, 0)
    _, a, b = lanczos(H, 3, nu)
    Hr = col.red.Hr
    np.testing.assert_allclose(np.diag(Hr), a, atol=1e-12)
    np.testing.assert_allclose(np.diag(Hr, 1), b, atol=1e-12)
    np.testing.assert_allclose(np.triu(Hr, 2), 0, atol=1e-12)


def test_identity_overlap_reduces_to_krylov_diagonalisation():
    """P7: S = I, q > 0: s_j = e_j adds nothing; the result is Krylov diagonalisation on K_nu(H; e_j)."""
    H, S = random_symmetric_pair(40, 12, identity_s=True)
    p, q, j = 6, 6, 7
    mu, kT = 0.0, 0.2
    col = mka.solve_column(H, S, j, p, q)
    assert col.basis.seam_substituted and col.basis.nu_eff == p + q
    Q, a, b = lanczos(H, j, p + q)
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    e, Y = np.linalg.eigh(T)
    Vl = Q @ Y
    rho_ref = Vl @ (mka.fermi(e, mu, kT) * Vl[j, :])
    np.testing.assert_allclose(mka.rho_column(col, mka.fermi(col.eps, mu, kT), np.arange(40)), rho_ref, atol=1e-12)
    np.testing.assert_allclose(col.eps, e, atol=1e-12)


def galerkin_rho(H, S, W, j, mu, kT):
    """Galerkin density column on span(W): QR, then the generalized reduced problem."""
    Q, _ = np.linalg.qr(W)
    e, Y = scipy.linalg.eigh(Q.T @ H @ Q, Q.T @ S @ Q)
    Vg = Q @ Y
    return Vg @ (mka.fermi(e, mu, kT) * Vg[j, :])


@pytest.mark.parametrize("p,q", [(6, 0), (5, 1), (1, 1)])
def test_closed_form_subspaces(p, q):
    """q = 0: L = K_p(H; e_j) (generalized Arnoldi). q = 1: L = K_p(H; e_j) + span{s_j} exactly."""
    H, S = random_symmetric_pair(30, 21)
    j, mu, kT = 4, 0.1, 0.25
    col = mka.solve_column(H, S, j, p, q)
    e = np.zeros(30)
    e[j] = 1.0
    cols = [e]
    for _ in range(p - 1):
        v = H @ cols[-1]
        cols.append(v / np.linalg.norm(v))
    if q == 1:
        cols.append(np.linalg.solve(S, e))
    ref = galerkin_rho(H, S, np.array(cols).T, j, mu, kT)
    np.testing.assert_allclose(mka.rho_column(col, mka.fermi(col.eps, mu, kT), np.arange(30)), ref, atol=1e-10)


def test_cg_matches_dense_solve():
    H, S = random_symmetric_pair(50, 31, s_scale=0.3)
    b = np.random.default_rng(0).normal(size=50)
    x, it = mka.cg(S, b, tol=1e-13)
    np.testing.assert_allclose(x, np.linalg.solve(S, b), atol=1e-12)
    assert 1 <= it <= 50


def test_cg_rejects_indefinite_matrix():
    A = np.diag([1.0, -1.0, 2.0])
    with pytest.raises(mka.OracleError):
        mka.cg(A, np.array([0.0, 1.0, 0.0]))


def test_fermi_function():
    assert mka.fermi(0.3, 0.3, 0.1) == 0.5
    x = np.linspace(-2, 2, 41)
    np.testing.assert_allclose(mka.fermi(x, 0.1, 0.2), 1.0 / (1.0 + np.exp((x - 0.1) / 0.2)), rtol=0, atol=1e-15)
    assert mka.fermi(-1e4, 0.0, 0.1) == 1.0 and mka.fermi(1e4, 0.0, 0.1) == 0.0


def _pi_dimer():
    """Two atoms on the z axis at the reference bond length in a large box."""
    from synth import SK_CARBON_LIKE
    pos = np.array([[5.0, 5.0, 5.0], [5.0, 5.0, 5.0 + SK_CARBON_LIKE.d0]])
    return pos, np.array([20.0, 20.0, 20.0]), SK_CARBON_LIKE


def _pi_dimer_closed_form(sk, mu, kT):
    """The p_x (or p_y) orbitals of a z-axis dimer see only the pp-pi couplings (direction cosine 0):
    the 2x2 pencil H = [[Ep, V], [V, Ep]], S = [[1, s], [s, 1]] with V = pp-pi of H, s = pp-pi of S
    at the reference length. Its eigenvectors are (1, +-1) / sqrt(2 (1 +- s)), so the levels are
    (Ep +- V) / (1 +- s), both with weight 1/2, and rho_{j'j} = f_+ / (2 (1 + s)) +- f_- / (2 (1 - s))
    for j' = j and for j' the same orbital on the other atom."""
    V, s = sk.V[3], sk.Sv[3]
    e_plus, e_minus = (sk.Ep + V) / (1 + s), (sk.Ep - V) / (1 - s)
    f = lambda e: 1.0 / (1.0 + np.exp((e - mu) / kT))
    same = f(e_plus) / (2 * (1 + s)) + f(e_minus) / (2 * (1 - s))
    other = f(e_plus) / (2 * (1 + s)) - f(e_minus) / (2 * (1 - s))
    return np.sort([e_plus, e_minus]), same, other


def test_pi_dimer_closed_form():
    pos, box, sk = _pi_dimer()
    mu, kT = 1.0, 0.1
    levels, same, other = _pi_dimer_closed_form(sk, mu, kT)
    res = system.solve_atom(pos, box, sk, 3.0, 0, 2, 2)
    rho, _, _ = system.density([res], mu, kT)
    for o in (1, 2):                                     # p_x and p_y columns of atom 0
        c = res.data[o]
        assert c.nu_eff == 2                             # the pi block is invariant: the basis closes
        np.testing.assert_allclose(c.eps, levels, rtol=0, atol=1e-13)
        np.testing.assert_allclose(c.w, [0.5, 0.5], rtol=0, atol=1e-13)
        k_self, k_other = list(res.neigh).index(0), list(res.neigh).index(1)
        assert abs(rho[0][k_self, o, o] - same) < 1e-13
        assert abs(rho[0][k_other, o, o] - other) < 1e-13


def test_single_atom_cluster():
    """R below the bond length: the cluster is the atom alone, H_c = diag(Es, Ep, Ep, Ep), S_c = I.
    Every column closes at nu_eff = 1 (s_j = e_j is already in the span) with its on-site level and
    weight 1; rho is f of that level on the diagonal and zero elsewhere, the pattern atoms outside
    the cluster included (reading A16)."""
    from synth import SK_CARBON_LIKE as sk
    pos, box = lattice_positions("diamond", 3.567, 3, 0.05, 0.0, 3)
    mu, kT = 0.5, 0.1
    res = system.solve_atom(pos, box, sk, 1.0, 7, 3, 3)
    assert list(res.cluster) == [7] and len(res.neigh) > 1
    rho, _, _ = system.density([res], mu, kT)
    onsite = [sk.Es, sk.Ep, sk.Ep, sk.Ep]
    k_self = list(res.neigh).index(7)
    expect = np.zeros_like(rho[0])
    for o in range(4):
        c = res.data[o]
        assert c.nu_eff == 1
        assert abs(c.eps[0] - onsite[o]) < 1e-14 and abs(c.w[0] - 1.0) < 1e-14
        expect[k_self, o, o] = 1.0 / (1.0 + np.exp((onsite[o] - mu) / kT))
    np.testing.assert_allclose(rho[0], expect, rtol=0, atol=1e-14)


def _s_projector(H, S, j, p):
    """Pi_p = Q (Q^T S Q)^{-1} Q^T S: the S-orthogonal projector onto K_p(H; e_j), from an explicit,
    Euclidean-QR-orthonormalised Krylov matrix (no S-orthogonalisation, no Gram-Schmidt of the oracle)."""
    m = H.shape[0]
    e = np.zeros(m)
    e[j] = 1.0
    cols = [e]
    for _ in range(p - 1):
        v = H @ cols[-1]
        cols.append(v / np.linalg.norm(v))
    Q, _ = np.linalg.qr(np.array(cols).T)
    return Q @ np.linalg.solve(Q.T @ S @ Q, Q.T @ S), Q


def reading_a_subspace(H, S, j, p, q):
    """Closed form of the seam reading for any q: L = K_p(H; e_j) (+) K_q(H_hat; t) with
    t = (I - Pi_p) s_j and H_hat = (I - Pi_p) H. Every vector the second chain adds is S-orthogonal
    to K_p(H; e_j), so H acting on it leaves that space only through its Pi_p part, which lies in the
    span already; hence the recursion of Eqs. EQ-KN-HUN / EQ-CALC-S-INV spans exactly this sum."""
    m = H.shape[0]
    Pi, Q = _s_projector(H, S, j, p)
    e = np.zeros(m)
    e[j] = 1.0
    t = np.linalg.solve(S, e)
    t = t - Pi @ t
    T = [t / np.linalg.norm(t)]
    for _ in range(q - 1):
        v = H @ T[-1]
        v = v - Pi @ v
        T.append(v / np.linalg.norm(v))
    return np.hstack([Q, np.array(T).T])


def reading_b_subspace(H, S, j, p, q):
    """The literal direct sum K_p(H; e_j) + K_q(H; s_j): a separate chain on s_j."""
    m = H.shape[0]
    _, Q = _s_projector(H, S, j, p)
    e = np.zeros(m)
    e[j] = 1.0
    s = np.linalg.solve(S, e)
    T = [s / np.linalg.norm(s)]
    for _ in range(q - 1):
        v = H @ T[-1]
        T.append(v / np.linalg.norm(v))
    return np.hstack([Q, np.array(T).T])


@pytest.mark.parametrize("p,q,seed", [(3, 2, 41), (4, 3, 42), (5, 5, 43), (6, 4, 44)])
def test_second_chain_closed_form(p, q, seed):
    """q >= 2: the oracle's seam recursion spans K_p(H; e_j) (+) K_q((I - Pi_p) H; (I - Pi_p) s_j),
    built here from explicit Krylov matrices and the S-projector formula. rho, G and the Ritz levels
    of the Galerkin problem on that span match the oracle; the literal direct sum (a second chain on
    s_j itself) does not, so the pin tells the two readings apart."""
    m = 40
    H, S = random_symmetric_pair(m, seed)
    j, mu, kT, z = 5, 0.1, 0.25, 0.3 + 0.4j
    col = mka.solve_column(H, S, j, p, q)
    assert col.basis.nu_eff == p + q
    W = reading_a_subspace(H, S, j, p, q)
    Qw, _ = np.linalg.qr(W)
    e, Y = scipy.linalg.eigh(Qw.T @ H @ Qw, Qw.T @ S @ Qw)
    Vg = Qw @ Y
    rows = np.arange(m)
    f = mka.fermi(col.eps, mu, kT)
    np.testing.assert_allclose(col.eps, e, atol=1e-10)
    np.testing.assert_allclose(mka.rho_column(col, f, rows), Vg @ (mka.fermi(e, mu, kT) * Vg[j, :]), atol=1e-10)
    np.testing.assert_allclose(mka.greens_column(col, z, rows), Vg @ (Vg[j, :] / (z - e)), atol=1e-10)
    rho_b = galerkin_rho(H, S, reading_b_subspace(H, S, j, p, q), j, mu, kT)
    assert np.abs(mka.rho_column(col, f, rows) - rho_b).max() > 1e-6


def test_second_chain_pin_catches_h_on_s():
    """A plausible slip in the seam recursion (H acting on s_j instead of on u_{p+1}) is caught by the
    closed form: the planted variant builds the reading-B span and misses it by far more than 1e-10."""
    m, p, q, j = 40, 4, 3, 5
    H, S = random_symmetric_pair(m, 45)
    mu, kT = 0.1, 0.25
    W = reading_a_subspace(H, S, j, p, q)
    ref = galerkin_rho(H, S, W, j, mu, kT)
    planted = galerkin_rho(H, S, reading_b_subspace(H, S, j, p, q), j, mu, kT)
    assert np.abs(planted - ref).max() > 1e-6


@pytest.mark.parametrize("p,q,seed", [(3, 2, 41), (4, 3, 42), (5, 5, 43)])
def test_reading_b_is_the_direct_sum(p, q, seed):
    """mode "B": the oracle's basis spans exactly K_p(H; e_j) + K_q(H; s_j) (explicit Krylov matrices of
    e_j and of s_j, QR of their union): eps, rho and G of the Galerkin problem match at 1e-10, and differ
    from reading A's."""
    m = 40
    H, S = random_symmetric_pair(m, seed)
    j, mu, kT, z = 5, 0.1, 0.25, 0.3 + 0.4j
    col = mka.solve_column(H, S, j, p, q, mode="B")
    assert col.basis.nu_eff == p + q
    Qw, _ = np.linalg.qr(reading_b_subspace(H, S, j, p, q))
    e, Y = scipy.linalg.eigh(Qw.T @ H @ Qw, Qw.T @ S @ Qw)
    Vg = Qw @ Y
    rows = np.arange(m)
    f = mka.fermi(col.eps, mu, kT)
    np.testing.assert_allclose(col.eps, e, atol=1e-10)
    np.testing.assert_allclose(mka.rho_column(col, f, rows), Vg @ (mka.fermi(e, mu, kT) * Vg[j, :]), atol=1e-10)
    np.testing.assert_allclose(mka.greens_column(col, z, rows), Vg @ (Vg[j, :] / (z - e)), atol=1e-10)
    cA = mka.solve_column(H, S, j, p, q, mode="A")
    assert np.abs(mka.rho_column(cA, mka.fermi(cA.eps, mu, kT), rows) - mka.rho_column(col, f, rows)).max() > 1e-6
    # the identities that hold for any subspace containing e_j and s_j hold for B as well
    assert abs(col.w.sum() - 1.0) < 1e-12
    np.testing.assert_allclose(mka.rho_column(col, np.ones_like(col.eps), rows), np.linalg.solve(S, np.eye(m)[:, j]),
                               atol=1e-11)
