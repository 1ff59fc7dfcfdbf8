"""Oracle: the multiple Arnoldi method for one column j, then mu, rho, G and the band energy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Plain dense FP64 numpy, one column at a time, in the paper's order (Sec. 2):

1. inner CG for s_j = S^{-1} e_j (standard Hestenes-Stiefel CG, x0 = 0);
2. the S-orthonormal basis u_1..u_nu of L_nu^(j) = K_p(H; e_j) (+) K_q(H; s_j)
   (Eqs. EQ-SUBSPACE-MULTI-KRY, EQ-REC-UN, EQ-KN-HUN, EQ-MGram-Schmidt,
   EQ-CALC-S-INV);
3. the Galerkin reduced problem on that basis (Eq. EQ-SUB-EIG-VEC);
4. per-column eigen data eps_alpha, w_alpha; the Fermi-Dirac occupation, mu by
   bisection on the electron count (Sec. 2, after Eq. EQ-DM);
5. rho_ij (Eq. EQ-DM), G_ij(z) (Eq. EQ-SOLUTION-SUB-GZ), E_elec (Eq. EQ-ENE).

Readings where the paper is garbled or silent (each one is listed in the
design notes):

* Seam (Eq. EQ-CALC-S-INV): the vector that follows u_p is s_j, i.e.
  l_{p+1} = s_j minus its S-projection on u_1..u_p; H keeps acting on the
  latest u_n afterwards. u_1..u_p span K_p(H; e_j).
* Gram-Schmidt: the modified form the text names, run twice ("twice is
  enough"); coefficients (S u_m)^T l with S u_m stored.
* Breakdown: when the new vector keeps no more than tau = 1e-10 of its S-norm
  before projection, it is dropped. A dropped s_j (it already lies in the
  span, e.g. S = I) is replaced by H u_n, continuing the first chain. A first
  chain that closes before reaching p hands over to s_j at once. Any other
  breakdown ends the basis with nu_eff < nu.
* Reduced problem: S_r = U^T S U is formed explicitly and the generalized
  nu x nu problem is solved by Cholesky reduction (it equals the paper's
  standard problem when U^T S U = I).
* Occupation f(x) = 1 / (1 + exp((x - mu)/kT)), evaluated as
  (1 - tanh((x - mu) / (2 kT))) / 2. Two electrons per orbital state; the
  electron count is 2 sum_j sum_alpha f(eps_alpha^(j)) w_alpha^(j).
* Bisection: bracket [min eps - 40 kT, max eps + 40 kT]; stop when the bracket
  is at most 1e-12 eV wide or after 200 halvings; return the midpoint.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg

BREAKDOWN_TAU = 1e-10
GS_PASSES = 2


class OracleError(RuntimeError):
    pass


def cg(A: np.ndarray, b: np.ndarray, tol: float = 1e-13, maxit: int = 500,
       x0: np.ndarray | None = None) -> tuple[np.ndarray, int]:
    """Standard CG for A x = b (A SPD), the inner loop that gives s_j = S^{-1} e_j (Sec. 2).

    Stops when ||r||_2 <= tol * ||b||_2 (recursively updated residual).
    Returns (x, iterations). Raises OracleError when p^T A p <= 0 (A not SPD)
    or after maxit iterations.
    """
    x = np.zeros_like(b) if x0 is None else x0.astype(np.float64).copy()
    r = b - A @ x
    p = r.copy()
    rr = r @ r
    bnorm = np.sqrt(b @ b)
    for it in range(maxit + 1):
        if np.sqrt(rr) <= tol * bnorm:
            return x, it
        if it == maxit:
            break
        Ap = A @ p
        pAp = p @ Ap
        if not pAp > 0:
            raise OracleError("CG: p^T S p <= 0, S is not positive definite")
        alpha = rr / pAp
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = r @ r
        p = r + (rr_new / rr) * p
        rr = rr_new
    raise OracleError(f"CG did not converge in {maxit} iterations")


@dataclass
class Basis:
    U: np.ndarray        # m x nu_eff, S-orthonormal columns u_n (Eq. EQ-SUBS-MEMBERS)
    SU: np.ndarray       # S u_n
    K: np.ndarray        # k_n = H u_n (Eq. EQ-KN-HUN)
    nu_eff: int
    seam_at: int         # index n (1-based) of the vector built from s_j, 0 if none
    seam_substituted: bool


def multiple_arnoldi_basis(H: np.ndarray, S: np.ndarray, j: int, s: np.ndarray, p: int, q: int,
                           tau: float = BREAKDOWN_TAU, passes: int = GS_PASSES, mode: str = "A") -> Basis:
    """S-orthonormal basis of L_nu^(j) = K_p(H; e_j) (+) K_q(H; s_j) (Sec. 2).

    Each new vector l is S-orthogonalised against u_1..u_{n-1} (Eq.
    EQ-MGram-Schmidt, modified form, `passes` times), normalised in the S-norm
    (Eq. EQ-REC-UN), and k_n = H u_n is formed (Eq. EQ-KN-HUN). The next l is
    k_n, except after u_p where it is s_j (Eq. EQ-CALC-S-INV, seam reading in
    the module docstring). Breakdown handling as in the module docstring.

    mode "B" (the literal direct sum of Eq. EQ-SUBSPACE-MULTI-KRY): after the seam
    the next vector is H applied to the previous raw vector of the s_j chain
    (s_j, H s_j, H^2 s_j, ..., each scaled to unit 2-norm), not to the
    orthogonalised u_n, so the span is exactly K_p(H; e_j) + K_q(H; s_j). A raw
    vector that breaks down ends the basis (it and every later power lie in the span).
    """
    if p < 1 or q < 0:
        raise OracleError("need p >= 1 and q >= 0")
    if mode not in ("A", "B"):
        raise OracleError("mode is 'A' or 'B'")
    m = H.shape[0]
    nu = p + q
    U, SU, K = [], [], []
    l = np.zeros(m)
    l[j] = 1.0                      # l_1 := e_j
    src = "e"
    seam_done = q == 0
    seam_at = 0
    substituted = False
    raw = None                     # mode B: the current raw vector of the s_j chain
    n = 0
    while n < nu:
        beta_pre = np.sqrt(max(l @ (S @ l), 0.0))
        for _ in range(passes):
            for mm in range(n):
                c = SU[mm] @ l        # (S u_m)^T l
                l = l - c * U[mm]
        Sl = S @ l
        beta = np.sqrt(max(l @ Sl, 0.0))
        if not beta > tau * beta_pre:
            if src == "r":
                break
            if src == "s":
                # s_j already lies in the span: continue the first chain with H u_n.
                l = K[n - 1].copy()
                src = "H"
                substituted = True
                seam_at = 0
                continue
            if not seam_done:
                # The first chain closed before u_p: start the second chain now.
                l = s.copy()
                src = "s"
                seam_done = True
                seam_at = n + 1
                continue
            break
        u = l / beta                   # Eq. EQ-REC-UN
        U.append(u)
        SU.append(Sl / beta)
        K.append(H @ u)                # Eq. EQ-KN-HUN
        n += 1
        if mode == "B" and src in ("s", "r"):
            raw = H @ (s if src == "s" else raw)   # the next power of the s_j chain, from the raw vector
            raw = raw / np.linalg.norm(raw)
            l = raw.copy()
            src = "r"
        elif n == p and not seam_done:
            l = s.copy()               # Eq. EQ-CALC-S-INV: the next vector is s_j
            src = "s"
            seam_done = True
            seam_at = n + 1
        else:
            l = K[-1].copy()
            src = "H"
    if n == 0:
        raise OracleError("empty basis")
    return Basis(np.array(U).T, np.array(SU).T, np.array(K).T, n, seam_at, substituted)


@dataclass
class Reduced:
    Hr: np.ndarray
    Sr: np.ndarray
    eps: np.ndarray      # ascending subspace eigenlevels eps_alpha
    C: np.ndarray        # nu_eff x nu_eff, v_alpha = sum_n C_{n alpha} u_n (Eq. EQ-SUB-EIG-VEC)


def reduced_problem(B: Basis) -> Reduced:
    """Galerkin reduced problem on the basis (Eq. EQ-SUB-EIG-VEC and the text after it).

    H_r = U^T H U = U^T K and S_r = U^T S U, each symmetrised as (A + A^T)/2;
    S_r = L L^T (Cholesky); L^{-1} H_r L^{-T} = Y diag(eps) Y^T (LAPACK
    symmetric eigensolver through numpy); C = L^{-T} Y.
    """
    Hr = B.U.T @ B.K
    Sr = B.U.T @ B.SU
    Hr = 0.5 * (Hr + Hr.T)
    Sr = 0.5 * (Sr + Sr.T)
    try:
        L = np.linalg.cholesky(Sr)
    except np.linalg.LinAlgError as e:
        raise OracleError("reduced overlap matrix is not positive definite") from e
    X = scipy.linalg.solve_triangular(L, Hr, lower=True)          # L^{-1} Hr
    A = scipy.linalg.solve_triangular(L, X.T, lower=True).T       # L^{-1} Hr L^{-T}
    A = 0.5 * (A + A.T)
    eps, Y = np.linalg.eigh(A)
    C = scipy.linalg.solve_triangular(L.T, Y, lower=False)        # L^{-T} Y
    return Reduced(Hr, Sr, eps, C)


@dataclass
class Column:
    j: int               # local index of the column in its cluster
    s: np.ndarray        # s_j = S^{-1} e_j (CG)
    cg_iters: int
    basis: Basis
    red: Reduced
    eps: np.ndarray      # eps_alpha, length nu_eff
    V: np.ndarray        # m x nu_eff, columns v_alpha
    w: np.ndarray        # w_alpha = V_{j alpha} (S V)_{j alpha}
    hv_j: np.ndarray     # (H V)_{j alpha}


def solve_column(H: np.ndarray, S: np.ndarray, j: int, p: int, q: int, cg_tol: float = 1e-13,
                 x0: np.ndarray | None = None, mode: str = "A") -> Column:
    """One column of the work flow, Eq. EQ-WORK-FLOW first brace: {u_n} => {v_alpha, eps_alpha}."""
    e = np.zeros(H.shape[0])
    e[j] = 1.0
    s, it = cg(S, e, tol=cg_tol, x0=x0)
    B = multiple_arnoldi_basis(H, S, j, s, p, q, mode=mode)
    R = reduced_problem(B)
    V = B.U @ R.C
    SV = B.SU @ R.C
    HV = B.K @ R.C
    w = V[j, :] * SV[j, :]
    return Column(j, s, it, B, R, R.eps, V, w, HV[j, :])


def fermi(x, mu: float, kT: float):
    """Fermi-Dirac occupation 1/(1 + exp((x - mu)/kT)) written as (1 - tanh((x - mu)/(2kT)))/2."""
    return 0.5 * (1.0 - np.tanh((np.asarray(x) - mu) / (2.0 * kT)))


def electron_count(eps: np.ndarray, w: np.ndarray, mu: float, kT: float) -> float:
    """2 sum_j sum_alpha f(eps_alpha^(j)) w_alpha^(j) = 2 Tr(rho S) (spin-unpolarised).

    `eps` and `w` hold every column's levels, flattened; entries with w = 0 and
    any eps (padding for nu_eff < nu) contribute nothing.
    """
    return float(2.0 * np.sum(fermi(eps, mu, kT) * w))


def find_mu(eps: np.ndarray, w: np.ndarray, n_electrons: float, kT: float, tol: float = 1e-12,
            maxit: int = 200) -> float:
    """Chemical potential by bisection on the total electron number (Sec. 2, after Eq. EQ-DM)."""
    eps = np.asarray(eps, dtype=np.float64).ravel()
    w = np.asarray(w, dtype=np.float64).ravel()
    valid = w != 0
    lo = float(eps[valid].min()) - 40.0 * kT
    hi = float(eps[valid].max()) + 40.0 * kT
    for _ in range(maxit):
        if hi - lo <= tol:
            break
        mid = 0.5 * (lo + hi)
        if electron_count(eps, w, mid, kT) < n_electrons:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def rho_column(col: Column, f: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """rho_ij = sum_alpha f(eps_alpha) V_{i alpha} V_{j alpha} for i in `rows` (Eq. EQ-DM)."""
    return col.V[rows, :] @ (f * col.V[col.j, :])


def greens_column(col: Column, z: complex, rows: np.ndarray) -> np.ndarray:
    """G_ij(z) = sum_alpha V_{i alpha} V_{j alpha} / (z - eps_alpha) for i in `rows` (Eq. EQ-SOLUTION-SUB-GZ)."""
    return col.V[rows, :].astype(np.complex128) @ (col.V[col.j, :] / (z - col.eps))


def column_energy(col: Column, f: np.ndarray, H: np.ndarray, rows: np.ndarray) -> float:
    """E^(j) = sum_i rho_ij H_ji over the selected rows (Eq. EQ-ENE partial sum)."""
    return float(rho_column(col, f, rows) @ H[col.j, rows])


def dos(eps: np.ndarray, w: np.ndarray, energies, eta: float) -> np.ndarray:
    """Density of states from the subspace Green's function (Sec. 3, DOS discussion):
    D(E) = -(1/pi) Im sum_j (G(E + i eta) S)_jj, with sum_i G_ji(z) S_ij = sum_alpha w_alpha / (z - eps_alpha)
    for the column's Galerkin pairs (Eq. EQ-SOLUTION-SUB-GZ and w_alpha = v_alpha,j (S v_alpha)_j).
    `eps`, `w`: every column's levels and weights (entries with w = 0 add nothing). One value per
    state (no spin factor)."""
    eps = np.asarray(eps, dtype=np.float64).ravel()
    w = np.asarray(w, dtype=np.float64).ravel()
    out = np.empty(len(energies))
    for k, E in enumerate(energies):
        z = complex(E, eta)
        out[k] = -np.imag(np.sum(w / (z - eps))) / np.pi
    return out
