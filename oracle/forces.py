"""Oracle: the energy density matrix and the forces (Sec. 2, after Eq. EQ-DM; Eqs. EQ-FORCE, EQ-FORCE-PART).

TEST INFRASTRUCTURE ONLY (see the package docstring).

For each column j of the selected atoms, on the pattern i of j's row (S_ij != 0; the same
pattern as H here, one cutoff rc for both):

    pi_ij  = sum_alpha f(eps_alpha) eps_alpha v_alpha,i v_alpha,j
    F_K    = -2 sum_j sum_i ( rho_ij dH_ji/dR_K - pi_ij dS_ji/dR_K )

(two electrons per orbital state, as for E_band = 2 Tr[rho H]). Reading of the sign: the
paper prints the S term with a plus sign inside the braces; the derivative of the
grand potential Omega = -2 kT sum_n ln(1 + exp(-(eps_n - mu)/kT)) at fixed mu is
dOmega = 2 sum_n f_n c_n^T (dH - eps_n dS) c_n = 2 (Tr[rho dH] - Tr[pi dS]) (the generalized
Hellmann-Feynman theorem with S c^T c = 1), which fixes the minus sign; the tests pin it
by finite differences of Omega.

dH_ji/dR_K is nonzero only for the two atoms of the block: for j on atom b and i on atom a,
H_ji is the SK block of d = R_a - R_b (minimum image), so dH_ji/dR_a = dB/dd and
dH_ji/dR_b = -dB/dd; on-site blocks do not depend on positions.
"""
from __future__ import annotations

import numpy as np

from . import mka
from .sk import min_image


def sk_block_grad(d: np.ndarray, V, d0: float) -> np.ndarray:
    """d/dd of the 4x4 two-centre block of `sk.sk_block` for displacement d: result [3 (l), 4, 4].

    With r = |d|, c = d / r, s(r) = exp(-2 (r/d0 - 1)): dr/dd_l = c_l, dc_k/dd_l = (delta_kl - c_k c_l)/r,
    ds/dd_l = -(2/d0) s c_l, applied to each entry of the table (product rule)."""
    r = float(np.sqrt(d @ d))
    c = d / r
    s = np.exp(-2.0 * (r / d0 - 1.0))
    ds = -(2.0 / d0) * s * c                       # [l]
    dc = (np.eye(3) - np.outer(c, c)) / r          # dc[k, l] = dc_k / dd_l
    ss, sp, pps, ppp = V
    G = np.zeros((3, 4, 4))
    for l in range(3):
        G[l, 0, 0] = ss * ds[l]
        for k in range(3):
            v = sp * (dc[k, l] * s + c[k] * ds[l])
            G[l, 0, 1 + k] = v
            G[l, 1 + k, 0] = -v
            for m in range(3):
                G[l, 1 + k, 1 + m] = ((pps - ppp) * ((dc[k, l] * c[m] + c[k] * dc[m, l]) * s + c[k] * c[m] * ds[l])
                                      + (ppp * ds[l] if k == m else 0.0))
    return G


def energy_density(results, mu: float, kT: float) -> list[np.ndarray]:
    """pi blocks per atom, the layout of `system.density`'s rho: blocks[k, c, r] = pi_{(a,r),(b,c)}."""
    out = []
    for r in results:
        blocks = np.zeros((len(r.neigh), 4, 4))
        for o, c in enumerate(r.data):
            fe = mka.fermi(c.eps, mu, kT) * c.eps
            blocks[:, o, :] = (c.Vrows @ (fe * c.vj)).reshape(-1, 4)
        out.append(blocks)
    return out


def forces(pos: np.ndarray, box: np.ndarray, sk, results, rho: list, pi: list) -> np.ndarray:
    """F_K of Eq. EQ-FORCE summed over the columns of `results` (atoms b), [N, 3]."""
    F = np.zeros((pos.shape[0], 3))
    for res, rb, pb in zip(results, rho, pi):
        b = res.atom
        for k, a in enumerate(res.neigh):
            if a == b:
                continue
            d = min_image(pos[a] - pos[b], box)
            gH = sk_block_grad(d, sk.V, sk.d0)       # d H_ba / d d, H_ba[c][r] = H_{(b,c),(a,r)} = H_ji
            gS = sk_block_grad(d, sk.Sv, sk.d0)
            g = -2.0 * (np.einsum("lcr,cr->l", gH, rb[k]) - np.einsum("lcr,cr->l", gS, pb[k]))
            F[a] += g
            F[b] -= g
    return F


def grand_potential(eps: np.ndarray, mu: float, kT: float) -> float:
    """Omega = -2 kT sum_n ln(1 + exp(-(eps_n - mu)/kT)) of a set of levels (two electrons per state)."""
    x = -(np.asarray(eps) - mu) / kT
    return float(-2.0 * kT * np.sum(np.logaddexp(0.0, x)))
