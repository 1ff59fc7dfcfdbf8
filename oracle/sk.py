"""Oracle: Slater-Koster sp tight-binding H and S, and the real-space projection.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's Hamiltonians (NRL, extended Hueckel) are not available; the model
is the textbook two-centre Slater-Koster sp table (Slater & Koster 1954) with
the orbital order s, px, py, pz of the paper's composite index (Sec. 1).
For atoms a, b with displacement d = r_b - r_a (minimum image), |d| <= rc, and
direction cosines (l, m, n) = d/|d|, the 4x4 block <mu_a|nu_b> is

    [s][s]     = ss_sigma
    [s][p_k]   =  c_k sp_sigma
    [p_k][s]   = -c_k sp_sigma
    [p_k][p_m] =  c_k c_m (pp_sigma - pp_pi) + delta_km pp_pi

each two-centre integral scaled by exp(-2 (|d|/d0 - 1)). On-site blocks are
diag(Es, Ep, Ep, Ep) for H and the unit matrix for S.

Real-space projection (Sec. 3): the cluster of atom a is every atom b whose
minimum-image distance from a is at most R (a included), and the projected
matrices P H P, P S P are the restrictions of the periodic H and S to the
cluster's orbitals. This module builds them densely from positions, pair by
pair, without a neighbour list.
"""
from __future__ import annotations

import numpy as np


def min_image(d: np.ndarray, box: np.ndarray) -> np.ndarray:
    """Minimum-image displacement in a cubic/orthorhombic periodic box."""
    return d - box * np.round(d / box)


def sk_block(d: np.ndarray, V, d0: float) -> np.ndarray:
    """4x4 two-centre block <mu_a|nu_b> for displacement d = r_b - r_a (textbook SK sp table)."""
    dist = float(np.sqrt(d @ d))
    c = d / dist
    scale = np.exp(-2.0 * (dist / d0 - 1.0))
    ss, sp, pps, ppp = (v * scale for v in V)
    B = np.empty((4, 4))
    B[0, 0] = ss
    B[0, 1:] = c * sp
    B[1:, 0] = -c * sp
    B[1:, 1:] = np.outer(c, c) * (pps - ppp) + np.eye(3) * ppp
    return B


def onsite_blocks(sk) -> tuple[np.ndarray, np.ndarray]:
    return np.diag([sk.Es, sk.Ep, sk.Ep, sk.Ep]).astype(np.float64), np.eye(4)


def cluster_atoms(pos: np.ndarray, box: np.ndarray, a: int, R: float) -> np.ndarray:
    """Sorted indices of the atoms within minimum-image distance R of atom a (a included)."""
    d = min_image(pos - pos[a], box)
    r2 = np.einsum("ij,ij->i", d, d)
    return np.nonzero(r2 <= R * R)[0].astype(np.int64)


def neighbour_atoms(pos: np.ndarray, box: np.ndarray, a: int, rc: float) -> np.ndarray:
    """Sorted atoms b with H_ab != 0: a itself and every atom within rc (the pattern of a's rows)."""
    return cluster_atoms(pos, box, a, rc)


def sk_blocks(d: np.ndarray, V, d0: float) -> np.ndarray:
    """`sk_block` for many displacements at once: d is [n, 3], result [n, 4, 4]."""
    dist = np.sqrt(np.einsum("ij,ij->i", d, d))
    c = d / dist[:, None]
    scale = np.exp(-2.0 * (dist / d0 - 1.0))
    ss, sp, pps, ppp = (v * scale for v in V)
    B = np.empty((d.shape[0], 4, 4))
    B[:, 0, 0] = ss
    B[:, 0, 1:] = c * sp[:, None]
    B[:, 1:, 0] = -c * sp[:, None]
    B[:, 1:, 1:] = c[:, :, None] * c[:, None, :] * (pps - ppp)[:, None, None] + np.eye(3) * ppp[:, None, None]
    return B


def cluster_matrices(pos: np.ndarray, box: np.ndarray, atoms: np.ndarray, sk) -> tuple[np.ndarray, np.ndarray]:
    """Dense P H P and P S P on the orbitals of `atoms` (4 per atom, s px py pz).

    Local orbital index 4*t + o belongs to atoms[t], orbital o. Every pair of
    cluster atoms within rc (minimum image) gets its two-centre blocks.
    """
    n = len(atoms)
    Hon, Son = onsite_blocks(sk)
    H4 = np.zeros((n, n, 4, 4))
    S4 = np.zeros((n, n, 4, 4))
    idx = np.arange(n)
    H4[idx, idx] = Hon
    S4[idx, idx] = Son
    d = min_image(pos[atoms][None, :, :] - pos[atoms][:, None, :], box)   # d[t, u] = r_u - r_t
    r2 = np.einsum("tuk,tuk->tu", d, d)
    t, u = np.nonzero((r2 <= sk.rc * sk.rc) & (idx[:, None] != idx[None, :]))
    H4[t, u] = sk_blocks(d[t, u], sk.V, sk.d0)
    S4[t, u] = sk_blocks(d[t, u], sk.Sv, sk.d0)
    Hc = H4.transpose(0, 2, 1, 3).reshape(4 * n, 4 * n)
    Sc = S4.transpose(0, 2, 1, 3).reshape(4 * n, 4 * n)
    return Hc, Sc


def global_bsr(pos: np.ndarray, box: np.ndarray, sk) -> dict:
    """The periodic H and S of the whole system as 4x4-block CSR (brute force over all pairs).

    Rows are atoms; each row's block columns are ascending and include the
    diagonal. Returns row_ptr (N+1), col (nnzb), H, S ([nnzb, 4, 4]).
    Only for systems small enough for an O(N^2) pair scan.
    """
    N = pos.shape[0]
    Hon, Son = onsite_blocks(sk)
    row_ptr = [0]
    cols, Hb, Sb = [], [], []
    for a in range(N):
        nb = neighbour_atoms(pos, box, a, sk.rc)
        for b in nb:
            if b == a:
                Hb.append(Hon)
                Sb.append(Son)
            else:
                d = min_image(pos[b] - pos[a], box)
                Hb.append(sk_block(d, sk.V, sk.d0))
                Sb.append(sk_block(d, sk.Sv, sk.d0))
            cols.append(b)
        row_ptr.append(len(cols))
    return {"row_ptr": np.array(row_ptr, dtype=np.int64), "col": np.array(cols, dtype=np.int64),
            "H": np.array(Hb).reshape(-1, 4, 4), "S": np.array(Sb).reshape(-1, 4, 4)}


def bsr_to_dense(row_ptr: np.ndarray, col: np.ndarray, blocks: np.ndarray) -> np.ndarray:
    N = len(row_ptr) - 1
    A = np.zeros((4 * N, 4 * N))
    for a in range(N):
        for k in range(row_ptr[a], row_ptr[a + 1]):
            b = col[k]
            A[4 * a:4 * a + 4, 4 * b:4 * b + 4] = blocks[k]
    return A
