"""Oracle: the whole work flow of Eq. EQ-WORK-FLOW over a set of atoms of a periodic system.

TEST INFRASTRUCTURE ONLY (see the package docstring).

For each selected atom a (its four columns j = 4a + o, o = s, px, py, pz share
one cluster): the cluster C_a (Sec. 3 real-space projection, by radius R),
dense P H P and P S P (optionally rounded to the storage format), one
`mka.solve_column` per column. Then mu by bisection over the selected columns'
(eps, w), and rho_ij, G_ij(z) and E_elec on the pattern i in H-row(j).

Output layout (the same as the library's): for atom b and each block k of
H's row b (neighbour atom a = col[k], columns ascending, a = b included),
``rho[k, c, r] = rho_{(a, r), (b, c)}``: block k holds the part of column
j = 4b + c on atom a's orbitals r. Then E^(j) = sum_k sum_r rho[k,c,r] H[k][c][r].
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import mka, sk as skmod
from .rounding import round_storage


@dataclass
class ColumnData:
    """What rho, G, E and mu need from one column: its levels and V on the pattern rows."""
    eps: np.ndarray              # eps_alpha, ascending, length nu_eff
    w: np.ndarray                # w_alpha
    Vrows: np.ndarray            # [len(rows), nu_eff] V restricted to the pattern rows
    vj: np.ndarray               # V_{j alpha}
    cg_iters: int
    nu_eff: int


@dataclass
class AtomResult:
    atom: int
    cluster: np.ndarray          # sorted global atom ids of C_a
    neigh: np.ndarray            # sorted global atom ids of H-row a (pattern), a included
    rows: np.ndarray             # local orbital indices of the pattern atoms (4 per atom)
    Hrow: np.ndarray             # [4, len(rows)] H_{j, i} for the 4 columns j and pattern i
    data: list                   # 4 x ColumnData
    nu: int
    cols: list | None = None     # 4 x mka.Column (full basis), only when asked for

    def eps_w(self) -> tuple[np.ndarray, np.ndarray]:
        """(eps, w) padded to nu per column; padding has w = 0."""
        eps = np.zeros((4, self.nu))
        w = np.zeros((4, self.nu))
        for o, c in enumerate(self.data):
            n = len(c.eps)
            eps[o, :n] = c.eps
            w[o, :n] = c.w
        return eps, w


def solve_atom(pos: np.ndarray, box: np.ndarray, skp, R: float, a: int, p: int, q: int,
               storage: str = "fp64", cg_tol: float = 1e-13, keep_full: bool = False, mode: str = "A",
               onsite_shift: np.ndarray | None = None) -> AtomResult:
    """`onsite_shift` [N] (eV) is added to the diagonal of every atom's on-site H block (a CSC potential)."""
    cl = skmod.cluster_atoms(pos, box, a, R)
    Hc, Sc = skmod.cluster_matrices(pos, box, cl, skp)
    if onsite_shift is not None:
        Hc = Hc + np.diag(np.repeat(np.asarray(onsite_shift)[cl], 4))
    Hc = round_storage(Hc, storage)
    Sc = round_storage(Sc, storage)
    t = int(np.searchsorted(cl, a))
    nb = skmod.neighbour_atoms(pos, box, a, skp.rc)
    loc = np.minimum(np.searchsorted(cl, nb), len(cl) - 1)
    inside = np.repeat(cl[loc] == nb, 4)        # pattern atoms beyond R lie outside the projection
    rows = (4 * loc[:, None] + np.arange(4)[None, :]).ravel()
    cols = [mka.solve_column(Hc, Sc, 4 * t + o, p, q, cg_tol=cg_tol, mode=mode) for o in range(4)]
    # v_alpha lives on the cluster: its rows outside the cluster are zero.
    data = [ColumnData(c.eps, c.w, c.V[rows, :] * inside[:, None], c.V[c.j, :], c.cg_iters, c.basis.nu_eff)
            for c in cols]
    Hrow = np.stack([Hc[4 * t + o, rows] * inside for o in range(4)])
    return AtomResult(a, cl, nb, rows, Hrow, data, p + q, cols if keep_full else None)


def solve_atoms(pos, box, skp, R, atoms, p, q, storage="fp64", cg_tol=1e-13, keep_full=True,
                mode="A") -> list[AtomResult]:
    return [solve_atom(pos, box, skp, R, int(a), p, q, storage, cg_tol, keep_full, mode) for a in atoms]


def stack_eps_w(results: list[AtomResult]) -> tuple[np.ndarray, np.ndarray]:
    """(eps, w) as [n_columns, nu], columns in atom order then orbital order."""
    e, w = zip(*(r.eps_w() for r in results))
    return np.concatenate(e), np.concatenate(w)


def find_mu(results: list[AtomResult], n_electrons: float, kT: float) -> float:
    eps, w = stack_eps_w(results)
    return mka.find_mu(eps, w, n_electrons, kT)


def density(results: list[AtomResult], mu: float, kT: float) -> tuple[list[np.ndarray], float, float]:
    """rho blocks per atom ([n_neigh, 4, 4] in the layout above), E_band and electron count.

    E_band = 2 sum_j sum_{i in pattern(j)} rho_ij H_ji (Eq. EQ-ENE, two electrons
    per orbital state); electron count = 2 sum_j sum_alpha f w.
    """
    rho_all = []
    e_band = 0.0
    n_el = 0.0
    for r in results:
        blocks = np.zeros((len(r.neigh), 4, 4))
        for o, c in enumerate(r.data):
            f = mka.fermi(c.eps, mu, kT)
            col = c.Vrows @ (f * c.vj)                  # Eq. EQ-DM, length 4 * n_neigh, atom-major
            blocks[:, o, :] = col.reshape(-1, 4)
            e_band += 2.0 * float(col @ r.Hrow[o])
            n_el += 2.0 * float(np.sum(f * c.w))
        rho_all.append(blocks)
    return rho_all, e_band, n_el


def band_energy_from_levels(results: list[AtomResult], mu: float, kT: float) -> float:
    """2 sum_j sum_alpha f eps w: equals E_band when p >= 1 (Tr[rho H] = Tr[pi S], Sec. 3)."""
    e = 0.0
    for r in results:
        for c in r.data:
            e += 2.0 * float(np.sum(mka.fermi(c.eps, mu, kT) * c.eps * c.w))
    return e


def greens(results: list[AtomResult], z: complex) -> list[np.ndarray]:
    """G_ij(z) blocks per atom, same layout as rho (complex128)."""
    out = []
    for r in results:
        blocks = np.zeros((len(r.neigh), 4, 4), dtype=np.complex128)
        for o, c in enumerate(r.data):
            g = c.Vrows.astype(np.complex128) @ (c.vj / (z - c.eps))   # Eq. EQ-SOLUTION-SUB-GZ
            blocks[:, o, :] = g.reshape(-1, 4)
        out.append(blocks)
    return out
