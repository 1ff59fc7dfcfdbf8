"""Seeded synthetic tight-binding systems shaped like the paper's workloads.

This module is the one piece shared by the FP64 oracle and the CUDA path. It
holds no arithmetic of the multiple Arnoldi method: it only draws atom
positions (perfect lattice, random vacancies, Gaussian displacements) and
names the Slater-Koster parameter sets, cluster radii, subspace sizes and
temperatures of the five workloads. Each side builds H and S from these
positions with its own code.

The paper's systems (NRL gold, extended-Hueckel PFO polymer; Sec. 3) cannot be
rebuilt here; these carbon-like sp systems keep their order-N structure: a
sparse 4x4-block H and S (s, px, py, pz per atom, Sec. 1 index convention),
S close to the unit matrix, local clusters of 80-270 atoms (Sec. 3 real-space
projection).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

# Slater-Koster two-centre parameters (eV for H, dimensionless for S), given at
# the reference bond length d0 and scaled by exp(-2 (d/d0 - 1)) up to a hard
# cutoff rc (Angstrom). V and Sv are (ss-sigma, sp-sigma, pp-sigma, pp-pi).


@dataclass(frozen=True)
class SKParams:
    Es: float
    Ep: float
    V: tuple
    Sv: tuple
    d0: float
    rc: float

    def as_array(self) -> np.ndarray:
        """Packed as [Es, Ep, V0..V3, Sv0..Sv3, d0, rc] (the C ABI's order)."""
        return np.array([self.Es, self.Ep, *self.V, *self.Sv, self.d0, self.rc], dtype=np.float64)


SK_CARBON_LIKE = SKParams(Es=-5.0, Ep=1.0, V=(-4.0, 4.5, 5.5, -1.8), Sv=(0.10, -0.12, -0.15, 0.05),
                          d0=1.54, rc=2.6)
# Metallic variant for the fcc workload: same functional form, shifted on-site
# levels so that the Fermi level lies inside a band. rc = 3.4 A keeps the
# first fcc shell (2.83 A at a = 4.0) inside the cutoff.
SK_FCC_METAL = replace(SK_CARBON_LIKE, Es=-2.0, Ep=0.5, rc=3.4)


@dataclass(frozen=True)
class Workload:
    name: str
    lattice: str          # "diamond" or "fcc"
    a: float              # cubic lattice constant (A)
    ncell: int            # cubic cells per edge
    sigma: float          # Gaussian displacement per Cartesian component (A)
    vacancy: float        # probability that a lattice site is left empty
    seed: int
    sk: SKParams
    R: float              # cluster radius (A)
    p: int
    q: int
    kT: float             # eV
    electrons_per_atom: float = 4.0

    @property
    def nu(self) -> int:
        return self.p + self.q


WORKLOADS = {
    # 512-atom diamond (4^3 cells), the small full-oracle case.
    "diamond512": Workload("diamond512", "diamond", 3.567, 4, 0.05, 0.0, 1, SK_CARBON_LIKE, 6.0, 15, 15, 0.1),
    # fcc 20^3 cells with 5% vacancies (about 30,400 atoms): uneven clusters.
    "fcc32k": Workload("fcc32k", "fcc", 4.0, 20, 0.08, 0.05, 2, SK_FCC_METAL, 7.0, 15, 15, 0.05),
    # 10^6-atom amorphous-like diamond (50^3 cells), p = q = 20.
    "diamond1m": Workload("diamond1m", "diamond", 3.567, 50, 0.15, 0.0, 3, SK_CARBON_LIKE, 7.0, 20, 20, 0.1),
    # 10,077,696-atom diamond (108^3 cells), the one-GPU full-scale system.
    "diamond10m": Workload("diamond10m", "diamond", 3.567, 108, 0.1, 0.0, 5, SK_CARBON_LIKE, 6.0, 15, 15, 0.1),
    # 262,144-atom cut of the same material (32^3 cells): the per-atom work of diamond10m on a
    # system small enough for full profiler captures.
    "diamond262k": Workload("diamond262k", "diamond", 3.567, 32, 0.1, 0.0, 6, SK_CARBON_LIKE, 6.0, 15, 15, 0.1),
}

_BASIS = {
    "diamond": np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0],
                         [.25, .25, .25], [.25, .75, .75], [.75, .25, .75], [.75, .75, .25]]),
    "fcc": np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]]),
}


def lattice_positions(lattice: str, a: float, ncell: int, sigma: float, vacancy: float,
                      seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Atom positions (N x 3, float64, wrapped into [0, L)) and the periodic box (3,).

    Sites are the conventional cubic cells in (ix, iy, iz) order, basis atom
    fastest. With one numpy PCG64 generator seeded by `seed`: first each site
    is dropped with probability `vacancy` (one uniform draw per site, only if
    vacancy > 0), then each kept atom gets an independent N(0, sigma^2)
    displacement per Cartesian component.
    """
    basis = _BASIS[lattice]
    g = np.arange(ncell, dtype=np.float64)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    sites = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    rng = np.random.Generator(np.random.PCG64(seed))
    if vacancy > 0:
        keep = rng.random(sites.shape[0]) >= vacancy
        sites = sites[keep]
    if sigma > 0:
        sites = sites + rng.normal(0.0, sigma, size=sites.shape)
    L = a * ncell
    box = np.array([L, L, L], dtype=np.float64)
    pos = np.mod(sites, box)
    # np.mod can return L itself for tiny negative inputs; fold that back to 0.
    pos[pos >= box] -= L
    return np.ascontiguousarray(pos), box


def workload_positions(w: Workload) -> tuple[np.ndarray, np.ndarray]:
    return lattice_positions(w.lattice, w.a, w.ncell, w.sigma, w.vacancy, w.seed)


def sample_atoms(n_atoms: int, n_sample: int, seed: int) -> np.ndarray:
    """Sorted distinct atom indices drawn uniformly without replacement."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_sample = min(n_sample, n_atoms)
    return np.sort(rng.choice(n_atoms, size=n_sample, replace=False)).astype(np.int64)


def random_symmetric_pair(m: int, seed: int, density: float = 0.5, s_scale: float = 0.1,
                          identity_s: bool = False) -> tuple[np.ndarray, np.ndarray]:
    """A small dense random H (symmetric) and S (SPD, S = I + small symmetric part).

    Used for tiny brute-force systems where the whole space is one cluster.
    Entries are dropped with probability 1 - density to give a sparse pattern.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    A = rng.normal(size=(m, m))
    A = A * (rng.random((m, m)) < density)
    H = 0.5 * (A + A.T) + np.diag(rng.normal(size=m))
    if identity_s:
        S = np.eye(m)
    else:
        B = rng.normal(size=(m, m)) * (rng.random((m, m)) < density)
        B = 0.5 * (B + B.T)
        B *= s_scale / max(1.0, np.abs(np.linalg.eigvalsh(B)).max())
        S = np.eye(m) + B
    return H, S
