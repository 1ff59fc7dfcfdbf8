"""Several processes, one system: the data plane of the whole-system work flow across GPUs.

The columns j are independent (Eq. EQ-WORK-FLOW, first brace): each process sweeps
one contiguous range of atoms on its own GPU (``mka_sweep_create`` over that range,
``mka_plan_run_sweep`` for its batches) with no exchange at all. The global steps
need only small exchanges, all of vectors of chunk sums that the library computes
(``mka_sweep_chunk_sums``):

* the level range, once (min / max of the processes' ranges);
* one sum of the chunk-count vector per root-finder step (Sec. 2: mu from the total
  electron number of all columns);
* the chunk vectors of the electron count and band energy at the final mu.

Ranges start on chunk boundaries (``atom_ranges``), so every chunk sum is computed by
exactly one process, from the same entries in the same order as a single process over
the whole system would; the zero-padded vectors' sum over processes is therefore exact,
and adding it in chunk order reproduces the single-process mu and energies bit for bit.

This module only orchestrates: it compares a sum with the target and narrows a bracket
(bisection, then the Illinois secant), step for step as ``mka_sweep_find_mu`` does on one
device; every sum over levels runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np

MAX_HALVINGS = 200


def atom_ranges(n_atoms: int, world: int, chunk_atoms: int) -> list[tuple[int, int]]:
    """Contiguous, chunk-aligned atom ranges of `world` processes (chunks shared out evenly)."""
    n_chunks = (n_atoms + chunk_atoms - 1) // chunk_atoms
    bounds = [min(n_atoms, (n_chunks * r // world) * chunk_atoms) for r in range(world + 1)]
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


class SweepPart:
    """One process's sweep seen through the two calls the global steps need."""

    def __init__(self, mka, sweep):
        self.mka, self.sweep = mka, sweep
        self.chunk0 = mka.mka_sweep_info(sweep)["chunk0"]

    def level_range(self) -> tuple[float, float]:
        return self.mka.mka_sweep_level_range(self.sweep)

    def chunk_sums(self, mu: float, kT: float, levels: bool = False, rho: bool = False) -> tuple[int, dict]:
        return self.chunk0, self.mka.mka_sweep_chunk_sums(self.sweep, mu, kT, levels=levels, rho=rho)


def _all_reduce(values: np.ndarray, op: str, group, device) -> np.ndarray:
    """Reduce over the processes of `group` (None: this process alone)."""
    if group is None:
        return values
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(values, dtype=np.float64)).to(device)
    dist.all_reduce(t, op={"sum": dist.ReduceOp.SUM, "min": dist.ReduceOp.MIN, "max": dist.ReduceOp.MAX}[op],
                    group=group)
    return t.cpu().numpy()


def _ordered_sum(v: np.ndarray) -> float:
    """Left-to-right sum, the order the device root finder adds its chunk sums in."""
    t = 0.0
    for x in v.tolist():
        t += x
    return t


def gather_chunks(parts, n_chunks_total: int, key: str, mu: float, kT: float, group=None, device="cpu",
                  levels=False, rho=False) -> np.ndarray:
    """The whole system's vector of chunk sums `key` at mu: each part fills its chunks, zeros elsewhere,
    and the vectors are summed over processes (exact: one nonzero term per entry)."""
    full = np.zeros(n_chunks_total)
    for p in parts:
        c0, sums = p.chunk_sums(mu, kT, levels=levels, rho=rho)
        full[c0:c0 + len(sums[key])] += sums[key]
    return _all_reduce(full, "sum", group, device)


SECANT_KT = 16.0   # bisection while the bracket is wider than this many kT, then the secant


def find_mu(parts, n_chunks_total: int, n_electrons: float, kT: float, tol: float = 1e-12, group=None,
            device="cpu") -> tuple[float, int]:
    """mu with N(mu) = n_electrons over every column of all processes; (mu, steps).

    The library's root finder step for step (mka_sweep_find_mu): bracket [min eps - 40 kT, max eps + 40 kT]
    over levels with nonzero weight (N = 0 at its lower end), its upper end evaluated first, bisection
    while the bracket is wider than 16 kT, then regula falsi with the Illinois rule (after two moves of the
    same end by the secant the other end's f is halved), the midpoint when the secant leaves the bracket;
    the count at each point is the chunk-ordered sum; a point where it equals n_electrons exactly closes
    the bracket on it; mu = the bracket's midpoint once it is no wider than tol. Python floats round like
    the device's IEEE operations, so the points agree bit for bit."""
    rng = np.array([[*p.level_range()] for p in parts])
    lo = float(_all_reduce(np.array([rng[:, 0].min()]), "min", group, device)[0]) - 40.0 * kT
    hi = float(_all_reduce(np.array([rng[:, 1].max()]), "max", group, device)[0]) + 40.0 * kT
    flo, fhi, side, rf = -float(n_electrons), 0.0, 0, False
    x = hi
    it = 0
    while it < MAX_HALVINGS and hi - lo > tol:
        t = _ordered_sum(gather_chunks(parts, n_chunks_total, "count", x, kT, group, device))
        fx = t - n_electrons
        if fx == 0.0:                  # x is a root to rounding: the bracket closes on it
            lo = hi = x
            it += 1
            break
        if fx < 0:
            lo, flo = x, fx
            if rf and side == -1:
                fhi = 0.5 * fhi
            side = -1
        else:
            hi, fhi = x, fx
            if rf and side == 1:
                flo = 0.5 * flo
            side = 1
        it += 1
        x, rf = 0.5 * (lo + hi), False
        if not (hi - lo > SECANT_KT * kT):
            sx = (lo * fhi - hi * flo) / (fhi - flo)
            if lo < sx < hi:
                x, rf = sx, True
    return 0.5 * (lo + hi), it


def totals(parts, n_chunks_total: int, mu: float, kT: float, rho: bool = True, group=None, device="cpu") -> dict:
    """Electron count, band energy from the levels (2 sum f eps w) and, after mka_sweep_density at mu on
    every process, the band energy of Eq. EQ-ENE (2 sum rho_ij H_ji), each a chunk-ordered sum."""
    out = {}
    keys = ["count", "e_levels"] + (["e_rho"] if rho else [])
    for k in keys:
        out[k] = _ordered_sum(gather_chunks(parts, n_chunks_total, k, mu, kT, group, device, levels=True, rho=rho))
    return {"n_electrons": out["count"], "e_band_levels": out["e_levels"], "e_band": out.get("e_rho")}
