"""Oracle: many atoms at once in a process pool started with 'spawn'.

TEST INFRASTRUCTURE ONLY (see the package docstring). 'spawn' keeps the pool
safe beside a process that already holds a CUDA context.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

from . import system as osys


def _work(args):
    pos, box, skp, R, atoms, p, q, storage, cg_tol = args[:9]
    mode = args[9] if len(args) > 9 else "A"
    return [osys.solve_atom(pos, box, skp, R, int(a), p, q, storage, cg_tol, mode=mode) for a in atoms]


def solve_atoms_parallel(pos, box, skp, R, atoms, p, q, storage="fp64", cg_tol=1e-13, workers=None, mode="A"):
    atoms = list(np.asarray(atoms, dtype=np.int64))
    workers = workers or min(16, os.cpu_count() or 1)
    if len(atoms) <= 4 or workers == 1:
        return _work((pos, box, skp, R, atoms, p, q, storage, cg_tol, mode))
    chunks = [atoms[i::workers] for i in range(workers)]
    chunks = [c for c in chunks if c]
    ctx = mp.get_context("spawn")
    # one BLAS thread per worker process (the workers already fill the cores); the children inherit this
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        with ctx.Pool(len(chunks)) as pool:
            parts = pool.map(_work, [(pos, box, skp, R, c, p, q, storage, cg_tol, mode) for c in chunks])
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    by_atom = {r.atom: r for part in parts for r in part}
    return [by_atom[int(a)] for a in atoms]
