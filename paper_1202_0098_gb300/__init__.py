"""GB300-native multiple Arnoldi method (Hoshi et al., arXiv:1202.0098).

The compute path is the in-tree CUDA library ``_build/libmka.so`` (C ABI in
``include/mka.h``); ``mka`` is its ctypes binding with the same entry-point
names, and ``warm_start`` trains the learned CG start with the library's own
kernels.

A direct solve of some columns, then mu, rho and the band energy::

    import numpy as np, torch
    from paper_1202_0098_gb300 import build, mka
    from synth import SK_CARBON_LIKE, lattice_positions

    build.build()                                   # nvcc, sm_103a, in-tree
    pos, box = lattice_positions("diamond", 3.567, 4, 0.05, 0.0, 1)
    sys_ = mka.mka_build_system(pos, box, SK_CARBON_LIKE, "fp64", cluster_radius=6.0)
    atoms = np.arange(64, dtype=np.int64)           # 4 columns (s, px, py, pz) per atom
    res = mka.mka_solve_columns(sys_, atoms, mka.solve_params(15, 15, keep_vectors=True))
    mu = mka.mka_find_mu(res, 4.0 * len(atoms), 0.1)
    rho = torch.empty(mka.mka_result_info(res)["n_blocks"] * 16, dtype=torch.float64, device="cuda")
    e_band, n_elec = mka.mka_density_energy(sys_, res, mu, 0.1, rho.data_ptr())
    mka.mka_result_destroy(res)
    mka.mka_system_destroy(sys_)

Batches of thousands of atoms go through a plan (one graph-captured launch
sequence per batch; ``mka.mka_autotune`` picks its launch shape)::

    prm = mka.solve_params(15, 15, arith="mixed", cg_tol=1e-7, keep_vectors=True)
    plan = mka.mka_plan_create(sys_, 65536, prm, mka.mka_autotune(sys_, prm, atoms, 4.0 * len(atoms), 0.1))
    mka.mka_plan_run(plan, batch, 4.0 * len(batch), 0.1, rho_ptr)
    mu, e_band, n_elec = mka.mka_plan_scalars(plan)
"""
from . import build, mka

__all__ = ["build", "mka"]
