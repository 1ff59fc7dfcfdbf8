"""Thin ctypes binding of libmka (include/mka.h), function for function.

Argument marshalling only: every step of the method runs in the library's
CUDA kernels. Device buffers are passed as raw pointers (for example
``torch.Tensor.data_ptr()`` of a CUDA tensor), streams as ``cudaStream_t``
integers (``torch.cuda.current_stream().cuda_stream``). There is no CPU
fallback: if the shared library is not built, importing this module's
functions raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MKA_OK, MKA_ERR_INVALID_ARG, MKA_ERR_NOT_SPD, MKA_ERR_NO_CONVERGENCE, MKA_ERR_BREAKDOWN = 0, 1, 2, 3, 4
MKA_ERR_OOM, MKA_ERR_CUDA, MKA_ERR_TIMEOUT, MKA_ERR_CLUSTER_TOO_LARGE = 5, 6, 7, 8
MKA_FP64, MKA_MIXED_FP32, MKA_MIXED_BF16 = 0, 1, 2
STORAGE = {"fp64": MKA_FP64, "fp32": MKA_MIXED_FP32, "bf16": MKA_MIXED_BF16}
MKA_MAX_CLUSTER_ATOMS = 512
MKA_MAX_NU = 320
MKA_STATIC_SCRATCH_BYTES = 64 << 20

# Every symbol include/mka.h declares (checked by the tests).
EXPORTED = [
    "mka_build_system", "mka_build_system_bsr", "mka_system_info", "mka_system_copy_bsr", "mka_cluster_sizes",
    "mka_system_destroy", "mka_spmv", "mka_solve_columns", "mka_solve_columns_static", "mka_result_info", "mka_result_copy_levels",
    "mka_result_device_levels", "mka_result_destroy", "mka_find_mu", "mka_density_energy", "mka_greens",
    "mka_plan_create", "mka_plan_run", "mka_plan_scalars", "mka_plan_kernel_ms", "mka_plan_result", "mka_plan_info", "mka_plan_destroy",
    "mka_autotune", "mka_mlp_num_params", "mka_mlp_create", "mka_mlp_destroy", "mka_mlp_set_params",
    "mka_mlp_get_params", "mka_mlp_forward", "mka_mlp_gradients", "mka_mlp_train_step", "mka_warm_start_features",
    "mka_cg_patch_targets", "mka_system_set_warm_start", "mka_result_copy_warm_start",
    "mka_sweep_create", "mka_sweep_info", "mka_plan_run_sweep", "mka_sweep_status", "mka_sweep_level_range",
    "mka_sweep_find_mu", "mka_sweep_density", "mka_sweep_forces", "mka_sweep_chunk_sums", "mka_sweep_device_levels",
    "mka_sweep_destroy", "mka_forces", "mka_dos", "mka_system_shift_onsite", "mka_autotune_batch",
    "mka_kernel_launches", "mka_last_error", "mka_status_string",
]


class MkaError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: status {status}: {message}")
        self.status = status


class mka_sk_params(C.Structure):
    _fields_ = [("Es", C.c_double), ("Ep", C.c_double), ("V", C.c_double * 4), ("Sv", C.c_double * 4),
                ("d0", C.c_double), ("rc", C.c_double)]


class mka_tuning(C.Structure):
    _fields_ = [("threads", C.c_int), ("ctas_per_sm", C.c_int), ("order_by_size", C.c_int)]


class mka_solve_params(C.Structure):
    _fields_ = [("p", C.c_int), ("q", C.c_int), ("arith", C.c_int), ("use_warm_start", C.c_int),
                ("cg_tol", C.c_double), ("cg_maxit", C.c_int), ("keep_vectors", C.c_int), ("keep_s", C.c_int),
                ("s_start", C.c_void_p), ("subspace", C.c_int)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None) -> C.CDLL:
    """Load libmka (built in-tree by ``__graft_entry__.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libmka is not built ({path}); run __graft_entry__.build() first")
    lib = C.CDLL(path)
    P, I64, I32, D = C.c_void_p, C.c_int64, C.c_int, C.c_double
    sig = {
        "mka_build_system": [P, I64, P, P, I32, D, P, P],
        "mka_build_system_bsr": [P, I64, P, P, P, I64, P, P, I32, D, P, P],
        "mka_system_info": [P, P, P, P, P],
        "mka_system_copy_bsr": [P, P, P, P, P],
        "mka_cluster_sizes": [P, P, I64, P],
        "mka_spmv": [P, I32, I32, P, P, I32, P],
        "mka_solve_columns": [P, P, I64, P, P, P],
        "mka_solve_columns_static": [P, P, I64, I32, I32, D, I32, I32, P, P, P, P, P, P],
        "mka_result_info": [P, P, P, P],
        "mka_result_copy_levels": [P, P, P, P, P, P],
        "mka_result_device_levels": [P, P, P],
        "mka_find_mu": [P, D, D, D, P],
        "mka_density_energy": [P, P, D, D, P, P, P],
        "mka_greens": [P, P, D, D, P],
        "mka_plan_create": [P, I64, P, P, P, P],
        "mka_plan_run": [P, P, I64, D, D, P],
        "mka_plan_scalars": [P, P, P, P],
        "mka_plan_result": [P, P],
        "mka_plan_kernel_ms": [P, P, P],
        "mka_plan_info": [P, P, P, P],
        "mka_autotune": [P, P, P, I64, D, D, C.c_char_p, P, P],
        "mka_mlp_create": [C.c_uint64, P],
        "mka_mlp_set_params": [P, P],
        "mka_mlp_get_params": [P, P, I32],
        "mka_mlp_forward": [P, P, P, I64, P],
        "mka_mlp_gradients": [P, P, P, I64, P, P, P],
        "mka_mlp_train_step": [P, P, P, I64, C.c_float, P, P],
        "mka_warm_start_features": [P, P, I64, P, P, P],
        "mka_cg_patch_targets": [P, P, I64, I32, D, P, P, P, P],
        "mka_system_set_warm_start": [P, P],
        "mka_result_copy_warm_start": [P, P],
        "mka_sweep_create": [P, I64, I64, I32, D, D, I32, I64, I32, P, P],
        "mka_sweep_forces": [P, P, D, D, P, P],
        "mka_forces": [P, P, D, D, P, P],
        "mka_dos": [P, P, I64, P, I32, D, P, P],
        "mka_system_shift_onsite": [P, P, P],
        "mka_autotune_batch": [P, P, P, P, I32, I64, D, D, C.c_char_p, P, P],
        "mka_sweep_info": [P, P, P, P, P],
        "mka_plan_run_sweep": [P, P, P, I64],
        "mka_sweep_status": [P, P, P],
        "mka_sweep_level_range": [P, P, P],
        "mka_sweep_find_mu": [P, D, D, D, P],
        "mka_sweep_density": [P, P, D, D, P, P],
        "mka_sweep_chunk_sums": [P, D, D, P, P, P],
        "mka_sweep_device_levels": [P, P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.mka_system_destroy.argtypes = [P]
    lib.mka_system_destroy.restype = None
    lib.mka_mlp_num_params.argtypes = []
    lib.mka_mlp_num_params.restype = C.c_int64
    lib.mka_mlp_destroy.argtypes = [P]
    lib.mka_mlp_destroy.restype = None
    lib.mka_plan_destroy.argtypes = [P]
    lib.mka_plan_destroy.restype = None
    lib.mka_sweep_destroy.argtypes = [P]
    lib.mka_sweep_destroy.restype = None
    lib.mka_result_destroy.argtypes = [P]
    lib.mka_result_destroy.restype = None
    lib.mka_kernel_launches.argtypes = []
    lib.mka_kernel_launches.restype = C.c_int64
    lib.mka_last_error.argtypes = []
    lib.mka_last_error.restype = C.c_char_p
    lib.mka_status_string.argtypes = [C.c_int]
    lib.mka_status_string.restype = C.c_char_p
    _lib = lib
    return lib


def _check(st: int, where: str):
    if st != MKA_OK:
        msg = load().mka_last_error().decode(errors="replace")
        raise MkaError(st, where, msg)


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def sk_struct(sk) -> mka_sk_params:
    """From an object with Es, Ep, V, Sv, d0, rc (e.g. synth.SKParams)."""
    s = mka_sk_params()
    s.Es, s.Ep, s.d0, s.rc = sk.Es, sk.Ep, sk.d0, sk.rc
    for i in range(4):
        s.V[i] = sk.V[i]
        s.Sv[i] = sk.Sv[i]
    return s


# ---- entry points, same names as the C ABI ------------------------------------------------

def mka_build_system(pos: np.ndarray, box: np.ndarray, sk, storage: str = "fp64", cluster_radius: float = 6.0,
                     stream: int = 0) -> C.c_void_p:
    lib = load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    box = np.ascontiguousarray(box, dtype=np.float64)
    out = C.c_void_p()
    skp = sk_struct(sk)
    _check(lib.mka_build_system(_ptr(pos), pos.shape[0], _ptr(box), C.byref(skp), STORAGE[storage],
                                float(cluster_radius), C.c_void_p(stream), C.byref(out)), "mka_build_system")
    return out


def mka_build_system_bsr(pos, box, row_ptr, col, valH, valS, storage="fp64", cluster_radius=6.0, stream=0):
    lib = load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    box = np.ascontiguousarray(box, dtype=np.float64)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    valH = np.ascontiguousarray(valH, dtype=np.float64)
    valS = np.ascontiguousarray(valS, dtype=np.float64)
    out = C.c_void_p()
    _check(lib.mka_build_system_bsr(_ptr(pos), pos.shape[0], _ptr(box), _ptr(row_ptr), _ptr(col), col.shape[0],
                                    _ptr(valH), _ptr(valS), STORAGE[storage], float(cluster_radius),
                                    C.c_void_p(stream), C.byref(out)), "mka_build_system_bsr")
    return out


def mka_system_info(sys) -> dict:
    n, nnzb, st, mrb = C.c_int64(), C.c_int64(), C.c_int(), C.c_int()
    _check(load().mka_system_info(sys, C.byref(n), C.byref(nnzb), C.byref(st), C.byref(mrb)), "mka_system_info")
    return {"n_atoms": n.value, "nnzb": nnzb.value, "storage": st.value, "max_row_blocks": mrb.value}


def mka_system_copy_bsr(sys, values: bool = True) -> dict:
    info = mka_system_info(sys)
    n, nnzb = info["n_atoms"], info["nnzb"]
    row_ptr = np.empty(n + 1, np.int32)
    col = np.empty(nnzb, np.int32)
    H = np.empty((nnzb, 4, 4)) if values else None
    S = np.empty((nnzb, 4, 4)) if values else None
    _check(load().mka_system_copy_bsr(sys, _ptr(row_ptr), _ptr(col), _ptr(H), _ptr(S)), "mka_system_copy_bsr")
    return {"row_ptr": row_ptr, "col": col, "H": H, "S": S}


def mka_cluster_sizes(sys, atoms: np.ndarray | None = None) -> np.ndarray:
    n = mka_system_info(sys)["n_atoms"] if atoms is None else len(atoms)
    a = None if atoms is None else np.ascontiguousarray(atoms, dtype=np.int64)
    out = np.empty(n, np.int32)
    _check(load().mka_cluster_sizes(sys, _ptr(a), n, _ptr(out)), "mka_cluster_sizes")
    return out


def mka_system_destroy(sys):
    if sys:
        load().mka_system_destroy(sys)


def mka_spmv(sys, which: int, x_dtype: int, x_ptr: int, y_ptr: int, k: int = 1, stream: int = 0):
    _check(load().mka_spmv(sys, which, x_dtype, C.c_void_p(x_ptr), C.c_void_p(y_ptr), k, C.c_void_p(stream)),
           "mka_spmv")


def solve_params(p: int, q: int, arith: str = "fp64", cg_tol: float = 1e-12, cg_maxit: int = 500,
                 keep_vectors: bool = True, use_warm_start: bool = False, subspace: str = "A", keep_s: bool = False,
                 s_start=None) -> mka_solve_params:
    prm = mka_solve_params()
    prm.subspace = {"A": 0, "B": 1}[subspace]
    prm.keep_s = int(keep_s)
    prm.s_start = s_start.value if isinstance(s_start, C.c_void_p) else s_start
    prm.p, prm.q = p, q
    prm.arith = MKA_FP64 if arith == "fp64" else MKA_MIXED_FP32
    prm.use_warm_start = int(use_warm_start)
    prm.cg_tol = cg_tol
    prm.cg_maxit = cg_maxit
    prm.keep_vectors = int(keep_vectors)
    return prm


def mka_solve_columns(sys, atoms: np.ndarray | None, prm: mka_solve_params, stream: int = 0) -> C.c_void_p:
    a = None if atoms is None else np.ascontiguousarray(atoms, dtype=np.int64)
    n = 0 if a is None else a.shape[0]
    out = C.c_void_p()
    _check(load().mka_solve_columns(sys, _ptr(a), n, C.byref(prm), C.c_void_p(stream), C.byref(out)),
           "mka_solve_columns")
    return out


def mka_solve_columns_static(sys, atoms: np.ndarray, p: int, q: int, cg_tol: float, cg_maxit: int,
                             max_cluster_atoms: int, eps_ptr: int, w_ptr: int, nu_eff_ptr: int, cg_iters_ptr: int,
                             status_ptr: int, stream: int = 0):
    """Allocation-free solve into caller device buffers (see include/mka.h)."""
    a = np.ascontiguousarray(atoms, dtype=np.int64)
    V = C.c_void_p
    _check(load().mka_solve_columns_static(sys, _ptr(a), a.shape[0], p, q, float(cg_tol), cg_maxit,
                                           max_cluster_atoms, V(eps_ptr), V(w_ptr), V(nu_eff_ptr), V(cg_iters_ptr),
                                           V(status_ptr), V(stream)), "mka_solve_columns_static")


def mka_result_info(res) -> dict:
    nc, nu, nb = C.c_int64(), C.c_int(), C.c_int64()
    _check(load().mka_result_info(res, C.byref(nc), C.byref(nu), C.byref(nb)), "mka_result_info")
    return {"n_cols": nc.value, "nu": nu.value, "n_blocks": nb.value}


def mka_result_copy_levels(res, check: bool = True) -> dict:
    info = mka_result_info(res)
    nc, nu = info["n_cols"], info["nu"]
    eps = np.empty((nc, nu))
    w = np.empty((nc, nu))
    nu_eff = np.empty(nc, np.int32)
    it = np.empty(nc, np.int32)
    status = np.empty(nc, np.int32)
    st = load().mka_result_copy_levels(res, _ptr(eps), _ptr(w), _ptr(nu_eff), _ptr(it), _ptr(status))
    if check:
        _check(st, "mka_result_copy_levels")
    return {"eps": eps, "w": w, "nu_eff": nu_eff, "cg_iters": it, "status": status, "aggregate": st}


def mka_result_device_levels(res) -> tuple[int, int]:
    e, w = C.c_void_p(), C.c_void_p()
    _check(load().mka_result_device_levels(res, C.byref(e), C.byref(w)), "mka_result_device_levels")
    return e.value, w.value


def mka_result_destroy(res):
    if res:
        load().mka_result_destroy(res)


def mka_find_mu(res, n_electrons: float, kT: float, tol: float = 1e-12) -> float:
    mu = C.c_double()
    _check(load().mka_find_mu(res, float(n_electrons), float(kT), float(tol), C.byref(mu)), "mka_find_mu")
    return mu.value


def mka_density_energy(sys, res, mu: float, kT: float, rho_ptr: int | None = None) -> tuple[float, float]:
    e, n = C.c_double(), C.c_double()
    _check(load().mka_density_energy(sys, res, float(mu), float(kT), C.c_void_p(rho_ptr) if rho_ptr else None,
                                     C.byref(e), C.byref(n)), "mka_density_energy")
    return e.value, n.value


def mka_greens(sys, res, z: complex, g_ptr: int):
    _check(load().mka_greens(sys, res, float(z.real), float(z.imag), C.c_void_p(g_ptr)), "mka_greens")


def mka_system_shift_onsite(sys, shift: np.ndarray, stream: int = 0):
    a = np.ascontiguousarray(shift, dtype=np.float64)
    _check(load().mka_system_shift_onsite(sys, _ptr(a), C.c_void_p(stream)), "mka_system_shift_onsite")


def mka_dos(eps_ptr: int, w_ptr: int, n_levels: int, energies, eta: float, stream: int = 0) -> np.ndarray:
    """Density of states at `energies` from levels and weights in device memory (see include/mka.h)."""
    e = np.ascontiguousarray(energies, dtype=np.float64)
    out = np.empty(e.shape[0])
    _check(load().mka_dos(C.c_void_p(eps_ptr), C.c_void_p(w_ptr), int(n_levels), _ptr(e), e.shape[0], float(eta),
                          C.c_void_p(stream), _ptr(out)), "mka_dos")
    return out


def tuning(threads: int = 256, ctas_per_sm: int = 0, order_by_size: bool = False) -> mka_tuning:
    t = mka_tuning()
    t.threads, t.ctas_per_sm, t.order_by_size = threads, ctas_per_sm, int(order_by_size)
    return t


def mka_plan_create(sys, max_atoms: int, prm: mka_solve_params, tune: mka_tuning | None = None,
                    stream: int = 0) -> C.c_void_p:
    out = C.c_void_p()
    _check(load().mka_plan_create(sys, int(max_atoms), C.byref(prm), C.byref(tune) if tune is not None else None,
                                  C.c_void_p(stream), C.byref(out)), "mka_plan_create")
    return out


def mka_plan_run(plan, atoms: np.ndarray, n_electrons: float, kT: float, rho_ptr: int | None = None):
    a = np.ascontiguousarray(atoms, dtype=np.int64)
    _check(load().mka_plan_run(plan, _ptr(a), a.shape[0], float(n_electrons), float(kT),
                               C.c_void_p(rho_ptr) if rho_ptr else None), "mka_plan_run")


def mka_plan_scalars(plan) -> tuple[float, float, float]:
    mu, e, n = C.c_double(), C.c_double(), C.c_double()
    _check(load().mka_plan_scalars(plan, C.byref(mu), C.byref(e), C.byref(n)), "mka_plan_scalars")
    return mu.value, e.value, n.value


def mka_plan_kernel_ms(plan) -> tuple[float, float]:
    """(per-atom kernel ms, batched reduced-problem kernel ms) of the last batch."""
    a, r = C.c_float(), C.c_float()
    _check(load().mka_plan_kernel_ms(plan, C.byref(a), C.byref(r)), "mka_plan_kernel_ms")
    return a.value, r.value


def mka_plan_result(plan) -> C.c_void_p:
    out = C.c_void_p()
    _check(load().mka_plan_result(plan, C.byref(out)), "mka_plan_result")
    return out


def mka_plan_info(plan) -> dict:
    t, g, c = mka_tuning(), C.c_int(), C.c_int()
    _check(load().mka_plan_info(plan, C.byref(t), C.byref(g), C.byref(c)), "mka_plan_info")
    return {"threads": t.threads, "ctas_per_sm": t.ctas_per_sm, "order_by_size": t.order_by_size, "grid": g.value,
            "ctas_per_sm_used": c.value}


def mka_plan_destroy(plan):
    if plan:
        load().mka_plan_destroy(plan)


def mka_autotune(sys, prm: mka_solve_params, sample: np.ndarray, n_electrons: float, kT: float,
                 cache_path: str | None = None, stream: int = 0) -> mka_tuning:
    a = np.ascontiguousarray(sample, dtype=np.int64)
    out = mka_tuning()
    _check(load().mka_autotune(sys, C.byref(prm), _ptr(a), a.shape[0], float(n_electrons), float(kT),
                               cache_path.encode() if cache_path else None, C.c_void_p(stream), C.byref(out)),
           "mka_autotune")
    return out


def mka_autotune_batch(sys, prm: mka_solve_params, tune: mka_tuning | None, candidates, first_atom: int,
                       electrons_per_atom: float, kT: float, cache_path: str | None = None, stream: int = 0) -> int:
    c = np.ascontiguousarray(candidates, dtype=np.int64)
    out = C.c_int64()
    _check(load().mka_autotune_batch(sys, C.byref(prm), C.byref(tune) if tune is not None else None, _ptr(c),
                                     c.shape[0], int(first_atom), float(electrons_per_atom), float(kT),
                                     cache_path.encode() if cache_path else None, C.c_void_p(stream), C.byref(out)),
           "mka_autotune_batch")
    return out.value


# ---- whole-system sweep ------------------------------------------------------------------

def mka_sweep_create(sys, atom_begin: int, atom_end: int, nu: int, win_lo: float, win_hi: float, kp: int,
                     chunk_atoms: int = 4096, stream: int = 0, with_forces: bool = False) -> C.c_void_p:
    out = C.c_void_p()
    _check(load().mka_sweep_create(sys, int(atom_begin), int(atom_end), int(nu), float(win_lo), float(win_hi), int(kp),
                                   int(chunk_atoms), int(with_forces), C.c_void_p(stream), C.byref(out)),
           "mka_sweep_create")
    return out


def mka_sweep_forces(sw, plan, mu: float, kT: float, forces_ptr: int) -> int:
    n = C.c_int64()
    _check(load().mka_sweep_forces(sw, plan, float(mu), float(kT), C.c_void_p(forces_ptr), C.byref(n)),
           "mka_sweep_forces")
    return n.value


def mka_forces(sys, res, mu: float, kT: float, pi_ptr: int | None = None, forces_ptr: int | None = None):
    _check(load().mka_forces(sys, res, float(mu), float(kT), C.c_void_p(pi_ptr) if pi_ptr else None,
                             C.c_void_p(forces_ptr) if forces_ptr else None), "mka_forces")


def mka_sweep_info(sw) -> dict:
    c0, nc, nb, by = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
    _check(load().mka_sweep_info(sw, C.byref(c0), C.byref(nc), C.byref(nb), C.byref(by)), "mka_sweep_info")
    return {"chunk0": c0.value, "n_chunks": nc.value, "n_blocks": nb.value, "bytes": by.value}


def mka_plan_run_sweep(plan, sw, atoms: np.ndarray):
    a = np.ascontiguousarray(atoms, dtype=np.int64)
    _check(load().mka_plan_run_sweep(plan, sw, _ptr(a), a.shape[0]), "mka_plan_run_sweep")


def mka_sweep_status(sw) -> tuple[int, int]:
    st, ov = C.c_int64(), C.c_int64()
    _check(load().mka_sweep_status(sw, C.byref(st), C.byref(ov)), "mka_sweep_status")
    return st.value, ov.value


def mka_sweep_level_range(sw) -> tuple[float, float]:
    lo, hi = C.c_double(), C.c_double()
    _check(load().mka_sweep_level_range(sw, C.byref(lo), C.byref(hi)), "mka_sweep_level_range")
    return lo.value, hi.value


def mka_sweep_find_mu(sw, n_electrons: float, kT: float, tol: float = 1e-12) -> float:
    mu = C.c_double()
    _check(load().mka_sweep_find_mu(sw, float(n_electrons), float(kT), float(tol), C.byref(mu)), "mka_sweep_find_mu")
    return mu.value


def mka_sweep_density(sw, plan, mu: float, kT: float, rho_ptr: int) -> int:
    n = C.c_int64()
    _check(load().mka_sweep_density(sw, plan, float(mu), float(kT), C.c_void_p(rho_ptr), C.byref(n)),
           "mka_sweep_density")
    return n.value


def mka_sweep_chunk_sums(sw, mu: float, kT: float, levels: bool = True, rho: bool = False) -> dict:
    nc = mka_sweep_info(sw)["n_chunks"]
    cnt = np.empty(nc)
    el = np.empty(nc) if levels else None
    er = np.empty(nc) if rho else None
    _check(load().mka_sweep_chunk_sums(sw, float(mu), float(kT), _ptr(cnt), _ptr(el), _ptr(er)), "mka_sweep_chunk_sums")
    return {"count": cnt, "e_levels": el, "e_rho": er}


def mka_sweep_device_levels(sw) -> tuple[int, int]:
    e, w = C.c_void_p(), C.c_void_p()
    _check(load().mka_sweep_device_levels(sw, C.byref(e), C.byref(w)), "mka_sweep_device_levels")
    return e.value, w.value


def mka_sweep_destroy(sw):
    if sw:
        load().mka_sweep_destroy(sw)


# ---- learned warm start ------------------------------------------------------------------

def mka_mlp_num_params() -> int:
    return int(load().mka_mlp_num_params())


def mka_mlp_create(seed: int = 0) -> C.c_void_p:
    out = C.c_void_p()
    _check(load().mka_mlp_create(C.c_uint64(seed), C.byref(out)), "mka_mlp_create")
    return out


def mka_mlp_destroy(net):
    if net:
        load().mka_mlp_destroy(net)


def mka_mlp_set_params(net, params: np.ndarray):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(load().mka_mlp_set_params(net, _ptr(p)), "mka_mlp_set_params")


def mka_mlp_get_params(net, bf16_rounded: bool = False) -> np.ndarray:
    p = np.empty(mka_mlp_num_params(), np.float32)
    _check(load().mka_mlp_get_params(net, _ptr(p), int(bf16_rounded)), "mka_mlp_get_params")
    return p


def mka_mlp_forward(net, x_ptr: int, y_ptr: int, B: int, stream: int = 0):
    _check(load().mka_mlp_forward(net, C.c_void_p(x_ptr), C.c_void_p(y_ptr), B, C.c_void_p(stream)), "mka_mlp_forward")


def mka_mlp_gradients(net, x_ptr: int, t_ptr: int, B: int, grad_ptr: int | None, loss_ptr: int | None,
                      stream: int = 0):
    V = C.c_void_p
    _check(load().mka_mlp_gradients(net, V(x_ptr), V(t_ptr), B, V(grad_ptr) if grad_ptr else None,
                                    V(loss_ptr) if loss_ptr else None, V(stream)), "mka_mlp_gradients")


def mka_mlp_train_step(net, x_ptr: int, t_ptr: int, B: int, lr: float, loss_ptr: int | None = None,
                       stream: int = 0):
    V = C.c_void_p
    _check(load().mka_mlp_train_step(net, V(x_ptr), V(t_ptr), B, C.c_float(lr), V(loss_ptr) if loss_ptr else None,
                                     V(stream)), "mka_mlp_train_step")


def mka_warm_start_features(sys, atoms: np.ndarray, x_ptr: int, patch_ptr: int, stream: int = 0):
    a = np.ascontiguousarray(atoms, dtype=np.int64)
    _check(load().mka_warm_start_features(sys, _ptr(a), a.shape[0], C.c_void_p(x_ptr), C.c_void_p(patch_ptr),
                                          C.c_void_p(stream)), "mka_warm_start_features")


def mka_cg_patch_targets(sys, atoms: np.ndarray, arith: str, cg_tol: float, patch_ptr: int, y_ptr: int,
                         iters_ptr: int | None = None, stream: int = 0):
    a = np.ascontiguousarray(atoms, dtype=np.int64)
    V = C.c_void_p
    _check(load().mka_cg_patch_targets(sys, _ptr(a), a.shape[0], MKA_FP64 if arith == "fp64" else MKA_MIXED_FP32,
                                       float(cg_tol), V(patch_ptr), V(y_ptr), V(iters_ptr) if iters_ptr else None,
                                       V(stream)), "mka_cg_patch_targets")


def mka_system_set_warm_start(sys, net):
    _check(load().mka_system_set_warm_start(sys, net), "mka_system_set_warm_start")


def mka_result_copy_warm_start(res) -> np.ndarray:
    n = mka_result_info(res)["n_cols"]
    out = np.empty(n, np.int32)
    _check(load().mka_result_copy_warm_start(res, _ptr(out)), "mka_result_copy_warm_start")
    return out


def mka_kernel_launches() -> int:
    return int(load().mka_kernel_launches())


def mka_last_error() -> str:
    return load().mka_last_error().decode(errors="replace")


def mka_status_string(st: int) -> str:
    return load().mka_status_string(st).decode(errors="replace")
