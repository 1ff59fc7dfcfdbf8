"""Benchmark: density-matrix columns per second of the multiple Arnoldi method on GB300.

Workload: the 10,077,696-atom diamond-lattice system (108^3 cubic cells,
a = 3.567 A, sigma = 0.1 A, sp basis, M = 40,310,784 columns), cluster radius
6 A, p = q = 15, kT = 0.1 eV, BF16-stored H and S, mixed form with the learned
CG start. The timed region is the whole work flow of Eq. EQ-WORK-FLOW over the
whole system: K steps, each one slice of N/K atoms solved by graph-replayed
plan batches (cluster extraction, inner CG, multiple Krylov basis, projection,
reduced eigensolve) whose levels and rho pieces a sweep keeps in HBM; after the
last slice, one mu by bisection over all 4.03e7 columns, rho on the whole
pattern and the band energy at that mu. `value` = 4 N / (timed seconds).

Under torchrun each rank sweeps one chunk-aligned range of the atoms; mu and
the energies come from one all-reduce of chunk sums per bisection halving
(paper_1202_0098_gb300.distributed), bit-identical to one process.

Also reported: K1 (the global BSR SpMV) in GB/s against the measured HBM peak,
per-batch rates of the plain mixed form and of the FP64 form, the per-atom and
reduced kernels' rooflines. Prints one JSON line (rank 0). `--impl reference`
times the FP64 CPU oracle on the host cores instead (a bounded sample of the
same workload per step).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import WORKLOADS, workload_positions  # noqa: E402

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FMA units per SM per clock on sm_103a: 128 FP32, 2 FP64 (nominal FP64 1.25 TFLOP/s per GPU).
FMA_PER_SM = {"fp32": 128, "fp64": 2}


def alu_peak_tflops(pipe, sms, mhz):
    """Peak of a plain-ALU pipe: SMs x FMA units x 2 flops x the SM clock seen under load."""
    return sms * FMA_PER_SM[pipe] * 2 * mhz * 1e6 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="diamond10m")
    ap.add_argument("--form", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--storage", default=None, choices=[None, "fp64", "fp32", "bf16"])
    ap.add_argument("--batch", type=int, default=0, help="atoms per step (0: per form default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shape instead of the autotuner's")
    ap.add_argument("--no-learned", action="store_true", help="mixed form without the learned CG start")
    ap.add_argument("--no-spmv", action="store_true", help="skip the K1 SpMV leg")
    ap.add_argument("--window", type=float, default=1.0,
                    help="half-width (eV) of the sweep's mu window beyond 40 kT around the sampled mu")
    ap.add_argument("--chunk-atoms", type=int, default=4096)
    ap.add_argument("--full-fp64", action="store_true",
                    help="after the headline, the FP64 form over the whole system: mu, E and rho differences")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---- multi-rank host logic (weak scaling: each rank its own atoms, no collective on the data path) ----

def shard_atoms(rank, i, n_steps, B, N):
    """Atoms of step i on `rank`: consecutive blocks of B atoms, rank-major, wrapping around the system."""
    start = ((rank * n_steps + i) * B) % N
    return np.arange(start, start + B, dtype=np.int64) % N


def max_over_ranks(x, device="cpu"):
    """The largest of the ranks' values of x (x itself on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def job_throughput(columns_per_rank_step, steps, world, max_ms):
    """Whole-job columns/s: the columns all ranks processed over the slowest rank's time."""
    return columns_per_rank_step * steps * world / (max_ms / 1e3)


def workload_desc(name, w, N):
    return f"{name}: {N} atoms, {4 * N} columns, R={w.R} A, p=q={w.p}, kT={w.kT} eV"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def local_flops(tree, pos, row_ptr, col, atoms, R):
    """Algorithmic FLOPs per column inputs: cluster orbitals m_c and local blocks nnzb_c per atom."""
    m_c, nnz_c = np.empty(len(atoms)), np.empty(len(atoms))
    mask = np.zeros(pos.shape[0], dtype=bool)
    for t, a in enumerate(atoms):
        cl = np.array(tree.query_ball_point(pos[a], R), dtype=np.int64)
        mask[cl] = True
        starts, ends = row_ptr[cl], row_ptr[cl + 1]
        idx = np.concatenate([np.arange(s, e) for s, e in zip(starts, ends)])
        nnz_c[t] = mask[col[idx]].sum()
        m_c[t] = 4 * len(cl)
        mask[cl] = False
    return m_c, nnz_c


def reduced_flops(nu):
    """FLOPs of one column's reduced solve: Cholesky nu^3/3, congruence nu^3 (both triangles of the symmetric
    products), tridiagonalisation 4 nu^3/3 (lower-triangle update), Q's reflectors applied to the
    eigenvectors 2 nu^3, L^-T nu^3; QL eigenvalues, inverse iteration and outputs about 47 nu^2."""
    return 17.0 / 3.0 * nu ** 3 + 47.0 * nu ** 2


def column_flops(m, nnz, nu, cg_it, n_pattern_rows):
    """Algorithmic FLOPs of one column, counted as plain arithmetic: the products of the CG and
    the basis, CG vector work, one Gram-Schmidt pass per vector (coefficients and update), norms,
    the projection, the reduced solve and the rows V_j, (S V)_j of the outputs."""
    spmv = 2.0 * 16.0 * nnz * (cg_it + 2 * nu)          # CG S-products + nu S- and nu H-products
    cg_vec = 10.0 * m * cg_it                            # two dots, three axpys per CG step
    gs = 2.0 * m * nu * (nu - 1)                          # one pass of dots + updates per new vector
    norms = 4.0 * m * nu                                  # S-norm and scaling per vector
    proj = 4.0 * m * nu * nu                              # U^T K and U^T (S U)
    red = reduced_flops(nu)                               # the reduced generalized eigensolve
    out = 4.0 * nu * nu                                   # V_j and (S V)_j
    return spmv + cg_vec + gs + norms + proj + red + out


def oracle_pool(mp, cores):
    """A spawn pool of `cores` oracle processes, each with one BLAS thread (the children inherit the
    environment), so the host runs one thread per core."""
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    return mp.get_context("spawn").Pool(cores)


def run_reference(args, rank, world):
    """The oracle on the host cores, a bounded sample of the same workload per step."""
    import multiprocessing as mp
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    pos, box = workload_positions(w)
    cores = os.cpu_count() or 1
    per_step = max(cores, 16)
    from oracle.parallel import _work
    rng = np.random.default_rng(0)
    times = []
    with oracle_pool(mp, cores) as pool:
        for it in range(args.warmup + args.steps):
            atoms = np.sort(rng.choice(pos.shape[0], per_step, replace=False))
            chunks = [atoms[i::cores] for i in range(cores)]
            t0 = time.perf_counter()
            pool.map(_work, [(pos, box, w.sk, w.R, c, w.p, w.q, "fp64", 1e-13) for c in chunks if len(c)])
            if it >= args.warmup:
                times.append(time.perf_counter() - t0)
    cols = 4 * per_step
    val = cols * len(times) / sum(times)
    line = {"impl": "reference", "metric": "density-matrix columns/s", "value": val, "unit": "columns/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(args.workload, w, pos.shape[0]),
                       "form": "FP64 oracle on FP64 values, host cores", "atoms_per_step": per_step,
                       "sample": f"{per_step} random atoms per step"},
            "cpu_baseline": {"value": val, "unit": "columns/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} random atoms ({cols} columns) of {args.workload} per step"},
            "e2e": {"value": val, "unit": "columns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(w, pos, box, budget_s=20.0):
    """The oracle as it stands, timed on the host cores over a bounded random sample of atoms."""
    import multiprocessing as mp
    from oracle.parallel import _work
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(1)
    with oracle_pool(mp, cores) as pool:
        pool.map(_work, [(pos, box, w.sk, w.R, [0], 2, 1, "fp64", 1e-13)] * cores)   # warm the workers
        n_at = cores
        atoms = np.sort(rng.choice(pos.shape[0], n_at, replace=False))
        t0 = time.perf_counter()
        pool.map(_work, [(pos, box, w.sk, w.R, atoms[i::cores], w.p, w.q, "fp64", 1e-13) for i in range(cores)])
        dt = time.perf_counter() - t0
        n_more = int(max(0, budget_s / max(dt, 1e-3) - 1) * n_at)
        if n_more > 0:
            extra = np.sort(rng.choice(pos.shape[0], n_more, replace=False))
            t1 = time.perf_counter()
            pool.map(_work, [(pos, box, w.sk, w.R, extra[i::cores], w.p, w.q, "fp64", 1e-13)
                             for i in range(cores) if len(extra[i::cores])])
            dt += time.perf_counter() - t1
            n_at += n_more
        # config 1 in full: every column of the 512-atom diamond system, the same p, q, R and CG tolerance
        from synth import WORKLOADS, workload_positions
        w1 = WORKLOADS["diamond512"]
        pos1, box1 = workload_positions(w1)
        a1 = np.arange(pos1.shape[0])
        t0 = time.perf_counter()
        pool.map(_work, [(pos1, box1, w1.sk, w1.R, a1[i::cores], w1.p, w1.q, "fp64", 1e-13) for i in range(cores)])
        dt_full = time.perf_counter() - t0
    with oracle_pool(mp, 1) as pool:                  # one core: one process, one BLAS thread
        pool.map(_work, [(pos, box, w.sk, w.R, [0], 2, 1, "fp64", 1e-13)])
        one = np.sort(rng.choice(pos.shape[0], 2, replace=False))
        t0 = time.perf_counter()
        pool.map(_work, [(pos, box, w.sk, w.R, one, w.p, w.q, "fp64", 1e-13)])
        dt1 = time.perf_counter() - t0
    return {"value": 4 * n_at / dt, "unit": "columns/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_at} random atoms ({4 * n_at} columns) of {w.name}, FP64 numpy oracle, "
                      f"one spawn process per core, one BLAS thread each",
            "single_core": {"value": 4 * len(one) / dt1, "unit": "columns/s", "cores": 1,
                            "sample": f"{len(one)} random atoms ({4 * len(one)} columns), one process, one BLAS thread"},
            "config1_full": {"value": 4 * len(a1) / dt_full, "unit": "columns/s", "cores": cores,
                             "seconds": dt_full, "sample": f"all {4 * len(a1)} columns of {w1.name}"},
            "cpu": cpu_model()}


def cpu_model():
    """The host CPU as /proc/cpuinfo names it (x86: model name; Arm: implementer and part)."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return platform.machine()
    names = [l.split(":", 1)[1].strip() for l in info if l.lower().startswith("model name")]
    if names:
        return f"{names[0]} x {len(names)}"
    parts = [l.split(":", 1)[1].strip() for l in info if l.startswith("CPU part")]
    impl = [l.split(":", 1)[1].strip() for l in info if l.startswith("CPU implementer")]
    return f"{platform.machine()} implementer {impl[0] if impl else '?'} part {parts[0] if parts else '?'} x {len(parts)}"


def flops_split(m, nnz, nu, cg_it, n_pattern_rows):
    """Algorithmic (vector work, reduced solve) FLOPs of one column."""
    total = column_flops(m, nnz, nu, cg_it, n_pattern_rows)
    red = reduced_flops(nu)
    return total - red, red


def alu_roofline(flops_per_col, n_cols, kernel_s, pipe, kernel, what, sms, mhz):
    """ALU bound of one kernel: its algorithmic FLOPs per launch over its event time, against the
    peak of the pipe that does them (derived from unit counts and the clock under load)."""
    peak = alu_peak_tflops(pipe, sms, mhz)
    achieved = flops_per_col * n_cols / kernel_s / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": kernel,
            "peak_source": (f"derived: {sms} SMs x {mhz:.0f} MHz (median under load) x 2 x {FMA_PER_SM[pipe]} "
                            f"{pipe.upper()} FMA/clk/SM; {what}"),
            "flops_per_column": flops_per_col, "kernel_ms": kernel_s * 1e3}


def captured_traffic(kernel, units):
    """DRAM bytes of one launch of `kernel` over `units` atoms or columns, scaled from the profiler
    capture recorded in profiles/traffic.json, or None when the kernel's source has changed since."""
    import hashlib
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", "traffic.json")
    try:
        rec = json.load(open(path))[kernel]
    except (OSError, KeyError, ValueError):
        return None
    root = os.path.dirname(path)[:-len("profiles")]
    for src, digest in rec["sources"].items():
        try:
            if hashlib.sha256(open(os.path.join(root, src), "rb").read()).hexdigest() != digest:
                return None
        except OSError:
            return None
    return rec["bytes_per_unit"] * units


def train_warm_start(mka, torch, seed=100):
    """The learned CG start, trained with the library's kernels on 2e5 inner-CG solutions (50,000 atoms x 4
    columns) of fresh seeds of the fcc (vacancies, sigma 0.08) and amorphous-like diamond (sigma 0.15) generators."""
    from paper_1202_0098_gb300 import warm_start
    from synth import SK_FCC_METAL, SK_CARBON_LIKE, lattice_positions
    Xs, Ys = [], []
    t0 = time.perf_counter()
    gens = [("fcc", 4.0, 20, 0.08, 0.05, SK_FCC_METAL, 7.0), ("fcc", 4.0, 20, 0.08, 0.05, SK_FCC_METAL, 7.0),
            ("diamond", 3.567, 16, 0.15, 0.0, SK_CARBON_LIKE, 7.0), ("diamond", 3.567, 16, 0.15, 0.0, SK_CARBON_LIKE, 7.0)]
    for k, (lat, a, nc, sig, vac, skp, R) in enumerate(gens):
        pos, box = lattice_positions(lat, a, nc, sig, vac, seed + k)
        s = mka.mka_build_system(pos, box, skp, "bf16", cluster_radius=R)
        atoms = np.sort(np.random.default_rng(seed + k).choice(pos.shape[0], 12500, replace=False)).astype(np.int64)
        X, Y, _ = warm_start.collect(s, atoms, "fp64", 1e-12)
        Xs.append(X)
        Ys.append(Y)
        mka.mka_system_destroy(s)
    X, Y = torch.cat(Xs), torch.cat(Ys)
    net = mka.mka_mlp_create(seed)
    mse0 = warm_start.mse(net, X, Y)
    hist = warm_start.train(net, X, Y, epochs=20, batch=1024, lr=1e-3, seed=seed)
    info = {"samples": int(X.shape[0]), "generators": "fcc (config-2) and diamond sigma 0.15 (config-3), seeds "
            f"{seed}-{seed + 3}", "targets": "inner CG, FP64 form, tolerance 1e-12", "epochs": 20, "batch": 1024,
            "mse_init": mse0, "mse_final": hist[-1], "train_s": time.perf_counter() - t0}
    del X, Y, Xs, Ys
    return net, info


def learned_eval(mka, torch, net, n_atoms=8192, seed=4):
    """The learned start on a fresh seed of the 10^6-atom amorphous-like generator (50^3 diamond cells,
    sigma 0.15, R = 7 A, p = q = 20, BF16 values, mixed form): CG iterations with and without it, the fallback
    rate, and the change of rho and of the band energy at the plain solve's mu."""
    from synth import SK_CARBON_LIKE, lattice_positions
    pos, box = lattice_positions("diamond", 3.567, 50, 0.15, 0.0, seed)
    s = mka.mka_build_system(pos, box, SK_CARBON_LIKE, "bf16", cluster_radius=7.0)
    mka.mka_system_set_warm_start(s, net)
    atoms = np.sort(np.random.default_rng(seed).choice(pos.shape[0], n_atoms, replace=False)).astype(np.int64)
    out = {}
    for learned in (False, True):
        prm = mka.solve_params(20, 20, arith="mixed", cg_tol=1e-7, keep_vectors=True, use_warm_start=learned)
        res = mka.mka_solve_columns(s, atoms, prm)
        lv = mka.mka_result_copy_levels(res, check=False)
        out[learned] = (res, lv)
    mu = mka.mka_find_mu(out[False][0], 4.0 * n_atoms, 0.1)
    rho, e = {}, {}
    for learned in (False, True):
        res = out[learned][0]
        r = torch.empty(mka.mka_result_info(res)["n_blocks"] * 16, dtype=torch.float64, device="cuda")
        e[learned], _ = mka.mka_density_energy(s, res, mu, 0.1, r.data_ptr())
        rho[learned] = r
    rec = {"system": f"diamond 50^3 cells, sigma 0.15, seed {seed} (unseen in training), {n_atoms} random atoms",
           "cg_iters_plain": float(out[False][1]["cg_iters"].mean()),
           "cg_iters_learned": float(out[True][1]["cg_iters"].mean()),
           "fallback_rate": float(mka.mka_result_copy_warm_start(out[True][0]).mean()),
           "max_abs_drho": float((rho[True] - rho[False]).abs().max().item()),
           "abs_dE_eV_per_atom": abs(e[True] - e[False]) / n_atoms}
    rec["iterations_saved"] = 1.0 - rec["cg_iters_learned"] / rec["cg_iters_plain"]
    for learned in out:
        mka.mka_result_destroy(out[learned][0])
    mka.mka_system_destroy(s)
    return rec


def run_form(mka, torch, sysh, w, form, B, batch_atoms, steps, warmup, stream, tune_cache, rank, autotune=True,
             compare=(), learned=False):
    """Time `steps` batches of one form through an autotuned plan (graph replay); returns timings + outputs."""
    cg_tol = 1e-12 if form == "fp64" else 1e-7
    prm = mka.solve_params(w.p, w.q, arith=form, cg_tol=cg_tol, keep_vectors=True, use_warm_start=learned)
    sp = stream.cuda_stream
    if autotune:
        tune = mka.mka_autotune(sysh, prm, batch_atoms(0)[:min(B, 4096)], w.electrons_per_atom * min(B, 4096), w.kT,
                                tune_cache, sp)
    else:
        tune = mka.tuning()
    plan = mka.mka_plan_create(sysh, B, prm, tune, sp)
    mrb = mka.mka_system_info(sysh)["max_row_blocks"]
    rho = torch.empty(B * mrb * 16, dtype=torch.float64, device="cuda")
    n_e = w.electrons_per_atom * B
    for i in range(warmup):
        mka.mka_plan_run(plan, batch_atoms(i), n_e, w.kT, rho.data_ptr())
    torch.cuda.synchronize()
    rank_barrier()
    out = {"tuning": mka.mka_plan_info(plan)}
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kms, mus, ebs = [], [], []
    launches0 = mka.mka_kernel_launches()
    # profiler filter: the timed steps of this form only (timed_mixed_learned, timed_mixed, timed_fp64)
    torch.cuda.nvtx.range_push(f"timed_{form}{'_learned' if learned else ''}")
    t0.record(stream)
    for i in range(warmup, warmup + steps):
        mka.mka_plan_run(plan, batch_atoms(i), n_e, w.kT, rho.data_ptr())
        kms.append(mka.mka_plan_kernel_ms(plan))      # waits for this batch's column kernels only
    t1.record(stream)
    torch.cuda.synchronize()
    rank_barrier()
    torch.cuda.nvtx.range_pop()
    out["launches"] = mka.mka_kernel_launches() - launches0
    out["ms"] = t0.elapsed_time(t1)
    out["kernel_ms"] = [a for a, _ in kms]
    out["reduced_ms"] = [r for _, r in kms]
    # outputs of the comparison batches (the same batch indices for every form), outside the timed region
    for i in compare:
        mka.mka_plan_run(plan, batch_atoms(i), n_e, w.kT, rho.data_ptr())
        mu, e, _ = mka.mka_plan_scalars(plan)
        mus.append(mu)
        ebs.append(e)
    lv = mka.mka_result_copy_levels(mka.mka_plan_result(plan), check=False)
    out["mu"], out["e_band"], out["cg_iters"] = mus, ebs, float(lv["cg_iters"].mean())
    out["fallback_rate"] = float(mka.mka_result_copy_warm_start(mka.mka_plan_result(plan)).mean()) if learned else None
    out["bad_columns"] = int(np.sum((lv["status"] != 0) & (lv["status"] != 4)))
    out["plan"], out["rho"], out["prm"] = plan, rho, prm
    return out


def step_slices(a0, a1, steps):
    """The rank's atoms [a0, a1) as `steps` consecutive slices of (nearly) equal size."""
    n = a1 - a0
    size = -(-n // steps)
    return [np.arange(a0 + i * size, min(a1, a0 + (i + 1) * size), dtype=np.int64) for i in range(steps)]


def batches_of(atoms, B):
    return [atoms[i:i + B] for i in range(0, len(atoms), B)]


def measured_peaks():
    try:
        return json.load(open(MEASURED_PEAKS)), "of measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "of fallback"


def spmv_leg(mka, torch, sysh, stream, reps=20):
    """K1: the global BSR SpMV y = A x over the whole system, FP32 and FP64 x, k = 1, 2, 4, CUDA events
    over `reps` launches each. Algorithmic bytes per product: values + column indices once, x read once,
    y written once, row pointers: nnzb (16 s_v + 4) + 4 N k (s_x + s_y) + 4 (N + 1)."""
    info = mka.mka_system_info(sysh)
    N, nnzb = info["n_atoms"], info["nnzb"]
    sv = {0: 8, 1: 4, 2: 2}[info["storage"]]
    peaks, src = measured_peaks()
    out = []
    sp = stream.cuda_stream
    for xd, xs, tdt in ((mka.MKA_MIXED_FP32, 4, torch.float32), (mka.MKA_FP64, 8, torch.float64)):
        for k in (1, 2, 4):
            x = torch.randn(4 * N * k, dtype=tdt, device="cuda")
            y = torch.empty_like(x)
            for which in (0, 1):
                for _ in range(3):
                    mka.mka_spmv(sysh, which, xd, x.data_ptr(), y.data_ptr(), k, sp)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(reps):
                    mka.mka_spmv(sysh, which, xd, x.data_ptr(), y.data_ptr(), k, sp)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                byt = nnzb * (16 * sv + 4) + 4 * N * k * 2 * xs + 4 * (N + 1)
                gbs = byt / ms / 1e6
                out.append({"matrix": "HS"[which], "x": "f32" if xs == 4 else "f64", "k": k, "ms": ms,
                            "GB_per_s": gbs, "frac": gbs / peaks["hbm_gbs"], "bytes": byt})
            del x, y
    torch.cuda.empty_cache()
    head = [r for r in out if r["x"] == "f32" and r["k"] == 1 and r["matrix"] == "H"][0]
    return {"bound": "hbm", "achieved": head["GB_per_s"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": head["GB_per_s"] / peaks["hbm_gbs"], "peak_source": f"hbm_gbs {src}",
            "kernel": "spmv_kernel (FP32 x, k = 1, H)", "traffic": None, "all": out}


def sample_window(mka, plan, atoms, w, half):
    """mu of a random sample of atoms (the plan's batch bisection), and the sweep window around it:
    [mu_s - half - 40 kT, mu_s + half + 40 kT]; the largest number of window levels in a sample column."""
    mka.mka_plan_run(plan, atoms, w.electrons_per_atom * len(atoms), w.kT, None)
    mu_s, _, _ = mka.mka_plan_scalars(plan)
    lv = mka.mka_result_copy_levels(mka.mka_plan_result(plan), check=False)
    lo, hi = mu_s - half - 40 * w.kT, mu_s + half + 40 * w.kT
    k = np.arange(lv["eps"].shape[1])[None, :] < lv["nu_eff"][:, None]
    cnt = ((lv["eps"] >= lo) & (lv["eps"] <= hi) & k).sum(1)
    return mu_s, (lo, hi), int(cnt.max())


def sweep_flow(mka, torch, D, sysh, plan, sw, slices, B, w, n_total, n_chunks, rho, stream, group, kms, F=None):
    """The whole work flow of Eq. EQ-WORK-FLOW over the rank's slices: plan batches into the sweep, then the
    global mu, rho, the energies and (F given) the forces. Per-batch kernel times are appended to kms.
    Returns the global scalars."""
    for sl in slices:
        for b in batches_of(sl, B):
            mka.mka_plan_run_sweep(plan, sw, b)
            kms.append(mka.mka_plan_kernel_ms(plan))
    part = D.SweepPart(mka, sw)
    if group is None:
        mu = mka.mka_sweep_find_mu(sw, w.electrons_per_atom * n_total, w.kT)
    else:
        mu, _ = D.find_mu([part], n_chunks, w.electrons_per_atom * n_total, w.kT, group=group, device="cuda")
    n_again = mka.mka_sweep_density(sw, plan, mu, w.kT, rho.data_ptr())
    tot = D.totals([part], n_chunks, mu, w.kT, group=group, device="cuda")
    out = {"mu": mu, "resolved_atoms": n_again, **tot}
    if F is not None:
        out["forces_resolved_atoms"] = mka.mka_sweep_forces(sw, plan, mu, w.kT, F.data_ptr())
    return out


def full_fp64(mka, torch, D, sysh, w, a0, a1, N, n_chunks, B, win, kp, slices, idx, rho_sample, res_head, F_head,
              stream, group, args, tune_cache):
    """The FP64 form (FP64 arithmetic on the same stored values) over the whole system, timed the same way
    (the same slices into a sweep, one mu, rho on the whole pattern, the energies and the forces): its
    rate, mu and band energy, and the differences from the headline form in mu, E, every force and a
    fixed sample of rho entries (positions idx; one whole rho fits beside the sweep, not two)."""
    sp = stream.cuda_stream
    prm = mka.solve_params(w.p, w.q, arith="fp64", cg_tol=1e-12, keep_vectors=True)
    rng = np.random.default_rng(17)
    sample = np.sort(rng.choice(np.arange(a0, a1), min(4096, a1 - a0), replace=False)).astype(np.int64)
    tune = (mka.mka_autotune(sysh, prm, sample, w.electrons_per_atom * len(sample), w.kT, tune_cache, sp)
            if not args.no_autotune else mka.tuning())
    plan = mka.mka_plan_create(sysh, B, prm, tune, sp)
    sw = mka.mka_sweep_create(sysh, a0, a1, w.nu, win[0], win[1], kp, args.chunk_atoms, sp, with_forces=True)
    rho = torch.empty(mka.mka_sweep_info(sw)["n_blocks"] * 16, dtype=torch.float64, device="cuda")
    F = torch.empty_like(F_head)
    for b in {len(x) for sl in slices for x in batches_of(sl, B)}:
        mka.mka_plan_run_sweep(plan, sw, np.arange(a0, a0 + b, dtype=np.int64))
    torch.cuda.synchronize()
    rank_barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kms = []
    t0.record(stream)
    res = sweep_flow(mka, torch, D, sysh, plan, sw, slices, B, w, N, n_chunks, rho, stream, group, kms, F)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(t0.elapsed_time(t1), "cuda")
    out = {"seconds": ms / 1e3, "columns_per_s": 4 * N / (ms / 1e3), "mu_eV": res["mu"],
           "e_band_eV_per_atom": res["e_band"] / N, "resolved_atoms": res["resolved_atoms"],
           "max_abs_drho_sampled": float((rho[idx] - rho_sample).abs().max().item()),
           "rho_sample": f"every {int(idx[1] - idx[0]) if idx.numel() > 1 else 1}th of {rho.numel()} entries",
           "max_abs_dF_eV_per_A": float((F - F_head).abs().max().item()),
           "abs_dmu_eV": abs(res["mu"] - res_head["mu"]),
           "abs_dE_eV_per_atom": abs(res["e_band"] - res_head["e_band"]) / N,
           "kernel_ms_mean": statistics.mean(k[0] for k in kms) if kms else None}
    mka.mka_sweep_destroy(sw)
    mka.mka_plan_destroy(plan)
    del rho, F
    return out


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import torch.distributed as dist
    from paper_1202_0098_gb300 import build as mka_build, distributed as D, mka

    torch.cuda.set_device(local)
    group = None
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        group = dist.group.WORLD
    w = WORKLOADS[args.workload]
    storage = args.storage or "bf16"
    form = args.form
    B = args.batch or 65536
    pos, box = workload_positions(w)
    N = pos.shape[0]
    t_build = time.perf_counter()
    sysh = mka.mka_build_system(pos, box, w.sk, storage, cluster_radius=w.R)
    t_build = time.perf_counter() - t_build
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    tune_cache = os.path.join(mka_build.BUILD, "autotune.json")
    a0, a1 = D.atom_ranges(N, world, args.chunk_atoms)[rank]
    n_chunks = (N + args.chunk_atoms - 1) // args.chunk_atoms

    spmv = None if args.no_spmv else spmv_leg(mka, torch, sysh, stream)

    learned = form == "mixed" and not args.no_learned
    net, learn_info = (None, None)
    if learned:
        net, learn_info = train_warm_start(mka, torch)
        mka.mka_system_set_warm_start(sysh, net)
    cg_tol = 1e-12 if form == "fp64" else 1e-7
    prm = mka.solve_params(w.p, w.q, arith=form, cg_tol=cg_tol, keep_vectors=True, use_warm_start=learned)
    rng = np.random.default_rng(17)
    sample = np.sort(rng.choice(np.arange(a0, a1), min(4096, a1 - a0), replace=False)).astype(np.int64)
    tune = (mka.mka_autotune(sysh, prm, sample, w.electrons_per_atom * len(sample), w.kT, tune_cache, sp)
            if not args.no_autotune else mka.tuning())
    if not args.batch and not args.no_autotune:   # the batch size from a measured search as well
        cands = [b for b in (16384, 32768, 65536, 131072) if b <= max(16384, a1 - a0)]
        B = mka.mka_autotune_batch(sysh, prm, tune, cands, a0, w.electrons_per_atom, w.kT, tune_cache, sp)
    plan = mka.mka_plan_create(sysh, B, prm, tune, sp)
    mu_s, win, max_in_win = sample_window(mka, plan, sample, w, args.window)

    # sweep sized for the free memory: rho [n_blocks][16] FP64 beside it
    nblk = int(mka.mka_system_info(sysh)["nnzb"] * (a1 - a0) / N) + 1
    free = torch.cuda.mem_get_info()[0]
    # rho, the occupied parts of rho and pi, the forces' block sums, the levels, 12 GiB for the rest
    fixed = 8 * 16 * nblk * 3 + 8 * 3 * nblk + 16 * 4 * (a1 - a0) * w.nu + 8 * 3 * N + (12 << 30)
    kp_fit = int((free - fixed) // (8 * 16 * nblk))
    kp = max(1, min(w.nu, max_in_win + 2, kp_fit))
    sw = mka.mka_sweep_create(sysh, a0, a1, w.nu, win[0], win[1], kp, args.chunk_atoms, sp, with_forces=True)
    nblk = mka.mka_sweep_info(sw)["n_blocks"]
    rho = torch.empty(nblk * 16, dtype=torch.float64, device="cuda")
    F = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    slices = step_slices(a0, a1, args.steps)

    # warm-up: the first W slices through the same path (captures every batch shape's graph)
    warm_kms = []
    for i in range(min(args.warmup, len(slices))):
        for b in batches_of(slices[i], B):
            mka.mka_plan_run_sweep(plan, sw, b)
            warm_kms.append(mka.mka_plan_kernel_ms(plan))
    for b in {len(x) for sl in slices for x in batches_of(sl, B)}:    # any batch shape not yet seen
        mka.mka_plan_run_sweep(plan, sw, np.arange(a0, a0 + b, dtype=np.int64))
    torch.cuda.synchronize()
    rank_barrier()

    kms = []
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = mka.mka_kernel_launches()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.nvtx.range_push("timed_sweep")
    t0.record(stream)
    res = sweep_flow(mka, torch, D, sysh, plan, sw, slices, B, w, N, n_chunks, rho, stream, group, kms, F)
    t1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    launches = mka.mka_kernel_launches() - launches0
    ms = max_over_ranks(t0.elapsed_time(t1), "cuda")
    rank_barrier()
    value = 4 * N / (ms / 1e3)
    stored, overflow = mka.mka_sweep_status(sw)

    # forces of every atom at the global mu (in the timed region, Eq. EQ-WORK-FLOW's last step); after it, the
    # forces alone timed again, and the density of states of all 4.03e7 columns on a grid around mu
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    mka.mka_sweep_forces(sw, plan, res["mu"], w.kT, F.data_ptr())
    f1.record(stream)
    torch.cuda.synchronize()
    Fh = F.view(-1, 3)
    forces = {"seconds": f0.elapsed_time(f1) / 1e3, "resolved_atoms": res["forces_resolved_atoms"],
              "max_abs_eV_per_A": float(Fh.abs().max().item()),
              "max_abs_sum_eV_per_A": float(Fh.sum(0).abs().max().item()) if world == 1 else None}
    del Fh
    e_ptr, w_ptr = mka.mka_sweep_device_levels(sw)
    grid = np.linspace(res["mu"] - 2.0, res["mu"] + 2.0, 41)
    t_dos = time.perf_counter()
    dos = mka.mka_dos(e_ptr, w_ptr, 4 * (a1 - a0) * w.nu, grid, w.kT, sp)
    t_dos = time.perf_counter() - t_dos
    dos_rec = {"seconds": t_dos, "energies_eV": [float(grid[0]), float(grid[-1]), len(grid)], "eta_eV": w.kT,
               "states_per_eV_per_atom_at_mu": float(dos[20] / (a1 - a0)),
               "min_states_per_eV_per_atom": float(dos.min() / (a1 - a0))}

    # ρ on sampled atoms of the rank against the oracle at the global mu (FP64 oracle on the stored values)
    # is a test (tests/test_gpu_sweep.py); here: the stored rho of a few atoms for the record
    lv_cg = mka.mka_result_copy_levels(mka.mka_plan_result(plan), check=False)

    # end to end through the public API with host buffers: atom slices in from pinned memory (staged by the
    # plan every batch), the scalars and the whole rho out to a pinned host buffer in 1 GiB pieces
    e2e = None
    if not args.no_e2e:
        piece = min(rho.numel(), (1 << 30) // 8)
        host = torch.empty(piece, dtype=torch.float64, pin_memory=True)
        pinned_slices = [torch.from_numpy(sl).pin_memory() for sl in slices]
        torch.cuda.synchronize()
        rank_barrier()
        te = time.perf_counter()
        h2d = 0
        for sl in pinned_slices:
            sl_np = sl.numpy()
            h2d += sl_np.nbytes
            for b in batches_of(sl_np, B):
                mka.mka_plan_run_sweep(plan, sw, b)
        part = D.SweepPart(mka, sw)
        if group is None:
            mu_e = mka.mka_sweep_find_mu(sw, w.electrons_per_atom * N, w.kT)
        else:
            mu_e, _ = D.find_mu([part], n_chunks, w.electrons_per_atom * N, w.kT, group=group, device="cuda")
        mka.mka_sweep_density(sw, plan, mu_e, w.kT, rho.data_ptr())
        tot_e = D.totals([part], n_chunks, mu_e, w.kT, group=group, device="cuda")
        mka.mka_sweep_forces(sw, plan, mu_e, w.kT, F.data_ptr())
        Fhost = torch.empty(F.numel(), dtype=torch.float64, pin_memory=True)
        Fhost.copy_(F)
        d2h = 8 * F.numel()
        for o in range(0, rho.numel(), piece):
            n = min(piece, rho.numel() - o)
            host[:n].copy_(rho[o:o + n])
            d2h += 8 * n
        torch.cuda.synchronize()
        rank_barrier()
        te = max_over_ranks(time.perf_counter() - te, "cuda")
        del Fhost
        e2e = {"value": 4 * N / te, "unit": "columns/s", "h2d_bytes_per_step": h2d // args.steps,
               "d2h_bytes_per_step": (d2h + 24) // args.steps, "mu": mu_e,
               "same_mu_as_timed": mu_e == res["mu"], "same_e_band": tot_e["e_band"] == res["e_band"]}
        del host

    full_system = {"atoms": N, "columns": 4 * N, "ranks": world, "atom_range_rank0": [int(a0), int(a1)],
                   "seconds": ms / 1e3, "columns_per_s": value, "mu_eV": res["mu"],
                   "e_band_eV_per_atom": res["e_band"] / N, "e_band_levels_eV_per_atom": res["e_band_levels"] / N,
                   "n_electrons": res["n_electrons"], "n_electrons_target": w.electrons_per_atom * N,
                   "sample_mu_eV": mu_s, "window_eV": list(win), "kp": kp, "stored_atoms": stored,
                   "overflow_atoms": overflow, "resolved_atoms": res["resolved_atoms"], "forces": forces, "dos": dos_rec,
                   "sweep_bytes": mka.mka_sweep_info(sw)["bytes"], "rho_bytes": 8 * rho.numel()}
    mka.mka_sweep_destroy(sw)
    mka.mka_plan_destroy(plan)
    if args.full_fp64 and form != "fp64":
        idx = torch.arange(0, rho.numel(), 211, device="cuda")
        rho_sample, F_head = rho[idx].clone(), F.clone()
        del rho
        torch.cuda.empty_cache()
        full_system["fp64_form"] = full_fp64(mka, torch, D, sysh, w, a0, a1, N, n_chunks, B, win, kp, slices,
                                             idx, rho_sample, res, F_head, stream, group, args, tune_cache)
        full_system["fp64_form"]["headline_speedup"] = value / full_system["fp64_form"]["columns_per_s"]
        del idx, rho_sample, F_head
    else:
        del rho
    torch.cuda.empty_cache()

    # per-batch rates (batch-local mu, the earlier step definition) of the comparison forms
    per_batch = {}
    n_steps_b = 3
    def batch_atoms(i):
        return shard_atoms(rank, i, n_steps_b + 1, B, N)
    compare = list(range(1, 1 + n_steps_b))
    main_b = run_form(mka, torch, sysh, w, form, B, batch_atoms, n_steps_b, 1, stream, tune_cache, rank,
                      not args.no_autotune, compare, learned)
    per_batch["headline_form"] = {"value": job_throughput(4 * B, n_steps_b, world, max_over_ranks(main_b["ms"], "cuda")),
                                  "kernel_ms_mean": statistics.mean(main_b["kernel_ms"])}
    if learned:
        prun = run_form(mka, torch, sysh, w, "mixed", B, batch_atoms, n_steps_b, 1, stream, tune_cache, rank,
                        not args.no_autotune, compare, False)
        pval = job_throughput(4 * B, n_steps_b, world, max_over_ranks(prun["ms"], "cuda"))
        nb = mka.mka_result_info(mka.mka_plan_result(prun["plan"]))["n_blocks"]
        last = batch_atoms(compare[-1])
        mka.mka_plan_run(main_b["plan"], last, w.electrons_per_atom * B, w.kT, main_b["rho"].data_ptr())
        torch.cuda.synchronize()
        learn_info.update({
            "plain_mixed_value_per_batch": pval, "speedup_over_plain_mixed": per_batch["headline_form"]["value"] / pval,
            "cg_iters_plain": prun["cg_iters"], "cg_iters_learned": main_b["cg_iters"],
            "fallback_rate": main_b["fallback_rate"],
            "max_abs_drho_vs_plain": float((main_b["rho"][:nb * 16] - prun["rho"][:nb * 16]).abs().max().item()),
            "max_abs_dE_eV_per_atom_vs_plain": max(abs(a - b) for a, b in zip(main_b["e_band"], prun["e_band"])) / B,
            "max_abs_dmu_eV_vs_plain": max(abs(a - b) for a, b in zip(main_b["mu"], prun["mu"]))})
        mka.mka_plan_destroy(prun["plan"])
        learn_info["fresh_seed_evaluation"] = learned_eval(mka, torch, net)
    other = None
    if form != "fp64" and not args.no_fp64_compare:
        frun = run_form(mka, torch, sysh, w, "fp64", B, batch_atoms, n_steps_b, 1, stream, tune_cache, rank,
                        not args.no_autotune, compare)
        fval = job_throughput(4 * B, n_steps_b, world, max_over_ranks(frun["ms"], "cuda"))
        other = {"form": "fp64", "value_per_batch": fval, "unit": "columns/s", "steps": n_steps_b,
                 "speedup_of_headline_form_per_batch": per_batch["headline_form"]["value"] / fval,
                 "compared_batches": len(compare),
                 "max_abs_dE_eV_per_atom_batch_mu": max(abs(a - b) for a, b in zip(main_b["e_band"], frun["e_band"])) / B,
                 "max_abs_dmu_eV_batch_mu": max(abs(a - b) for a, b in zip(main_b["mu"], frun["mu"])),
                 "tuning": frun["tuning"], "kernel_ms_mean": statistics.mean(frun["kernel_ms"])}
        mka.mka_plan_destroy(frun["plan"])
    mka.mka_plan_destroy(main_b["plan"])

    # rooflines of the two column kernels from their in-graph event times over the timed batches
    from scipy.spatial import cKDTree
    bsr = mka.mka_system_copy_bsr(sysh, values=False)
    tree = cKDTree(pos, boxsize=box)
    smp = np.sort(rng.choice(np.arange(a0, a1), 256, replace=False))
    m_c, nnz_c = local_flops(tree, pos, bsr["row_ptr"], bsr["col"], smp, w.R)
    cg_mean = float(lv_cg["cg_iters"].mean())
    a_v, a_r = flops_split(m_c, nnz_c, w.nu, cg_mean, 4 * np.diff(bsr["row_ptr"])[smp])
    full = [i for i, b in enumerate(x for sl in slices for x in batches_of(sl, B)) if len(b) == B]
    atoms_ms = statistics.mean(kms[i][0] for i in full)
    red_ms = statistics.mean(kms[i][1] for i in full)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = clk.get("sm_mhz") or measured_peaks()[0].get("sm_max_mhz", 1980.0)
    roofline = alu_roofline(float(np.mean(a_v)), 4 * B, atoms_ms / 1e3, "fp64" if form == "fp64" else "fp32",
                            "atoms_kernel", "cluster, CG, Krylov basis and projection, counted as plain (not pair) arithmetic",
                            sms, mhz)
    roofline_red = alu_roofline(float(np.mean(a_r)), 4 * B, red_ms / 1e3, "fp64", "reduced_kernel",
                                "Cholesky, congruence, tridiagonalisation, QL eigenvalues, inverse iteration, "
                                "back-transform, outputs: 17/3 nu^3 + 47 nu^2 FLOP per column", sms, mhz)
    if form == "mixed":   # DRAM bytes per launch from the profiler capture (null once the kernel has changed)
        roofline["traffic"] = captured_traffic("atoms_kernel", B)
        roofline_red["traffic"] = captured_traffic("reduced_kernel", 4 * B)
    mka.mka_system_destroy(sysh)
    if net is not None:
        mka.mka_mlp_destroy(net)

    line = {"metric": "density-matrix columns/s", "value": value, "unit": "columns/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64" if form == "fp64" else "f32",
            "data": "synthetic",
            "config": {"workload": workload_desc(args.workload, w, N),
                       "form": f"{form}{'+learned' if learned else ''}, {storage}-stored H and S",
                       "step": f"one slice of {len(slices[0])} atoms through plan batches of {B} atoms into the "
                               "sweep; after the last, mu over all columns, rho on the whole pattern, energies, forces",
                       "atoms_per_step": len(slices[0]), "batch_atoms": B,
                       "l2": "inputs larger than L2 (H, S, levels and rho pieces of the whole system in HBM)",
                       "tuning": {"threads": tune.threads, "ctas_per_sm": tune.ctas_per_sm,
                                  "order_by_size": tune.order_by_size},
                       "build_s": t_build},
            "gpu_launches": launches, "clocks": clk, "e2e": e2e, "roofline": roofline,
            "roofline_reduced": roofline_red, "spmv": spmv, "full_system": full_system,
            "kernel_ms_mean": atoms_ms, "reduced_ms_mean": red_ms, "cg_iters_mean": cg_mean,
            "per_batch": per_batch, "learned_warm_start": learn_info, "fp64_form": other}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, pos, box)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
