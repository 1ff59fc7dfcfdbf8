"""Benchmark: density-matrix columns per second of the multiple Arnoldi method on GB300.

Workload: the 10,077,696-atom diamond-lattice system (108^3 cubic cells,
a = 3.567 A, sigma = 0.1 A, sp basis, M = 40,310,784 columns), cluster radius
6 A, p = q = 15, kT = 0.1 eV. One step is one pass of the whole per-column work
flow over a batch of consecutive atoms (4 columns each): cluster extraction,
inner CG, multiple Krylov basis, projection, reduced eigensolve, mu by
bisection over the batch, rho on the H pattern and the band energy. Each rank
streams its own batches (weak scaling; no collective on the data path).

Prints one JSON line (rank 0). `--impl reference` times the FP64 CPU oracle
on the host cores instead (a bounded sample of the same workload per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import WORKLOADS, workload_positions  # noqa: E402

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 / FP32 FMA peaks of a GB300: 152 SMs x (2 FP64 | 128 FP32 FMA per clock) x 2 flops at the
# 1.98 GHz seen under load; nominal FP64 1.25 TFLOP/s.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 1.98e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 1.98e9 / 1e12


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


def column_flops(m, nnz, nu, cg_it, n_pattern_rows):
    """Algorithmic FLOPs of one column, counted as plain arithmetic: the products of the CG and
    the basis, CG vector work, one Gram-Schmidt pass per vector (coefficients and update), norms,
    the projection, the reduced solve and the rows V_j, (S V)_j of the outputs."""
    spmv = 2.0 * 16.0 * nnz * (cg_it + 2 * nu)          # CG S-products + nu S- and nu H-products
    cg_vec = 10.0 * m * cg_it                            # two dots, three axpys per CG step
    gs = 2.0 * m * nu * (nu - 1)                          # one pass of dots + updates per new vector
    norms = 4.0 * m * nu                                  # S-norm and scaling per vector
    proj = 4.0 * m * nu * nu                              # U^T K and U^T (S U)
    red = 12.3 * nu ** 3                                  # Cholesky, two triangular solves, eig, back-transform
    out = 4.0 * nu * nu                                   # V_j and (S V)_j
    return spmv + cg_vec + gs + norms + proj + red + out


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
    ctx = mp.get_context("spawn")
    rng = np.random.default_rng(0)
    times = []
    with ctx.Pool(cores) as pool:
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
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
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
    return {"value": 4 * n_at / dt, "unit": "columns/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_at} random atoms ({4 * n_at} columns) of {w.name}, FP64 numpy oracle, "
                      f"one spawn process per core"}


def flops_split(m, nnz, nu, cg_it, n_pattern_rows):
    """Algorithmic (vector work, reduced solve) FLOPs of one column: the reduced solve is 12.3 nu^3."""
    total = column_flops(m, nnz, nu, cg_it, n_pattern_rows)
    red = 12.3 * nu ** 3
    return total - red, red


def alu_roofline(flops_per_col, n_cols, kernel_s, pipe, kernel, what):
    """ALU bound of one kernel: its algorithmic FLOPs per launch over its event time, against the
    peak of the pipe that does them (derived from unit counts and the clock under load)."""
    peak = FP64_PEAK_TFLOPS if pipe == "fp64" else FP32_PEAK_TFLOPS
    achieved = flops_per_col * n_cols / kernel_s / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": kernel,
            "peak_source": (f"derived: 152 SMs x 1.98 GHz x 2 x {2 if pipe == 'fp64' else 128} "
                            f"{'FP64' if pipe == 'fp64' else 'FP32'} FMA/clk/SM; {what}"),
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
        X, Y, _ = warm_start.collect(s, atoms, "mixed", 1e-7)
        Xs.append(X)
        Ys.append(Y)
        mka.mka_system_destroy(s)
    X, Y = torch.cat(Xs), torch.cat(Ys)
    net = mka.mka_mlp_create(seed)
    mse0 = warm_start.mse(net, X, Y)
    hist = warm_start.train(net, X, Y, epochs=20, batch=1024, lr=1e-3, seed=seed)
    info = {"samples": int(X.shape[0]), "generators": "fcc (config-2) and diamond sigma 0.15 (config-3), seeds "
            f"{seed}-{seed + 3}", "epochs": 20, "batch": 1024, "mse_init": mse0, "mse_final": hist[-1],
            "train_s": time.perf_counter() - t0}
    del X, Y, Xs, Ys
    return net, info


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


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import torch.distributed as dist
    from paper_1202_0098_gb300 import build as mka_build, mka

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
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
    tune_cache = os.path.join(mka_build.BUILD, "autotune.json")
    n_steps = args.warmup + args.steps

    def batch_atoms(i):
        return shard_atoms(rank, i, n_steps, B, N)

    compare = list(range(args.warmup, args.warmup + max(1, min(args.steps, 3))))
    learned = form == "mixed" and not args.no_learned
    net, learn_info = (None, None)
    if learned:
        net, learn_info = train_warm_start(mka, torch)
        mka.mka_system_set_warm_start(sysh, net)
    main_run = run_form(mka, torch, sysh, w, form, B, batch_atoms, args.steps, args.warmup, stream, tune_cache, rank,
                        not args.no_autotune, compare, learned)
    ms = max_over_ranks(main_run["ms"], "cuda")
    value = job_throughput(4 * B, args.steps, world, ms)

    # clocks during a second pass of the same timed batches
    clocks = ClockSampler(local)
    clocks.start()
    plan = main_run["plan"]
    n_e = w.electrons_per_atom * B
    for i in range(args.warmup, n_steps):
        mka.mka_plan_run(plan, batch_atoms(i), n_e, w.kT, main_run["rho"].data_ptr())
    torch.cuda.synchronize()
    clk = clocks.stop()

    # end to end through the public API with host buffers: host atoms in; mu, E, levels and rho out
    e2e = None
    if not args.no_e2e:
        rho_h = torch.empty(main_run["rho"].numel(), dtype=torch.float64, pin_memory=True)
        torch.cuda.synchronize()
        rank_barrier()
        te = time.perf_counter()
        d2h = 0
        for i in range(args.warmup, n_steps):
            mka.mka_plan_run(plan, batch_atoms(i), n_e, w.kT, main_run["rho"].data_ptr())
            mka.mka_plan_scalars(plan)
            lv = mka.mka_result_copy_levels(mka.mka_plan_result(plan), check=False)
            nb = mka.mka_result_info(mka.mka_plan_result(plan))["n_blocks"]
            rho_h[:nb * 16].copy_(main_run["rho"][:nb * 16])
            d2h += nb * 16 * 8 + sum(v.nbytes for k, v in lv.items() if hasattr(v, "nbytes")) + 24
        torch.cuda.synchronize()
        rank_barrier()
        te = max_over_ranks(time.perf_counter() - te, "cuda")
        e2e = {"value": job_throughput(4 * B, args.steps, world, 1e3 * te), "unit": "columns/s",
               "h2d_bytes_per_step": 16 * B + 8,
               "d2h_bytes_per_step": d2h // args.steps}

    # the mixed form without the learned start on the same batches: what the network gains
    if learned:
        fsteps = max(1, min(args.steps, 3))
        prun = run_form(mka, torch, sysh, w, "mixed", B, batch_atoms, fsteps, 1, stream, tune_cache, rank,
                        not args.no_autotune, compare, False)
        pval = job_throughput(4 * B, fsteps, world, max_over_ranks(prun["ms"], "cuda"))
        # both plans' rho buffers on the same (last compared) batch
        last = batch_atoms(compare[-1])
        mka.mka_plan_run(main_run["plan"], last, w.electrons_per_atom * B, w.kT, main_run["rho"].data_ptr())
        torch.cuda.synchronize()
        nb = mka.mka_result_info(mka.mka_plan_result(prun["plan"]))["n_blocks"]
        learn_info.update({
            "plain_mixed_value": pval, "speedup_over_plain_mixed": value / pval,
            "cg_iters_plain": prun["cg_iters"], "cg_iters_learned": main_run["cg_iters"],
            "fallback_rate": main_run["fallback_rate"],
            "max_abs_drho_vs_plain": float((main_run["rho"][:nb * 16] - prun["rho"][:nb * 16]).abs().max().item()),
            "max_abs_dE_eV_per_atom_vs_plain": max(abs(a - b) for a, b in zip(main_run["e_band"], prun["e_band"])) / B,
            "max_abs_dmu_eV_vs_plain": max(abs(a - b) for a, b in zip(main_run["mu"], prun["mu"]))})
        mka.mka_plan_destroy(prun["plan"])

    # the FP64 form on the same stored values and batches: speed and agreement of mu / E
    other = None
    if form != "fp64" and not args.no_fp64_compare:
        fsteps = max(1, min(args.steps, 3))
        frun = run_form(mka, torch, sysh, w, "fp64", B, batch_atoms, fsteps, 1, stream, tune_cache, rank,
                        not args.no_autotune, compare)
        fval = job_throughput(4 * B, fsteps, world, max_over_ranks(frun["ms"], "cuda"))
        de = max(abs(a - b) for a, b in zip(main_run["e_band"], frun["e_band"])) / B
        dmu = max(abs(a - b) for a, b in zip(main_run["mu"], frun["mu"]))
        other = {"form": "fp64", "value": fval, "unit": "columns/s", "steps": fsteps,
                 "speedup_of_headline": value / fval, "compared_batches": len(compare),
                 "max_abs_dE_eV_per_atom": de, "max_abs_dmu_eV": dmu,
                 "tuning": frun["tuning"], "kernel_ms_mean": statistics.mean(frun["kernel_ms"])}
        mka.mka_plan_destroy(frun["plan"])

    # roofline of the per-atom kernel from its in-graph event time
    from scipy.spatial import cKDTree
    bsr = mka.mka_system_copy_bsr(sysh, values=False)
    tree = cKDTree(pos, boxsize=box)
    fv = fr = 0.0
    for i in range(args.warmup, n_steps):
        atoms = batch_atoms(i)[::max(1, B // 256)]
        m_c, nnz_c = local_flops(tree, pos, bsr["row_ptr"], bsr["col"], atoms, w.R)
        rows = 4 * np.diff(bsr["row_ptr"])[atoms]
        a_v, a_r = flops_split(m_c, nnz_c, w.nu, main_run["cg_iters"], rows)
        fv += float(np.mean(a_v)) / args.steps
        fr += float(np.mean(a_r)) / args.steps
    roofline = alu_roofline(fv, 4 * B, statistics.mean(main_run["kernel_ms"]) / 1e3,
                            "fp64" if form == "fp64" else "fp32", "atoms_kernel",
                            "cluster, CG, Krylov basis and projection, counted as plain (not pair) arithmetic")
    roofline_red = alu_roofline(fr, 4 * B, statistics.mean(main_run["reduced_ms"]) / 1e3, "fp64", "reduced_kernel",
                                "Cholesky, congruence, tridiagonalisation, QL with vectors, back-transform, "
                                "outputs: 12.3 nu^3 FLOP per column")
    if form == "mixed":   # DRAM bytes per launch from the profiler capture (null once the kernel has changed)
        roofline["traffic"] = captured_traffic("atoms_kernel", B)
        roofline_red["traffic"] = captured_traffic("reduced_kernel", 4 * B)
    mka.mka_plan_destroy(plan)
    mka.mka_system_destroy(sysh)
    if net is not None:
        mka.mka_mlp_destroy(net)

    line = {"metric": "density-matrix columns/s", "value": value, "unit": "columns/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if form == "fp64" else "f32",
            "data": "synthetic",
            "config": {"workload": workload_desc(args.workload, w, N),
                       "form": f"{form}{'+learned' if learned else ''}, {storage}-stored H and S",
                       "atoms_per_step": B, "columns_per_step": 4 * B,
                       "step": "one graph-replayed batch: per-atom kernel, mu bisection over the batch, rho, E",
                       "l2": "inputs larger than L2 (H,S of the whole system in HBM; each step a new batch of atoms)",
                       "tuning": main_run["tuning"], "build_s": t_build},
            "gpu_launches": main_run["launches"], "clocks": clk, "e2e": e2e, "roofline": roofline,
            "roofline_reduced": roofline_red,
            "kernel_ms_mean": statistics.mean(main_run["kernel_ms"]),
            "reduced_ms_mean": statistics.mean(main_run["reduced_ms"]), "cg_iters_mean": main_run["cg_iters"],
            "bad_columns": main_run["bad_columns"], "learned_warm_start": learn_info, "fp64_form": other,
            "mu_first_compared": main_run["mu"][0], "e_band_per_atom_first_compared": main_run["e_band"][0] / B}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, pos, box)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
