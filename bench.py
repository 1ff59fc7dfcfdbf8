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
    ap.add_argument("--form", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--storage", default=None, choices=[None, "fp64", "fp32", "bf16"])
    ap.add_argument("--batch", type=int, default=0, help="atoms per step (0: per form default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


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
    """Algorithmic FLOPs of one column (counted in the design doc terms)."""
    spmv = 2.0 * 16.0 * nnz * (cg_it + 2 * nu)          # CG S-products + nu S- and nu H-products
    cg_vec = 10.0 * m * cg_it                            # two dots, three axpys per CG step
    gs = 4.0 * m * nu * (nu - 1)                          # CGS2: two passes of dots + updates
    norms = 4.0 * m * nu                                  # S-norm and scaling per vector
    proj = 4.0 * m * nu * nu                              # U^T K and U^T (S U)
    red = 12.3 * nu ** 3                                  # Cholesky, two triangular solves, eig, back-transform
    out = 2.0 * nu * nu * (n_pattern_rows + 2)            # V pattern rows, V_j and (S V)_j
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
            "config": {"workload": f"{args.workload}: FP64 CPU oracle, {per_step} random atoms per step"},
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


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import torch.distributed as dist
    from paper_1202_0098_gb300 import mka

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = WORKLOADS[args.workload]
    storage = args.storage or ("fp64" if args.form == "fp64" else "bf16")
    B = args.batch or (8192 if args.form == "fp64" else 65536)
    pos, box = workload_positions(w)
    N = pos.shape[0]
    t_build = time.perf_counter()
    sysh = mka.mka_build_system(pos, box, w.sk, storage, cluster_radius=w.R)
    t_build = time.perf_counter() - t_build
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    cg_tol = 1e-12 if args.form == "fp64" else 1e-7
    prm = mka.solve_params(w.p, w.q, arith="fp64" if args.form == "fp64" else "mixed", cg_tol=cg_tol,
                           keep_vectors=True)
    n_steps = args.warmup + args.steps

    def batch_atoms(i):
        start = ((rank * n_steps + i) * B) % N
        return (np.arange(start, start + B, dtype=np.int64) % N)

    def step(i, host=False):
        atoms = batch_atoms(i)
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record(stream)
        res = mka.mka_solve_columns(sysh, atoms, prm, stream=sp)
        ev[1].record(stream)
        mu = mka.mka_find_mu(res, w.electrons_per_atom * B, w.kT)
        nb = mka.mka_result_info(res)["n_blocks"]
        rho = torch.empty(nb * 16, dtype=torch.float64, device="cuda")
        e_band, n_el = mka.mka_density_energy(sysh, res, mu, w.kT, rho.data_ptr())
        out = None
        if host:
            out = (rho.cpu(), mka.mka_result_copy_levels(res, check=False))
        mka.mka_result_destroy(res)
        return ev, mu, e_band, nb, out

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    kevs, mus, ebs = [], [], []
    launches0 = mka.mka_kernel_launches()
    for i in range(args.warmup, n_steps):
        ev, mu, eb, nb, _ = step(i)
        kevs.append(ev)
        mus.append(mu)
        ebs.append(eb)
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    launches = mka.mka_kernel_launches() - launches0
    ms = t0.elapsed_time(t1)
    if world > 1:
        tt = torch.tensor([ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    cols_total = 4 * B * args.steps * world
    value = cols_total / (ms / 1e3)
    solve_ms = [a.elapsed_time(b) for a, b in kevs]

    # end to end through the public API with host buffers (host atoms in, rho and levels out)
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        te = time.perf_counter()
        h2d = d2h = 0
        cg_its = []
        for i in range(args.warmup, n_steps):
            ev, mu, eb, nb, out = step(i, host=True)
            h2d += 8 * B + 8 * (B + 1)
            d2h += out[0].numel() * 8 + 4 * B * w.nu * 8 * 2 + 4 * B * 4 * 3
            cg_its.append(float(out[1]["cg_iters"].mean()))
        torch.cuda.synchronize()
        te = time.perf_counter() - te
        e2e = {"value": 4 * B * args.steps * world / te, "unit": "columns/s",
               "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps}

    # roofline of the per-atom kernel: algorithmic FLOPs of the timed batches / its event time
    from scipy.spatial import cKDTree
    bsr = mka.mka_system_copy_bsr(sysh)
    tree = cKDTree(pos, boxsize=box)
    cg_mean = statistics.mean(cg_its) if e2e else 20.0
    flops = 0.0
    for i in range(args.warmup, n_steps):
        atoms = batch_atoms(i)[::max(1, B // 256)]
        m_c, nnz_c = local_flops(tree, pos, bsr["row_ptr"], bsr["col"], atoms, w.R)
        rows = 4 * np.diff(bsr["row_ptr"])[atoms]
        flops += column_flops(m_c, nnz_c, w.nu, cg_mean, rows).mean() * 4 * B
    achieved = flops / (sum(solve_ms) / 1e3) / 1e12
    peak = FP64_PEAK_TFLOPS if args.form == "fp64" else FP32_PEAK_TFLOPS
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "atoms_kernel",
                "peak_source": "derived: 152 SMs x FMA/clk x 2 x 1.98 GHz (FP64 2, FP32 128 FMA/clk/SM)"}
    mka.mka_system_destroy(sysh)

    line = {"metric": "density-matrix columns/s", "value": value, "unit": "columns/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.form == "fp64" else "f32",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {N} atoms, {4 * N} columns, R={w.R} A, p=q={w.p}, "
                                   f"kT={w.kT} eV, {args.form} form, {storage} storage",
                       "atoms_per_step": B, "columns_per_step": 4 * B, "l2": "inputs larger than L2 "
                       "(H,S of the whole system in HBM; each step a new batch of atoms)",
                       "build_s": t_build},
            "gpu_launches": launches, "clocks": clk, "e2e": e2e, "roofline": roofline,
            "solve_ms_per_step": sum(solve_ms) / len(solve_ms), "cg_iters_mean": cg_mean, "mu_last": mus[-1],
            "e_band_per_atom_last": ebs[-1] / B}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, pos, box)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
