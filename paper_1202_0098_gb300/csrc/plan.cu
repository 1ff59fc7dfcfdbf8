// Persistent, graph-captured batches of columns (plans) and the autotuner.
//
// A plan owns every buffer one batch of the work flow needs (Eq. EQ-WORK-FLOW:
// the per-column brace, mu by bisection, rho and the band energy), sized once for
// at most `max_atoms` atoms, so that running a batch allocates nothing and never
// waits on the host. A batch is one CUDA graph: copy of the atom list and its
// output offsets from pinned staging, optional ordering of the work queue by
// descending cluster size (uneven clusters finish together), the persistent
// per-atom kernel, a fixed-length device bisection for mu, and the density /
// energy kernels. The graph is captured the first time a batch shape (atom count,
// electron count, kT, rho buffer) is seen and replayed afterwards.
//
// The autotuner times candidate launch shapes (CTA size, resident CTAs per SM,
// size ordering) on a sample batch and keeps the fastest, optionally cached in a
// small JSON file keyed by GPU, storage, arithmetic, subspace size and cluster size.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "mka_internal.h"

namespace mka {
namespace {

constexpr int kSizeBins = MKA_MAX_CLUSTER_ATOMS + 1;
constexpr int kHalvings = 64;   // bracket width / 2^64: below 1e-12 eV for any bracket narrower than 1.8e7 eV

__global__ void size_hist_kernel(const int32_t* sizes, int64_t n, int32_t* bins) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&bins[min(max(sizes[i], 0), kSizeBins - 1)], 1);
}

// Exclusive scan of the bins from the largest size down: bins[s] = first slot of size s.
__global__ void size_scan_kernel(int32_t* bins) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int32_t run = 0;
    for (int s = kSizeBins - 1; s >= 0; --s) {
      const int32_t c = bins[s];
      bins[s] = run;
      run += c;
    }
  }
}

__global__ void size_scatter_kernel(const int32_t* sizes, int64_t n, int32_t* bins, int32_t* order) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t pos = atomicAdd(&bins[min(max(sizes[i], 0), kSizeBins - 1)], 1);
    order[pos] = (int32_t)i;
  }
}

struct GraphEntry {
  int64_t n = 0;
  int kind = PLAN_BATCH;
  const mka_sweep* sw = nullptr;
  double n_electrons = 0, kT = 0, mu = 0;
  double* rho = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;
  bool forces = false;
  bool same(int64_t n_, const PlanMode& m) const {
    return n == n_ && kind == m.kind && sw == m.sw && n_electrons == m.n_electrons && kT == m.kT && mu == m.mu &&
           rho == m.rho && forces == m.forces;
  }
};

}  // namespace
}  // namespace mka

struct mka_plan {
  mka_system* sys = nullptr;
  cudaStream_t stream = nullptr;
  mka_solve_params prm{};
  mka_tuning tune{};
  int64_t max_atoms = 0;
  int max_cl = 0;
  mka::AtomsConfig cf{};
  int grid = 0;
  mka_result* res = nullptr;       // owned; its sizes follow the last run
  char* scratch = nullptr;
  int* counter = nullptr;
  int32_t* order = nullptr;
  int32_t* sizes = nullptr;
  int32_t* bins = nullptr;
  void* mu_buf = nullptr;
  double* dev_out = nullptr;       // [0] mu, then density partials (max_atoms), E, N
  int64_t* h_stage = nullptr;      // pinned: atoms [max_atoms], block offsets [max_atoms + 1]
  cudaEvent_t staged = nullptr;
  cudaStream_t capture = nullptr;  // private stream the graphs are captured on (never executes work)
  cudaEvent_t k0 = nullptr, k1 = nullptr;   // recorded around the per-atom kernel inside every graph
  cudaEvent_t k2 = nullptr;        // recorded after the batched reduced problems
  double* red = nullptr;           // reduced-problem buffer of max_atoms atoms
  float* warm = nullptr;           // learned start: X [4A][132], Y [4A][68], network work buffers
  int32_t* patch = nullptr;        // [A][17]
  std::vector<mka::GraphEntry> graphs;
};

using namespace mka;

namespace {

mka_status plan_alloc(mka_plan* P) {
  mka_result* r = new mka_result();
  P->res = r;
  r->sys = P->sys;
  r->stream = P->stream;
  r->p = P->prm.p;
  r->q = P->prm.q;
  r->nu = P->prm.p + P->prm.q;
  r->arith = P->prm.arith;
  r->keep = 1;
  const int64_t A = P->max_atoms, nu = r->nu;
  const int64_t max_blocks = A * std::max(1, P->sys->max_row_blocks);
  MKA_CUDA_TRY(cudaMalloc(&r->d_sel, sizeof(int64_t) * A));
  MKA_CUDA_TRY(cudaMalloc(&r->d_blk_off, sizeof(int64_t) * (A + 1)));
  MKA_CUDA_TRY(cudaMalloc(&r->d_eps, sizeof(double) * 4 * A * nu));
  MKA_CUDA_TRY(cudaMalloc(&r->d_w, sizeof(double) * 4 * A * nu));
  MKA_CUDA_TRY(cudaMalloc(&r->d_nu_eff, sizeof(int32_t) * 4 * A));
  MKA_CUDA_TRY(cudaMalloc(&r->d_cg_iters, sizeof(int32_t) * 4 * A));
  MKA_CUDA_TRY(cudaMalloc(&r->d_status, sizeof(int32_t) * 4 * A));
  MKA_CUDA_TRY(cudaMalloc(&r->d_vp, sizeof(double) * max_blocks * 16 * nu));
  MKA_CUDA_TRY(cudaMalloc(&r->d_cv, kept_buffer_bytes(4 * A, (int)nu)));
  MKA_CUDA_TRY(cudaMalloc(&P->scratch, P->cf.slot_bytes * (size_t)P->grid + 256));
  MKA_CUDA_TRY(cudaMalloc(&P->red, red_buffer_bytes(4 * A, (int)nu)));
  MKA_CUDA_TRY(cudaMalloc(&P->counter, 256));
  MKA_CUDA_TRY(cudaMalloc(&P->order, sizeof(int32_t) * A));
  MKA_CUDA_TRY(cudaMalloc(&P->sizes, sizeof(int32_t) * A));
  MKA_CUDA_TRY(cudaMalloc(&P->bins, sizeof(int32_t) * kSizeBins));
  MKA_CUDA_TRY(cudaMalloc(&P->mu_buf, mu_buffer_bytes()));
  MKA_CUDA_TRY(cudaMalloc(&P->dev_out, sizeof(double) * (A + 4 + kMaxRedBlocks)));   // mu, partials, E, N, count partials
  MKA_CUDA_TRY(cudaMallocHost(&P->h_stage, sizeof(int64_t) * (2 * A + 1)));
  MKA_CUDA_TRY(cudaEventCreateWithFlags(&P->staged, cudaEventDisableTiming));
  MKA_CUDA_TRY(cudaStreamCreateWithFlags(&P->capture, cudaStreamNonBlocking));
  MKA_CUDA_TRY(cudaEventCreate(&P->k0));
  MKA_CUDA_TRY(cudaEventCreate(&P->k1));
  MKA_CUDA_TRY(cudaEventCreate(&P->k2));
  if (P->prm.use_warm_start) {
    MKA_CUDA_TRY(cudaMalloc(&r->d_fallback, sizeof(int32_t) * 4 * A));
    MKA_CUDA_TRY(cudaMalloc(&P->warm, sizeof(float) * (4 * A * (132 + 68) + mlp_work_floats(4 * A))));
    MKA_CUDA_TRY(cudaMalloc(&P->patch, sizeof(int32_t) * 17 * A));
  }
  return MKA_OK;
}

// Enqueue one batch of n atoms (already staged) on the capture stream (recorded into a graph).
mka_status plan_enqueue(mka_plan* P, int64_t n, const PlanMode& m) {
  cudaStream_t st = P->capture;
  mka_result* r = P->res;
  MKA_CUDA_TRY(cudaMemcpyAsync(r->d_sel, P->h_stage, sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
  MKA_CUDA_TRY(cudaMemcpyAsync(r->d_blk_off, P->h_stage + P->max_atoms, sizeof(int64_t) * (n + 1),
                               cudaMemcpyHostToDevice, st));
  MKA_CUDA_TRY(cudaMemsetAsync(P->counter, 0, sizeof(int), st));
  const int32_t* order = nullptr;
  if (P->tune.order_by_size) {
    mka_status s = launch_cluster_sizes(P->sys, r->d_sel, n, P->sizes, st);
    if (s) return s;
    MKA_CUDA_TRY(cudaMemsetAsync(P->bins, 0, sizeof(int32_t) * kSizeBins, st));
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 1024);
    size_hist_kernel<<<blocks, 256, 0, st>>>(P->sizes, n, P->bins);
    size_scan_kernel<<<1, 32, 0, st>>>(P->bins);
    size_scatter_kernel<<<blocks, 256, 0, st>>>(P->sizes, n, P->bins, P->order);
    count_launches(3);
    MKA_CUDA_TRY(cudaGetLastError());
    order = P->order;
  }
  AtomsLaunchArgs a{};
  if (P->prm.use_warm_start) {
    const int64_t rows = 4 * n;
    float* X = P->warm;
    float* Y = X + 4 * P->max_atoms * 132;
    float* W = Y + 4 * P->max_atoms * 68;
    mka_status sw = features_enqueue(P->sys, r->d_sel, n, X, P->patch, st);
    if (!sw) sw = mlp_forward_enqueue(P->sys->warm, X, rows, W, W + rows * 128, W + 2 * rows * 128, W + 3 * rows * 128, Y, st);
    if (sw) return sw;
    a.x0 = Y;
    a.patch = P->patch;
    a.fallback = r->d_fallback;
  }
  a.sel = r->d_sel;
  a.order = order;
  a.n_sel = n;
  a.p = P->prm.p;
  a.q = P->prm.q;
  a.cg_tol = P->prm.cg_tol;
  a.cg_maxit = P->prm.cg_maxit;
  a.eps = r->d_eps;
  a.w = r->d_w;
  a.nu_eff = r->d_nu_eff;
  a.cg_iters = r->d_cg_iters;
  a.status = r->d_status;
  a.keep = 1;
  a.vp = r->d_vp;
  a.blk_off = r->d_blk_off;
  a.scratch = P->scratch;
  a.counter = P->counter;
  a.red = P->red;
  a.cv = r->d_cv;
  a.col0 = 0;
  a.mode_b = P->prm.subspace == MKA_SUBSPACE_B;
  a.grid = (int)std::min<int64_t>(n, P->grid);
  MKA_CUDA_TRY(cudaEventRecordWithFlags(P->k0, st, cudaEventRecordExternal));
  mka_status s = atoms_launch(P->sys, P->prm.arith, P->cf, a, st);
  if (s) return s;
  MKA_CUDA_TRY(cudaEventRecordWithFlags(P->k1, st, cudaEventRecordExternal));
  s = reduced_for(P->sys, a, st);
  if (s) return s;
  MKA_CUDA_TRY(cudaEventRecordWithFlags(P->k2, st, cudaEventRecordExternal));
  const int nu = r->nu;
  if (m.kind == PLAN_SWEEP)
    return sweep_pack_enqueue(m.sw, r->d_sel, r->d_blk_off, r->d_vp, r->d_cv, r->d_eps, r->d_w, r->d_nu_eff, n, nu, st);
  if (m.kind == PLAN_AT_MU)
    return sweep_at_mu_enqueue(m.sw, r->d_sel, r->d_blk_off, r->d_vp, r->d_cv, r->d_eps, n, nu, m.mu, m.kT, m.rho,
                               m.forces, st);
  s = find_mu_enqueue(r->d_eps, r->d_w, 4 * n * nu, m.n_electrons, m.kT, 1e-12, kHalvings, P->mu_buf, P->dev_out, st);
  if (s) return s;
  return density_enqueue(P->sys, r->d_sel, r->d_blk_off, r->d_vp, r->d_cv, r->d_eps, r->d_w, n, nu, P->dev_out, m.kT,
                         m.rho, P->dev_out + 1, st);
}

}  // namespace

extern "C" {

void mka_plan_destroy(mka_plan* P) {
  if (!P) return;
  for (auto& g : P->graphs) cudaGraphExecDestroy(g.exec);
  if (P->staged) cudaEventDestroy(P->staged);
  if (P->capture) cudaStreamDestroy(P->capture);
  if (P->k0) cudaEventDestroy(P->k0);
  if (P->k1) cudaEventDestroy(P->k1);
  if (P->k2) cudaEventDestroy(P->k2);
  cudaFreeHost(P->h_stage);
  cudaFree(P->scratch);
  cudaFree(P->red);
  cudaFree(P->counter);
  cudaFree(P->order);
  cudaFree(P->sizes);
  cudaFree(P->bins);
  cudaFree(P->mu_buf);
  cudaFree(P->dev_out);
  cudaFree(P->warm);
  cudaFree(P->patch);
  mka_result_destroy(P->res);
  delete P;
}

mka_status mka_plan_create(mka_system* sys, int64_t max_atoms, const mka_solve_params* prm, const mka_tuning* tune,
                           void* stream, mka_plan** out) {
  if (!out) return fail(MKA_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!sys || !prm || max_atoms < 1) return fail(MKA_ERR_INVALID_ARG, "system, params and max_atoms >= 1 are required");
  if (prm->p < 1 || prm->q < 0 || prm->p + prm->q > MKA_MAX_NU)
    return fail(MKA_ERR_INVALID_ARG, "need p >= 1, q >= 0, p + q <= MKA_MAX_NU");
  if (prm->arith != MKA_FP64 && prm->arith != MKA_MIXED_FP32)
    return fail(MKA_ERR_INVALID_ARG, "arith must be MKA_FP64 or MKA_MIXED_FP32");
  if (!(prm->cg_tol > 0) || prm->cg_maxit < 1) return fail(MKA_ERR_INVALID_ARG, "need cg_tol > 0, cg_maxit >= 1");
  if (prm->subspace != MKA_SUBSPACE_A && prm->subspace != MKA_SUBSPACE_B)
    return fail(MKA_ERR_INVALID_ARG, "subspace must be MKA_SUBSPACE_A or MKA_SUBSPACE_B");
  if (prm->s_start || prm->keep_s) return fail(MKA_ERR_INVALID_ARG, "keep_s and s_start are for direct solves");
  if (prm->use_warm_start && !sys->warm)
    return fail(MKA_ERR_INVALID_ARG, "use_warm_start needs a network attached with mka_system_set_warm_start");
  mka_tuning t{256, 0, 0};
  if (tune) t = *tune;
  if (t.threads == 0) t.threads = 256;
  if (t.threads != 128 && t.threads != 256 && t.threads != 512)
    return fail(MKA_ERR_INVALID_ARG, "tuning.threads must be 128, 256 or 512");
  if (t.ctas_per_sm < 0) return fail(MKA_ERR_INVALID_ARG, "tuning.ctas_per_sm must be >= 0");
  mka_plan* P = new mka_plan();
  P->sys = sys;
  P->stream = (cudaStream_t)stream;
  P->prm = *prm;
  P->tune = t;
  P->max_atoms = max_atoms;
  // largest cluster of the whole system sizes every work slot (computed once per system)
  if (sys->max_cluster < 0) {
    std::vector<int32_t> sz(sys->n_atoms);
    mka_status s0 = mka_cluster_sizes(sys, nullptr, sys->n_atoms, sz.data());
    if (s0) {
      delete P;
      return s0;
    }
    sys->max_cluster = *std::max_element(sz.begin(), sz.end());
  }
  mka_status s = MKA_OK;
  P->max_cl = sys->max_cluster;
  if (P->max_cl > MKA_MAX_CLUSTER_ATOMS) {
    delete P;
    return fail(MKA_ERR_CLUSTER_TOO_LARGE, "a cluster of the system exceeds MKA_MAX_CLUSTER_ATOMS");
  }
  s = atoms_config(sys, prm->p + prm->q, prm->arith, P->max_cl, t.threads, t.ctas_per_sm, &P->cf);
  if (s) {
    delete P;
    return s;
  }
  P->grid = (int)std::min<int64_t>(P->max_atoms, P->cf.grid_max);
  s = plan_alloc(P);
  if (s) {
    mka_plan_destroy(P);
    return s;
  }
  *out = P;
  return MKA_OK;
}

mka_status mka_plan_run(mka_plan* P, const int64_t* atoms, int64_t n_sel, double n_electrons, double kT,
                        double* rho_out) {
  PlanMode m;
  m.kind = PLAN_BATCH;
  m.n_electrons = n_electrons;
  m.kT = kT;
  m.rho = rho_out;
  return plan_run_mode(P, atoms, n_sel, m);
}

}  // extern "C"

int64_t mka::plan_max_atoms(const mka_plan* P) { return P->max_atoms; }

mka_status mka::plan_run_mode(mka_plan* P, const int64_t* atoms, int64_t n_sel, const PlanMode& m) {
  if (!P || !atoms || n_sel < 1 || n_sel > P->max_atoms)
    return fail(MKA_ERR_INVALID_ARG, "plan, host atoms and 1 <= n_sel <= max_atoms are required");
  if (m.kind != PLAN_SWEEP && !(m.kT > 0)) return fail(MKA_ERR_INVALID_ARG, "need kT > 0");
  const mka_system* sys = P->sys;
  for (int64_t t = 0; t < n_sel; ++t)
    if (atoms[t] < 0 || atoms[t] >= sys->n_atoms) return fail(MKA_ERR_INVALID_ARG, "atom index out of range");
  if (m.kind != PLAN_BATCH) {
    mka_status sc = sweep_check_atoms(m.sw, sys, P->prm.p + P->prm.q, atoms, n_sel);
    if (sc) return sc;
  }
  // the previous batch's copies must have read the staging buffer before it is refilled
  MKA_CUDA_TRY(cudaEventSynchronize(P->staged));
  int64_t* off = P->h_stage + P->max_atoms;
  off[0] = 0;
  for (int64_t t = 0; t < n_sel; ++t) {
    P->h_stage[t] = atoms[t];
    off[t + 1] = off[t] + (sys->h_row_ptr[atoms[t] + 1] - sys->h_row_ptr[atoms[t]]);
  }
  mka_result* r = P->res;
  r->n_sel = n_sel;
  r->n_cols = 4 * n_sel;
  r->n_blocks = off[n_sel];
  r->h_sel.assign(atoms, atoms + n_sel);
  r->h_blk_off.assign(off, off + n_sel + 1);
  GraphEntry* g = nullptr;
  for (auto& e : P->graphs)
    if (e.same(n_sel, m)) g = &e;
  if (!g) {
    cudaGraph_t graph = nullptr;
    const int64_t k0 = mka_kernel_launches();
    MKA_CUDA_TRY(cudaStreamBeginCapture(P->capture, cudaStreamCaptureModeThreadLocal));
    mka_status s = plan_enqueue(P, n_sel, m);
    cudaError_t e = cudaStreamEndCapture(P->capture, &graph);
    const int64_t kernels = mka_kernel_launches() - k0;
    count_launches(-kernels);    // captured, not executed
    if (s) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    GraphEntry ge;
    ge.n = n_sel;
    ge.kind = m.kind;
    ge.sw = m.sw;
    ge.n_electrons = m.n_electrons;
    ge.kT = m.kT;
    ge.mu = m.mu;
    ge.rho = m.rho;
    ge.forces = m.forces;
    ge.kernels = kernels;
    e = cudaGraphInstantiate(&ge.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    P->graphs.push_back(ge);
    g = &P->graphs.back();
  }
  if (m.kind != PLAN_BATCH) {
    mka_status sj = sweep_join_before(m.sw, P->stream);
    if (sj) return sj;
  }
  MKA_CUDA_TRY(cudaGraphLaunch(g->exec, P->stream));
  count_launches(g->kernels);
  MKA_CUDA_TRY(cudaEventRecord(P->staged, P->stream));
  if (m.kind != PLAN_BATCH) return sweep_join_after(m.sw, P->stream);
  return MKA_OK;
}

extern "C" {

mka_status mka_plan_scalars(mka_plan* P, double* mu, double* e_band, double* n_elec) {
  if (!P) return fail(MKA_ERR_INVALID_ARG, "plan is NULL");
  double h[3] = {0, 0, 0};
  const int64_t n = P->res->n_sel;
  MKA_CUDA_TRY(cudaMemcpyAsync(&h[0], P->dev_out, sizeof(double), cudaMemcpyDeviceToHost, P->stream));
  MKA_CUDA_TRY(cudaMemcpyAsync(&h[1], P->dev_out + 1 + n, 2 * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
  MKA_CUDA_TRY(cudaStreamSynchronize(P->stream));
  if (mu) *mu = h[0];
  if (e_band) *e_band = h[1];
  if (n_elec) *n_elec = h[2];
  return MKA_OK;
}

mka_status mka_plan_kernel_ms(mka_plan* P, float* atoms_ms, float* reduced_ms) {
  if (!P) return fail(MKA_ERR_INVALID_ARG, "plan is NULL");
  MKA_CUDA_TRY(cudaEventSynchronize(P->k2));
  if (atoms_ms) MKA_CUDA_TRY(cudaEventElapsedTime(atoms_ms, P->k0, P->k1));
  if (reduced_ms) MKA_CUDA_TRY(cudaEventElapsedTime(reduced_ms, P->k1, P->k2));
  return MKA_OK;
}

mka_status mka_plan_result(mka_plan* P, mka_result** res) {
  if (!P || !res) return fail(MKA_ERR_INVALID_ARG, "plan and res are required");
  *res = P->res;
  return MKA_OK;
}

mka_status mka_plan_info(const mka_plan* P, mka_tuning* tune, int* grid, int* ctas_per_sm_used) {
  if (!P) return fail(MKA_ERR_INVALID_ARG, "plan is NULL");
  if (tune) *tune = P->tune;
  if (grid) *grid = P->grid;
  if (ctas_per_sm_used) *ctas_per_sm_used = P->cf.per_sm;
  return MKA_OK;
}

mka_status mka_autotune(mka_system* sys, const mka_solve_params* prm, const int64_t* sample, int64_t n_sample,
                        double n_electrons, double kT, const char* cache_path, void* stream, mka_tuning* out) {
  if (!sys || !prm || !sample || n_sample < 1 || !out) return fail(MKA_ERR_INVALID_ARG, "bad autotune arguments");
  int dev = 0;
  cudaDeviceProp prop{};
  MKA_CUDA_TRY(cudaGetDevice(&dev));
  MKA_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
  std::vector<int32_t> sz(n_sample);
  mka_status s = mka_cluster_sizes(sys, sample, n_sample, sz.data());
  if (s) return s;
  const int max_cl = *std::max_element(sz.begin(), sz.end());
  std::ostringstream key;
  key << prop.name << "|storage=" << sys->storage << "|arith=" << prm->arith << "|nu=" << prm->p + prm->q
      << "|subspace=" << prm->subspace
      << "|maxcl=" << (max_cl / 16) * 16 << "|nsample=" << n_sample;
  const std::string k = key.str();
  std::vector<std::string> lines;
  if (cache_path) {
    std::ifstream f(cache_path);
    std::string line;
    while (std::getline(f, line)) {
      if (line.find("\"key\"") == std::string::npos) continue;
      lines.push_back(line);
      if (line.find("\"key\": \"" + k + "\"") != std::string::npos) {
        mka_tuning t{};
        if (sscanf(line.c_str() + line.find("\"threads\""), "\"threads\": %d, \"ctas_per_sm\": %d, \"order_by_size\": %d",
                   &t.threads, &t.ctas_per_sm, &t.order_by_size) == 3) {
          *out = t;
          return MKA_OK;
        }
      }
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int threads_c[3] = {128, 256, 512};
  const int ctas_c[3] = {0, 1, 2};
  double best = 1e300;
  mka_tuning best_t{256, 0, 0};
  cudaEvent_t e0, e1;
  MKA_CUDA_TRY(cudaEventCreate(&e0));
  MKA_CUDA_TRY(cudaEventCreate(&e1));
  for (int ti = 0; ti < 3; ++ti)
    for (int ci = 0; ci < 3; ++ci)
      for (int ord = 0; ord < 2; ++ord) {
        mka_tuning t{threads_c[ti], ctas_c[ci], ord};
        mka_plan* P = nullptr;
        if (mka_plan_create(sys, n_sample, prm, &t, stream, &P) != MKA_OK) continue;   // shape does not fit
        if (ctas_c[ci] > 0 && P->cf.per_sm < ctas_c[ci]) {   // same as a smaller cap
          mka_plan_destroy(P);
          continue;
        }
        float ms = 0, tot = 0;
        bool ok = mka_plan_run(P, sample, n_sample, n_electrons, kT, nullptr) == MKA_OK;   // capture + warm
        for (int rep = 0; ok && rep < 2; ++rep) {
          cudaEventRecord(e0, st);
          ok = mka_plan_run(P, sample, n_sample, n_electrons, kT, nullptr) == MKA_OK;
          cudaEventRecord(e1, st);
          cudaEventSynchronize(e1);
          cudaEventElapsedTime(&ms, e0, e1);
          tot += ms;
        }
        mka_plan_destroy(P);
        if (ok && tot < best) {
          best = tot;
          best_t = t;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *out = best_t;
  if (cache_path) {
    std::ofstream f(cache_path, std::ios::trunc);
    f << "{\"entries\": [\n";
    for (auto& l : lines) {
      if (l.find("\"key\": \"" + k + "\"") != std::string::npos) continue;
      std::string x = l;
      while (!x.empty() && (x.back() == ',' || x.back() == ' ')) x.pop_back();
      f << x << ",\n";
    }
    f << "{\"key\": \"" << k << "\", \"threads\": " << best_t.threads << ", \"ctas_per_sm\": " << best_t.ctas_per_sm
      << ", \"order_by_size\": " << best_t.order_by_size << ", \"ms\": " << best / 2.0 << "}\n]}\n";
  }
  return MKA_OK;
}

mka_status mka_autotune_batch(mka_system* sys, const mka_solve_params* prm, const mka_tuning* tune,
                              const int64_t* candidates, int n_candidates, int64_t first_atom,
                              double electrons_per_atom, double kT, const char* cache_path, void* stream,
                              int64_t* out_batch) {
  if (!sys || !prm || !candidates || n_candidates < 1 || !out_batch || first_atom < 0 || first_atom >= sys->n_atoms)
    return fail(MKA_ERR_INVALID_ARG, "bad batch-autotune arguments");
  for (int i = 0; i < n_candidates; ++i)
    if (candidates[i] < 1 || candidates[i] > sys->n_atoms) return fail(MKA_ERR_INVALID_ARG, "candidate batch out of range");
  mka_tuning t = tune ? *tune : mka_tuning{256, 0, 0};
  int dev = 0;
  cudaDeviceProp prop{};
  MKA_CUDA_TRY(cudaGetDevice(&dev));
  MKA_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
  std::ostringstream key;
  key << prop.name << "|storage=" << sys->storage << "|arith=" << prm->arith << "|nu=" << prm->p + prm->q
      << "|subspace=" << prm->subspace << "|atoms=" << sys->n_atoms << "|threads=" << t.threads
      << "|ctas=" << t.ctas_per_sm << "|order=" << t.order_by_size << "|batch_of";
  for (int i = 0; i < n_candidates; ++i) key << ":" << candidates[i];
  const std::string k = key.str();
  std::vector<std::string> lines;
  if (cache_path) {
    std::ifstream f(cache_path);
    std::string line;
    while (std::getline(f, line)) {
      if (line.find("\"key\"") == std::string::npos) continue;
      lines.push_back(line);
      if (line.find("\"key\": \"" + k + "\"") != std::string::npos) {
        long long b = 0;
        const size_t pos = line.find("\"batch\"");
        if (pos != std::string::npos && sscanf(line.c_str() + pos, "\"batch\": %lld", &b) == 1 && b > 0) {
          *out_batch = b;
          return MKA_OK;
        }
      }
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  MKA_CUDA_TRY(cudaEventCreate(&e0));
  MKA_CUDA_TRY(cudaEventCreate(&e1));
  double best = -1.0;
  int64_t best_b = candidates[0];
  std::vector<int64_t> atoms;
  for (int i = 0; i < n_candidates; ++i) {
    const int64_t B = candidates[i];
    atoms.resize(B);
    for (int64_t a = 0; a < B; ++a) atoms[a] = (first_atom + a) % sys->n_atoms;
    mka_plan* P = nullptr;
    if (mka_plan_create(sys, B, prm, &t, stream, &P) != MKA_OK) continue;   // does not fit
    bool ok = mka_plan_run(P, atoms.data(), B, electrons_per_atom * B, kT, nullptr) == MKA_OK;   // capture + warm
    float ms = 0;
    if (ok) {
      cudaEventRecord(e0, st);
      ok = mka_plan_run(P, atoms.data(), B, electrons_per_atom * B, kT, nullptr) == MKA_OK;
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
    }
    mka_plan_destroy(P);
    const double rate = ok && ms > 0 ? 4.0 * B / (ms / 1e3) : -1.0;
    if (rate > best) {
      best = rate;
      best_b = B;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best < 0) return fail(MKA_ERR_OOM, "no candidate batch size fits");
  *out_batch = best_b;
  if (cache_path) {
    std::ofstream f(cache_path, std::ios::trunc);
    f << "{\"entries\": [\n";
    for (auto& l : lines) {
      if (l.find("\"key\": \"" + k + "\"") != std::string::npos) continue;
      std::string x = l;
      while (!x.empty() && (x.back() == ',' || x.back() == ' ')) x.pop_back();
      f << x << ",\n";
    }
    f << "{\"key\": \"" << k << "\", \"batch\": " << best_b << ", \"columns_per_s\": " << best << "}\n]}\n";
  }
  return MKA_OK;
}

}  // extern "C"
