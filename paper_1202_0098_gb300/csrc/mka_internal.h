// Internal definitions shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/mka.h"

namespace mka {

// Thread-local error text for mka_last_error().
void set_error(const std::string& msg);
mka_status fail(mka_status st, const std::string& msg);
mka_status cuda_fail(cudaError_t e, const char* what);

#define MKA_CUDA_TRY(expr)                                   \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) return ::mka::cuda_fail(_e, #expr); \
  } while (0)

// Device-side periodic cell list used by the cluster extraction (radius R).
struct CellList {
  int n[3];            // cells per dimension, >= 1
  double len[3];       // cell edge (>= R)
  int32_t* start;      // device [ncells + 1]
  int32_t* atoms;      // device [n_atoms], atom ids grouped by cell, ascending inside a cell
};

}  // namespace mka

struct mka_system {
  int64_t n_atoms = 0;
  int64_t nnzb = 0;
  double box[3] = {0, 0, 0};
  double R = 0;                 // cluster radius
  int storage = MKA_FP64;
  int max_row_blocks = 0;
  cudaStream_t stream = nullptr;
  // device
  int32_t* d_row_ptr = nullptr;
  int32_t* d_col = nullptr;
  void* d_valH = nullptr;       // storage-typed [nnzb][16]
  void* d_valS = nullptr;
  double* d_pos = nullptr;      // [n_atoms][3], wrapped into the box
  float* d_posf = nullptr;      // the same rounded to FP32 (distance prefilter)
  mka_mlp* warm = nullptr;      // network used when a solve asks for the learned warm start (not owned)
  mka_sk_params sk{};           // the model's Slater-Koster parameters (forces need their derivatives)
  bool have_sk = false;         // false for a caller's BSR matrices: no forces
  int max_cluster = -1;         // largest cluster over all atoms (-1: not computed yet)
  mka::CellList cells{};
  // host copies of the pattern
  std::vector<int32_t> h_row_ptr, h_col;
};

typedef struct mka_plan mka_plan;
typedef struct mka_sweep mka_sweep;

struct mka_result {
  mka_system* sys = nullptr;
  cudaStream_t stream = nullptr;
  int64_t n_sel = 0;
  int64_t n_cols = 0;
  int nu = 0, p = 0, q = 0, arith = MKA_FP64;
  int keep = 0;
  int64_t n_blocks = 0;
  int64_t* d_sel = nullptr;       // selected atoms
  int64_t* d_blk_off = nullptr;   // [n_sel + 1] output block offsets
  double* d_eps = nullptr;        // [n_cols][nu]
  double* d_w = nullptr;          // [n_cols][nu]
  int32_t* d_nu_eff = nullptr;
  int32_t* d_cg_iters = nullptr;
  int32_t* d_status = nullptr;
  double* d_vp = nullptr;         // kept pattern rows of U [n_blocks][4 c][4 r][nu]
  double* d_cv = nullptr;         // kept C and V_j, lane-interleaved [n_cols / 32][kept_block_doubles][32]
  double* d_mu_state = nullptr;   // bisection bracket and partial sums
  int32_t* d_fallback = nullptr;  // [n_cols] warm-start fallback flags (learned start only)
  int s_cap = 0;                  // kept s_j: atoms per cluster slot (0: not kept)
  int32_t* d_s_cl = nullptr;      // [n_sel][s_cap] cluster atom ids, ascending, -1 beyond the count
  double* d_s = nullptr;          // [n_cols][4 s_cap] s_j on those atoms' orbitals
  std::vector<int64_t> h_sel;
  std::vector<int64_t> h_blk_off;
};

namespace mka {

// Configuration of the per-atom kernel for a system, subspace size, arithmetic and CTA size.
struct AtomsConfig {
  int threads = 256;       // CTA size
  int per_sm = 0;          // resident CTAs per SM used
  int grid_max = 0;        // SMs x per_sm
  size_t smem = 0;         // dynamic shared memory per CTA
  size_t slot_bytes = 0;   // global work slot per CTA
  int mcap = 0;            // 4 x largest cluster
  int lnnz_cap = 0;        // local block capacity
  int clcap = 0;           // cluster list capacity: the power of two at or above the largest cluster
};

// Arguments of one launch of the per-atom kernel over a selection.
struct AtomsLaunchArgs {
  const int64_t* sel = nullptr;    // device selected atoms
  const int32_t* order = nullptr;  // device work order (selection indices) or NULL
  int64_t n_sel = 0;
  int p = 0, q = 0;
  double cg_tol = 0;
  int cg_maxit = 0;
  double* eps = nullptr;
  double* w = nullptr;
  int32_t* nu_eff = nullptr;
  int32_t* cg_iters = nullptr;
  int32_t* status = nullptr;
  int keep = 0;
  double* vp = nullptr;
  const int64_t* blk_off = nullptr;
  char* scratch = nullptr;         // grid x slot_bytes
  int* counter = nullptr;          // zero in stream order before the launch
  int grid = 0;
  const float* x0 = nullptr;       // learned CG start on the patch [4 n_sel][68], or NULL
  const int32_t* patch = nullptr;  // [n_sel][17]
  int32_t* fallback = nullptr;     // [4 n_sel] or NULL
  int cg_only = 0;                 // 1: stop after CG, write s_j on the patch into cg_target
  int mode_b = 0;                  // 1: the literal direct sum K_p(H; e_j) + K_q(H; s_j)
  const int32_t* prev_cl = nullptr;  // earlier s_j as the CG start (see the kernel's Args)
  const double* prev_s = nullptr;
  int prev_cap = 0;
  int32_t* keep_cl = nullptr;        // keep this solve's s_j
  double* keep_s = nullptr;
  int keep_cap = 0;
  float* cg_target = nullptr;      // [4 n_sel][68]
  // reduced problems of the selection, lane-interleaved: [ceil(4 n_sel / 32)][red_block_doubles(nu)][32]
  // (not used with cg_only)
  double* red = nullptr;
  // kept C and V_j (NULL: not kept), lane-interleaved by absolute column index col0 + local column
  double* cv = nullptr;
  int64_t col0 = 0;
};

// Per-column doubles of the reduced-problem buffer: H_r and S_r (nu x nu each), then the
// row j of U and of S U (nu each), then nu x nu of scratch for the reduced kernel (the
// eigenvectors of the tridiagonal matrix).
__host__ __device__ constexpr size_t red_block_doubles(int nu) { return (size_t)3 * nu * nu + (size_t)2 * nu; }
// Per-column doubles of the kept reduced solution: C (nu x nu, columns in ascending order of
// eps) and the row V_j = (row j of U) C; rho_ij = U_i . (C diag(f) V_j).
__host__ __device__ constexpr size_t kept_block_doubles(int nu) { return (size_t)nu * nu + (size_t)nu; }
inline size_t kept_buffer_bytes(int64_t n_cols, int nu) {
  return sizeof(double) * kept_block_doubles(nu) * 32 * (size_t)((n_cols + 31) / 32);
}
// Bytes of the reduced-problem buffer for n_cols columns.
inline size_t red_buffer_bytes(int64_t n_cols, int nu) {
  return sizeof(double) * red_block_doubles(nu) * 32 * (size_t)((n_cols + 31) / 32);
}
// The batched reduced problems (reduced.cu): one lane per column over the buffer filled by
// the per-atom kernel; writes eps, w (ranked), the final status and nu_eff, and (cv != NULL)
// the kept C and V_j of column col0 + c.
mka_status reduced_launch(double* red, int64_t n_cols, int nu, int32_t* status, int32_t* nu_eff, double* eps,
                          double* w, double* cv, int64_t col0, cudaStream_t st);

// Learned warm start (mlp.cu).
mka_status features_enqueue(const mka_system* sys, const int64_t* d_sel, int64_t n, float* X, int32_t* patch,
                            cudaStream_t st);
mka_status mlp_forward_enqueue(const mka_mlp* net, const float* X, int64_t B, float* Z1, float* H1, float* Z2,
                               float* H2, float* Y, cudaStream_t st);
int64_t mlp_work_floats(int64_t B);   // floats of forward/backward work buffers for B rows

mka_status atoms_config(const mka_system* sys, int nu, int arith, int max_cl, int threads, int ctas_per_sm,
                        AtomsConfig* out);
// The batched reduced problems of a selection the per-atom kernel has just processed.
mka_status reduced_for(const mka_system* sys, const AtomsLaunchArgs& a, cudaStream_t st);
mka_status atoms_launch(const mka_system* sys, int arith, const AtomsConfig& cf, const AtomsLaunchArgs& a,
                        cudaStream_t st);

// Kernels launched from the C entry points (defined in the .cu files).
mka_status launch_cluster_sizes(const mka_system* sys, const int64_t* d_sel, int64_t n_sel, int32_t* d_sizes,
                                cudaStream_t st);
mka_status launch_columns(mka_system* sys, mka_result* res, const mka_solve_params* prm, int max_cluster_atoms,
                          cudaStream_t st);
mka_status launch_find_mu(mka_result* res, double n_electrons, double kT, double tol, double* mu_out);
mka_status launch_density(mka_system* sys, mka_result* res, double mu, double kT, double* rho_out,
                          double* e_band, double* n_elec);
mka_status launch_greens(mka_system* sys, mka_result* res, double z_re, double z_im, double* g_out);
mka_status launch_spmv(const mka_system* sys, int which, int x_dtype, const void* x, void* y, int k,
                       cudaStream_t st);
mka_status launch_onsite_shift(mka_system* sys, const double* shift_host, cudaStream_t st);
mka_status launch_dos(const double* eps, const double* w, int64_t n, const double* energies, int n_e, double eta,
                      cudaStream_t st, double* dos_host);

// Stream-ordered (no host synchronisation, no allocation) variants used by plans and graphs.
size_t mu_buffer_bytes();
mka_status find_mu_enqueue(const double* eps, const double* w, int64_t n, double n_electrons, double kT, double tol,
                           int halvings, void* buf, double* mu_dev_out, cudaStream_t st);
mka_status density_enqueue(const mka_system* sys, const int64_t* sel, const int64_t* blk_off, const double* vp,
                           const double* cv, const double* eps, const double* w, int64_t n_sel, int nu,
                           const double* mu_dev, double kT, double* rho_out, double* tmp, cudaStream_t st);
// rho at a host mu into the system's pattern order (blocks from out_base on) and 2 sum rho H per atom
// into e_atom[atom - e_base].
mka_status density_global_enqueue(const mka_system* sys, const int64_t* sel, const int64_t* blk_off, const double* vp,
                                  const double* cv, const double* eps, int64_t n_sel, int nu, double mu, double kT,
                                  double* rho, int64_t out_base, double* e_atom, int64_t e_base, cudaStream_t st);
// Largest grid of the fixed-order reductions (4 CTAs per SM); sizes their partial-sum buffers.
constexpr int kMaxRedBlocks = 4096;
// tmp of density_enqueue holds n_sel + 2 + kDensityTmpExtra doubles.
constexpr int kDensityTmpExtra = kMaxRedBlocks;

size_t storage_bytes(int storage);

// ---- whole-system sweeps (sweep.cu) ----
// What a plan does with a batch after its column kernels.
enum PlanModeKind { PLAN_BATCH = 0, PLAN_SWEEP = 1, PLAN_AT_MU = 2 };
struct PlanMode {
  int kind = PLAN_BATCH;
  mka_sweep* sw = nullptr;     // PLAN_SWEEP / PLAN_AT_MU: the sweep the batch belongs to
  double mu = 0;               // PLAN_AT_MU: chemical potential
  double kT = 0;               // PLAN_BATCH / PLAN_AT_MU
  double n_electrons = 0;      // PLAN_BATCH
  double* rho = nullptr;       // PLAN_BATCH: batch layout; PLAN_AT_MU: the sweep's global layout
  bool forces = false;         // PLAN_AT_MU: force contributions of the batch's blocks instead of rho
};
// Runs one batch of a plan in the given mode (validation, staging, graph capture / replay).
mka_status plan_run_mode(mka_plan* P, const int64_t* atoms, int64_t n_sel, const PlanMode& m);
// Largest batch of a plan.
int64_t plan_max_atoms(const mka_plan* P);
// Kernels a plan captures for a sweep: pack the batch's kept data into the sweep (levels, window,
// occupied sum, partially occupied products), or write rho at a given mu into the sweep's layout.
mka_status sweep_pack_enqueue(mka_sweep* sw, const int64_t* sel, const int64_t* blk_off, const double* vp,
                              const double* cv, const double* eps, const double* w, const int32_t* nu_eff,
                              int64_t n_sel, int nu, cudaStream_t st);
mka_status sweep_at_mu_enqueue(mka_sweep* sw, const int64_t* sel, const int64_t* blk_off, const double* vp,
                               const double* cv, const double* eps, int64_t n_sel, int nu, double mu, double kT,
                               double* rho, bool forces, cudaStream_t st);
// Forces (forces.cu): per-block contributions g = -2 sum_{c,r} (rho dH/dd - pi dS/dd) of the selected atoms'
// blocks (batch layout when out_base < 0, else the system's blocks from out_base on), pi on the pattern
// (may be NULL); and F_K from the blocks of atoms [a0, a1) for every atom of the system.
mka_status force_blocks_enqueue(const mka_system* sys, const int64_t* sel, const int64_t* blk_off, const double* vp,
                                const double* cv, const double* eps, int64_t n_sel, int nu, double mu, double kT,
                                int64_t out_base, double* pi, double* g, cudaStream_t st);
mka_status force_gather_enqueue(const mka_system* sys, const double* g, int64_t a0, int64_t a1, int64_t blk0, double* F,
                                cudaStream_t st);
// Stream ordering between a sweep's stream and a plan's stream around a plan's batch.
mka_status sweep_join_before(mka_sweep* sw, cudaStream_t plan_stream);
mka_status sweep_join_after(mka_sweep* sw, cudaStream_t plan_stream);
// Host-side check of a batch against the sweep's atom range.
mka_status sweep_check_atoms(const mka_sweep* sw, const mka_system* sys, int nu, const int64_t* atoms, int64_t n);

// Kernel launches of this library (mka_kernel_launches).
extern std::atomic<int64_t> g_kernel_launches;
inline void count_launches(int64_t n = 1) { g_kernel_launches.fetch_add(n, std::memory_order_relaxed); }

}  // namespace mka
