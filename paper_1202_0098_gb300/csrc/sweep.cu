// Whole-system sweeps: every column's levels, one chemical potential, then rho (Eq. EQ-WORK-FLOW).
//
// A plan solves the system batch by batch; after each batch's column kernels a packing kernel
// stores, at the system's own positions:
//   - the levels eps_alpha and weights w_alpha of every column (what the bisection for mu needs);
//   - for every pattern entry (i, j) the occupied part sum_{eps_alpha < win_lo} v_alpha,i v_alpha,j
//     and the products v_alpha,i v_alpha,j of the (at most kp) levels inside [win_lo, win_hi].
// The Fermi-Dirac occupation f(x) = (1 - tanh((x - mu) / 2kT)) / 2 is exactly 1 in FP64 for
// x < mu - 40 kT and exactly 0 for x > mu + 40 kT, so for any mu in [win_lo + 40 kT, win_hi - 40 kT]
// rho_ij(mu) = occupied + sum_window f(eps_alpha) v_alpha,i v_alpha,j is Eq. EQ-DM with only the
// rounding order changed, and rho costs one pass over HBM instead of a second solve of every
// column. Atoms whose columns have more than kp levels in the window, and all atoms when mu is
// outside that range, are solved again at mu.
//
// Sums (electron count, band energy) run per chunk of consecutive atoms of the whole system, in a
// fixed order inside the chunk (thread-strided, then a fixed tree), and the chunk sums are added in
// chunk order. A process that sweeps a range starting on a chunk boundary therefore reproduces a
// whole-system process's chunk sums exactly, and the bisection (Sec. 2) gives the same mu.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "mka_internal.h"
#include "sk_grad.cuh"

namespace mka {
namespace {

constexpr int kChunkThreads = 256;
constexpr int kRangeBlocks = 1024;
constexpr int kMaxHalvings = 200;

// The root finder's state: the bracket [lo, hi] with f = N - N_e at its ends, the next point x, the
// side that moved last (-1 lo, +1 hi) and whether x came from the secant (rf).
struct BisState {
  double lo, hi, target, kT, tol, last, iters, x, flo, fhi, side, rf;
};
constexpr double kSecantKT = 16.0;   // bisection while the bracket is wider than this many kT

__device__ __forceinline__ double fermi_f(double x, double mu, double r2kT) {   // r2kT = 1 / (2 kT)
  const double y = (x - mu) * r2kT;
  if (y > 20.0) return 0.0;
  if (y < -20.0) return 1.0;
  return 0.5 * (1.0 - tanh(y));
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order sum over the CTA (warp xor trees, then the warps' sums in warp order); valid in thread 0.
__device__ __forceinline__ double cta_sum(double v, double* red) {
  v = warp_sum_t(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
  __syncthreads();
  return s;
}

struct PackArgs {
  const int64_t* sel;
  const int64_t* blk_off;
  const double* vp;
  const double* cv;
  const double* eps;
  const double* w;
  const int32_t* nu_eff;
  const int32_t* row_ptr;
  int nu, kp;
  double win_lo, win_hi;
  int64_t a0, blk0;
  double* g_eps;
  double* g_w;
  uint16_t* g_win;
  uint8_t* g_flag;
  double* g_occ;
  double* g_part;
  double* g_occ_pi;          // occupied part of pi (NULL: not kept)
};

// One CTA per atom of the batch. Shared memory: g_below [4][nu] = C diag(1_below) V_j and
// W [4][nu][kp] = C[:, window] diag(V_j[window]), so that for a kept pattern row U_i of the basis
// occupied = U_i . g_below and product_a = U_i . W[:, a].
__global__ void __launch_bounds__(128) sweep_pack_kernel(const PackArgs A) {
  extern __shared__ double sm[];
  __shared__ int s_lo[4], s_cnt[4], s_over;
  const int nu = A.nu, kp = A.kp;
  const int64_t t = blockIdx.x;
  const int64_t atom = A.sel[t];
  const int64_t la = atom - A.a0;
  for (int i = threadIdx.x; i < 4 * nu; i += blockDim.x) {
    A.g_eps[4 * la * nu + i] = A.eps[4 * t * nu + i];
    A.g_w[4 * la * nu + i] = A.w[4 * t * nu + i];
  }
  if (threadIdx.x < 4) {
    const int c = threadIdx.x;
    const int ne = A.nu_eff[4 * t + c];
    const double* e = A.eps + (4 * t + c) * nu;
    int lo = 0, hi = 0;
    for (int a = 0; a < ne; ++a) {      // levels ascend: below the window, then inside it
      lo += e[a] < A.win_lo;
      hi += e[a] <= A.win_hi;
    }
    s_lo[c] = lo;
    s_cnt[c] = hi - lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) s_over = (s_cnt[0] > kp) || (s_cnt[1] > kp) || (s_cnt[2] > kp) || (s_cnt[3] > kp);
  __syncthreads();
  if (s_over) {                         // solved again at mu; nothing of rho is stored
    if (threadIdx.x < 4) {
      A.g_win[2 * (4 * la + threadIdx.x)] = 0;
      A.g_win[2 * (4 * la + threadIdx.x) + 1] = 0;
    }
    if (threadIdx.x == 0) A.g_flag[la] = 3;
    return;
  }
  double* gb = sm;
  double* W = sm + 4 * nu;
  double* gbp = W + (size_t)4 * nu * kp;     // pi's occupied part: C diag(eps 1_below) V_j
  for (int i = threadIdx.x; i < 4 * nu; i += blockDim.x) {
    const int c = i / nu, n = i % nu;
    const int64_t col = 4 * t + c;
    const double* b = A.cv + (size_t)(col >> 5) * kept_block_doubles(nu) * 32 + (col & 31);
    const int lo = s_lo[c], cnt = s_cnt[c];
    const double* ec = A.eps + (4 * t + c) * nu;
    double g = 0.0, gp = 0.0;
    for (int a = 0; a < lo; ++a) {
      const double cv = b[(size_t)(n * nu + a) * 32] * b[(size_t)(nu * nu + a) * 32];
      g += cv;
      gp += cv * ec[a];
    }
    gb[i] = g;
    if (A.g_occ_pi) gbp[i] = gp;
    for (int a = 0; a < kp; ++a)
      W[(size_t)(c * nu + n) * kp + a] =
          a < cnt ? b[(size_t)(n * nu + lo + a) * 32] * b[(size_t)(nu * nu + lo + a) * 32] : 0.0;
  }
  if (threadIdx.x < 4) {
    A.g_win[2 * (4 * la + threadIdx.x)] = (uint16_t)s_lo[threadIdx.x];
    A.g_win[2 * (4 * la + threadIdx.x) + 1] = (uint16_t)s_cnt[threadIdx.x];
  }
  __syncthreads();
  const int nrow = A.row_ptr[atom + 1] - A.row_ptr[atom];
  const int64_t gk0 = (int64_t)A.row_ptr[atom] - A.blk0;
  const int64_t bk0 = A.blk_off[t];
  for (int i = threadIdx.x; i < nrow * 16; i += blockDim.x) {
    const int k = i >> 4, c = (i >> 2) & 3, r = i & 3;
    const double* u = A.vp + ((bk0 + k) * 16 + c * 4 + r) * (int64_t)nu;
    const double* g = gb + c * nu;
    const double* Wc = W + (size_t)c * nu * kp;
    double occ = 0.0;
    for (int n = 0; n < nu; ++n) occ += u[n] * g[n];
    const int64_t e = (gk0 + k) * 16 + c * 4 + r;
    A.g_occ[e] = occ;
    if (A.g_occ_pi) {
      const double* gp = gbp + c * nu;
      double op = 0.0;
      for (int n = 0; n < nu; ++n) op += u[n] * gp[n];
      A.g_occ_pi[e] = op;
    }
    double* out = A.g_part + e * kp;
    for (int a = 0; a < kp; ++a) {
      double s = 0.0;
      for (int n = 0; n < nu; ++n) s += u[n] * Wc[n * kp + a];
      out[a] = s;
    }
  }
  if (threadIdx.x == 0) A.g_flag[la] = 1;
}

// Stored and overflowed atoms of the range (integer counts: the order does not matter).
__global__ void sweep_flag_count_kernel(const uint8_t* flag, int64_t n, unsigned long long* out) {
  unsigned long long st = 0, ov = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    st += flag[i] & 1;
    ov += (flag[i] >> 1) & 1;
  }
  st = warp_sum_t(st);
  ov = warp_sum_t(ov);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out, st);
    atomicAdd(out + 1, ov);
  }
}

// Per-block min / max of the levels with nonzero weight.
__global__ void sweep_range_kernel(const double* eps, const double* w, int64_t n, double* partial) {
  __shared__ double rmin[32], rmax[32];
  double mn = INFINITY, mx = -INFINITY;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (w[i] != 0.0) {
      mn = fmin(mn, eps[i]);
      mx = fmax(mx, eps[i]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    rmin[threadIdx.x >> 5] = mn;
    rmax[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      mn = fmin(mn, rmin[k]);
      mx = fmax(mx, rmax[k]);
    }
    partial[2 * blockIdx.x] = mn;
    partial[2 * blockIdx.x + 1] = mx;
  }
}

struct ChunkArgs {
  const double* eps;
  const double* w;
  const double* eatom;
  int nu;
  int64_t a0, a1, chunk_atoms, chunk0;
  double mu;                 // used when S == NULL
  const BisState* S;         // root finder: mu = the state's next point; nothing once converged
  double kT;
  double* count;             // [n_chunks] 2 sum f w
  double* e_levels;          // [n_chunks] 2 sum f eps w (may be NULL)
  double* e_rho;             // [n_chunks] sum of the atoms' 2 sum rho H (may be NULL)
};

// One CTA per chunk: entries of the chunk's atoms, thread t takes chunk-relative entries t, t + 256, ...
__global__ void __launch_bounds__(kChunkThreads) sweep_chunk_kernel(const ChunkArgs A) {
  __shared__ double red[kChunkThreads / 32];
  double mu = A.mu, kT = A.kT;
  if (A.S) {
    if (!(A.S->hi - A.S->lo > A.S->tol)) return;
    mu = A.S->x;
    kT = A.S->kT;
  }
  const double r2kT = 0.5 / kT;        // one division per thread, a product per level
  const int64_t gi = blockIdx.x;
  const int64_t g = A.chunk0 + gi;
  const int64_t lo = max(A.a0, g * A.chunk_atoms), hi = min(A.a1, (g + 1) * A.chunk_atoms);
  const int64_t e0 = 4 * (lo - A.a0) * A.nu, e1 = 4 * (hi - A.a0) * A.nu;
  double c = 0.0, el = 0.0, er = 0.0;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const double wi = A.w[e];
    if (wi != 0.0) {
      const double x = A.eps[e];
      const double f = fermi_f(x, mu, r2kT);
      c += f * wi;
      if (A.e_levels) el += f * x * wi;
    }
  }
  if (A.e_rho)
    for (int64_t a = lo - A.a0 + threadIdx.x; a < hi - A.a0; a += blockDim.x) er += A.eatom[a];
  const double cs = cta_sum(c, red);
  const double es = A.e_levels ? cta_sum(el, red) : 0.0;
  const double rs = A.e_rho ? cta_sum(er, red) : 0.0;
  if (threadIdx.x == 0) {
    A.count[gi] = 2.0 * cs;
    if (A.e_levels) A.e_levels[gi] = 2.0 * es;
    if (A.e_rho) A.e_rho[gi] = rs;
  }
}

// One step of the root finder for N(mu) = N_e: the count at x is the chunk sums added in chunk order;
// the bracket end on its side moves to x. The next point is the midpoint while the bracket is wider
// than 16 kT, then the secant through the ends (regula falsi, with the Illinois rule: after two moves
// of the same end by the secant, the other end's f is halved), the midpoint when the secant leaves the
// bracket; a point where the count equals N_e exactly closes the bracket on it. IEEE-rounded
// operations throughout (no contraction), so that a host driver doing the same
// arithmetic on the same chunk sums takes the same points bit for bit.
__global__ void sweep_bisect_step_kernel(const double* count, int64_t n_chunks, BisState* S) {
  if (!(S->hi - S->lo > S->tol)) return;
  double t = 0.0;
  for (int64_t k = 0; k < n_chunks; ++k) t += count[k];
  const double x = S->x, fx = __dsub_rn(t, S->target);
  if (fx == 0.0) {                     // x is a root to rounding: the bracket closes on it
    S->lo = x;
    S->hi = x;
    S->flo = 0.0;
    S->fhi = 0.0;
    S->last = t;
    S->iters += 1;
    return;
  }
  if (fx < 0.0) {
    S->lo = x;
    S->flo = fx;
    if (S->rf != 0.0 && S->side == -1.0) S->fhi = __dmul_rn(0.5, S->fhi);
    S->side = -1.0;
  } else {
    S->hi = x;
    S->fhi = fx;
    if (S->rf != 0.0 && S->side == 1.0) S->flo = __dmul_rn(0.5, S->flo);
    S->side = 1.0;
  }
  S->last = t;
  S->iters += 1;
  const double lo = S->lo, hi = S->hi, mid = __dmul_rn(0.5, __dadd_rn(lo, hi));
  double nx = mid, rf = 0.0;
  if (!(__dsub_rn(hi, lo) > __dmul_rn(kSecantKT, S->kT))) {
    const double sx = __ddiv_rn(__dsub_rn(__dmul_rn(lo, S->fhi), __dmul_rn(hi, S->flo)), __dsub_rn(S->fhi, S->flo));
    if (lo < sx && sx < hi) {
      nx = sx;
      rf = 1.0;
    }
  }
  S->x = nx;
  S->rf = rf;
}

struct RhoArgs {
  const double* eps;
  const uint16_t* win;
  const uint8_t* flag;
  const double* occ;
  const double* part;
  const int32_t* row_ptr;
  const void* valH;
  int storage;
  int nu, kp;
  int64_t a0, n, blk0;
  double mu, kT;
  double* rho;
  double* eatom;
};

__device__ __forceinline__ double h_value(const void* v, int storage, int64_t i) {
  if (storage == MKA_FP64) return reinterpret_cast<const double*>(v)[i];
  if (storage == MKA_MIXED_FP32) return reinterpret_cast<const float*>(v)[i];
  return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(v)[i]);
}

// rho from the stored pieces: one warp per atom, lanes over its 16 x (row length) entries; the
// window's occupations in shared memory [warp][4][kp]; 2 sum rho H per atom.
__global__ void __launch_bounds__(256) sweep_rho_kernel(const RhoArgs A) {
  extern __shared__ double fsm[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int kp = A.kp, nu = A.nu;
  double* f = fsm + (size_t)wid * 4 * kp;
  for (int64_t la = (int64_t)blockIdx.x * nw + wid; la < A.n; la += (int64_t)gridDim.x * nw) {
    if (A.flag[la] != 1) continue;     // overflowed: solved again instead
    for (int i = lane; i < 4 * kp; i += 32) {
      const int c = i / kp, a = i % kp;
      const uint16_t* wn = A.win + 2 * (4 * la + c);
      f[i] = a < wn[1] ? fermi_f(A.eps[(4 * la + c) * nu + wn[0] + a], A.mu, 0.5 / A.kT) : 0.0;
    }
    __syncwarp();
    const int64_t atom = A.a0 + la;
    const int64_t k0 = A.row_ptr[atom];
    const int nrow = A.row_ptr[atom + 1] - (int)k0;
    const int64_t gk0 = k0 - A.blk0;
    double e = 0.0;
    for (int i = lane; i < nrow * 16; i += 32) {
      const int k = i >> 4, c = (i >> 2) & 3;
      const int64_t idx = (gk0 + k) * 16 + (i & 15);
      double s = A.occ[idx];
      const double* p = A.part + idx * kp;
      for (int a = 0; a < kp; ++a) s += f[c * kp + a] * p[a];
      A.rho[idx] = s;
      e += s * h_value(A.valH, A.storage, (k0 + k) * 16 + (i & 15));
    }
    e = warp_sum_t(e);
    if (lane == 0) A.eatom[la] = 2.0 * e;
    __syncwarp();
  }
}

// Forces from the stored pieces: one warp per atom, lanes 0-15 on one block's 16 entries and 16-31 on the
// next; rho and pi at mu, the entries' contributions -2 (rho dH/dd - pi dS/dd) summed per block by a fixed
// xor tree into g[block] (3 doubles).
struct ForceArgs {
  const double* eps;
  const uint16_t* win;
  const uint8_t* flag;
  const double* occ;
  const double* occ_pi;
  const double* part;
  const int32_t* row_ptr;
  const int32_t* col;
  const double* pos;
  double box[3];
  double Vh[4], Vs[4], d0;
  int nu, kp;
  int64_t a0, n, blk0;
  double mu, kT;
  double* g;
};

__global__ void __launch_bounds__(256) sweep_force_kernel(const ForceArgs A) {
  extern __shared__ double fsm[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int kp = A.kp, nu = A.nu;
  double* f = fsm + (size_t)wid * 8 * kp;         // [4][kp] occupations, then [4][kp] f eps
  double* fe = f + 4 * kp;
  for (int64_t la = (int64_t)blockIdx.x * nw + wid; la < A.n; la += (int64_t)gridDim.x * nw) {
    if (A.flag[la] != 1) continue;
    for (int i = lane; i < 4 * kp; i += 32) {
      const int c = i / kp, a = i % kp;
      const uint16_t* wn = A.win + 2 * (4 * la + c);
      const double x = a < wn[1] ? A.eps[(4 * la + c) * nu + wn[0] + a] : 0.0;
      const double fx = a < wn[1] ? fermi_f(x, A.mu, 0.5 / A.kT) : 0.0;
      f[i] = fx;
      fe[i] = fx * x;
    }
    __syncwarp();
    const int64_t atom = A.a0 + la;
    const int64_t k0 = A.row_ptr[atom];
    const int nrow = A.row_ptr[atom + 1] - (int)k0;
    const int64_t gk0 = k0 - A.blk0;
    const double ax = A.pos[3 * atom], ay = A.pos[3 * atom + 1], az = A.pos[3 * atom + 2];
    for (int base = 0; base < nrow * 16; base += 32) {
      const int i = base + lane;
      const bool on = i < nrow * 16;
      const int k = i >> 4, c = (i >> 2) & 3, r = i & 3;
      double e[3] = {0.0, 0.0, 0.0};
      if (on) {
        const int64_t idx = (gk0 + k) * 16 + (i & 15);
        double rho = A.occ[idx], pi = A.occ_pi[idx];
        const double* p = A.part + idx * kp;
        for (int a = 0; a < kp; ++a) {
          rho += f[c * kp + a] * p[a];
          pi += fe[c * kp + a] * p[a];
        }
        const int64_t b = A.col[k0 + k];
        if (b != atom) {
          double d[3] = {A.pos[3 * b] - ax, A.pos[3 * b + 1] - ay, A.pos[3 * b + 2] - az};
          for (int q = 0; q < 3; ++q) d[q] -= A.box[q] * rint(d[q] / A.box[q]);
          double gh[3], gs[3];
          sk_entry_grad(d, A.Vh, A.d0, c, r, gh);
          sk_entry_grad(d, A.Vs, A.d0, c, r, gs);
          for (int q = 0; q < 3; ++q) e[q] = -2.0 * (rho * gh[q] - pi * gs[q]);
        }
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < 3; ++q) e[q] += __shfl_xor_sync(0xffffffffu, e[q], o);
      if (on && (lane & 15) == 0)
        for (int q = 0; q < 3; ++q) A.g[(gk0 + k) * 3 + q] = e[q];
    }
    __syncwarp();
  }
}

size_t pack_smem_bytes(int nu, int kp) { return sizeof(double) * 4 * (size_t)nu * (kp + 2); }

}  // namespace
}  // namespace mka

struct mka_sweep {
  mka_system* sys = nullptr;
  cudaStream_t stream = nullptr;
  int nu = 0, kp = 0;
  double win_lo = 0, win_hi = 0;
  int64_t a0 = 0, a1 = 0, n = 0;        // atom range [a0, a1), n = a1 - a0
  int64_t blk0 = 0, nblk = 0;           // pattern blocks of the range
  int64_t chunk_atoms = 0, chunk0 = 0, n_chunks = 0;
  double* d_eps = nullptr;              // [4 n][nu]
  double* d_w = nullptr;
  uint16_t* d_win = nullptr;            // [4 n][2]: first window level, count
  uint8_t* d_flag = nullptr;            // [n]: 1 stored, 3 stored and overflowed
  double* d_occ = nullptr;              // [nblk][16]
  double* d_part = nullptr;             // [nblk][16][kp]
  double* d_eatom = nullptr;            // [n] 2 sum rho H of the atom's columns (after a density)
  double* d_occ_pi = nullptr;           // [nblk][16] occupied part of pi (sweeps made for forces)
  double* d_g = nullptr;                // [nblk][3] force contribution of each block
  double* d_chunk = nullptr;            // [3][n_chunks]
  double* d_range = nullptr;            // [2 kRangeBlocks]
  mka::BisState* d_state = nullptr;
  unsigned long long* d_counts = nullptr;
  cudaEvent_t ev = nullptr;
  double rho_mu = NAN, rho_kT = NAN;
  int64_t bytes = 0;
};

using namespace mka;

namespace mka {

mka_status sweep_check_atoms(const mka_sweep* sw, const mka_system* sys, int nu, const int64_t* atoms, int64_t n) {
  if (sw->sys != sys) return fail(MKA_ERR_INVALID_ARG, "the plan and the sweep belong to different systems");
  if (sw->nu != nu) return fail(MKA_ERR_INVALID_ARG, "the plan's p + q differs from the sweep's nu");
  for (int64_t t = 0; t < n; ++t)
    if (atoms[t] < sw->a0 || atoms[t] >= sw->a1) return fail(MKA_ERR_INVALID_ARG, "atom outside the sweep's range");
  return MKA_OK;
}

mka_status sweep_pack_enqueue(mka_sweep* sw, const int64_t* sel, const int64_t* blk_off, const double* vp,
                              const double* cv, const double* eps, const double* w, const int32_t* nu_eff,
                              int64_t n_sel, int nu, cudaStream_t st) {
  PackArgs A{};
  A.sel = sel;
  A.blk_off = blk_off;
  A.vp = vp;
  A.cv = cv;
  A.eps = eps;
  A.w = w;
  A.nu_eff = nu_eff;
  A.row_ptr = sw->sys->d_row_ptr;
  A.nu = nu;
  A.kp = sw->kp;
  A.win_lo = sw->win_lo;
  A.win_hi = sw->win_hi;
  A.a0 = sw->a0;
  A.blk0 = sw->blk0;
  A.g_eps = sw->d_eps;
  A.g_w = sw->d_w;
  A.g_win = sw->d_win;
  A.g_flag = sw->d_flag;
  A.g_occ = sw->d_occ;
  A.g_part = sw->d_part;
  A.g_occ_pi = sw->d_occ_pi;
  sweep_pack_kernel<<<(unsigned)n_sel, 128, pack_smem_bytes(nu, sw->kp), st>>>(A);
  count_launches();
  MKA_CUDA_TRY(cudaGetLastError());
  return MKA_OK;
}

mka_status sweep_at_mu_enqueue(mka_sweep* sw, const int64_t* sel, const int64_t* blk_off, const double* vp,
                               const double* cv, const double* eps, int64_t n_sel, int nu, double mu, double kT,
                               double* rho, bool forces, cudaStream_t st) {
  if (forces)
    return force_blocks_enqueue(sw->sys, sel, blk_off, vp, cv, eps, n_sel, nu, mu, kT, sw->blk0, nullptr, sw->d_g, st);
  return density_global_enqueue(sw->sys, sel, blk_off, vp, cv, eps, n_sel, nu, mu, kT, rho, sw->blk0, sw->d_eatom,
                                sw->a0, st);
}

}  // namespace mka

namespace {

// Work on `from` before this point is ordered before later work on `to`.
mka_status join(cudaStream_t from, cudaStream_t to, cudaEvent_t ev) {
  if (from == to) return MKA_OK;
  MKA_CUDA_TRY(cudaEventRecord(ev, from));
  MKA_CUDA_TRY(cudaStreamWaitEvent(to, ev, 0));
  return MKA_OK;
}

mka_status flag_counts(mka_sweep* sw, int64_t* stored, int64_t* overflow) {
  cudaStream_t st = sw->stream;
  MKA_CUDA_TRY(cudaMemsetAsync(sw->d_counts, 0, 2 * sizeof(unsigned long long), st));
  const int blocks = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (sw->n + 255) / 256));
  sweep_flag_count_kernel<<<blocks, 256, 0, st>>>(sw->d_flag, sw->n, sw->d_counts);
  count_launches();
  MKA_CUDA_TRY(cudaGetLastError());
  unsigned long long h[2];
  MKA_CUDA_TRY(cudaMemcpyAsync(h, sw->d_counts, sizeof(h), cudaMemcpyDeviceToHost, st));
  MKA_CUDA_TRY(cudaStreamSynchronize(st));
  if (stored) *stored = (int64_t)h[0];
  if (overflow) *overflow = (int64_t)h[1];
  return MKA_OK;
}

mka_status chunk_launch(mka_sweep* sw, double mu, double kT, const BisState* S, bool levels, bool rho) {
  ChunkArgs A{};
  A.eps = sw->d_eps;
  A.w = sw->d_w;
  A.eatom = sw->d_eatom;
  A.nu = sw->nu;
  A.a0 = sw->a0;
  A.a1 = sw->a1;
  A.chunk_atoms = sw->chunk_atoms;
  A.chunk0 = sw->chunk0;
  A.mu = mu;
  A.S = S;
  A.kT = kT;
  A.count = sw->d_chunk;
  A.e_levels = levels ? sw->d_chunk + sw->n_chunks : nullptr;
  A.e_rho = rho ? sw->d_chunk + 2 * sw->n_chunks : nullptr;
  sweep_chunk_kernel<<<(unsigned)sw->n_chunks, kChunkThreads, 0, sw->stream>>>(A);
  count_launches();
  MKA_CUDA_TRY(cudaGetLastError());
  return MKA_OK;
}

}  // namespace

extern "C" {

void mka_sweep_destroy(mka_sweep* sw) {
  if (!sw) return;
  cudaFree(sw->d_eps);
  cudaFree(sw->d_w);
  cudaFree(sw->d_win);
  cudaFree(sw->d_flag);
  cudaFree(sw->d_occ);
  cudaFree(sw->d_part);
  cudaFree(sw->d_eatom);
  cudaFree(sw->d_occ_pi);
  cudaFree(sw->d_g);
  cudaFree(sw->d_chunk);
  cudaFree(sw->d_range);
  cudaFree(sw->d_state);
  cudaFree(sw->d_counts);
  if (sw->ev) cudaEventDestroy(sw->ev);
  delete sw;
}

mka_status mka_sweep_create(mka_system* sys, int64_t atom_begin, int64_t atom_end, int nu, double win_lo,
                            double win_hi, int kp, int64_t chunk_atoms, int with_forces, void* stream, mka_sweep** out) {
  if (!out) return fail(MKA_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!sys) return fail(MKA_ERR_INVALID_ARG, "system is NULL");
  if (atom_begin < 0 || atom_end > sys->n_atoms || atom_begin >= atom_end)
    return fail(MKA_ERR_INVALID_ARG, "need 0 <= atom_begin < atom_end <= n_atoms");
  if (nu < 1 || nu > MKA_MAX_NU) return fail(MKA_ERR_INVALID_ARG, "need 1 <= nu <= MKA_MAX_NU");
  if (kp < 1 || kp > nu) return fail(MKA_ERR_INVALID_ARG, "need 1 <= kp <= nu");
  if (pack_smem_bytes(nu, kp) > (size_t)200 * 1024)
    return fail(MKA_ERR_INVALID_ARG, "kp too large for nu: the packing kernel holds 32 nu (kp + 2) bytes in shared memory");
  if (!(win_lo < win_hi)) return fail(MKA_ERR_INVALID_ARG, "need win_lo < win_hi");
  if (chunk_atoms < 1) return fail(MKA_ERR_INVALID_ARG, "need chunk_atoms >= 1");
  if (with_forces && !sys->have_sk) return fail(MKA_ERR_INVALID_ARG, "forces need the Slater-Koster model (mka_build_system)");
  mka_sweep* sw = new mka_sweep();
  sw->sys = sys;
  sw->stream = (cudaStream_t)stream;
  sw->nu = nu;
  sw->kp = kp;
  sw->win_lo = win_lo;
  sw->win_hi = win_hi;
  sw->a0 = atom_begin;
  sw->a1 = atom_end;
  sw->n = atom_end - atom_begin;
  sw->blk0 = sys->h_row_ptr[atom_begin];
  sw->nblk = (int64_t)sys->h_row_ptr[atom_end] - sw->blk0;
  sw->chunk_atoms = chunk_atoms;
  sw->chunk0 = atom_begin / chunk_atoms;
  sw->n_chunks = (atom_end - 1) / chunk_atoms - sw->chunk0 + 1;
  const int64_t n = sw->n;
  cudaError_t e = cudaSuccess;
  int64_t bytes = 0;
#define ALLOC(ptr, b)                                 \
  if (e == cudaSuccess) {                             \
    e = cudaMalloc(&(ptr), (size_t)(b));              \
    bytes += (int64_t)(b);                            \
  }
  ALLOC(sw->d_eps, sizeof(double) * 4 * n * nu);
  ALLOC(sw->d_w, sizeof(double) * 4 * n * nu);
  ALLOC(sw->d_win, sizeof(uint16_t) * 2 * 4 * n);
  ALLOC(sw->d_flag, n);
  ALLOC(sw->d_occ, sizeof(double) * 16 * sw->nblk);
  ALLOC(sw->d_part, sizeof(double) * 16 * sw->nblk * kp);
  ALLOC(sw->d_eatom, sizeof(double) * n);
  if (with_forces) {
    ALLOC(sw->d_occ_pi, sizeof(double) * 16 * sw->nblk);
    ALLOC(sw->d_g, sizeof(double) * 3 * sw->nblk);
  }
  ALLOC(sw->d_chunk, sizeof(double) * 3 * sw->n_chunks);
  ALLOC(sw->d_range, sizeof(double) * 2 * kRangeBlocks);
  ALLOC(sw->d_state, sizeof(BisState));
  ALLOC(sw->d_counts, 2 * sizeof(unsigned long long));
#undef ALLOC
  if (e == cudaSuccess) e = cudaMemsetAsync(sw->d_flag, 0, n, sw->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(sw->d_eatom, 0, sizeof(double) * n, sw->stream);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sw->ev, cudaEventDisableTiming);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sweep_pack_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)pack_smem_bytes(nu, kp));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sweep_rho_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * 8 * 4 * kp));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sweep_force_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * 8 * 8 * kp));
  if (e != cudaSuccess) {
    const bool oom = e == cudaErrorMemoryAllocation;
    cudaGetLastError();
    mka_sweep_destroy(sw);
    return oom ? fail(MKA_ERR_OOM, "mka_sweep_create: " + std::to_string(bytes) + " bytes of device memory do not fit")
               : cuda_fail(e, "mka_sweep_create");
  }
  sw->bytes = bytes;
  *out = sw;
  return MKA_OK;
}

mka_status mka_sweep_info(const mka_sweep* sw, int64_t* chunk0, int64_t* n_chunks, int64_t* n_blocks, int64_t* bytes) {
  if (!sw) return fail(MKA_ERR_INVALID_ARG, "sweep is NULL");
  if (chunk0) *chunk0 = sw->chunk0;
  if (n_chunks) *n_chunks = sw->n_chunks;
  if (n_blocks) *n_blocks = sw->nblk;
  if (bytes) *bytes = sw->bytes;
  return MKA_OK;
}

mka_status mka_plan_run_sweep(mka_plan* plan, mka_sweep* sw, const int64_t* atoms, int64_t n_sel) {
  if (!plan || !sw) return fail(MKA_ERR_INVALID_ARG, "plan and sweep are required");
  PlanMode m;
  m.kind = PLAN_SWEEP;
  m.sw = sw;
  return plan_run_mode(plan, atoms, n_sel, m);
}

mka_status mka_sweep_status(mka_sweep* sw, int64_t* n_stored, int64_t* n_overflow) {
  if (!sw) return fail(MKA_ERR_INVALID_ARG, "sweep is NULL");
  return flag_counts(sw, n_stored, n_overflow);
}

mka_status mka_sweep_level_range(mka_sweep* sw, double* lo, double* hi) {
  if (!sw || !lo || !hi) return fail(MKA_ERR_INVALID_ARG, "sweep, lo and hi are required");
  cudaStream_t st = sw->stream;
  const int64_t n = 4 * sw->n * sw->nu;
  const int blocks = (int)std::min<int64_t>(kRangeBlocks, std::max<int64_t>(1, (n + 255) / 256));
  sweep_range_kernel<<<blocks, 256, 0, st>>>(sw->d_eps, sw->d_w, n, sw->d_range);
  count_launches();
  MKA_CUDA_TRY(cudaGetLastError());
  std::vector<double> h(2 * blocks);
  MKA_CUDA_TRY(cudaMemcpyAsync(h.data(), sw->d_range, sizeof(double) * 2 * blocks, cudaMemcpyDeviceToHost, st));
  MKA_CUDA_TRY(cudaStreamSynchronize(st));
  double mn = INFINITY, mx = -INFINITY;
  for (int b = 0; b < blocks; ++b) {
    mn = std::min(mn, h[2 * b]);
    mx = std::max(mx, h[2 * b + 1]);
  }
  if (!(mn <= mx)) return fail(MKA_ERR_INVALID_ARG, "no level with nonzero weight in the sweep");
  *lo = mn;
  *hi = mx;
  return MKA_OK;
}

mka_status mka_sweep_find_mu(mka_sweep* sw, double n_electrons, double kT, double tol, double* mu) {
  if (!sw || !mu) return fail(MKA_ERR_INVALID_ARG, "sweep and mu are required");
  if (!(kT > 0) || !(tol > 0)) return fail(MKA_ERR_INVALID_ARG, "need kT > 0 and tol > 0");
  int64_t stored = 0;
  mka_status s = flag_counts(sw, &stored, nullptr);
  if (s) return s;
  if (stored != sw->n)
    return fail(MKA_ERR_INVALID_ARG, std::to_string(sw->n - stored) + " atoms of the sweep's range are not stored yet");
  double lo = 0, hi = 0;
  s = mka_sweep_level_range(sw, &lo, &hi);
  if (s) return s;
  BisState h{};
  h.lo = lo - 40.0 * kT;
  h.hi = hi + 40.0 * kT;
  h.target = n_electrons;
  h.kT = kT;
  h.tol = tol;
  h.x = h.hi;                 // first point: every level occupied (N(lo) = 0 needs no pass)
  h.flo = -n_electrons;
  h.fhi = 0.0;
  h.side = 0.0;
  h.rf = 0.0;
  cudaStream_t st = sw->stream;
  MKA_CUDA_TRY(cudaMemcpyAsync(sw->d_state, &h, sizeof(h), cudaMemcpyHostToDevice, st));
  for (int i = 0; i < kMaxHalvings; ++i) {
    // both kernels return at once when the bracket is already narrower than tol (the loop's bound is
    // the bisection's worst case; the secant phase usually ends it after a few steps)
    s = chunk_launch(sw, 0.0, kT, sw->d_state, false, false);
    if (s) return s;
    sweep_bisect_step_kernel<<<1, 1, 0, st>>>(sw->d_chunk, sw->n_chunks, sw->d_state);
    count_launches();
    MKA_CUDA_TRY(cudaGetLastError());
  }
  MKA_CUDA_TRY(cudaMemcpyAsync(&h, sw->d_state, sizeof(h), cudaMemcpyDeviceToHost, st));
  MKA_CUDA_TRY(cudaStreamSynchronize(st));
  *mu = 0.5 * (h.lo + h.hi);
  return MKA_OK;
}

mka_status mka_sweep_density(mka_sweep* sw, mka_plan* plan, double mu, double kT, double* rho, int64_t* n_resolved) {
  if (!sw || !rho) return fail(MKA_ERR_INVALID_ARG, "sweep and rho are required");
  if (!(kT > 0)) return fail(MKA_ERR_INVALID_ARG, "need kT > 0");
  int64_t stored = 0, overflow = 0;
  mka_status s = flag_counts(sw, &stored, &overflow);
  if (s) return s;
  if (stored != sw->n)
    return fail(MKA_ERR_INVALID_ARG, std::to_string(sw->n - stored) + " atoms of the sweep's range are not stored yet");
  const bool inside = sw->win_lo + 40.0 * kT <= mu && mu <= sw->win_hi - 40.0 * kT;
  cudaStream_t st = sw->stream;
  if (inside) {
    RhoArgs A{};
    A.eps = sw->d_eps;
    A.win = sw->d_win;
    A.flag = sw->d_flag;
    A.occ = sw->d_occ;
    A.part = sw->d_part;
    A.row_ptr = sw->sys->d_row_ptr;
    A.valH = sw->sys->d_valH;
    A.storage = sw->sys->storage;
    A.nu = sw->nu;
    A.kp = sw->kp;
    A.a0 = sw->a0;
    A.n = sw->n;
    A.blk0 = sw->blk0;
    A.mu = mu;
    A.kT = kT;
    A.rho = rho;
    A.eatom = sw->d_eatom;
    int dev = 0, sms = 0;
    MKA_CUDA_TRY(cudaGetDevice(&dev));
    MKA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t blocks = std::min<int64_t>((sw->n + 7) / 8, (int64_t)sms * 8);
    sweep_rho_kernel<<<(unsigned)std::max<int64_t>(1, blocks), 256, sizeof(double) * 8 * 4 * sw->kp, st>>>(A);
    count_launches();
    MKA_CUDA_TRY(cudaGetLastError());
  }
  const int64_t n_again = inside ? overflow : sw->n;
  if (n_again > 0) {
    if (!plan) return fail(MKA_ERR_INVALID_ARG, std::to_string(n_again) + " atoms must be solved again at mu; pass a plan");
    std::vector<int64_t> again;
    again.reserve(n_again);
    if (inside) {
      std::vector<uint8_t> fl(sw->n);
      MKA_CUDA_TRY(cudaMemcpyAsync(fl.data(), sw->d_flag, sw->n, cudaMemcpyDeviceToHost, st));
      MKA_CUDA_TRY(cudaStreamSynchronize(st));
      for (int64_t i = 0; i < sw->n; ++i)
        if (fl[i] & 2) again.push_back(sw->a0 + i);
    } else {
      for (int64_t i = 0; i < sw->n; ++i) again.push_back(sw->a0 + i);
    }
    const int64_t B = plan_max_atoms(plan);
    PlanMode m;
    m.kind = PLAN_AT_MU;
    m.sw = sw;
    m.mu = mu;
    m.kT = kT;
    m.rho = rho;
    for (size_t off = 0; off < again.size(); off += (size_t)B) {
      const int64_t cnt = std::min<int64_t>(B, (int64_t)again.size() - (int64_t)off);
      s = plan_run_mode(plan, again.data() + off, cnt, m);
      if (s) return s;
    }
  }
  sw->rho_mu = mu;
  sw->rho_kT = kT;
  if (n_resolved) *n_resolved = n_again;
  return MKA_OK;
}

mka_status mka_sweep_forces(mka_sweep* sw, mka_plan* plan, double mu, double kT, double* forces, int64_t* n_resolved) {
  if (!sw || !forces) return fail(MKA_ERR_INVALID_ARG, "sweep and forces are required");
  if (!sw->d_g) return fail(MKA_ERR_INVALID_ARG, "the sweep was created without forces");
  if (!(kT > 0)) return fail(MKA_ERR_INVALID_ARG, "need kT > 0");
  int64_t stored = 0, overflow = 0;
  mka_status s = flag_counts(sw, &stored, &overflow);
  if (s) return s;
  if (stored != sw->n)
    return fail(MKA_ERR_INVALID_ARG, std::to_string(sw->n - stored) + " atoms of the sweep's range are not stored yet");
  const bool inside = sw->win_lo + 40.0 * kT <= mu && mu <= sw->win_hi - 40.0 * kT;
  cudaStream_t st = sw->stream;
  const mka_system* sys = sw->sys;
  if (inside) {
    ForceArgs A{};
    A.eps = sw->d_eps;
    A.win = sw->d_win;
    A.flag = sw->d_flag;
    A.occ = sw->d_occ;
    A.occ_pi = sw->d_occ_pi;
    A.part = sw->d_part;
    A.row_ptr = sys->d_row_ptr;
    A.col = sys->d_col;
    A.pos = sys->d_pos;
    for (int q = 0; q < 3; ++q) A.box[q] = sys->box[q];
    for (int q = 0; q < 4; ++q) {
      A.Vh[q] = sys->sk.V[q];
      A.Vs[q] = sys->sk.Sv[q];
    }
    A.d0 = sys->sk.d0;
    A.nu = sw->nu;
    A.kp = sw->kp;
    A.a0 = sw->a0;
    A.n = sw->n;
    A.blk0 = sw->blk0;
    A.mu = mu;
    A.kT = kT;
    A.g = sw->d_g;
    int dev = 0, sms = 0;
    MKA_CUDA_TRY(cudaGetDevice(&dev));
    MKA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t blocks = std::min<int64_t>((sw->n + 7) / 8, (int64_t)sms * 8);
    sweep_force_kernel<<<(unsigned)std::max<int64_t>(1, blocks), 256, sizeof(double) * 8 * 8 * sw->kp, st>>>(A);
    count_launches();
    MKA_CUDA_TRY(cudaGetLastError());
  }
  const int64_t n_again = inside ? overflow : sw->n;
  if (n_again > 0) {
    if (!plan) return fail(MKA_ERR_INVALID_ARG, std::to_string(n_again) + " atoms must be solved again at mu; pass a plan");
    std::vector<int64_t> again;
    again.reserve(n_again);
    if (inside) {
      std::vector<uint8_t> fl(sw->n);
      MKA_CUDA_TRY(cudaMemcpyAsync(fl.data(), sw->d_flag, sw->n, cudaMemcpyDeviceToHost, st));
      MKA_CUDA_TRY(cudaStreamSynchronize(st));
      for (int64_t i = 0; i < sw->n; ++i)
        if (fl[i] & 2) again.push_back(sw->a0 + i);
    } else {
      for (int64_t i = 0; i < sw->n; ++i) again.push_back(sw->a0 + i);
    }
    const int64_t B = plan_max_atoms(plan);
    PlanMode m;
    m.kind = PLAN_AT_MU;
    m.sw = sw;
    m.mu = mu;
    m.kT = kT;
    m.forces = true;
    for (size_t off = 0; off < again.size(); off += (size_t)B) {
      const int64_t cnt = std::min<int64_t>(B, (int64_t)again.size() - (int64_t)off);
      s = plan_run_mode(plan, again.data() + off, cnt, m);
      if (s) return s;
    }
  }
  s = force_gather_enqueue(sys, sw->d_g, sw->a0, sw->a1, sw->blk0, forces, st);
  if (s) return s;
  if (n_resolved) *n_resolved = n_again;
  return MKA_OK;
}

mka_status mka_sweep_chunk_sums(mka_sweep* sw, double mu, double kT, double* count, double* e_levels, double* e_rho) {
  if (!sw) return fail(MKA_ERR_INVALID_ARG, "sweep is NULL");
  if (!(kT > 0)) return fail(MKA_ERR_INVALID_ARG, "need kT > 0");
  if (e_rho && !(sw->rho_mu == mu && sw->rho_kT == kT))
    return fail(MKA_ERR_INVALID_ARG, "e_rho needs mka_sweep_density at the same mu and kT first");
  mka_status s = chunk_launch(sw, mu, kT, nullptr, e_levels != nullptr, e_rho != nullptr);
  if (s) return s;
  const int64_t nc = sw->n_chunks;
  cudaStream_t st = sw->stream;
  if (count) MKA_CUDA_TRY(cudaMemcpyAsync(count, sw->d_chunk, sizeof(double) * nc, cudaMemcpyDeviceToHost, st));
  if (e_levels) MKA_CUDA_TRY(cudaMemcpyAsync(e_levels, sw->d_chunk + nc, sizeof(double) * nc, cudaMemcpyDeviceToHost, st));
  if (e_rho) MKA_CUDA_TRY(cudaMemcpyAsync(e_rho, sw->d_chunk + 2 * nc, sizeof(double) * nc, cudaMemcpyDeviceToHost, st));
  MKA_CUDA_TRY(cudaStreamSynchronize(st));
  return MKA_OK;
}

mka_status mka_sweep_device_levels(const mka_sweep* sw, const double** eps, const double** w) {
  if (!sw) return fail(MKA_ERR_INVALID_ARG, "sweep is NULL");
  if (eps) *eps = sw->d_eps;
  if (w) *w = sw->d_w;
  return MKA_OK;
}

}  // extern "C"

namespace mka {
// Orders a plan's work on `plan_stream` after the sweep's earlier work, and the sweep's later work after it.
mka_status sweep_join_before(mka_sweep* sw, cudaStream_t plan_stream) { return join(sw->stream, plan_stream, sw->ev); }
mka_status sweep_join_after(mka_sweep* sw, cudaStream_t plan_stream) { return join(plan_stream, sw->stream, sw->ev); }
}  // namespace mka
