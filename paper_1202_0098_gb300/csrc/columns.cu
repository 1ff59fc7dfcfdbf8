// Per-column hot path of the multiple Arnoldi method on sm_103a.
//
// One CTA owns one atom a at a time and runs its four columns j = 4a + o
// (o = s, px, py, pz) together, because they share the cluster C_a of the
// real-space projection (Sec. 3). Per atom, in one persistent launch over a
// device work queue:
//   1. cluster extraction: atoms within R of a (minimum image) from the cell
//      list, sorted by atom id; the cluster-local 4x4-block pattern of
//      P H P / P S P is built in shared memory (local column, global block id);
//   2. inner CG for S s_j = e_j (Sec. 2, standard CG, x0 = 0);
//   3. the S-orthonormal basis of K_p(H; e_j) (+) K_q(H; s_j): S-orthogonalise,
//      normalise, k_n = H u_n, next vector k_n or s_j after u_p (Eqs.
//      EQ-REC-UN, EQ-KN-HUN, EQ-MGram-Schmidt, EQ-CALC-S-INV); Gram-Schmidt is
//      the classical form run twice, coefficients (S u_m)^T l with S u_m kept;
//   4. the projection H_r = U^T K, S_r = U^T (S U), symmetrised, and the
//      reduced generalized problem (Eq. EQ-SUB-EIG-VEC): Cholesky of S_r,
//      L^{-1} H_r L^{-T}, parallel cyclic Jacobi eigensolve, C = L^{-T} Y;
//   5. per column: ascending eps_alpha, w_alpha = V_{j alpha} (S V)_{j alpha},
//      and (optionally) the pattern rows of V for rho and G.
// Breakdown rule: a new vector that keeps no more than 1e-10 of its S-norm
// (S-norm before projection taken from the Pythagorean sum of the removed
// coefficients) is dropped; a dropped s_j is replaced by H u_n, a first chain
// that closes before u_p hands over to s_j, any other breakdown ends the basis.
//
// Vectors (U, S U, K = H U and the CG/Arnoldi work vectors) live in a per-CTA
// global scratch slot, [row][4 columns] interleaved so that one thread owns a
// row of all four columns; the cluster pattern, reductions and the nu x nu
// matrices live in shared memory. Arithmetic type T is double for the FP64
// form and float for the mixed form (values of any storage type are decoded
// to T on load); the projection and the reduced solve are FP64 in both.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "mka_internal.h"

namespace mka {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxCl = MKA_MAX_CLUSTER_ATOMS;  // power of two (bitonic sort size bound)
static_assert((kMaxCl & (kMaxCl - 1)) == 0, "cluster cap must be a power of two");

enum ColStatus { ST_OK = 0, ST_NOT_SPD = MKA_ERR_NOT_SPD, ST_NOCONV = MKA_ERR_NO_CONVERGENCE,
                 ST_BREAKDOWN = MKA_ERR_BREAKDOWN, ST_TOOLARGE = MKA_ERR_CLUSTER_TOO_LARGE };
enum Src { SRC_E = 0, SRC_H = 1, SRC_S = 2 };
enum Act { ACT_NONE = 0, ACT_LOAD_K = 1, ACT_LOAD_S = 2 };

// ---- value loads: one row (4 entries) of a 4x4 block, decoded ----------------
template <typename TV, typename T>
struct RowLoad;
template <typename T>
struct RowLoad<double, T> {
  static __device__ __forceinline__ void load(const double* v, int64_t blk, int i, T out[4]) {
    const double2* p = reinterpret_cast<const double2*>(v + blk * 16 + i * 4);
    double2 a = __ldg(p), b = __ldg(p + 1);
    out[0] = (T)a.x; out[1] = (T)a.y; out[2] = (T)b.x; out[3] = (T)b.y;
  }
};
template <typename T>
struct RowLoad<float, T> {
  static __device__ __forceinline__ void load(const float* v, int64_t blk, int i, T out[4]) {
    float4 a = __ldg(reinterpret_cast<const float4*>(v + blk * 16 + i * 4));
    out[0] = (T)a.x; out[1] = (T)a.y; out[2] = (T)a.z; out[3] = (T)a.w;
  }
};
template <typename T>
struct RowLoad<__nv_bfloat16, T> {
  static __device__ __forceinline__ void load(const __nv_bfloat16* v, int64_t blk, int i, T out[4]) {
    uint2 a = __ldg(reinterpret_cast<const uint2*>(v + blk * 16 + i * 4));
    out[0] = (T)__uint_as_float(a.x << 16); out[1] = (T)__uint_as_float(a.x & 0xFFFF0000u);
    out[2] = (T)__uint_as_float(a.y << 16); out[3] = (T)__uint_as_float(a.y & 0xFFFF0000u);
  }
};

// ---- kernel arguments ----------------------------------------------------------
template <typename TV>
struct Args {
  // system
  int64_t n_atoms;
  const int32_t* row_ptr;
  const int32_t* col;
  const TV* valH;
  const TV* valS;
  const double* pos;
  double box[3];
  double R2;
  int ncell[3];
  double cell_len[3];
  const int32_t* cell_start;
  const int32_t* cell_atoms;
  // work
  const int64_t* sel;
  int64_t n_sel;
  int* work_counter;
  // method
  int p, q, nu;
  double cg_tol;
  int cg_maxit;
  double tau;
  // scratch
  char* scratch;
  size_t slot_bytes;
  int mcap;            // 4 x (largest cluster of the selection)
  int lnnz_cap;        // local-block capacity per cluster
  // outputs
  double* eps;
  double* w;
  int32_t* nu_eff;
  int32_t* cg_iters;
  int32_t* status;
  int keep;
  double* vp;
  const int64_t* blk_off;
  int32_t* self_k;
};

// ---- small CTA helpers -------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums a[0..3] over the CTA; the result lands in out[0..3] (shared) for every thread.
__device__ __forceinline__ void cta_sum4(double a[4], double* red, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 4; ++c) a[c] = warp_sum(a[c]);
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < 4; ++c) red[wid * 4 + c] = a[c];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0;
    for (int k = 0; k < kWarps; ++k) s += red[k * 4 + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Binary search of atom id c in the sorted cluster list; -1 when absent.
__device__ __forceinline__ int find_local(const int* cl, int n, int c) {
  int lo = 0, hi = n - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int v = cl[mid];
    if (v == c) return mid;
    if (v < c) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

__device__ __forceinline__ double min_image(double d, double L) { return d - L * rint(d / L); }

__device__ __forceinline__ int cell_range(int c, int n, int out[3]) {
  if (n < 3) {
    for (int i = 0; i < n; ++i) out[i] = i;
    return n;
  }
  out[0] = (c + n - 1) % n;
  out[1] = c;
  out[2] = (c + 1) % n;
  return 3;
}

__device__ __forceinline__ int cell_coord(double x, double len, int n) {
  int v = (int)floor(x / len);
  return v < 0 ? 0 : (v >= n ? n - 1 : v);
}

// Atoms within R of atom a (minimum image) appended to cl via the shared counter;
// returns the count (which may exceed kMaxCl: then nothing beyond kMaxCl is stored).
template <typename TV>
__device__ int gather_cluster(const Args<TV>& A, int64_t a, int* cl, int* cnt) {
  if (threadIdx.x == 0) *cnt = 0;
  __syncthreads();
  const double px = A.pos[3 * a], py = A.pos[3 * a + 1], pz = A.pos[3 * a + 2];
  int rx[3], ry[3], rz[3];
  const int nx = cell_range(cell_coord(px, A.cell_len[0], A.ncell[0]), A.ncell[0], rx);
  const int ny = cell_range(cell_coord(py, A.cell_len[1], A.ncell[1]), A.ncell[1], ry);
  const int nz = cell_range(cell_coord(pz, A.cell_len[2], A.ncell[2]), A.ncell[2], rz);
  const int ncells = nx * ny * nz;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int ci = wid; ci < ncells; ci += kWarps) {
    const int ix = ci / (ny * nz), iy = (ci / nz) % ny, iz = ci % nz;
    const int c = (rx[ix] * A.ncell[1] + ry[iy]) * A.ncell[2] + rz[iz];
    const int s0 = A.cell_start[c], s1 = A.cell_start[c + 1];
    for (int k = s0 + lane; k < s1; k += 32) {
      const int b = A.cell_atoms[k];
      const double dx = min_image(A.pos[3 * b] - px, A.box[0]);
      const double dy = min_image(A.pos[3 * b + 1] - py, A.box[1]);
      const double dz = min_image(A.pos[3 * b + 2] - pz, A.box[2]);
      const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
      if (r2 <= A.R2) {
        const int idx = atomicAdd(cnt, 1);
        if (idx < kMaxCl) cl[idx] = b;
      }
    }
  }
  __syncthreads();
  return *cnt;
}

// Ascending bitonic sort of cl[0..n) (n <= kMaxCl), padding with INT_MAX.
__device__ void sort_cluster(int* cl, int n) {
  int N = 2;
  while (N < n) N <<= 1;
  for (int i = n + threadIdx.x; i < N; i += blockDim.x) cl[i] = 0x7fffffff;
  __syncthreads();
  for (int k = 2; k <= N; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const int x = cl[i], y = cl[ixj];
          const bool up = (i & k) == 0;
          if ((x > y) == up) {
            cl[i] = y;
            cl[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

// y = A x on the cluster (all four columns), rows 4t + i; x, y are [m][4].
template <typename TV, typename T>
__device__ __forceinline__ void spmm4(const TV* __restrict__ val, const int* lrow, const int* lcol,
                                      const int* lblk, int ncl, const T* __restrict__ x, T* __restrict__ y) {
  const int m = 4 * ncl;
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    const int t = r >> 2, i = r & 3;
    T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    for (int e = lrow[t]; e < lrow[t + 1]; ++e) {
      T v[4];
      RowLoad<TV, T>::load(val, lblk[e], i, v);
      const T* xb = x + (size_t)lcol[e] * 16;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        a0 += v[k] * xb[4 * k + 0];
        a1 += v[k] * xb[4 * k + 1];
        a2 += v[k] * xb[4 * k + 2];
        a3 += v[k] * xb[4 * k + 3];
      }
    }
    y[4 * r + 0] = a0;
    y[4 * r + 1] = a1;
    y[4 * r + 2] = a2;
    y[4 * r + 3] = a3;
  }
  __syncthreads();
}

// Per-column dot products over the cluster rows, accumulated in double.
template <typename T>
__device__ __forceinline__ void dot4(const T* a, const T* b, int m, double* red, double* out) {
  double acc[4] = {0, 0, 0, 0};
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] += (double)a[4 * r + c] * (double)b[4 * r + c];
  }
  cta_sum4(acc, red, out);
}

// ---- shared state of one atom --------------------------------------------------------
struct AtomState {
  int n[4], src[4], seam_done[4], active[4], accept[4], act[4], next_s[4];
  int it[4], cg_active[4], status[4];
  double beta_inv[4], csum[4], rr[4], alpha[4], beta_cg[4];
  double tmp4[4];
  int ncl, t0, flag, n_max;
};

// Parallel cyclic Jacobi on the symmetric nv x nv matrix A (leading dimension ld) in
// shared memory; accumulates the rotations into Y (starts as I). Round-robin
// ordering: ceil(nv/2) disjoint (p, q) pairs per round, nv' - 1 rounds per sweep.
__device__ void jacobi_eig(double* A, double* Y, int nv, int ld, double* cs, double* red, int* flag) {
  const int np = (nv + 1) / 2;           // pairs per round
  const int n2 = 2 * np;                 // even number of players (one dummy when nv is odd)
  for (int i = threadIdx.x; i < nv * nv; i += blockDim.x) Y[(i / nv) * ld + i % nv] = (i / nv == i % nv) ? 1.0 : 0.0;
  __syncthreads();
  for (int sweep = 0; sweep < 40; ++sweep) {
    // convergence: largest off-diagonal entry vs largest diagonal entry
    double off = 0, dia = 0;
    for (int i = threadIdx.x; i < nv * nv; i += blockDim.x) {
      const int r = i / nv, c = i % nv;
      const double v = fabs(A[r * ld + c]);
      if (r == c) dia = fmax(dia, v); else off = fmax(off, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
      off = fmax(off, __shfl_xor_sync(0xffffffffu, off, o));
      dia = fmax(dia, __shfl_xor_sync(0xffffffffu, dia, o));
    }
    if ((threadIdx.x & 31) == 0) {
      red[(threadIdx.x >> 5) * 2] = off;
      red[(threadIdx.x >> 5) * 2 + 1] = dia;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double o2 = 0, d2 = 0;
      for (int k = 0; k < kWarps; ++k) {
        o2 = fmax(o2, red[2 * k]);
        d2 = fmax(d2, red[2 * k + 1]);
      }
      *flag = (o2 <= 1e-17 * d2) || o2 == 0.0;
    }
    __syncthreads();
    if (*flag) break;
    for (int round = 0; round < n2 - 1; ++round) {
      // rotation angles of this round's pairs
      for (int k = threadIdx.x; k < np; k += blockDim.x) {
        int pp, qq;
        if (k == 0) {
          pp = 0;
          qq = 1 + round;
        } else {
          pp = 1 + (round + k) % (n2 - 1);
          qq = 1 + (round - k + n2 - 1) % (n2 - 1);
        }
        if (pp > qq) { const int t = pp; pp = qq; qq = t; }
        double c = 1.0, s = 0.0;
        if (qq < nv) {
          const double apq = A[pp * ld + qq];
          if (apq != 0.0) {
            const double app = A[pp * ld + pp], aqq = A[qq * ld + qq];
            const double theta = (aqq - app) / (2.0 * apq);
            const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        }
        cs[4 * k + 0] = c;
        cs[4 * k + 1] = s;
        reinterpret_cast<int*>(cs)[8 * k + 4] = pp;   // indices packed behind (c, s)
        reinterpret_cast<int*>(cs)[8 * k + 5] = qq;
      }
      __syncthreads();
      // A <- A J (columns p, q) and Y <- Y J
      for (int idx = threadIdx.x; idx < np * nv; idx += blockDim.x) {
        const int k = idx / nv, r = idx % nv;
        const int pp = reinterpret_cast<int*>(cs)[8 * k + 4], qq = reinterpret_cast<int*>(cs)[8 * k + 5];
        if (qq >= nv) continue;
        const double c = cs[4 * k], s = cs[4 * k + 1];
        const double ap = A[r * ld + pp], aq = A[r * ld + qq];
        A[r * ld + pp] = c * ap - s * aq;
        A[r * ld + qq] = s * ap + c * aq;
        const double yp = Y[r * ld + pp], yq = Y[r * ld + qq];
        Y[r * ld + pp] = c * yp - s * yq;
        Y[r * ld + qq] = s * yp + c * yq;
      }
      __syncthreads();
      // A <- J^T A (rows p, q)
      for (int idx = threadIdx.x; idx < np * nv; idx += blockDim.x) {
        const int k = idx / nv, r = idx % nv;
        const int pp = reinterpret_cast<int*>(cs)[8 * k + 4], qq = reinterpret_cast<int*>(cs)[8 * k + 5];
        if (qq >= nv) continue;
        const double c = cs[4 * k], s = cs[4 * k + 1];
        const double ap = A[pp * ld + r], aq = A[qq * ld + r];
        A[pp * ld + r] = c * ap - s * aq;
        A[qq * ld + r] = s * ap + c * aq;
      }
      __syncthreads();
    }
  }
}

// Reduced problem of one column: Hr, Sr in shared memory (nv x nv, leading dimension ld).
// On return eps_sorted[0..nv) ascending and C (ld) = L^{-T} Y with columns in that order.
// Returns false when S_r is not positive definite.
__device__ bool reduced_solve(double* Hr, double* Sr, double* Y, double* C, double* eps, int nv, int ld,
                              double* cs, double* red, int* flag) {
  // Cholesky S_r = L L^T in place (lower triangle of Sr), right-looking.
  for (int k = 0; k < nv; ++k) {
    if (threadIdx.x == 0) {
      const double d = Sr[k * ld + k];
      *flag = d > 0.0;
      Sr[k * ld + k] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    if (!*flag) return false;
    const double lkk = Sr[k * ld + k];
    for (int i = k + 1 + threadIdx.x; i < nv; i += blockDim.x) Sr[i * ld + k] /= lkk;
    __syncthreads();
    const int rem = nv - k - 1;
    for (int idx = threadIdx.x; idx < rem * rem; idx += blockDim.x) {
      const int i = k + 1 + idx / rem, j = k + 1 + idx % rem;
      if (j <= i) Sr[i * ld + j] -= Sr[i * ld + k] * Sr[j * ld + k];
    }
    __syncthreads();
  }
  // X = L^{-1} Hr (column by column, forward substitution) into C
  for (int n = threadIdx.x; n < nv; n += blockDim.x) {
    for (int i = 0; i < nv; ++i) {
      double v = Hr[i * ld + n];
      for (int k = 0; k < i; ++k) v -= Sr[i * ld + k] * C[k * ld + n];
      C[i * ld + n] = v / Sr[i * ld + i];
    }
  }
  __syncthreads();
  // A = L^{-1} X^T into Hr (A = L^{-1} Hr L^{-T})
  for (int n = threadIdx.x; n < nv; n += blockDim.x) {
    for (int i = 0; i < nv; ++i) {
      double v = C[n * ld + i];
      for (int k = 0; k < i; ++k) v -= Sr[i * ld + k] * Hr[k * ld + n];
      Hr[i * ld + n] = v / Sr[i * ld + i];
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nv * nv; idx += blockDim.x) {
    const int i = idx / nv, j = idx % nv;
    if (j > i) {
      const double v = 0.5 * (Hr[i * ld + j] + Hr[j * ld + i]);
      Hr[i * ld + j] = v;
      Hr[j * ld + i] = v;
    }
  }
  __syncthreads();
  jacobi_eig(Hr, Y, nv, ld, cs, red, flag);
  // ranks of the eigenvalues (ascending, ties by index)
  int* rank = reinterpret_cast<int*>(red);
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    const double e = Hr[i * ld + i];
    int r = 0;
    for (int k = 0; k < nv; ++k) {
      const double f = Hr[k * ld + k];
      r += (f < e) || (f == e && k < i);
    }
    rank[i] = r;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nv; i += blockDim.x) eps[rank[i]] = Hr[i * ld + i];
  // C = L^{-T} Y, column alpha stored at its rank
  for (int a = threadIdx.x; a < nv; a += blockDim.x) {
    const int ra = rank[a];
    for (int i = nv - 1; i >= 0; --i) {
      double v = Y[i * ld + a];
      for (int k = i + 1; k < nv; ++k) v -= Sr[k * ld + i] * C[k * ld + ra];
      C[i * ld + ra] = v / Sr[i * ld + i];
    }
  }
  __syncthreads();
  return true;
}

template <typename TV, typename T>
__global__ void __launch_bounds__(kThreads) atoms_kernel(const Args<TV> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ AtomState st;
  __shared__ double red[2 * kWarps * 4];
  __shared__ double sums[4];
  __shared__ double coef[MKA_MAX_NU * 4];
  __shared__ int64_t cur_atom;
  __shared__ int cnt;

  const int nu = A.nu;
  const int ld = nu + 1;
  int* cl = reinterpret_cast<int*>(smem_raw);                 // kMaxCl
  int* lrow = cl + kMaxCl;                                     // kMaxCl + 1
  int* lcol = lrow + kMaxCl + 1;                               // lnnz_cap
  int* lblk = lcol + A.lnnz_cap;                               // lnnz_cap
  size_t off = (size_t)(2 * kMaxCl + 1 + 2 * A.lnnz_cap) * sizeof(int);
  off = (off + 15) & ~(size_t)15;
  double* Hr = reinterpret_cast<double*>(smem_raw + off);     // nu x ld
  double* Sr = Hr + nu * ld;
  double* Y = Sr + nu * ld;
  double* C = Y + nu * ld;
  double* evals = C + nu * ld;                                 // nu
  double* cs = evals + nu;                                     // 4 x ceil(nu/2) (+ packed ints)

  const int m_cap = A.mcap;
  T* base = reinterpret_cast<T*>(A.scratch + (size_t)blockIdx.x * A.slot_bytes);
  T* U = base;                                   // [nu][m][4]
  T* SU = U + (size_t)nu * m_cap * 4;
  T* Kv = SU + (size_t)nu * m_cap * 4;
  T* l = Kv + (size_t)nu * m_cap * 4;            // [m][4]
  T* Sl = l + (size_t)m_cap * 4;
  T* kv = Sl + (size_t)m_cap * 4;
  T* sv = kv + (size_t)m_cap * 4;                // s_j (CG solution)
  T* rv = sv + (size_t)m_cap * 4;
  T* pv = rv + (size_t)m_cap * 4;
  T* Ap = pv + (size_t)m_cap * 4;

  for (;;) {
    if (threadIdx.x == 0) {
      const int64_t w = atomicAdd(A.work_counter, 1);
      cur_atom = w;
    }
    __syncthreads();
    const int64_t widx = cur_atom;
    if (widx >= A.n_sel) break;
    const int64_t atom = A.sel[widx];

    // ---- 1. cluster ----------------------------------------------------------------
    const int ncl_raw = gather_cluster(A, atom, cl, &cnt);
    if (ncl_raw > kMaxCl || 4 * ncl_raw > m_cap) {
      for (int c = threadIdx.x; c < 4; c += blockDim.x) {
        const int64_t col = 4 * widx + c;
        A.status[col] = ST_TOOLARGE;
        A.nu_eff[col] = 0;
        A.cg_iters[col] = 0;
      }
      for (int i = threadIdx.x; i < 4 * nu; i += blockDim.x) {
        A.eps[4 * widx * nu + i] = 0.0;
        A.w[4 * widx * nu + i] = 0.0;
      }
      __syncthreads();
      continue;
    }
    const int ncl = ncl_raw;
    sort_cluster(cl, ncl);
    // local pattern: count, prefix, fill
    for (int t = threadIdx.x; t < ncl; t += blockDim.x) {
      const int b = cl[t];
      int c = 0;
      for (int k = A.row_ptr[b]; k < A.row_ptr[b + 1]; ++k) c += find_local(cl, ncl, A.col[k]) >= 0;
      lrow[t + 1] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      lrow[0] = 0;
      for (int t = 0; t < ncl; ++t) lrow[t + 1] += lrow[t];
      st.ncl = ncl;
      st.t0 = find_local(cl, ncl, (int)atom);
      st.flag = lrow[ncl] <= A.lnnz_cap;
    }
    __syncthreads();
    if (!st.flag) {  // cannot happen with a capacity of (largest cluster) x (longest row)
      for (int c = threadIdx.x; c < 4; c += blockDim.x) A.status[4 * widx + c] = ST_TOOLARGE;
      __syncthreads();
      continue;
    }
    for (int t = threadIdx.x; t < ncl; t += blockDim.x) {
      const int b = cl[t];
      int e = lrow[t];
      for (int k = A.row_ptr[b]; k < A.row_ptr[b + 1]; ++k) {
        const int lc = find_local(cl, ncl, A.col[k]);
        if (lc >= 0) {
          lcol[e] = lc;
          lblk[e] = k;
          ++e;
        }
      }
    }
    const int m = 4 * ncl;
    const int t0 = st.t0;
    // ---- 2. inner CG: S s = e_j, x0 = 0 ----------------------------------------------
    for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
      const int r = i >> 2, c = i & 3;
      const T e = (r == 4 * t0 + c) ? (T)1 : (T)0;
      sv[i] = 0;
      rv[i] = e;
      pv[i] = e;
    }
    if (threadIdx.x < 4) {
      const int c = threadIdx.x;
      st.rr[c] = 1.0;
      st.it[c] = 0;
      st.status[c] = ST_OK;
      st.cg_active[c] = !(1.0 <= A.cg_tol);
    }
    __syncthreads();
    for (int it = 0; it < A.cg_maxit; ++it) {
      if (!(st.cg_active[0] | st.cg_active[1] | st.cg_active[2] | st.cg_active[3])) break;
      spmm4<TV, T>(A.valS, lrow, lcol, lblk, ncl, pv, Ap);
      dot4<T>(pv, Ap, m, red, sums);
      if (threadIdx.x < 4) {
        const int c = threadIdx.x;
        double a = 0.0;
        if (st.cg_active[c]) {
          if (!(sums[c] > 0.0)) {
            st.status[c] = ST_NOT_SPD;
            st.cg_active[c] = 0;
          } else {
            a = st.rr[c] / sums[c];
          }
        }
        st.alpha[c] = a;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
        const int c = i & 3;
        if (st.cg_active[c]) {
          const T a = (T)st.alpha[c];
          sv[i] += a * pv[i];
          rv[i] -= a * Ap[i];
        }
      }
      __syncthreads();
      dot4<T>(rv, rv, m, red, sums);
      if (threadIdx.x < 4) {
        const int c = threadIdx.x;
        if (st.cg_active[c]) {
          st.beta_cg[c] = sums[c] / st.rr[c];
          st.rr[c] = sums[c];
          st.it[c] += 1;
          if (sqrt(sums[c]) <= A.cg_tol) st.cg_active[c] = 0;
        }
      }
      __syncthreads();
      for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
        const int c = i & 3;
        if (st.cg_active[c]) pv[i] = rv[i] + (T)st.beta_cg[c] * pv[i];
      }
      __syncthreads();
    }
    if (threadIdx.x < 4) {
      const int c = threadIdx.x;
      if (st.cg_active[c] && st.status[c] == ST_OK) st.status[c] = ST_NOCONV;
      // ---- 3. basis state ----
      st.n[c] = 0;
      st.src[c] = SRC_E;
      st.seam_done[c] = (A.q == 0);
      st.active[c] = (st.status[c] == ST_OK);
    }
    for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
      const int r = i >> 2, c = i & 3;
      l[i] = (r == 4 * t0 + c) ? (T)1 : (T)0;
    }
    __syncthreads();

    // ---- 3. multiple Arnoldi basis ---------------------------------------------------------
    for (int guard = 0; guard < nu + 4; ++guard) {
      if (!(st.active[0] | st.active[1] | st.active[2] | st.active[3])) break;
      if (threadIdx.x == 0) {
        int nm = 0;
        for (int c = 0; c < 4; ++c) {
          st.csum[c] = 0.0;
          if (st.active[c]) nm = max(nm, st.n[c]);
        }
        st.n_max = nm;
      }
      __syncthreads();
      const int nmax = st.n_max;
      for (int pass = 0; pass < 2 && nmax > 0; ++pass) {
        // coefficients (S u_mm)^T l, one warp per mm
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int mm = wid; mm < nmax; mm += kWarps) {
          const T* su = SU + (size_t)mm * m_cap * 4;
          double acc[4] = {0, 0, 0, 0};
          for (int r = lane; r < m; r += 32) {
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[c] += (double)su[4 * r + c] * (double)l[4 * r + c];
          }
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[c] = warp_sum(acc[c]);
          if (lane < 4) {
            const int c = lane;
            coef[mm * 4 + c] = (st.active[c] && mm < st.n[c]) ? acc[c] : 0.0;
          }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
          const int r = i >> 2, c = i & 3;
          T v = l[i];
          for (int mm = 0; mm < nmax; ++mm) v -= (T)coef[mm * 4 + c] * U[(size_t)mm * m_cap * 4 + 4 * r + c];
          l[i] = v;
        }
        if (threadIdx.x < 4) {
          double s = 0;
          for (int mm = 0; mm < nmax; ++mm) s += coef[mm * 4 + threadIdx.x] * coef[mm * 4 + threadIdx.x];
          st.csum[threadIdx.x] += s;
        }
        __syncthreads();
      }
      spmm4<TV, T>(A.valS, lrow, lcol, lblk, ncl, l, Sl);
      dot4<T>(l, Sl, m, red, sums);
      if (threadIdx.x < 4) {
        const int c = threadIdx.x;
        st.accept[c] = 0;
        st.act[c] = ACT_NONE;
        if (st.active[c]) {
          const double b2 = fmax(sums[c], 0.0);
          const double beta = sqrt(b2);
          const double beta_pre = sqrt(b2 + st.csum[c]);
          if (beta > A.tau * beta_pre) {
            st.accept[c] = 1;
            st.beta_inv[c] = 1.0 / beta;
          } else if (st.src[c] == SRC_S) {
            st.act[c] = ACT_LOAD_K;   // s_j already in the span: continue with H u_n
            st.src[c] = SRC_H;
          } else if (!st.seam_done[c]) {
            st.act[c] = ACT_LOAD_S;   // first chain closed early: start the second chain
            st.src[c] = SRC_S;
            st.seam_done[c] = 1;
          } else {
            st.active[c] = 0;         // basis ends with nu_eff = n
          }
        }
      }
      __syncthreads();
      const bool any_acc = st.accept[0] | st.accept[1] | st.accept[2] | st.accept[3];
      if (any_acc) {
        for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
          const int r = i >> 2, c = i & 3;
          if (st.accept[c]) {
            const T bi = (T)st.beta_inv[c];
            const T u = l[i] * bi;
            const size_t o = (size_t)st.n[c] * m_cap * 4 + 4 * r + c;
            U[o] = u;
            SU[o] = Sl[i] * bi;
            l[i] = u;
          }
        }
        __syncthreads();
        spmm4<TV, T>(A.valH, lrow, lcol, lblk, ncl, l, kv);
        for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
          const int r = i >> 2, c = i & 3;
          if (st.accept[c]) Kv[(size_t)st.n[c] * m_cap * 4 + 4 * r + c] = kv[i];
        }
        __syncthreads();
      }
      if (threadIdx.x < 4) {
        const int c = threadIdx.x;
        st.next_s[c] = 0;
        if (st.accept[c]) {
          st.n[c] += 1;
          if (st.n[c] >= nu) {
            st.active[c] = 0;
          } else if (st.n[c] == A.p && !st.seam_done[c]) {
            st.next_s[c] = 1;         // the vector after u_p is s_j
            st.seam_done[c] = 1;
            st.src[c] = SRC_S;
          } else {
            st.src[c] = SRC_H;
          }
        }
      }
      __syncthreads();
      for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
        const int r = i >> 2, c = i & 3;
        if (!st.active[c]) continue;
        if (st.accept[c]) {
          l[i] = st.next_s[c] ? sv[i] : kv[i];
        } else if (st.act[c] == ACT_LOAD_K) {
          l[i] = Kv[(size_t)(st.n[c] - 1) * m_cap * 4 + 4 * r + c];
        } else if (st.act[c] == ACT_LOAD_S) {
          l[i] = sv[i];
        }
      }
      __syncthreads();
    }

    // ---- 4./5. projection, reduced solve, outputs, one column at a time ----------------
    for (int c = 0; c < 4; ++c) {
      const int64_t col = 4 * widx + c;
      const int nv = st.n[c];
      int stc = st.status[c];
      if (stc == ST_OK && nv < nu) stc = ST_BREAKDOWN;
      bool ok = (st.status[c] == ST_OK) && nv > 0;
      if (ok) {
        // Hr = U^T K, Sr = U^T SU, then symmetrised
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int e = wid; e < nv * nv; e += kWarps) {
          const int a = e / nv, b = e % nv;
          const T* ua = U + (size_t)a * m_cap * 4;
          const T* kb = Kv + (size_t)b * m_cap * 4;
          const T* sb = SU + (size_t)b * m_cap * 4;
          double h = 0, s = 0;
          for (int r = lane; r < m; r += 32) {
            const double u = (double)ua[4 * r + c];
            h += u * (double)kb[4 * r + c];
            s += u * (double)sb[4 * r + c];
          }
          h = warp_sum(h);
          s = warp_sum(s);
          if (lane == 0) {
            Hr[a * ld + b] = h;
            Sr[a * ld + b] = s;
          }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nv * nv; e += blockDim.x) {
          const int a = e / nv, b = e % nv;
          if (b > a) {
            const double h = 0.5 * (Hr[a * ld + b] + Hr[b * ld + a]);
            const double s = 0.5 * (Sr[a * ld + b] + Sr[b * ld + a]);
            Hr[a * ld + b] = h;
            Hr[b * ld + a] = h;
            Sr[a * ld + b] = s;
            Sr[b * ld + a] = s;
          }
        }
        __syncthreads();
        ok = reduced_solve(Hr, Sr, Y, C, evals, nv, ld, cs, red, &st.flag);
        if (!ok) stc = ST_NOT_SPD;
      }
      if (threadIdx.x == 0) {
        A.status[col] = stc;
        A.nu_eff[col] = ok ? nv : 0;
        A.cg_iters[col] = st.it[c];
      }
      // eps, w = V_j (S V)_j with V = U C
      const int jr = 4 * t0 + c;
      for (int a = threadIdx.x; a < nu; a += blockDim.x) {
        double e = 0.0, wv = 0.0;
        if (ok && a < nv) {
          double vj = 0.0, svj = 0.0;
          for (int n = 0; n < nv; ++n) {
            const double cn = C[n * ld + a];
            vj += (double)U[(size_t)n * m_cap * 4 + 4 * jr + c] * cn;
            svj += (double)SU[(size_t)n * m_cap * 4 + 4 * jr + c] * cn;
          }
          e = evals[a];
          wv = vj * svj;
        }
        A.eps[col * nu + a] = e;
        A.w[col * nu + a] = wv;
      }
      if (A.keep) {
        // pattern rows of V: blocks of the atom's own row, neighbour atom local index lcol
        const int e0 = lrow[t0], e1 = lrow[t0 + 1];
        const int64_t rbase = A.row_ptr[atom];
        const int nrow = A.row_ptr[atom + 1] - A.row_ptr[atom];
        // zero the whole output row first (blocks outside the cluster stay zero)
        for (int i = threadIdx.x; i < nrow * 4 * nu; i += blockDim.x) {
          const int k = i / (4 * nu), rem = i % (4 * nu);
          A.vp[((A.blk_off[widx] + k) * 16 + c * 4) * (int64_t)nu + rem] = 0.0;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < (e1 - e0) * 4 * nu; i += blockDim.x) {
          const int e = e0 + i / (4 * nu), rem = i % (4 * nu), r = rem / nu, a = rem % nu;
          const int k = (int)(lblk[e] - rbase);
          double v = 0.0;
          if (ok && a < nv) {
            const int row = 4 * lcol[e] + r;
            for (int n = 0; n < nv; ++n) v += (double)U[(size_t)n * m_cap * 4 + 4 * row + c] * C[n * ld + a];
          }
          A.vp[((A.blk_off[widx] + k) * 16 + c * 4 + r) * (int64_t)nu + a] = v;
        }
        if (threadIdx.x == 0 && c == 0) {
          int sk = -1;
          for (int e = e0; e < e1; ++e)
            if (lcol[e] == t0) sk = (int)(lblk[e] - rbase);
          A.self_k[widx] = sk;
        }
      }
      __syncthreads();
    }
  }
}

// One warp per atom: cluster size only.
__global__ void cluster_size_kernel(Args<double> A, int32_t* sizes) {
  const int lane = threadIdx.x & 31;
  const int64_t wglobal = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = wglobal; i < A.n_sel; i += wstride) {
    const int64_t a = A.sel[i];
    const double px = A.pos[3 * a], py = A.pos[3 * a + 1], pz = A.pos[3 * a + 2];
    int rx[3], ry[3], rz[3];
    const int nx = cell_range(cell_coord(px, A.cell_len[0], A.ncell[0]), A.ncell[0], rx);
    const int ny = cell_range(cell_coord(py, A.cell_len[1], A.ncell[1]), A.ncell[1], ry);
    const int nz = cell_range(cell_coord(pz, A.cell_len[2], A.ncell[2]), A.ncell[2], rz);
    int count = 0;
    for (int ci = 0; ci < nx * ny * nz; ++ci) {
      const int ix = ci / (ny * nz), iy = (ci / nz) % ny, iz = ci % nz;
      const int c = (rx[ix] * A.ncell[1] + ry[iy]) * A.ncell[2] + rz[iz];
      for (int k = A.cell_start[c] + lane; k < A.cell_start[c + 1]; k += 32) {
        const int b = A.cell_atoms[k];
        const double dx = min_image(A.pos[3 * b] - px, A.box[0]);
        const double dy = min_image(A.pos[3 * b + 1] - py, A.box[1]);
        const double dz = min_image(A.pos[3 * b + 2] - pz, A.box[2]);
        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        count += r2 <= A.R2;
      }
    }
    count = warp_sum(count);
    if (lane == 0) sizes[i] = count;
  }
}

template <typename TV>
void fill_system_args(Args<TV>& A, const mka_system* s) {
  A.n_atoms = s->n_atoms;
  A.row_ptr = s->d_row_ptr;
  A.col = s->d_col;
  A.valH = reinterpret_cast<const TV*>(s->d_valH);
  A.valS = reinterpret_cast<const TV*>(s->d_valS);
  A.pos = s->d_pos;
  for (int d = 0; d < 3; ++d) {
    A.box[d] = s->box[d];
    A.ncell[d] = s->cells.n[d];
    A.cell_len[d] = s->cells.len[d];
  }
  A.R2 = s->R * s->R;
  A.cell_start = s->cells.start;
  A.cell_atoms = s->cells.atoms;
}

size_t dyn_smem_bytes(int nu, int lnnz_cap) {
  size_t off = (size_t)(2 * kMaxCl + 1 + 2 * lnnz_cap) * sizeof(int);
  off = (off + 15) & ~(size_t)15;
  const int ld = nu + 1;
  return off + sizeof(double) * ((size_t)4 * nu * ld + nu + 4 * ((nu + 1) / 2 + 1));
}

template <typename TV, typename T>
mka_status run_columns(mka_system* sys, mka_result* res, const mka_solve_params* prm, int max_cl,
                       cudaStream_t st) {
  Args<TV> A{};
  fill_system_args(A, sys);
  A.sel = res->d_sel;
  A.n_sel = res->n_sel;
  A.p = prm->p;
  A.q = prm->q;
  A.nu = prm->p + prm->q;
  A.cg_tol = prm->cg_tol;
  A.cg_maxit = prm->cg_maxit;
  A.tau = 1e-10;
  A.mcap = 4 * std::max(1, std::min(max_cl, kMaxCl));
  A.lnnz_cap = std::max(1, std::min(max_cl, kMaxCl) * std::max(1, sys->max_row_blocks));
  A.eps = res->d_eps;
  A.w = res->d_w;
  A.nu_eff = res->d_nu_eff;
  A.cg_iters = res->d_cg_iters;
  A.status = res->d_status;
  A.keep = res->keep;
  A.vp = res->d_vp;
  A.blk_off = res->d_blk_off;
  A.self_k = res->d_self;

  const size_t smem = dyn_smem_bytes(A.nu, A.lnnz_cap);
  auto kern = atoms_kernel<TV, T>;
  MKA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, sms = 0, per_sm = 0;
  MKA_CUDA_TRY(cudaGetDevice(&dev));
  MKA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  MKA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
  if (per_sm < 1) return fail(MKA_ERR_INVALID_ARG, "per-atom working set does not fit in shared memory");
  const int64_t slots = std::min<int64_t>(res->n_sel, (int64_t)sms * per_sm);
  A.slot_bytes = sizeof(T) * ((size_t)3 * A.nu + 7) * A.mcap * 4;
  A.slot_bytes = (A.slot_bytes + 255) & ~(size_t)255;
  char* scratch = nullptr;
  int* counter = nullptr;
  MKA_CUDA_TRY(cudaMallocAsync(&scratch, A.slot_bytes * slots + 256, st));
  MKA_CUDA_TRY(cudaMallocAsync(&counter, sizeof(int), st));
  MKA_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int), st));
  A.scratch = scratch;
  A.work_counter = counter;
  kern<<<(unsigned)slots, kThreads, smem, st>>>(A);
  count_launches();
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(scratch, st);
  cudaFreeAsync(counter, st);
  if (e != cudaSuccess) return cuda_fail(e, "atoms_kernel launch");
  return MKA_OK;
}

}  // namespace

mka_status launch_cluster_sizes(const mka_system* sys, const int64_t* d_sel, int64_t n_sel, int32_t* d_sizes,
                                cudaStream_t st) {
  Args<double> A{};
  fill_system_args(A, sys);
  A.sel = d_sel;
  A.n_sel = n_sel;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((n_sel + 7) / 8, 152 * 16);
  cluster_size_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), threads, 0, st>>>(A, d_sizes);
  count_launches();
  MKA_CUDA_TRY(cudaGetLastError());
  return MKA_OK;
}

mka_status launch_columns(mka_system* sys, mka_result* res, const mka_solve_params* prm, int max_cl,
                          cudaStream_t st) {
  const bool mixed = prm->arith != MKA_FP64;
  switch (sys->storage) {
    case MKA_FP64:
      return mixed ? run_columns<double, float>(sys, res, prm, max_cl, st)
                   : run_columns<double, double>(sys, res, prm, max_cl, st);
    case MKA_MIXED_FP32:
      return mixed ? run_columns<float, float>(sys, res, prm, max_cl, st)
                   : run_columns<float, double>(sys, res, prm, max_cl, st);
    default:
      return mixed ? run_columns<__nv_bfloat16, float>(sys, res, prm, max_cl, st)
                   : run_columns<__nv_bfloat16, double>(sys, res, prm, max_cl, st);
  }
}

}  // namespace mka

// ---- fixed-scratch variant (mka_solve_columns_static) ------------------------------------
//
// The same per-atom kernel, FP64 form, with its work queue counter, the atom list
// and every per-CTA work slot carved out of one file-scope device array instead of
// memory allocated per call. Host code cannot use the array's name as a device
// address, so each device's address is looked up once with cudaGetSymbolAddress
// (with that device current) and cached.
static __device__ __align__(256) unsigned char g_static_scratch[MKA_STATIC_SCRATCH_BYTES];

namespace mka {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device (looked up on first use).
mka_status static_scratch_address(void** out) {
  int dev = 0;
  MKA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(MKA_ERR_INVALID_ARG, "device index beyond the supported range");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return MKA_OK;
}

template <typename TV>
mka_status run_columns_static(const mka_system* sys, const int64_t* h_atoms, int64_t n_sel, int p, int q,
                              double cg_tol, int cg_maxit, int max_cl, double* eps, double* w, int32_t* nu_eff,
                              int32_t* cg_iters, int32_t* status, cudaStream_t st) {
  char* base = nullptr;
  mka_status s = static_scratch_address(reinterpret_cast<void**>(&base));
  if (s) return s;
  Args<TV> A{};
  fill_system_args(A, sys);
  A.n_sel = n_sel;
  A.p = p;
  A.q = q;
  A.nu = p + q;
  A.cg_tol = cg_tol;
  A.cg_maxit = cg_maxit;
  A.tau = 1e-10;
  A.mcap = 4 * max_cl;
  A.lnnz_cap = std::max(1, max_cl * std::max(1, sys->max_row_blocks));
  A.eps = eps;
  A.w = w;
  A.nu_eff = nu_eff;
  A.cg_iters = cg_iters;
  A.status = status;
  A.keep = 0;
  // layout: [work counter | 256 B] [atom ids | rounded to 256 B] [per-CTA slots]
  const size_t sel_bytes = ((size_t)n_sel * sizeof(int64_t) + 255) & ~(size_t)255;
  A.slot_bytes = (sizeof(double) * ((size_t)3 * A.nu + 7) * A.mcap * 4 + 255) & ~(size_t)255;
  const size_t fixed = 256 + sel_bytes;
  if (fixed + A.slot_bytes > (size_t)MKA_STATIC_SCRATCH_BYTES)
    return fail(MKA_ERR_INVALID_ARG,
                "mka_solve_columns_static: one work slot (" + std::to_string(A.slot_bytes) + " B) plus the atom list (" +
                    std::to_string(sel_bytes) + " B) exceeds the fixed scratch of " +
                    std::to_string((size_t)MKA_STATIC_SCRATCH_BYTES) +
                    " B; pass fewer atoms, a smaller p + q or a smaller max_cluster_atoms");
  const int64_t slots_fit = (int64_t)(((size_t)MKA_STATIC_SCRATCH_BYTES - fixed) / A.slot_bytes);
  const size_t smem = dyn_smem_bytes(A.nu, A.lnnz_cap);
  auto kern = atoms_kernel<TV, double>;
  MKA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, sms = 0, per_sm = 0;
  MKA_CUDA_TRY(cudaGetDevice(&dev));
  MKA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  MKA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
  if (per_sm < 1) return fail(MKA_ERR_INVALID_ARG, "per-atom working set does not fit in shared memory");
  const int64_t grid = std::min<int64_t>(std::min<int64_t>(n_sel, slots_fit), (int64_t)sms * per_sm);
  A.work_counter = reinterpret_cast<int*>(base);
  A.sel = reinterpret_cast<const int64_t*>(base + 256);
  A.scratch = base + fixed;
  // The counter must start at zero; the atom list is copied in; slots need no clearing
  // (the kernel writes every slot entry before reading it).
  MKA_CUDA_TRY(cudaMemsetAsync(base, 0, 256, st));
  MKA_CUDA_TRY(cudaMemcpyAsync(base + 256, h_atoms, (size_t)n_sel * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  kern<<<(unsigned)grid, kThreads, smem, st>>>(A);
  count_launches();
  MKA_CUDA_TRY(cudaGetLastError());
  return MKA_OK;
}

}  // namespace
}  // namespace mka

extern "C" mka_status mka_solve_columns_static(const mka_system* sys, const int64_t* atoms, int64_t n_sel, int p,
                                               int q, double cg_tol, int cg_maxit, int max_cluster_atoms,
                                               double* eps, double* w, int32_t* nu_eff, int32_t* cg_iters,
                                               int32_t* status, void* stream) {
  using namespace mka;
  if (!sys || !atoms || n_sel < 1) return fail(MKA_ERR_INVALID_ARG, "system, a host atom list and n_sel >= 1 are required");
  if (!eps || !w || !nu_eff || !cg_iters || !status) return fail(MKA_ERR_INVALID_ARG, "every output buffer is required");
  if (p < 1 || q < 0 || p + q > MKA_MAX_NU) return fail(MKA_ERR_INVALID_ARG, "need p >= 1, q >= 0, p + q <= MKA_MAX_NU");
  if (!(cg_tol > 0) || cg_maxit < 1) return fail(MKA_ERR_INVALID_ARG, "need cg_tol > 0, cg_maxit >= 1");
  if (max_cluster_atoms < 1 || max_cluster_atoms > MKA_MAX_CLUSTER_ATOMS)
    return fail(MKA_ERR_INVALID_ARG, "max_cluster_atoms must be in [1, MKA_MAX_CLUSTER_ATOMS]");
  for (int64_t t = 0; t < n_sel; ++t)
    if (atoms[t] < 0 || atoms[t] >= sys->n_atoms) return fail(MKA_ERR_INVALID_ARG, "atom index out of range");
  cudaStream_t st = (cudaStream_t)stream;
  switch (sys->storage) {
    case MKA_FP64:
      return run_columns_static<double>(sys, atoms, n_sel, p, q, cg_tol, cg_maxit, max_cluster_atoms, eps, w, nu_eff,
                                        cg_iters, status, st);
    case MKA_MIXED_FP32:
      return run_columns_static<float>(sys, atoms, n_sel, p, q, cg_tol, cg_maxit, max_cluster_atoms, eps, w, nu_eff,
                                       cg_iters, status, st);
    default:
      return run_columns_static<__nv_bfloat16>(sys, atoms, n_sel, p, q, cg_tol, cg_maxit, max_cluster_atoms, eps, w,
                                               nu_eff, cg_iters, status, st);
  }
}
