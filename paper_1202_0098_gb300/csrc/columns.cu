// Per-column hot path of the multiple Arnoldi method on sm_103a.
//
// One CTA owns one atom a at a time and runs its four columns j = 4a + o
// (o = s, px, py, pz) together, because they share the cluster C_a of the
// real-space projection (Sec. 3). Per atom, in one persistent launch over a
// device work queue:
//   1. cluster extraction: atoms within R of a (minimum image) from the cell
//      list, sorted by atom id; the cluster-local 4x4-block pattern of
//      P H P / P S P is built in shared memory (local column, global block id);
//   2. inner CG for S s_j = e_j (Sec. 2, standard CG, from x0 = 0 or from a
//      learned guess on the 17-atom patch);
//   3. the S-orthonormal basis of K_p(H; e_j) (+) K_q(H; s_j): S-orthogonalise,
//      normalise, k_n = H u_n, next vector k_n or s_j after u_p (Eqs.
//      EQ-REC-UN, EQ-KN-HUN, EQ-MGram-Schmidt, EQ-CALC-S-INV); Gram-Schmidt is
//      one classical pass, coefficients (S u_m)^T l with S u_m kept, corrected to
//      first order by S_r - I (the seam vector gets two full FP64 passes);
//      optionally the s_j chain continues from its raw vectors H^k s_j (the
//      literal direct sum, reading B);
//   4. the projection H_r = U^T K, S_r = U^T (S U), accumulated while the basis
//      grows, written with row j of U and S U to the reduced-problem buffer;
//      the reduced generalized problem (Eq. EQ-SUB-EIG-VEC) and the per-column
//      outputs are the batched kernel of reduced.cu;
//   5. with kept vectors, the pattern rows of U (rho and G are
//      U_i . (C diag(x) V_j) from them and the reduced kernel's C and V_j).
// Breakdown rule: a new vector that keeps no more than 1e-10 of its S-norm
// (S-norm before projection taken from the Pythagorean sum of the removed
// coefficients) is dropped; a dropped s_j is replaced by H u_n, a first chain
// that closes before u_p hands over to s_j, any other breakdown ends the basis.
//
// The vector the SpMV gathers (CG: p; basis: l) lives in shared memory, [row][4 columns]
// interleaved so that one thread owns a row of all four columns; the basis U and S U, s_j,
// the streamed work vectors and S_r - I live in a per-CTA global slot. Arithmetic type T is
// double for the FP64 form and float for the mixed form (values of any storage type are
// decoded to T on load).
//
// Mixed form. s_j is nearly inside K_p(H; e_j): the seam vector keeps about 1%
// of its S-norm, so any perturbation of the first chain at FP32 rounding level
// turns the direction the second chain starts from by about 100 times as much.
// The basis is therefore carried as FP32 pairs (hi + lo, about 48 significant
// bits): H u takes error-free FP32 products and compensated sums on the hi part,
// the Gram-Schmidt update likewise, and only products with the lo parts are
// rounded. s_j is refined to FP64 accuracy by CG on the true residual (computed
// the same way) and orthogonalised in FP64 at the seam. S u, the Gram-Schmidt
// coefficients and the projected matrices are plain FP32 from the hi parts
// (their errors stay inside the span or enter the reduced problem unmagnified);
// the reduced solve, the mu bisection and all cross-thread sums are FP64.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "mka_internal.h"

namespace mka {
namespace {

constexpr int kMaxWarps = 16;   // CTAs of up to 512 threads
constexpr int kMaxCl = MKA_MAX_CLUSTER_ATOMS;  // power of two (bitonic sort size bound)
static_assert((kMaxCl & (kMaxCl - 1)) == 0, "cluster cap must be a power of two");

__host__ __device__ constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

enum ColStatus { ST_OK = 0, ST_NOT_SPD = MKA_ERR_NOT_SPD, ST_NOCONV = MKA_ERR_NO_CONVERGENCE,
                 ST_BREAKDOWN = MKA_ERR_BREAKDOWN, ST_TOOLARGE = MKA_ERR_CLUSTER_TOO_LARGE };
enum Src { SRC_E = 0, SRC_H = 1, SRC_S = 2, SRC_R = 3 };   // SRC_R: a raw power H^k s_j (reading B)
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
  const float* posf;      // positions rounded to FP32, for the distance prefilter
  double box[3];
  double R2;
  float pre_lo, pre_hi;   // FP32 prefilter: inside below pre_lo * R^2, outside above pre_hi * R^2
  int ncell[3];
  double cell_len[3];
  const int32_t* cell_start;
  const int32_t* cell_atoms;
  // work
  const int64_t* sel;
  const int32_t* order;   // optional work order (selection indices), NULL = selection order
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
  int clcap;           // cluster list capacity (power of two)
  // outputs
  double* eps;
  double* w;
  int32_t* nu_eff;
  int32_t* cg_iters;
  int32_t* status;
  int keep;
  double* vp;
  const int64_t* blk_off;
  // learned warm start: predicted s_j on the 17-atom patch, or NULL for x0 = 0
  const float* x0;          // [4 n_sel][68]
  const int32_t* patch;     // [n_sel][17] atom ids (-1: none)
  int32_t* fallback;        // [4 n_sel]: 1 where the prediction was no better than x0 = 0 (may be NULL)
  // CG-only mode: stop after the inner CG and write s_j on the patch (training targets)
  int cg_only;
  float* cg_target;         // [4 n_sel][68]
  // 1: the s_j chain continues from its raw vector (the literal direct sum K_p(H; e_j) + K_q(H; s_j))
  int mode_b;
  // s_j of an earlier solve of the same atoms as the CG start: its clusters' atom ids [n_sel][prev_cap]
  // (ascending, -1 beyond the count) and values [4 n_sel][4 prev_cap] (NULL: not used)
  const int32_t* prev_cl;
  const double* prev_s;
  int prev_cap;
  // keep this solve's s_j the same way (NULL: not kept), keep_cap atoms per cluster
  int32_t* keep_cl;
  double* keep_s;
  int keep_cap;
  double* red;              // reduced-problem buffer, lane-interleaved per 32 columns
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
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k * 4 + threadIdx.x];
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

// Is atom b within R of the point (px, py, pz) (minimum image)? An FP32 test decides every
// candidate whose FP32 distance is clear of the boundary by more than its rounding error
// (relative margin max(1e-3, 1e-5 L / R) on R^2); the rest get the exact FP64 test.
__device__ __forceinline__ bool within_R(const double* pos, const float* posf, const double box[3], double R2,
                                         float pre_lo, float pre_hi, int b, double px, double py, double pz,
                                         float pxf, float pyf, float pzf) {
  const float Lx = (float)box[0], Ly = (float)box[1], Lz = (float)box[2];
  float fx = posf[3 * b] - pxf, fy = posf[3 * b + 1] - pyf, fz = posf[3 * b + 2] - pzf;
  fx -= Lx * rintf(fx / Lx);
  fy -= Ly * rintf(fy / Ly);
  fz -= Lz * rintf(fz / Lz);
  const float r2f = fx * fx + fy * fy + fz * fz;
  const float R2f = (float)R2;
  if (r2f < pre_lo * R2f) return true;
  if (r2f > pre_hi * R2f) return false;
  const double dx = pos[3 * b] - px - box[0] * rint((pos[3 * b] - px) / box[0]);
  const double dy = pos[3 * b + 1] - py - box[1] * rint((pos[3 * b + 1] - py) / box[1]);
  const double dz = pos[3 * b + 2] - pz - box[2] * rint((pos[3 * b + 2] - pz) / box[2]);
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  return r2 <= R2;
}

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
// returns the count (which may exceed A.clcap: then nothing beyond A.clcap is stored).
template <typename TV>
__device__ int gather_cluster(const Args<TV>& A, int64_t a, int* cl, int* cnt) {
  if (threadIdx.x == 0) *cnt = 0;
  __syncthreads();
  const double px = A.pos[3 * a], py = A.pos[3 * a + 1], pz = A.pos[3 * a + 2];
  const float pxf = A.posf[3 * a], pyf = A.posf[3 * a + 1], pzf = A.posf[3 * a + 2];
  int rx[3], ry[3], rz[3];
  const int nx = cell_range(cell_coord(px, A.cell_len[0], A.ncell[0]), A.ncell[0], rx);
  const int ny = cell_range(cell_coord(py, A.cell_len[1], A.ncell[1]), A.ncell[1], ry);
  const int nz = cell_range(cell_coord(pz, A.cell_len[2], A.ncell[2]), A.ncell[2], rz);
  const int ncells = nx * ny * nz;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int ci = wid; ci < ncells; ci += (int)(blockDim.x >> 5)) {
    const int ix = ci / (ny * nz), iy = (ci / nz) % ny, iz = ci % nz;
    const int c = (rx[ix] * A.ncell[1] + ry[iy]) * A.ncell[2] + rz[iz];
    const int s0 = A.cell_start[c], s1 = A.cell_start[c + 1];
    for (int k = s0 + lane; k < s1; k += 32) {
      const int b = A.cell_atoms[k];
      if (within_R(A.pos, A.posf, A.box, A.R2, A.pre_lo, A.pre_hi, b, px, py, pz, pxf, pyf, pzf)) {
        const int idx = atomicAdd(cnt, 1);
        if (idx < A.clcap) cl[idx] = b;
      }
    }
  }
  __syncthreads();
  return *cnt;
}

// Ascending bitonic sort of cl[0..n) (n <= the list's power-of-two capacity), padding with INT_MAX.
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

// 16-byte (float) / 2 x 16-byte (double) access to one [row][4] entry of a work vector.
__device__ __forceinline__ void ld4(const float* p, float v[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void ld4(const double* p, double v[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, float a0, float a1, float a2, float a3) {
  *reinterpret_cast<float4*>(p) = make_float4(a0, a1, a2, a3);
}
__device__ __forceinline__ void st4(double* p, double a0, double a1, double a2, double a3) {
  reinterpret_cast<double2*>(p)[0] = make_double2(a0, a1);
  reinterpret_cast<double2*>(p)[1] = make_double2(a2, a3);
}

// y = A x on the cluster for the columns in `mask` (bit c = column c), rows 4t + i;
// x, y are [m][4] in shared memory; other columns of y are left untouched.
template <typename TV, typename T>
__device__ __forceinline__ void spmm4(const TV* __restrict__ val, const int* lrow, const uint16_t* lcol,
                                      const int* rbase, const uint8_t* loff, int ncl, const T* __restrict__ x, T* __restrict__ y,
                                      int mask) {
  const int m = 4 * ncl;
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    const int t = r >> 2, i = r & 3;
    const int rb = rbase[t];
    T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    const int e1 = lrow[t + 1];
#pragma unroll 4
    for (int e = lrow[t]; e < e1; ++e) {
      T v[4];
      RowLoad<TV, T>::load(val, rb + loff[e], i, v);
      const T* xb = x + (size_t)lcol[e] * 16;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        T xk[4];
        ld4(xb + 4 * k, xk);
        a0 += v[k] * xk[0];
        a1 += v[k] * xk[1];
        a2 += v[k] * xk[2];
        a3 += v[k] * xk[3];
      }
    }
    if (mask == 15) {
      st4(y + 4 * r, a0, a1, a2, a3);
    } else {
      if (mask & 1) y[4 * r + 0] = a0;
      if (mask & 2) y[4 * r + 1] = a1;
      if (mask & 4) y[4 * r + 2] = a2;
      if (mask & 8) y[4 * r + 3] = a3;
    }
  }
  __syncthreads();
}

// r = e_j - A (hi + lo) for x given as an FP32 pair: the hi part with error-free products and
// compensated sums as in resid4_comp, the small lo part (|lo| <= ulp(hi) / 2) in plain FP32.
template <typename TV>
__device__ void resid4_comp2(const TV* __restrict__ val, const int* lrow, const uint16_t* lcol, const int* rbase, const uint8_t* loff,
                             int ncl, const float* __restrict__ xh, const float* __restrict__ xl, float* __restrict__ r,
                             int jrow0) {
  for (int row = threadIdx.x; row < 4 * ncl; row += blockDim.x) {
    const int t = row >> 2, i = row & 3;
    const int rb = rbase[t];
    float hi[4] = {0, 0, 0, 0}, lo[4] = {0, 0, 0, 0}, sl[4] = {0, 0, 0, 0};
    for (int e = lrow[t]; e < lrow[t + 1]; ++e) {
      float v[4];
      RowLoad<TV, float>::load(val, rb + loff[e], i, v);
      const float* xb = xh + (size_t)lcol[e] * 16;
      const float* xc = xl + (size_t)lcol[e] * 16;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float xk[4], xs[4];
        ld4(xb + 4 * k, xk);
        ld4(xc + 4 * k, xs);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float p = __fmul_rn(v[k], xk[q]);
          const float pe = fmaf(v[k], xk[q], -p);
          const float s = __fadd_rn(hi[q], p);
          const float bb = __fsub_rn(s, hi[q]);
          const float err = __fadd_rn(__fsub_rn(hi[q], __fsub_rn(s, bb)), __fsub_rn(p, bb));
          hi[q] = s;
          lo[q] = __fadd_rn(lo[q], __fadd_rn(err, pe));
          sl[q] = fmaf(v[k], xs[q], sl[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float e = (row == jrow0 + q) ? 1.0f : 0.0f;
      r[4 * row + q] = __fsub_rn(__fsub_rn(__fsub_rn(e, hi[q]), lo[q]), sl[q]);
    }
  }
  __syncthreads();
}

// y = A x for x given as an FP32 pair (xh + xl), the result as an FP32 pair (yh + yl), for the
// columns in `mask`: the hi part with error-free products and compensated sums, the lo part in
// plain FP32, renormalised so that yh is the sum rounded to FP32 and |yl| <= ulp(yh) / 2
// (yl == nullptr: yh only). Other columns are left untouched.
template <typename TV>
__device__ void spmm4_pair(const TV* __restrict__ val, const int* lrow, const uint16_t* lcol, const int* rbase, const uint8_t* loff,
                           int ncl, const float* __restrict__ xh, const float* __restrict__ xl, float* __restrict__ yh,
                           float* __restrict__ yl, int mask) {
  for (int row = threadIdx.x; row < 4 * ncl; row += blockDim.x) {
    const int t = row >> 2, i = row & 3;
    const int rb = rbase[t];
    float hi[4] = {0, 0, 0, 0}, lo[4] = {0, 0, 0, 0};
    const int e1 = lrow[t + 1];
    for (int e = lrow[t]; e < e1; ++e) {
      float v[4];
      RowLoad<TV, float>::load(val, rb + loff[e], i, v);
      const float* xb = xh + (size_t)lcol[e] * 16;
      const float* xc = xl + (size_t)lcol[e] * 16;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float xk[4], xs[4];
        ld4(xb + 4 * k, xk);
        ld4(xc + 4 * k, xs);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float p = __fmul_rn(v[k], xk[q]);
          const float pe = fmaf(v[k], xk[q], -p);
          const float s = __fadd_rn(hi[q], p);
          const float bb = __fsub_rn(s, hi[q]);
          const float err = __fadd_rn(__fsub_rn(hi[q], __fsub_rn(s, bb)), __fsub_rn(p, bb));
          hi[q] = s;
          lo[q] = __fadd_rn(lo[q], __fadd_rn(err, fmaf(v[k], xs[q], pe)));
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (!(mask >> q & 1)) continue;
      const float s = __fadd_rn(hi[q], lo[q]);
      yh[4 * row + q] = s;
      if (yl) yl[4 * row + q] = __fsub_rn(lo[q], __fsub_rn(s, hi[q]));
    }
  }
  __syncthreads();
}

// yH = H x and yS = S x in one pass over the shared block pattern (x read once), for the
// columns in `mask`; FP64 form.
template <typename TV, typename T>
__device__ void spmm4_hs(const TV* __restrict__ valH, const TV* __restrict__ valS, const int* lrow,
                         const uint16_t* lcol, const int* rbase, const uint8_t* loff, int ncl, const T* __restrict__ x, T* __restrict__ yH,
                         T* __restrict__ yS, int mask) {
  for (int r = threadIdx.x; r < 4 * ncl; r += blockDim.x) {
    const int t = r >> 2, i = r & 3;
    const int rb = rbase[t];
    T h[4] = {0, 0, 0, 0}, s[4] = {0, 0, 0, 0};
    const int e1 = lrow[t + 1];
#pragma unroll 2
    for (int e = lrow[t]; e < e1; ++e) {
      T vh[4], vs[4];
      RowLoad<TV, T>::load(valH, rb + loff[e], i, vh);
      RowLoad<TV, T>::load(valS, rb + loff[e], i, vs);
      const T* xb = x + (size_t)lcol[e] * 16;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        T xk[4];
        ld4(xb + 4 * k, xk);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          h[q] += vh[k] * xk[q];
          s[q] += vs[k] * xk[q];
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (mask >> q & 1) {
        yH[4 * r + q] = h[q];
        yS[4 * r + q] = s[q];
      }
  }
  __syncthreads();
}

// The FP32-pair form of spmm4_hs: x = xh + xl; H x as a pair (yHh + yHl) with error-free
// products and compensated sums on the hi part (as spmm4_pair); S x in plain FP32 from the hi
// part (S u enters the coefficients, whose errors stay in the span, and S_r, unmagnified).
template <typename TV>
__device__ void spmm4_pair_hs(const TV* __restrict__ valH, const TV* __restrict__ valS, const int* lrow,
                              const uint16_t* lcol, const int* rbase, const uint8_t* loff, int ncl, const float* __restrict__ xh,
                              const float* __restrict__ xl, float* __restrict__ yHh, float* __restrict__ yHl,
                              float* __restrict__ yS, int mask) {
  for (int row = threadIdx.x; row < 4 * ncl; row += blockDim.x) {
    const int t = row >> 2, i = row & 3;
    const int rb = rbase[t];
    float hh[4] = {0, 0, 0, 0}, hl[4] = {0, 0, 0, 0}, sh[4] = {0, 0, 0, 0};
    const int e1 = lrow[t + 1];
    for (int e = lrow[t]; e < e1; ++e) {
      float vh[4], vs[4];
      RowLoad<TV, float>::load(valH, rb + loff[e], i, vh);
      RowLoad<TV, float>::load(valS, rb + loff[e], i, vs);
      const float* xb = xh + (size_t)lcol[e] * 16;
      const float* xc = xl + (size_t)lcol[e] * 16;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float xk[4], xs[4];
        ld4(xb + 4 * k, xk);
        ld4(xc + 4 * k, xs);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          {
            const float p = __fmul_rn(vh[k], xk[q]);
            const float pe = fmaf(vh[k], xk[q], -p);
            const float s = __fadd_rn(hh[q], p);
            const float bb = __fsub_rn(s, hh[q]);
            const float err = __fadd_rn(__fsub_rn(hh[q], __fsub_rn(s, bb)), __fsub_rn(p, bb));
            hh[q] = s;
            hl[q] = __fadd_rn(hl[q], __fadd_rn(err, fmaf(vh[k], xs[q], pe)));
          }
          sh[q] = fmaf(vs[k], xk[q], sh[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (!(mask >> q & 1)) continue;
      const float s = __fadd_rn(hh[q], hl[q]);
      yHh[4 * row + q] = s;
      yHl[4 * row + q] = __fsub_rn(hl[q], __fsub_rn(s, hh[q]));
      yS[4 * row + q] = sh[q];
    }
  }
  __syncthreads();
}

// Per-column dot products over the cluster rows: per-thread partial sums in T
// (a few terms each), combined across threads in FP64.
template <typename T>
__device__ __forceinline__ void dot4(const T* a, const T* b, int m, double* red, double* out) {
  T part[4] = {0, 0, 0, 0};
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
#pragma unroll
    for (int c = 0; c < 4; ++c) part[c] += a[4 * r + c] * b[4 * r + c];
  }
  double acc[4] = {(double)part[0], (double)part[1], (double)part[2], (double)part[3]};
  cta_sum4(acc, red, out);
}

// ---- shared state of one atom --------------------------------------------------------
struct AtomState {
  int n[4], src[4], seam_done[4], active[4], accept[4], act[4], next_s[4], proj[4], next_raw[4];
  int it[4], cg_active[4], status[4];
  double beta_inv[4], csum[4], rr[4], alpha[4], beta_cg[4], cg_stop[4];
  int ncl, t0, flag, n_max, proj_any, acc_mask, act_mask;
};

// One Gram-Schmidt coefficient sweep over u_0..u_{nmax-1} (one warp per vector, lanes over
// rows): coef[mm][c] = (S u_mm)^T l for columns whose basis holds mm (when do_coef), and, for
// columns with a pending projection column pn = n - 1, H_r[mm][pn] = u_mm^T (H u_pn) and
// S_r[mm][pn] = u_mm^T (S u_pn) written (with their mirror) to the reduced-problem buffer of
// column col0 + c, and S_r - I to Es ([4][nu][nu], FP32).
template <typename T>
__device__ void gs_sweep(const T* U, const T* SU, const T* L, const T* KV, const T* SV, int m, int m_cap, int nmax,
                         bool do_coef, const AtomState& st, double* coef, T* coefT, double* red, int64_t col0,
                         int nu, float* Es) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const bool proj = st.proj_any;
  for (int mm = wid; mm < nmax; mm += (int)(blockDim.x >> 5)) {
    const T* su = SU + (size_t)mm * m_cap * 4;
    const T* u = U + (size_t)mm * m_cap * 4;
    T pc[4] = {0, 0, 0, 0}, ph[4] = {0, 0, 0, 0}, ps[4] = {0, 0, 0, 0};
#pragma unroll 2
    for (int r = lane; r < m; r += 32) {
      if (do_coef) {
#pragma unroll
        for (int c = 0; c < 4; ++c) pc[c] += su[4 * r + c] * L[4 * r + c];
      }
      if (proj) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const T uv = u[4 * r + c];
          ph[c] += uv * KV[4 * r + c];
          ps[c] += uv * SV[4 * r + c];
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (do_coef) pc[c] = warp_sum(pc[c]);
      if (proj) {
        ph[c] = warp_sum(ph[c]);
        ps[c] = warp_sum(ps[c]);
      }
    }
    if (lane < 4) {
      const int c = lane;
      if (do_coef) {
        const bool use = st.active[c] && mm < st.n[c];
        coef[mm * 4 + c] = use ? (double)pc[c] : 0.0;
        coefT[mm * 4 + c] = use ? pc[c] : (T)0;
      }
      if (proj && st.proj[c] && mm < st.n[c]) {
        const int pn = st.n[c] - 1;
        const int64_t col = col0 + c;
        double* H = red + (size_t)(col >> 5) * red_block_doubles(nu) * 32 + (col & 31);
        double* S = H + (size_t)nu * nu * 32;
        H[(size_t)(mm * nu + pn) * 32] = (double)ph[c];
        H[(size_t)(pn * nu + mm) * 32] = (double)ph[c];
        S[(size_t)(mm * nu + pn) * 32] = (double)ps[c];
        S[(size_t)(pn * nu + mm) * 32] = (double)ps[c];
        const float ev = (float)(ps[c] - (mm == pn ? (T)1 : (T)0));
        Es[(c * nu + mm) * nu + pn] = ev;
        Es[(c * nu + pn) * nu + mm] = ev;
      }
    }
  }
  __syncthreads();
}

// The seam vector of the FP32 form in FP64: two classical Gram-Schmidt passes on s_j (FP64, in place)
// against the basis pairs for the columns in smask, the result left in l as a pair. Kept out of line:
// it runs once per atom, and inlined it would crowd the instruction cache of the basis loop.
__device__ __noinline__ void seam_fp64(const float* SU, const float* U, const float* Ulo, double* SJd, float* Lv,
                                       float* Llo, double* coef, AtomState& st, int m, int m_cap, int nmax, int smask) {
  using T = float;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  if (threadIdx.x < 4) st.csum[threadIdx.x] = (smask >> threadIdx.x & 1) ? 0.0 : st.csum[threadIdx.x];
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    for (int mm = wid; mm < nmax; mm += nwarp) {
      const T* su = SU + (size_t)mm * m_cap * 4;
      double acc[4] = {0, 0, 0, 0};
      for (int r = lane; r < m; r += 32)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (smask >> q & 1) acc[q] += (double)su[4 * r + q] * SJd[4 * r + q];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = warp_sum(acc[q]);
      if (lane < 4) coef[mm * 4 + lane] = ((smask >> lane & 1) && mm < st.n[lane]) ? acc[lane] : 0.0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
      const int r = i >> 2, q = i & 3;
      if (!(smask >> q & 1)) continue;
      double v = SJd[i];
      for (int mm = 0; mm < nmax; ++mm) {
        const size_t o = (size_t)mm * m_cap * 4 + 4 * r + q;
        const double cf = coef[mm * 4 + q];
        if (cf != 0.0) v -= cf * ((double)U[o] + (double)Ulo[o]);
      }
      SJd[i] = v;
    }
    if (threadIdx.x < 4 && (smask >> threadIdx.x & 1)) {
      double s2 = 0;
      for (int mm = 0; mm < nmax; ++mm) s2 += coef[mm * 4 + threadIdx.x] * coef[mm * 4 + threadIdx.x];
      st.csum[threadIdx.x] += s2;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < 4 * m; i += blockDim.x)
    if (smask >> (i & 3) & 1) {
      const T h = (T)SJd[i];
      Lv[i] = h;
      Llo[i] = (float)(SJd[i] - (double)h);
    }
  __syncthreads();
}

// s_j dropped as already in the span (columns in kmask): l becomes u_n, the last accepted vector, and
// KV = H u_n is formed again (KV held H applied to the dropped s_j). Kept out of line: it runs at most
// once per column, and inlined its product would crowd the instruction cache of the basis loop.
template <typename TV, typename T>
__device__ __noinline__ void reload_hu(const TV* __restrict__ valH, const int* lrow, const uint16_t* lcol,
                                       const int* rbase, const uint8_t* loff, int ncl, int m, int m_cap, int kmask,
                                       const AtomState& st, const T* U, const float* Ulo, T* Lv, float* Llo, T* KV,
                                       float* Klo) {
  for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
    const int r = i >> 2, c = i & 3;
    if (!(kmask >> c & 1)) continue;
    const size_t o = (size_t)(st.n[c] - 1) * m_cap * 4 + 4 * r + c;
    Lv[i] = U[o];
    if constexpr (sizeof(T) == 4) Llo[i] = Ulo[o];
  }
  __syncthreads();
  if constexpr (sizeof(T) == 4)
    spmm4_pair<TV>(valH, lrow, lcol, rbase, loff, ncl, Lv, Llo, KV, Klo, kmask);
  else
    spmm4<TV, T>(valH, lrow, lcol, rbase, loff, ncl, Lv, KV, kmask);
}

// Reading B: the next raw vector of the s_j chain for the columns in rmask, H applied to s_j (columns in
// pmask, copied from s_j first) or to the previous raw vector, scaled by a power of two near its inverse
// 2-norm (exact for both halves of a pair); left in RW (and RWlo). Kept out of line: it runs a few times
// per atom, and inlined its products would crowd the instruction cache of the basis loop.
template <typename TV, typename T>
__device__ __noinline__ void raw_chain_step(const TV* __restrict__ valH, const int* lrow, const uint16_t* lcol,
                                            const int* rbase, const uint8_t* loff, int ncl, int m, int pmask, int rmask,
                                            const T* SJ, const double* SJd, T* RW, T* RWN, float* RWlo, float* RWNlo,
                                            double* red, double* sums, T* scal) {
  for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
    const int c = i & 3;
    if (!(pmask >> c & 1)) continue;
    if constexpr (sizeof(T) == 4) {
      const float h = (float)SJd[i];
      RW[i] = h;
      RWlo[i] = (float)(SJd[i] - (double)h);
    } else {
      RW[i] = SJ[i];
    }
  }
  __syncthreads();
  if constexpr (sizeof(T) == 4)
    spmm4_pair<TV>(valH, lrow, lcol, rbase, loff, ncl, reinterpret_cast<const float*>(RW), RWlo,
                   reinterpret_cast<float*>(RWN), RWNlo, rmask);
  else
    spmm4<TV, T>(valH, lrow, lcol, rbase, loff, ncl, RW, RWN, rmask);
  dot4<T>(RWN, RWN, m, red, sums);
  if (threadIdx.x < 4) {
    const int c = threadIdx.x;
    scal[c] = (T)1;
    if (rmask >> c & 1) {
      const double nrm = sqrt(fmax(sums[c], 0.0));
      scal[c] = nrm > 0.0 ? (T)ldexp(1.0, -ilogb(nrm)) : (T)1;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
    const int c = i & 3;
    if (!(rmask >> c & 1)) continue;
    RW[i] = RWN[i] * scal[c];
    if constexpr (sizeof(T) == 4) RWlo[i] = RWNlo[i] * (float)scal[c];
  }
  __syncthreads();
}

// Resident CTAs per SM the register budget is cut for: the FP32 form at 256 threads runs five (48
// registers: 124.8 against 132.8 ms per 16,384 atoms at four, the kernel waits on memory and gains
// from the extra warps; six at 40 registers spill and lose); otherwise 1024 threads per SM.
template <typename T, int NT>
constexpr int atoms_min_blocks() { return (sizeof(T) == 4 && NT == 256) ? 5 : 1024 / NT; }

template <typename TV, typename T, int NT>
__global__ void __launch_bounds__(NT, atoms_min_blocks<T, NT>()) atoms_kernel(const Args<TV> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ AtomState st;
  __shared__ double red[2 * kMaxWarps * 4];
  __shared__ double sums[4];
  __shared__ T scal[12];                 // CG alpha [0..4), CG beta [4..8), 1 / beta of the basis [8..12)
  __shared__ int64_t cur_atom;
  __shared__ int cnt;

  const int nu = A.nu;
  const int m_cap = A.mcap;
  // cluster list, local row pointers and each local row's first global block; then per local
  // block its local column and its offset within the global row
  int* cl = reinterpret_cast<int*>(smem_raw);                            // clcap
  int* lrow = cl + A.clcap;                                               // clcap + 1
  int* rbase = lrow + A.clcap + 1;                                        // clcap
  uint16_t* lcol = reinterpret_cast<uint16_t*>(rbase + A.clcap);          // lnnz_cap
  uint8_t* loff = reinterpret_cast<uint8_t*>(lcol + A.lnnz_cap);          // lnnz_cap
  size_t off = (size_t)(3 * A.clcap + 1) * sizeof(int) + (size_t)A.lnnz_cap * (sizeof(uint16_t) + 1);
  off = (off + 15) & ~(size_t)15;
  // Shared memory holds the vector the SpMV gathers through the cluster pattern; the vectors
  // that are only streamed row by row live in the CTA's global slot.
  unsigned char* region = smem_raw + off;
  T* V0 = reinterpret_cast<T*>(region);     // CG: p     basis: l
  // FP32 form only: the low half of l
  float* Llo = reinterpret_cast<float*>(V0 + (size_t)m_cap * 4);
  // Gram-Schmidt coefficients [nu][4] in FP64 and in the arithmetic type
  double* coef = reinterpret_cast<double*>(region + (size_t)m_cap * 4 * (sizeof(T) + (sizeof(T) == 4 ? 4 : 0)));
  T* coefT = reinterpret_cast<T*>(coef + (size_t)nu * 4);

  char* slot = A.scratch + (size_t)blockIdx.x * A.slot_bytes;
  T* U = reinterpret_cast<T*>(slot);                 // [nu][m_cap][4]
  T* SU = U + (size_t)nu * m_cap * 4;                // [nu][m_cap][4]
  T* SJ = SU + (size_t)nu * m_cap * 4;               // s_j, [m_cap][4]
  double* SJd = reinterpret_cast<double*>(slot + align_up(sizeof(T) * ((size_t)2 * nu + 1) * m_cap * 4, 256));
  (void)SJd;   // FP32 arithmetic only: s_j in FP64 for the seam [m_cap][4]
  // S_r - I of the four columns' bases so far, [4][nu][nu] FP32
  float* Es = reinterpret_cast<float*>(reinterpret_cast<char*>(SJd) + align_up(sizeof(double) * 4 * (size_t)m_cap, 256));
  T* V1 = reinterpret_cast<T*>(reinterpret_cast<char*>(Es) + align_up(sizeof(float) * 4 * (size_t)nu * nu, 256));
  T* V2 = V1 + (size_t)m_cap * 4;   // V1: CG S p, basis S l then S u_{n-1}; V2: CG r, basis H u_{n-1}
  // FP32 arithmetic only: the low half of H u_{n-1} [m_cap][4], low halves of the basis [nu][m_cap][4]
  float* Klo = reinterpret_cast<float*>(V2 + (size_t)m_cap * 4);
  float* Ulo = Klo + (size_t)m_cap * 4;
  (void)Ulo;
  // reading B: the raw vector of the s_j chain and H applied to it, [m_cap][4] each (with low halves in
  // the FP32 form)
  T* RW = reinterpret_cast<T*>(reinterpret_cast<char*>(V2 + (size_t)m_cap * 4) +
                               align_up(sizeof(T) == 4 ? sizeof(float) * ((size_t)nu + 1) * m_cap * 4 : 0, 256));
  T* RWN = RW + (size_t)m_cap * 4;
  float* RWlo = reinterpret_cast<float*>(RWN + (size_t)m_cap * 4);
  float* RWNlo = RWlo + (size_t)m_cap * 4;
  (void)Llo;
  (void)Klo;

  for (;;) {
    if (threadIdx.x == 0) {
      const int64_t w = atomicAdd(A.work_counter, 1);
      cur_atom = w;
    }
    __syncthreads();
    if (cur_atom >= A.n_sel) break;
    const int64_t widx = A.order ? (int64_t)A.order[cur_atom] : cur_atom;
    const int64_t atom = A.sel[widx];

    // ---- 1. cluster ----------------------------------------------------------------
    const int ncl_raw = gather_cluster(A, atom, cl, &cnt);
    if (ncl_raw > A.clcap || 4 * ncl_raw > m_cap) {
      for (int c = threadIdx.x; c < 4; c += blockDim.x) {   // the reduced pass writes zero outputs
        const int64_t col = 4 * widx + c;
        A.status[col] = ST_TOOLARGE;
        A.nu_eff[col] = 0;
        A.cg_iters[col] = 0;
      }
      if (A.keep) {
        const int nrow = A.row_ptr[atom + 1] - A.row_ptr[atom];
        double* vpa = A.vp + A.blk_off[widx] * 16 * (int64_t)nu;
        for (int i = threadIdx.x; i < nrow * 16 * nu; i += blockDim.x) vpa[i] = 0.0;
      }
      __syncthreads();
      continue;
    }
    const int ncl = ncl_raw;
    sort_cluster(cl, ncl);
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
      for (int c = threadIdx.x; c < 4; c += blockDim.x) {
        A.status[4 * widx + c] = ST_TOOLARGE;
        A.nu_eff[4 * widx + c] = 0;
        A.cg_iters[4 * widx + c] = 0;
      }
      if (A.keep) {
        const int nrow = A.row_ptr[atom + 1] - A.row_ptr[atom];
        double* vpa = A.vp + A.blk_off[widx] * 16 * (int64_t)nu;
        for (int i = threadIdx.x; i < nrow * 16 * nu; i += blockDim.x) vpa[i] = 0.0;
      }
      __syncthreads();
      continue;
    }
    for (int t = threadIdx.x; t < ncl; t += blockDim.x) {
      const int b = cl[t];
      const int k0 = A.row_ptr[b];
      int e = lrow[t];
      rbase[t] = k0;
      for (int k = k0; k < A.row_ptr[b + 1]; ++k) {   // rows hold at most 255 blocks (checked at setup)
        const int lc = find_local(cl, ncl, A.col[k]);
        if (lc >= 0) {
          lcol[e] = (uint16_t)lc;
          loff[e] = (uint8_t)(k - k0);
          ++e;
        }
      }
    }
    const int m = 4 * ncl;
    const int t0 = st.t0;
    // ---- 2. inner CG: S s = e_j from x0 = 0 or the learned patch values ----------------
    T* P = V0;
    T* AP = V1;
    T* R = V2;
    for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
      SJ[i] = 0;
      P[i] = 0;
    }
    if (threadIdx.x < 4) {
      const int c = threadIdx.x;
      st.rr[c] = 1.0;
      st.it[c] = 0;
      st.status[c] = ST_OK;
      st.act[c] = 0;    // reused: warm-start fallback flag
    }
    __syncthreads();
    if (A.keep_cl)
      for (int t = threadIdx.x; t < A.keep_cap; t += blockDim.x) A.keep_cl[widx * A.keep_cap + t] = t < ncl ? cl[t] : -1;
    if (A.x0 || A.prev_s) {
      if (A.prev_s) {   // an earlier s_j on this atom's cluster, matched by atom id (atoms new to the cluster start at 0)
        const int32_t* pc = A.prev_cl + widx * A.prev_cap;
        int np = 0;
        while (np < A.prev_cap && pc[np] >= 0) ++np;
        for (int t = threadIdx.x; t < ncl; t += blockDim.x) {
          int lo = 0, hi = np - 1, f = -1;
          while (lo <= hi) {
            const int mid = (lo + hi) >> 1;
            if (pc[mid] == cl[t]) { f = mid; break; }
            if (pc[mid] < cl[t]) lo = mid + 1; else hi = mid - 1;
          }
          if (f < 0) continue;
#pragma unroll
          for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int o = 0; o < 4; ++o) {
              const T v = (T)A.prev_s[(4 * widx + c) * (4 * (int64_t)A.prev_cap) + 4 * f + o];
              SJ[4 * (4 * t + o) + c] = v;
              P[4 * (4 * t + o) + c] = v;
            }
        }
      } else {
        for (int i = threadIdx.x; i < 4 * 68; i += blockDim.x) {   // (column, patch atom, orbital)
          const int c = i / 68, rem = i % 68, k = rem >> 2, o = rem & 3;
          const int pa = A.patch[widx * 17 + k];
          const int lk = pa >= 0 ? find_local(cl, ncl, pa) : -1;
          if (lk < 0) continue;
          const T v = (T)A.x0[(4 * widx + c) * 68 + rem];
          SJ[4 * (4 * lk + o) + c] = v;
          P[4 * (4 * lk + o) + c] = v;
        }
      }
      __syncthreads();
      spmm4<TV, T>(A.valS, lrow, lcol, rbase, loff, ncl, P, AP, 15);
      for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
        const int r = i >> 2, c = i & 3;
        R[i] = ((r == 4 * t0 + c) ? (T)1 : (T)0) - AP[i];
      }
      __syncthreads();
      dot4<T>(R, R, m, red, sums);
      if (threadIdx.x < 4) {
        const int c = threadIdx.x;
        if (!(sums[c] < 1.0)) {
          st.act[c] = 1;         // no better than x0 = 0: start from zero
        } else {
          st.rr[c] = sums[c];
        }
      }
      __syncthreads();
      for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
        const int r = i >> 2, c = i & 3;
        if (st.act[c]) {
          SJ[i] = 0;
          R[i] = (r == 4 * t0 + c) ? (T)1 : (T)0;
        }
        P[i] = R[i];
      }
    } else {
      for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
        const int r = i >> 2, c = i & 3;
        const T e = (r == 4 * t0 + c) ? (T)1 : (T)0;
        R[i] = e;
        P[i] = e;
      }
    }
    if (threadIdx.x < 4) {
      st.cg_stop[threadIdx.x] = A.cg_tol;
      st.cg_active[threadIdx.x] = sqrt(st.rr[threadIdx.x]) > A.cg_tol;
    }
    __syncthreads();
    // Phase 0: CG to the tolerance. Phase 1 (FP32 arithmetic only): x is carried in FP64, its true
    // residual, recomputed with error-free products and compensated sums (x as an FP32 pair),
    // replaces the recursive one and CG on the correction continues until that residual has
    // dropped 10^6-fold (at most 20 iterations), which leaves s_j accurate far below FP32
    // rounding. The seam vector is s_j minus its projection on K_p(H; e_j), of which s_j is mostly
    // made, so its relative accuracy is that of s_j divided by the small remainder.
    constexpr int kPhases = sizeof(T) == 4 ? 2 : 1;
    for (int phase = 0; phase < kPhases; ++phase) {
      int maxit = A.cg_maxit;
      if (phase >= 1) {
        maxit = 20;
        if (phase == 1)
          for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) SJd[i] = (double)SJ[i];
        __syncthreads();
        for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
          const double x = SJd[i];
          const T h = (T)x;
          P[i] = h;
          AP[i] = (T)(x - (double)h);
        }
        __syncthreads();
        if constexpr (sizeof(T) == 4)
          resid4_comp2<TV>(A.valS, lrow, lcol, rbase, loff, ncl, reinterpret_cast<const float*>(P),
                           reinterpret_cast<const float*>(AP), reinterpret_cast<float*>(R), 4 * t0);
        dot4<T>(R, R, m, red, sums);
        if (threadIdx.x < 4) {
          const int c = threadIdx.x;
          st.rr[c] = sums[c];
          st.cg_stop[c] = 1e-6 * sqrt(sums[c]);
          st.cg_active[c] = (st.status[c] == ST_OK) && sums[c] > 0.0;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) P[i] = R[i];
        __syncthreads();
      }
      for (int it = 0; it < maxit; ++it) {
        const int cmask = st.cg_active[0] | (st.cg_active[1] << 1) | (st.cg_active[2] << 2) | (st.cg_active[3] << 3);
        if (!cmask) break;
        spmm4<TV, T>(A.valS, lrow, lcol, rbase, loff, ncl, P, AP, cmask);
        dot4<T>(P, AP, m, red, sums);
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
          scal[c] = (T)a;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
          const int c = i & 3;
          if (st.cg_active[c]) {
            const T a = scal[c];
            if (phase == 0) SJ[i] += a * P[i];
            else SJd[i] += st.alpha[c] * (double)P[i];
            R[i] -= a * AP[i];
          }
        }
        __syncthreads();
        dot4<T>(R, R, m, red, sums);
        if (threadIdx.x < 4) {
          const int c = threadIdx.x;
          if (st.cg_active[c]) {
            st.beta_cg[c] = sums[c] / st.rr[c];
            scal[4 + c] = (T)st.beta_cg[c];
            st.rr[c] = sums[c];
            st.it[c] += 1;
            if (sqrt(sums[c]) <= st.cg_stop[c]) st.cg_active[c] = 0;
          }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
          const int c = i & 3;
          if (st.cg_active[c]) P[i] = R[i] + scal[4 + c] * P[i];
        }
        __syncthreads();
      }
      if (threadIdx.x < 4) {
        const int c = threadIdx.x;
        // a column still running after the main phase did not converge; the refinement cap is no failure
        if (phase == 0 && st.cg_active[c] && st.status[c] == ST_OK) st.status[c] = ST_NOCONV;
        st.cg_active[c] = 0;
      }
      __syncthreads();
    }
    if (sizeof(T) == 4)
      for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) SJ[i] = (T)SJd[i];
    __syncthreads();
    if (A.fallback && threadIdx.x < 4) A.fallback[4 * widx + threadIdx.x] = st.act[threadIdx.x];
    if (A.keep_s)
      for (int i = threadIdx.x; i < 16 * A.keep_cap; i += blockDim.x) {   // (column, cluster atom, orbital)
        const int c = i / (4 * A.keep_cap), rem = i % (4 * A.keep_cap), t = rem >> 2, o = rem & 3;
        double v = 0.0;
        if (t < ncl) v = sizeof(T) == 4 ? SJd[4 * (4 * t + o) + c] : (double)SJ[4 * (4 * t + o) + c];
        A.keep_s[(4 * widx + c) * (4 * (int64_t)A.keep_cap) + rem] = v;
      }
    if (A.cg_only) {
      for (int i = threadIdx.x; i < 4 * 68; i += blockDim.x) {
        const int c = i / 68, rem = i % 68, k = rem >> 2, o = rem & 3;
        const int pa = A.patch[widx * 17 + k];
        const int lk = pa >= 0 ? find_local(cl, ncl, pa) : -1;
        A.cg_target[(4 * widx + c) * 68 + rem] = lk >= 0 ? (float)SJ[4 * (4 * lk + o) + c] : 0.0f;
      }
      if (threadIdx.x < 4) {
        const int c = threadIdx.x;
        int s = st.status[c];
        if (st.cg_active[c] && s == ST_OK) s = ST_NOCONV;
        A.status[4 * widx + c] = s;
        A.cg_iters[4 * widx + c] = st.it[c];
      }
      __syncthreads();
      continue;
    }
    // ---- 3. multiple Arnoldi basis, with the projection accumulated on the way ---------
    T* Lv = V0;
    T* SL = V1;
    T* KV = V2;
    if (threadIdx.x < 4) {
      const int c = threadIdx.x;
      if (st.cg_active[c] && st.status[c] == ST_OK) st.status[c] = ST_NOCONV;
      st.n[c] = 0;
      st.src[c] = SRC_E;
      st.seam_done[c] = (A.q == 0);
      st.active[c] = (st.status[c] == ST_OK);
      st.proj[c] = 0;
    }
    if (threadIdx.x == 0) st.proj_any = 0;
    for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
      const int r = i >> 2, c = i & 3;
      Lv[i] = (r == 4 * t0 + c) ? (T)1 : (T)0;
      if constexpr (sizeof(T) == 4) Llo[i] = 0.0f;
    }
    __syncthreads();
    for (int guard = 0; guard < nu + 4; ++guard) {
      if (!(st.active[0] | st.active[1] | st.active[2] | st.active[3])) break;
      if (threadIdx.x == 0) {
        int nm = 0;
        for (int c = 0; c < 4; ++c) {
          st.csum[c] = 0.0;
          if (st.active[c] || st.proj[c]) nm = max(nm, st.n[c]);
        }
        st.n_max = nm;
      }
      __syncthreads();
      const int nmax = st.n_max;
      // One classical Gram-Schmidt pass with the projector's first-order Gram correction: the
      // coefficients c = (S U)^T l become c - E c with E = S_r - I = U^T S U - I (formed by the
      // projection already), so that l - U (c - E c) is S-orthogonal to the basis up to O(E^2)
      // and to the errors of this pass, the non-orthogonality a second pass would remove.
      if (nmax > 0) {
        gs_sweep<T>(U, SU, Lv, KV, SL, m, m_cap, nmax, true, st, coef, coefT, A.red, 4 * widx, nu, Es);
        if (threadIdx.x < 4) {
          double s = 0;
          for (int mm = 0; mm < nmax; ++mm) s += coef[mm * 4 + threadIdx.x] * coef[mm * 4 + threadIdx.x];
          st.csum[threadIdx.x] += s;
          st.proj[threadIdx.x] = 0;
        }
        if (threadIdx.x == 0) st.proj_any = 0;
        for (int t = threadIdx.x; t < 4 * nmax; t += blockDim.x) {
          const int c = t & 3, mm = t >> 2, nc = st.n[c];
          if (mm >= nc) continue;
          const float* er = Es + (c * nu + mm) * nu;
          double corr = 0.0;
          for (int k = 0; k < nc; ++k) corr += (double)er[k] * coef[k * 4 + c];
          coefT[mm * 4 + c] = (T)(coef[mm * 4 + c] - corr);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
          const int r = i >> 2, c = i & 3;
          if constexpr (sizeof(T) == 4) {
            if (st.active[c]) {
              // l and the basis as FP32 pairs, the update with error-free products and
              // compensated sums; only the low parts' products are rounded
              float h = Lv[i], lo = Llo[i];
              const int nc = min(nmax, st.n[c]);
              for (int mm = 0; mm < nc; ++mm) {
                const size_t o = (size_t)mm * m_cap * 4 + 4 * r + c;
                const float cf = coefT[mm * 4 + c];
                const float uh = U[o];
                const float p = __fmul_rn(cf, uh);
                const float pe = fmaf(cf, uh, -p);
                const float s = __fsub_rn(h, p);
                const float bb = __fsub_rn(s, h);
                const float err = __fsub_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fadd_rn(p, bb));
                h = s;
                lo = __fsub_rn(__fadd_rn(lo, err), fmaf(cf, Ulo[o], pe));
              }
              const float s = __fadd_rn(h, lo);
              Lv[i] = s;
              Llo[i] = __fsub_rn(lo, __fsub_rn(s, h));
              continue;
            }
          }
          T v = Lv[i];
          for (int mm = 0; mm < nmax; ++mm) v -= coefT[mm * 4 + c] * U[(size_t)mm * m_cap * 4 + 4 * r + c];
          Lv[i] = v;
        }
        __syncthreads();
      }
      if constexpr (sizeof(T) == 4) {
        // the seam vector in FP64: two classical Gram-Schmidt passes on s_j (FP64) for the columns
        // whose l is s_j, replacing what the FP32 pass above made of them
        const int smask = (st.active[0] && st.src[0] == SRC_S) | ((st.active[1] && st.src[1] == SRC_S) << 1) |
                          ((st.active[2] && st.src[2] == SRC_S) << 2) | ((st.active[3] && st.src[3] == SRC_S) << 3);
        if (smask && nmax > 0) seam_fp64(SU, U, Ulo, SJd, Lv, Llo, coef, st, m, m_cap, nmax, smask);
      }
      const int amask = st.active[0] | (st.active[1] << 1) | (st.active[2] << 2) | (st.active[3] << 3);
      // S l and H l in one pass (H u_n = H l / beta for an accepted l); in the FP32 form H l as a
      // pair from the pair, S l in FP32.
      // KV held H u of the last accepted vector, whose projection the sweep above has taken.
      if constexpr (sizeof(T) == 4)
        spmm4_pair_hs<TV>(A.valH, A.valS, lrow, lcol, rbase, loff, ncl, Lv, Llo, KV, Klo, SL, amask);
      else
        spmm4_hs<TV, T>(A.valH, A.valS, lrow, lcol, rbase, loff, ncl, Lv, KV, SL, amask);
      dot4<T>(Lv, SL, m, red, sums);
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
            scal[8 + c] = (T)st.beta_inv[c];
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
      const int acc_mask = st.accept[0] | (st.accept[1] << 1) | (st.accept[2] << 2) | (st.accept[3] << 3);
      if (acc_mask) {
        for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
          const int r = i >> 2, c = i & 3;
          if (st.accept[c]) {
            const T bi = scal[8 + c];
            T u = Lv[i] * bi;
            T k = KV[i] * bi;
            const T su = SL[i] * bi;
            const size_t o = (size_t)st.n[c] * m_cap * 4 + 4 * r + c;
            if constexpr (sizeof(T) == 4) {   // u_n and H u_n as FP32 pairs
              const float ul = __fadd_rn(fmaf(Lv[i], bi, -u), __fmul_rn(Llo[i], bi));
              const float s = __fadd_rn(u, ul);
              const float lo = __fsub_rn(ul, __fsub_rn(s, u));
              u = s;
              Ulo[o] = lo;
              Llo[i] = lo;
              const float kl = __fadd_rn(fmaf(KV[i], bi, -k), __fmul_rn(Klo[i], bi));
              const float ks = __fadd_rn(k, kl);
              Klo[i] = __fsub_rn(kl, __fsub_rn(ks, k));
              k = ks;
            }
            U[o] = u;
            SU[o] = su;
            Lv[i] = u;
            KV[i] = k;                // H u_n
            SL[i] = su;               // S u_n, kept for the projection column
          }
        }
        __syncthreads();
      }
      if (threadIdx.x < 4) {
        const int c = threadIdx.x;
        st.next_s[c] = 0;
        st.next_raw[c] = 0;
        if (st.accept[c]) {
          const int prev = st.src[c];
          st.n[c] += 1;
          st.proj[c] = 1;
          if (st.n[c] >= nu) {
            st.active[c] = 0;
          } else if (A.mode_b && (prev == SRC_S || prev == SRC_R)) {
            // the next raw vector: H s_j, formed when s_j was loaded (1), or H applied to the previous
            // raw vector (2)
            st.next_raw[c] = prev == SRC_S ? 1 : 2;
            st.src[c] = SRC_R;
          } else if (st.n[c] == A.p && !st.seam_done[c]) {
            st.next_s[c] = 1;         // the vector after u_p is s_j
            st.seam_done[c] = 1;
            st.src[c] = SRC_S;
          } else {
            st.src[c] = SRC_H;
          }
        }
      }
      if (threadIdx.x == 0) st.proj_any = acc_mask != 0;
      __syncthreads();
      // s_j dropped as already in the span: the next vector is H u_n of the last accepted u_n,
      // recomputed here from the stored basis (KV now holds H applied to the dropped s_j)
      const int kmask = (st.act[0] == ACT_LOAD_K) | ((st.act[1] == ACT_LOAD_K) << 1) |
                        ((st.act[2] == ACT_LOAD_K) << 2) | ((st.act[3] == ACT_LOAD_K) << 3);
      if (kmask) reload_hu<TV, T>(A.valH, lrow, lcol, rbase, loff, ncl, m, m_cap, kmask, st, U, Ulo, Lv, Llo, KV, Klo);
      // reading B: the raw vectors of the s_j chain, each H applied to the one before, scaled by a power
      // of two near its inverse 2-norm (exact for both halves of a pair). The first, H s_j, is formed when
      // s_j is loaded as the next vector, from s_j as CG left it (the FP64 seam pass of the FP32 form
      // orthogonalises its copy of s_j in place); the later ones when the previous raw vector is accepted.
      int pmask = 0;                         // columns whose next vector is s_j
      if (A.mode_b)
        for (int c = 0; c < 4; ++c)
          pmask |= (st.active[c] && ((st.accept[c] && st.next_s[c]) || st.act[c] == ACT_LOAD_S)) << c;
      const int rmask = pmask | ((st.next_raw[0] == 2) | ((st.next_raw[1] == 2) << 1) | ((st.next_raw[2] == 2) << 2) |
                                 ((st.next_raw[3] == 2) << 3));
      if (rmask)
        raw_chain_step<TV, T>(A.valH, lrow, lcol, rbase, loff, ncl, m, pmask, rmask, SJ, SJd, RW, RWN, RWlo, RWNlo, red,
                              sums, scal);
      for (int i = threadIdx.x; i < 4 * m; i += blockDim.x) {
        const int c = i & 3;
        if (!st.active[c]) continue;
        if (st.next_raw[c]) {
          Lv[i] = RW[i];
          if constexpr (sizeof(T) == 4) Llo[i] = RWlo[i];
          continue;
        }
        if (st.accept[c]) {
          Lv[i] = st.next_s[c] ? SJ[i] : KV[i];
          if constexpr (sizeof(T) == 4) Llo[i] = st.next_s[c] ? 0.0f : Klo[i];
        } else if (st.act[c] == ACT_LOAD_K) {
          Lv[i] = KV[i];
          if constexpr (sizeof(T) == 4) Llo[i] = Klo[i];
        } else if (st.act[c] == ACT_LOAD_S) {
          Lv[i] = SJ[i];
          if constexpr (sizeof(T) == 4) Llo[i] = 0.0f;
        }
      }
      __syncthreads();
    }
    // projection columns still pending (the last accepted vector of each column)
    if (st.proj_any) {
      if (threadIdx.x == 0) {
        int nm = 0;
        for (int c = 0; c < 4; ++c)
          if (st.proj[c]) nm = max(nm, st.n[c]);
        st.n_max = nm;
      }
      __syncthreads();
      gs_sweep<T>(U, SU, Lv, KV, SL, m, m_cap, st.n_max, false, st, coef, coefT, A.red, 4 * widx, nu, Es);
    }

    // ---- 4. what the reduced problems need: row j of U and S U (H_r, S_r are in place) -------
    {
      double* red0 = A.red + (size_t)((4 * widx) >> 5) * red_block_doubles(nu) * 32;
      for (int i = threadIdx.x; i < 4 * 2 * nu; i += blockDim.x) {
        const int c = i / (2 * nu), k = i % (2 * nu), n = k % nu;
        const int64_t col = 4 * widx + c;
        if (n >= st.n[c]) continue;
        const T* src = (k < nu ? U : SU) + (size_t)n * m_cap * 4 + 4 * (4 * t0 + c) + c;
        red0[((size_t)2 * nu * nu + k) * 32 + (col & 31)] = (double)*src;
      }
    }
    for (int c = threadIdx.x; c < 4; c += blockDim.x) {
      const int64_t col = 4 * widx + c;
      A.status[col] = st.status[c];
      A.nu_eff[col] = st.n[c];
      A.cg_iters[col] = st.it[c];
    }
    if (A.keep) {
      // pattern rows of U (zero outside the cluster): rho_ij = U_i . (C diag(f) V_j)
      const int nrow = A.row_ptr[atom + 1] - A.row_ptr[atom];
      double* vpa = A.vp + A.blk_off[widx] * 16 * (int64_t)nu;
      for (int i = threadIdx.x; i < nrow * 16 * nu; i += blockDim.x) vpa[i] = 0.0;
      __syncthreads();
      const int e0 = lrow[t0], ne = lrow[t0 + 1] - e0;
      for (int i = threadIdx.x; i < 16 * ne * nu; i += blockDim.x) {
        const int n = i % nu, rem = i / nu, c = rem / (4 * ne), er = rem % (4 * ne), e = e0 + er / 4, r = er % 4;
        if (n >= st.n[c]) continue;
        const int k = loff[e];   // the atom's own row: offset = block index within the row
        vpa[((int64_t)k * 16 + c * 4 + r) * nu + n] = (double)U[(size_t)n * m_cap * 4 + 4 * (4 * (int)lcol[e] + r) + c];
      }
    }
    __syncthreads();
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
    const float pxf = A.posf[3 * a], pyf = A.posf[3 * a + 1], pzf = A.posf[3 * a + 2];
    int rx[3], ry[3], rz[3];
    const int nx = cell_range(cell_coord(px, A.cell_len[0], A.ncell[0]), A.ncell[0], rx);
    const int ny = cell_range(cell_coord(py, A.cell_len[1], A.ncell[1]), A.ncell[1], ry);
    const int nz = cell_range(cell_coord(pz, A.cell_len[2], A.ncell[2]), A.ncell[2], rz);
    int count = 0;
    for (int ci = 0; ci < nx * ny * nz; ++ci) {
      const int ix = ci / (ny * nz), iy = (ci / nz) % ny, iz = ci % nz;
      const int c = (rx[ix] * A.ncell[1] + ry[iy]) * A.ncell[2] + rz[iz];
      for (int k = A.cell_start[c] + lane; k < A.cell_start[c + 1]; k += 32)
        count += within_R(A.pos, A.posf, A.box, A.R2, A.pre_lo, A.pre_hi, A.cell_atoms[k], px, py, pz, pxf, pyf,
                          pzf);
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
  A.posf = s->d_posf;
  for (int d = 0; d < 3; ++d) {
    A.box[d] = s->box[d];
    A.ncell[d] = s->cells.n[d];
    A.cell_len[d] = s->cells.len[d];
  }
  A.R2 = s->R * s->R;
  const double lmax = std::max(s->box[0], std::max(s->box[1], s->box[2]));
  const double margin = std::max(1e-3, 1e-5 * lmax / s->R);
  A.pre_lo = (float)(1.0 - margin);
  A.pre_hi = (float)(1.0 + margin);
  A.cell_start = s->cells.start;
  A.cell_atoms = s->cells.atoms;
}

// Dynamic shared memory of atoms_kernel: cluster list and local pattern, then the [m_cap][4]
// vector the SpMV gathers (p in CG, l in the basis; its low half too in the FP32 form), then
// the Gram-Schmidt coefficients ([nu][4] in FP64 and in the arithmetic type).
size_t dyn_smem_bytes(int nu, int clcap, int lnnz_cap, int mcap, size_t elem) {
  size_t off = (size_t)(3 * clcap + 1) * sizeof(int) + (size_t)lnnz_cap * (sizeof(uint16_t) + 1);
  off = align_up(off, 16);
  return off + (size_t)mcap * 4 * elem + (elem == 4 ? (size_t)mcap * 4 * sizeof(float) : 0) +
         (size_t)nu * 4 * (sizeof(double) + elem);
}

// Per-CTA global work slot: U and S U ([nu][m_cap][4]) and s_j ([m_cap][4]) in the arithmetic
// type, then s_j in FP64 ([m_cap][4]), S_r - I of the four columns ([4][nu][nu] FP32), the two
// streamed work vectors ([m_cap][4] each, arithmetic type), (FP32 arithmetic) the low half of H u
// ([m_cap][4]) and of the basis vectors ([nu][m_cap][4]), then the raw vector of the s_j chain and H
// applied to it ([m_cap][4] each, arithmetic type) with their FP32 low halves.
size_t slot_bytes_for(int nu, int mcap, size_t elem) {
  return align_up(elem * ((size_t)2 * nu + 1) * mcap * 4, 256) + align_up(sizeof(double) * 4 * (size_t)mcap, 256) +
         align_up(sizeof(float) * 4 * (size_t)nu * nu, 256) + elem * 2 * (size_t)mcap * 4 +
         align_up(elem == 4 ? sizeof(float) * ((size_t)nu + 1) * mcap * 4 : 0, 256) +
         (2 * elem + 2 * sizeof(float)) * (size_t)mcap * 4 + 256;
}

template <typename TV, typename T, int NT>
mka_status config_t(const mka_system* sys, int nu, int max_cl, int ctas_per_sm, AtomsConfig* out) {
  AtomsConfig cf{};
  cf.threads = NT;
  if (sys->max_row_blocks > 255)
    return fail(MKA_ERR_INVALID_ARG, "rows of more than 255 blocks are not supported by the per-atom kernel");
  const int cl_atoms = std::max(1, std::min(max_cl, kMaxCl));
  cf.mcap = 4 * cl_atoms;
  cf.lnnz_cap = cl_atoms * std::max(1, sys->max_row_blocks);
  cf.clcap = 2;
  while (cf.clcap < cl_atoms) cf.clcap <<= 1;
  cf.smem = dyn_smem_bytes(nu, cf.clcap, cf.lnnz_cap, cf.mcap, sizeof(T));
  cf.slot_bytes = slot_bytes_for(nu, cf.mcap, sizeof(T));
  auto kern = atoms_kernel<TV, T, NT>;
  MKA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cf.smem));
  int dev = 0, sms = 0, per_sm = 0;
  MKA_CUDA_TRY(cudaGetDevice(&dev));
  MKA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  MKA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, cf.smem));
  if (per_sm < 1) return fail(MKA_ERR_INVALID_ARG, "per-atom working set does not fit in shared memory");
  if (ctas_per_sm > 0) per_sm = std::min(per_sm, ctas_per_sm);
  cf.per_sm = per_sm;
  cf.grid_max = sms * per_sm;
  *out = cf;
  return MKA_OK;
}

template <typename TV, typename T, int NT>
mka_status launch_t(const mka_system* sys, const AtomsConfig& cf, const AtomsLaunchArgs& a, cudaStream_t st) {
  Args<TV> A{};
  fill_system_args(A, sys);
  A.sel = a.sel;
  A.order = a.order;
  A.n_sel = a.n_sel;
  A.work_counter = a.counter;
  A.p = a.p;
  A.q = a.q;
  A.nu = a.p + a.q;
  A.cg_tol = a.cg_tol;
  A.cg_maxit = a.cg_maxit;
  A.tau = 1e-10;
  A.scratch = a.scratch;
  A.slot_bytes = cf.slot_bytes;
  A.mcap = cf.mcap;
  A.lnnz_cap = cf.lnnz_cap;
  A.clcap = cf.clcap;
  A.eps = a.eps;
  A.w = a.w;
  A.nu_eff = a.nu_eff;
  A.cg_iters = a.cg_iters;
  A.status = a.status;
  A.keep = a.keep;
  A.vp = a.vp;
  A.blk_off = a.blk_off;
  A.x0 = a.x0;
  A.patch = a.patch;
  A.fallback = a.fallback;
  A.cg_only = a.cg_only;
  A.cg_target = a.cg_target;
  A.mode_b = a.mode_b;
  A.prev_cl = a.prev_cl;
  A.prev_s = a.prev_s;
  A.prev_cap = a.prev_cap;
  A.keep_cl = a.keep_cl;
  A.keep_s = a.keep_s;
  A.keep_cap = a.keep_cap;
  A.red = a.red;
  if (!a.cg_only && !a.red) return fail(MKA_ERR_INVALID_ARG, "the per-atom kernel needs a reduced-problem buffer");
  atoms_kernel<TV, T, NT><<<(unsigned)a.grid, NT, cf.smem, st>>>(A);
  count_launches();
  MKA_CUDA_TRY(cudaGetLastError());
  return MKA_OK;
}

// Dispatch on (storage type, arithmetic, CTA size).
#define MKA_DISPATCH_T(CALL, TV, T, threads)        \
  ((threads) == 128 ? CALL(TV, T, 128) : (threads) == 512 ? CALL(TV, T, 512) : CALL(TV, T, 256))
#define MKA_DISPATCH(CALL, storage, mixed, threads)                                                        \
  ((storage) == MKA_FP64 ? ((mixed) ? MKA_DISPATCH_T(CALL, double, float, threads)                         \
                                    : MKA_DISPATCH_T(CALL, double, double, threads))                       \
   : (storage) == MKA_MIXED_FP32 ? ((mixed) ? MKA_DISPATCH_T(CALL, float, float, threads)                  \
                                            : MKA_DISPATCH_T(CALL, float, double, threads))                \
   : ((mixed) ? MKA_DISPATCH_T(CALL, __nv_bfloat16, float, threads)                                        \
              : MKA_DISPATCH_T(CALL, __nv_bfloat16, double, threads)))

}  // namespace

mka_status launch_cluster_sizes(const mka_system* sys, const int64_t* d_sel, int64_t n_sel, int32_t* d_sizes,
                                cudaStream_t st) {
  Args<double> A{};
  fill_system_args(A, sys);
  A.sel = d_sel;
  A.n_sel = n_sel;
  const int threads = 256;
  int dev = 0, sms = 0;
  MKA_CUDA_TRY(cudaGetDevice(&dev));
  MKA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t blocks = std::min<int64_t>((n_sel + 7) / 8, (int64_t)sms * 16);
  cluster_size_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), threads, 0, st>>>(A, d_sizes);
  count_launches();
  MKA_CUDA_TRY(cudaGetLastError());
  return MKA_OK;
}

mka_status atoms_config(const mka_system* sys, int nu, int arith, int max_cl, int threads, int ctas_per_sm,
                        AtomsConfig* out) {
  const bool mixed = arith != MKA_FP64;
#define MKA_CFG(TV, T, NT) config_t<TV, T, NT>(sys, nu, max_cl, ctas_per_sm, out)
  return MKA_DISPATCH(MKA_CFG, sys->storage, mixed, threads);
#undef MKA_CFG
}

mka_status reduced_for(const mka_system* sys, const AtomsLaunchArgs& a, cudaStream_t st) {
  return reduced_launch(a.red, 4 * a.n_sel, a.p + a.q, a.status, a.nu_eff, a.eps, a.w, a.keep ? a.cv : nullptr,
                        a.col0, st);
}

mka_status atoms_launch(const mka_system* sys, int arith, const AtomsConfig& cf, const AtomsLaunchArgs& a,
                        cudaStream_t st) {
  const bool mixed = arith != MKA_FP64;
#define MKA_LAUNCH(TV, T, NT) launch_t<TV, T, NT>(sys, cf, a, st)
  return MKA_DISPATCH(MKA_LAUNCH, sys->storage, mixed, cf.threads);
#undef MKA_LAUNCH
}

mka_status launch_columns(mka_system* sys, mka_result* res, const mka_solve_params* prm, int max_cl,
                          cudaStream_t st) {
  const int nu = prm->p + prm->q;
  AtomsConfig cf{};
  mka_status s = atoms_config(sys, nu, prm->arith, max_cl, 256, 0, &cf);
  if (s) return s;
  // atoms per chunk: the reduced-problem buffer of a chunk stays within 2 GiB
  const size_t per_atom = red_buffer_bytes(32, nu) / 8;
  const int64_t chunk = std::max<int64_t>(8, std::min<int64_t>(res->n_sel, ((size_t)2 << 30) / per_atom) & ~(int64_t)7);
  const int64_t grid = std::min<int64_t>(std::min(res->n_sel, chunk), cf.grid_max);
  char* scratch = nullptr;
  int* counter = nullptr;
  double* red = nullptr;
  MKA_CUDA_TRY(cudaMallocAsync(&scratch, cf.slot_bytes * grid + 256, st));
  MKA_CUDA_TRY(cudaMallocAsync(&counter, sizeof(int), st));
  MKA_CUDA_TRY(cudaMallocAsync(&red, red_buffer_bytes(4 * std::min(res->n_sel, chunk), nu), st));
  // learned warm start: features, then the network's prediction of s_j on each patch (per chunk)
  float* wbuf = nullptr;
  int32_t* patch = nullptr;
  const int64_t rows_max = 4 * std::min(res->n_sel, chunk);
  if (prm->use_warm_start) {
    MKA_CUDA_TRY(cudaMallocAsync(&wbuf, sizeof(float) * (rows_max * (132 + 68) + mlp_work_floats(rows_max)), st));
    MKA_CUDA_TRY(cudaMallocAsync(&patch, sizeof(int32_t) * 17 * std::min(res->n_sel, chunk), st));
  }
  for (int64_t off = 0; off < res->n_sel && !s; off += chunk) {
    const int64_t cnt = std::min(chunk, res->n_sel - off);
    AtomsLaunchArgs a{};
    if (prm->use_warm_start) {
      const int64_t rows = 4 * cnt;
      float* X = wbuf;
      float* Y = X + rows * 132;
      float* W = Y + rows * 68;
      s = features_enqueue(sys, res->d_sel + off, cnt, X, patch, st);
      if (!s) s = mlp_forward_enqueue(sys->warm, X, rows, W, W + rows * 128, W + 2 * rows * 128, W + 3 * rows * 128, Y, st);
      if (s) break;
      a.x0 = Y;
      a.patch = patch;
      a.fallback = res->d_fallback + 4 * off;
    }
    MKA_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int), st));
    a.sel = res->d_sel + off;
    a.order = nullptr;
    a.n_sel = cnt;
    a.p = prm->p;
    a.q = prm->q;
    a.cg_tol = prm->cg_tol;
    a.cg_maxit = prm->cg_maxit;
    a.eps = res->d_eps + 4 * off * nu;
    a.w = res->d_w + 4 * off * nu;
    a.nu_eff = res->d_nu_eff + 4 * off;
    a.cg_iters = res->d_cg_iters + 4 * off;
    a.status = res->d_status + 4 * off;
    a.keep = res->keep;
    a.vp = res->d_vp;
    a.blk_off = res->keep ? res->d_blk_off + off : nullptr;
    a.cv = res->d_cv;
    a.col0 = 4 * off;
    a.mode_b = prm->subspace == MKA_SUBSPACE_B;
    if (prm->s_start) {
      const mka_result* pr = prm->s_start;
      a.prev_cap = pr->s_cap;
      a.prev_cl = pr->d_s_cl + off * pr->s_cap;
      a.prev_s = pr->d_s + 4 * off * 4 * (int64_t)pr->s_cap;
    }
    if (res->d_s) {
      a.keep_cap = res->s_cap;
      a.keep_cl = res->d_s_cl + off * res->s_cap;
      a.keep_s = res->d_s + 4 * off * 4 * (int64_t)res->s_cap;
    }
    a.scratch = scratch;
    a.counter = counter;
    a.red = red;
    a.grid = (int)std::min<int64_t>(grid, cnt);
    s = atoms_launch(sys, prm->arith, cf, a, st);
    if (!s) s = reduced_for(sys, a, st);
  }
  cudaFreeAsync(scratch, st);
  cudaFreeAsync(counter, st);
  cudaFreeAsync(red, st);
  if (wbuf) cudaFreeAsync(wbuf, st);
  if (patch) cudaFreeAsync(patch, st);
  return s;
}

}  // namespace mka

// ---- fixed-scratch variant (mka_solve_columns_static) ------------------------------------
//
// The same per-atom kernel, FP64 form, with its work queue counter, the atom list
// and every per-CTA work slot carved out of one file-scope device array instead of
// memory allocated per call. Host code cannot use the array's name as a device
// address: every call looks the address up with cudaGetSymbolAddress on the current
// device (a table lookup that allocates nothing once the library's device code is
// loaded), so that a context created anew on that device (after cudaDeviceReset, or a
// released and re-created primary context) never sees a stale address.
static __device__ __align__(256) unsigned char g_static_scratch[MKA_STATIC_SCRATCH_BYTES];

namespace mka {
namespace {

// Device address of g_static_scratch in the current device's context.
mka_status static_scratch_address(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || !p) return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
  *out = p;
  return MKA_OK;
}

mka_status run_columns_static(const mka_system* sys, const int64_t* h_atoms, int64_t n_sel, int p, int q,
                              double cg_tol, int cg_maxit, int max_cl, double* eps, double* w, int32_t* nu_eff,
                              int32_t* cg_iters, int32_t* status, cudaStream_t st) {
  char* base = nullptr;
  mka_status s = static_scratch_address(reinterpret_cast<void**>(&base));
  if (s) return s;
  AtomsConfig cf{};
  s = atoms_config(sys, p + q, MKA_FP64, max_cl, 256, 0, &cf);
  if (s) return s;
  // layout: [work counter | 256 B] [atom ids of a chunk | rounded to 256 B] [reduced-problem buffer of
  // the chunk] [per-CTA slots]; the selection runs in chunks that leave room for at least one slot
  const int nu = p + q;
  const size_t total = (size_t)MKA_STATIC_SCRATCH_BYTES;
  const size_t per_atom = sizeof(int64_t) + red_buffer_bytes(32, nu) / 8;
  if (256 + cf.slot_bytes + 256 + red_buffer_bytes(4, nu) > total)
    return fail(MKA_ERR_INVALID_ARG,
                "mka_solve_columns_static: one work slot (" + std::to_string(cf.slot_bytes) +
                    " B) and one atom's reduced problems exceed the fixed scratch of " + std::to_string(total) +
                    " B; pass a smaller p + q or a smaller max_cluster_atoms");
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(n_sel, (int64_t)((total - 512 - cf.slot_bytes) / 2 / per_atom)));
  const size_t sel_bytes = align_up((size_t)chunk * sizeof(int64_t), 256);
  const size_t red_bytes = align_up(red_buffer_bytes(4 * chunk, nu), 256);
  const size_t fixed = 256 + sel_bytes + red_bytes;
  const int64_t slots_fit = (int64_t)((total - fixed) / cf.slot_bytes);
  if (slots_fit < 1) return fail(MKA_ERR_INVALID_ARG, "mka_solve_columns_static: the fixed scratch holds no work slot");
  for (int64_t off = 0; off < n_sel; off += chunk) {
    const int64_t cnt = std::min(chunk, n_sel - off);
    AtomsLaunchArgs a{};
    a.counter = reinterpret_cast<int*>(base);
    a.sel = reinterpret_cast<const int64_t*>(base + 256);
    a.red = reinterpret_cast<double*>(base + 256 + sel_bytes);
    a.scratch = base + fixed;
    a.order = nullptr;
    a.n_sel = cnt;
    a.p = p;
    a.q = q;
    a.cg_tol = cg_tol;
    a.cg_maxit = cg_maxit;
    a.eps = eps + 4 * off * nu;
    a.w = w + 4 * off * nu;
    a.nu_eff = nu_eff + 4 * off;
    a.cg_iters = cg_iters + 4 * off;
    a.status = status + 4 * off;
    a.keep = 0;
    a.grid = (int)std::min<int64_t>(std::min<int64_t>(cnt, slots_fit), cf.grid_max);
    // The counter must start at zero; the chunk's atom list is copied in; slots and the reduced
    // buffer need no clearing (every entry is written before it is read).
    MKA_CUDA_TRY(cudaMemsetAsync(base, 0, 256, st));
    MKA_CUDA_TRY(cudaMemcpyAsync(base + 256, h_atoms + off, (size_t)cnt * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    s = atoms_launch(sys, MKA_FP64, cf, a, st);
    if (!s) s = reduced_for(sys, a, st);
    if (s) return s;
  }
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
  return run_columns_static(sys, atoms, n_sel, p, q, cg_tol, cg_maxit, max_cluster_atoms, eps, w, nu_eff, cg_iters,
                            status, (cudaStream_t)stream);
}
