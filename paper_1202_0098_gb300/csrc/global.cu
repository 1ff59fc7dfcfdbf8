// Global (all-column) kernels: mu by bisection, the density matrix with the band
// energy, the subspace Green's function, and the global block-sparse product.
//
// mu (Sec. 2, after Eq. EQ-DM): the electron count 2 sum_j sum_alpha f w is
// evaluated by one launch per halving; the launch's blocks write fixed-order
// partial sums, and the last block to finish (ticket counter) adds them in
// block order and moves the bracket, so the result does not depend on timing.
// f(x) = (1 - tanh((x - mu) / (2 kT))) / 2; for |x - mu| / (2 kT) > 20 the FP64
// tanh is exactly +-1, so those terms take f = 0 or 1 without calling it.
//
// rho (Eq. EQ-DM), G (Eq. EQ-SOLUTION-SUB-GZ) and E (Eq. EQ-ENE) read the kept
// pattern rows of v_alpha (row block k of column j, [c][r][alpha]).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "mka_internal.h"

namespace mka {
namespace {

constexpr int kRedThreads = 256;
// Grid of the reductions: 4 CTAs per SM of the current device, at most kMaxRedBlocks (the size of
// the partial-sum buffers).
int red_blocks() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 152;
  return std::max(1, std::min(kMaxRedBlocks, 4 * sms));
}

__device__ __forceinline__ double fermi(double x, double mu, double kT) {
  const double y = (x - mu) / (2.0 * kT);
  if (y > 20.0) return 0.0;
  if (y < -20.0) return 1.0;
  return 0.5 * (1.0 - tanh(y));
}

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
  __syncthreads();
  return s;  // valid in thread 0
}

// Bisection state (device doubles): [0] lo, [1] hi, [2] target, [3] kT, [4] tol,
// [5] last count, [6] halvings done. partial[kMaxRedBlocks], ticket (unsigned).
struct MuState {
  double lo, hi, target, kT, tol, last, iters, pad;
};

// min / max of eps over entries with w != 0 (fixed-order two-level reduction).
__global__ void eps_range_kernel(const double* eps, const double* w, int64_t n, double* partial,
                                 unsigned* ticket, MuState* S) {
  __shared__ double rmin[kRedThreads / 32], rmax[kRedThreads / 32];
  __shared__ bool last;
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
    for (int k = 1; k < kRedThreads / 32; ++k) {
      mn = fmin(mn, rmin[k]);
      mx = fmax(mx, rmax[k]);
    }
    mn = fmin(mn, rmin[0]);
    mx = fmax(mx, rmax[0]);
    partial[2 * blockIdx.x] = mn;
    partial[2 * blockIdx.x + 1] = mx;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double a = INFINITY, b = -INFINITY;
    for (unsigned k = 0; k < gridDim.x; ++k) {
      a = fmin(a, partial[2 * k]);
      b = fmax(b, partial[2 * k + 1]);
    }
    S->lo = a - 40.0 * S->kT;
    S->hi = b + 40.0 * S->kT;
    S->iters = 0;
    *ticket = 0;
  }
}

// One halving: N(mid) = 2 sum f(eps; mid) w, then the bracket update.
__global__ void bisect_kernel(const double* eps, const double* w, int64_t n, double* partial, unsigned* ticket,
                              MuState* S) {
  __shared__ double red[kRedThreads / 32];
  __shared__ bool last;
  const double lo = S->lo, hi = S->hi;
  if (!(hi - lo > S->tol)) return;   // converged: every block leaves before touching the ticket
  const double mid = 0.5 * (lo + hi), kT = S->kT;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double wi = w[i];
    if (wi != 0.0) acc += fermi(eps[i], mid, kT) * wi;
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double t = 0.0;
    for (unsigned k = 0; k < gridDim.x; ++k) t += partial[k];
    const double count = 2.0 * t;
    if (count < S->target) S->lo = mid; else S->hi = mid;
    S->last = count;
    S->iters += 1;
    *ticket = 0;
  }
}

// Bracket state of a stream-ordered bisection (no host round trip): target, kT, tolerance,
// ticket cleared; the range kernel then sets lo / hi.
__global__ void mu_init_kernel(MuState* S, unsigned* ticket, double target, double kT, double tol) {
  S->target = target;
  S->kT = kT;
  S->tol = tol;
  S->iters = 0;
  *ticket = 0;
}

__global__ void mu_finish_kernel(const MuState* S, double* mu_out) { *mu_out = 0.5 * (S->lo + S->hi); }

// Column c of atom t: g = C diag(x) V_j for per-level weights x (ascending order of eps), from the
// kept C and V_j (lane-interleaved by column); thread per (c, n), g into shared memory [4][nu].
__device__ void column_weights(const double* cv, int64_t t, int nu, const double* x, double* g) {
  for (int i = threadIdx.x; i < 4 * nu; i += blockDim.x) {
    const int c = i / nu, n = i % nu;
    const int64_t col = 4 * t + c;
    const double* b = cv + (size_t)(col >> 5) * kept_block_doubles(nu) * 32 + (col & 31);
    double s = 0.0;
    for (int a = 0; a < nu; ++a) s += b[(size_t)(n * nu + a) * 32] * x[c * nu + a] * b[(size_t)(nu * nu + a) * 32];
    g[i] = s;
  }
  __syncthreads();
}

// rho / E: one CTA per selected atom, thread per (block k, c, r) of its row:
// rho_ij = sum_alpha f_alpha V_i alpha V_j alpha = U_i . g_j with g_j = C diag(f) V_j.
// Output layout: the batch's (blocks at blk_off[t], E of atom t at e_partial[t]) when out_base < 0;
// otherwise the system's pattern order from block out_base on (blocks at row_ptr[atom] - out_base,
// E at e_partial[atom - e_base]).
__global__ void density_kernel(const double* vp, const double* cv, const double* eps, const int64_t* blk_off,
                               const int64_t* sel, const int32_t* row_ptr, const void* valH, int storage,
                               int nu, double mu_host, const double* mu_dev, double kT, double* rho,
                               double* e_partial, int64_t out_base = -1, int64_t e_base = 0) {
  __shared__ double red[kRedThreads / 32];
  __shared__ double f[4 * MKA_MAX_NU];
  __shared__ double g[4 * MKA_MAX_NU];
  const double mu = mu_dev ? *mu_dev : mu_host;
  const int64_t t = blockIdx.x;
  const int64_t atom = sel[t];
  const int nrow = row_ptr[atom + 1] - row_ptr[atom];
  const int64_t b0 = blk_off[t];
  const int64_t ob = out_base < 0 ? b0 : (int64_t)row_ptr[atom] - out_base;
  for (int i = threadIdx.x; i < 4 * nu; i += blockDim.x) {
    const int c = i / nu;
    f[i] = fermi(eps[(4 * t + c) * nu + i % nu], mu, kT);
  }
  __syncthreads();
  column_weights(cv, t, nu, f, g);
  double e = 0.0;
  for (int i = threadIdx.x; i < nrow * 16; i += blockDim.x) {
    const int k = i >> 4, c = (i >> 2) & 3, r = i & 3;
    const double* u = vp + ((b0 + k) * 16 + c * 4 + r) * (int64_t)nu;
    double s = 0.0;
    for (int n = 0; n < nu; ++n) s += u[n] * g[c * nu + n];
    if (rho) rho[(ob + k) * 16 + c * 4 + r] = s;
    const int64_t gk = (int64_t)row_ptr[atom] + k;
    double h;
    if (storage == MKA_FP64) h = reinterpret_cast<const double*>(valH)[gk * 16 + c * 4 + r];
    else if (storage == MKA_MIXED_FP32) h = reinterpret_cast<const float*>(valH)[gk * 16 + c * 4 + r];
    else h = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(valH)[gk * 16 + c * 4 + r]);
    e += s * h;
  }
  const double s = block_sum(e, red);
  if (threadIdx.x == 0) e_partial[out_base < 0 ? t : atom - e_base] = 2.0 * s;
}

// G_ij(z) = sum_alpha V_i alpha V_j alpha / (z - eps_alpha) = U_i . (C diag(1 / (z - eps)) V_j).
__global__ void greens_kernel(const double* vp, const double* cv, const double* eps, const int64_t* blk_off,
                              const int64_t* sel, const int32_t* row_ptr, int nu, double zr, double zi, double* g) {
  __shared__ double xr[4 * MKA_MAX_NU], xi[4 * MKA_MAX_NU], gr[4 * MKA_MAX_NU], gi[4 * MKA_MAX_NU];
  const int64_t t = blockIdx.x;
  const int64_t atom = sel[t];
  const int nrow = row_ptr[atom + 1] - row_ptr[atom];
  const int64_t b0 = blk_off[t];
  for (int i = threadIdx.x; i < 4 * nu; i += blockDim.x) {
    const int c = i / nu;
    const double dr = zr - eps[(4 * t + c) * nu + i % nu];
    const double den = dr * dr + zi * zi;   // 1 / (z - e) = (dr - i zi) / den
    xr[i] = dr / den;
    xi[i] = -zi / den;
  }
  __syncthreads();
  column_weights(cv, t, nu, xr, gr);
  column_weights(cv, t, nu, xi, gi);
  for (int i = threadIdx.x; i < nrow * 16; i += blockDim.x) {
    const int k = i >> 4, c = (i >> 2) & 3, r = i & 3;
    const double* u = vp + ((b0 + k) * 16 + c * 4 + r) * (int64_t)nu;
    double sr = 0.0, si = 0.0;
    for (int n = 0; n < nu; ++n) {
      sr += u[n] * gr[c * nu + n];
      si += u[n] * gi[c * nu + n];
    }
    g[2 * ((b0 + k) * 16 + c * 4 + r)] = sr;
    g[2 * ((b0 + k) * 16 + c * 4 + r) + 1] = si;
  }
}

// Fixed-order sum of n doubles by one CTA (thread 0 adds the per-thread sums in order).
__global__ void sum_kernel(const double* x, int64_t n, double* out) {
  __shared__ double part[kRedThreads];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)blockDim.x; ++k) t += part[k];
    *out = t;
  }
}

// 2 sum f(eps; mu) w: per-block partial sums (fixed grid), added in order by sum_kernel.
__global__ void count_partial_kernel(const double* eps, const double* w, int64_t n, double mu_host, const double* mu_dev,
                                     double kT, double* partial) {
  __shared__ double red[kRedThreads / 32];
  const double mu = mu_dev ? *mu_dev : mu_host;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double wi = w[i];
    if (wi != 0.0) acc += fermi(eps[i], mu, kT) * wi;
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = 2.0 * s;
}

// ---- global BSR SpMV: four lanes per block row, one per output row of the 4x4 blocks ----
// Lane (a, i) computes y[4a + i][0..K) = sum over the row's blocks k of sum_jj val[k][i][jj] x[4 col[k] + jj][0..K).
// Each lane streams its row of every block (4 values: 8 bytes in BF16, 16 in FP32, 32 in FP64), so the four
// lanes of a block row read each block's values as one contiguous piece; the column index is read by all
// four (one request), and x through the read-only cache, one 16-byte vector per (block column, jj) row
// group. Blocks are taken four at a time with their loads issued before the arithmetic.
template <typename TV>
struct RowVals;
template <>
struct RowVals<__nv_bfloat16> {
  static __device__ __forceinline__ void load(const __nv_bfloat16* v, int64_t k, int i, float out[4]) {
    const uint2 a = __ldcs(reinterpret_cast<const uint2*>(v + k * 16 + i * 4));
    out[0] = __uint_as_float(a.x << 16);
    out[1] = __uint_as_float(a.x & 0xFFFF0000u);
    out[2] = __uint_as_float(a.y << 16);
    out[3] = __uint_as_float(a.y & 0xFFFF0000u);
  }
};
template <>
struct RowVals<float> {
  static __device__ __forceinline__ void load(const float* v, int64_t k, int i, float out[4]) {
    const float4 a = __ldcs(reinterpret_cast<const float4*>(v + k * 16 + i * 4));
    out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
  }
};
template <>
struct RowVals<double> {
  static __device__ __forceinline__ void load(const double* v, int64_t k, int i, double out[4]) {
    const double2 a = __ldcs(reinterpret_cast<const double2*>(v + k * 16 + i * 4));
    const double2 b = __ldcs(reinterpret_cast<const double2*>(v + k * 16 + i * 4) + 1);
    out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
  }
};

// x rows 4 cb .. 4 cb + 3, K values each: xv[jj][c].
template <typename TX, int K>
__device__ __forceinline__ void load_x(const TX* __restrict__ x, int64_t cb, TX xv[4][K]) {
  const TX* p = x + cb * 4 * K;
  if constexpr (sizeof(TX) == 4) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int t = 0; t < K; ++t) {        // 4 K floats = K float4
      const float4 a = __ldg(q + t);
      const float f[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) xv[(4 * t + u) / K][(4 * t + u) % K] = f[u];
    }
  } else {
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int t = 0; t < 2 * K; ++t) {    // 4 K doubles = 2 K double2
      const double2 a = __ldg(q + t);
      xv[(2 * t) / K][(2 * t) % K] = a.x;
      xv[(2 * t + 1) / K][(2 * t + 1) % K] = a.y;
    }
  }
}

template <typename TV, typename TX, int K>
__global__ void __launch_bounds__(256) spmv_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                                   const TV* __restrict__ val, const TX* __restrict__ x,
                                                   TX* __restrict__ y, int64_t n_rows) {
  using TL = typename std::conditional<std::is_same<TV, double>::value, double, float>::type;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < 4 * n_rows; g += stride) {
    const int64_t a = g >> 2;
    const int i = (int)(g & 3);
    const int k0 = __ldg(row_ptr + a), k1 = __ldg(row_ptr + a + 1);
    TX acc[K];
#pragma unroll
    for (int c = 0; c < K; ++c) acc[c] = 0;
    int k = k0;
    for (; k + 4 <= k1; k += 4) {
      int cb[4];
      TL v[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u) cb[u] = __ldg(col + k + u);
#pragma unroll
      for (int u = 0; u < 4; ++u) RowVals<TV>::load(val, k + u, i, v[u]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        TX xv[4][K];
        load_x<TX, K>(x, cb[u], xv);
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
#pragma unroll
          for (int c = 0; c < K; ++c) acc[c] = fma((TX)v[u][jj], xv[jj][c], acc[c]);
      }
    }
    for (; k < k1; ++k) {
      TL v[4];
      RowVals<TV>::load(val, k, i, v);
      TX xv[4][K];
      load_x<TX, K>(x, __ldg(col + k), xv);
#pragma unroll
      for (int jj = 0; jj < 4; ++jj)
#pragma unroll
        for (int c = 0; c < K; ++c) acc[c] = fma((TX)v[jj], xv[jj][c], acc[c]);
    }
    TX* yo = y + (4 * a + i) * K;
#pragma unroll
    for (int c = 0; c < K; ++c) yo[c] = acc[c];
  }
}

template <typename TV, typename TX>
mka_status spmv_dispatch_k(const mka_system* s, const TV* val, const void* x, void* y, int k, cudaStream_t st) {
  int dev = 0, sms = 0;
  MKA_CUDA_TRY(cudaGetDevice(&dev));
  MKA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((4 * s->n_atoms + 255) / 256, (int64_t)sms * 8));
  const TX* xx = reinterpret_cast<const TX*>(x);
  TX* yy = reinterpret_cast<TX*>(y);
  if (k == 1) spmv_kernel<TV, TX, 1><<<(unsigned)blocks, 256, 0, st>>>(s->d_row_ptr, s->d_col, val, xx, yy, s->n_atoms);
  else if (k == 2) spmv_kernel<TV, TX, 2><<<(unsigned)blocks, 256, 0, st>>>(s->d_row_ptr, s->d_col, val, xx, yy, s->n_atoms);
  else spmv_kernel<TV, TX, 4><<<(unsigned)blocks, 256, 0, st>>>(s->d_row_ptr, s->d_col, val, xx, yy, s->n_atoms);
  count_launches();
  MKA_CUDA_TRY(cudaGetLastError());
  return MKA_OK;
}

template <typename TV>
mka_status spmv_dispatch(const mka_system* s, const void* val, int x_dtype, const void* x, void* y, int k,
                         cudaStream_t st) {
  if (x_dtype == MKA_FP64) return spmv_dispatch_k<TV, double>(s, (const TV*)val, x, y, k, st);
  return spmv_dispatch_k<TV, float>(s, (const TV*)val, x, y, k, st);
}

// ---- density of states: D(E) = -(1/pi) Im sum_j (G(E + i eta) S)_jj = (eta/pi) sum w / ((E - eps)^2 + eta^2) ----
// Grid (level chunks, energy tiles of 256): a CTA stages its chunk's levels through shared memory
// 256 at a time, each thread one energy, and writes its chunk's sum; a second kernel adds the chunk
// sums in chunk order. FP64 throughout.
constexpr int kDosThreads = 256;
constexpr int64_t kDosChunk = 32768;   // levels per CTA

__global__ void __launch_bounds__(kDosThreads) dos_partial_kernel(const double* eps, const double* w, int64_t n,
                                                                  const double* energies, int n_e, double eta,
                                                                  double* partial) {
  __shared__ double se[kDosThreads], sw[kDosThreads];
  const int64_t l0 = (int64_t)blockIdx.x * kDosChunk, l1 = min(n, l0 + kDosChunk);
  const int k = blockIdx.y * kDosThreads + threadIdx.x;
  const double E = k < n_e ? energies[k] : 0.0;
  const double eta2 = eta * eta;
  double acc = 0.0;
  for (int64_t t0 = l0; t0 < l1; t0 += kDosThreads) {
    const int64_t t = t0 + threadIdx.x;
    se[threadIdx.x] = t < l1 ? eps[t] : 0.0;
    sw[threadIdx.x] = t < l1 ? w[t] : 0.0;
    __syncthreads();
    const int cnt = (int)(l1 - t0 < kDosThreads ? l1 - t0 : kDosThreads);
    for (int i = 0; i < cnt; ++i) {
      const double wi = sw[i];
      if (wi != 0.0) {
        const double d = E - se[i];
        acc += wi / (d * d + eta2);
      }
    }
    __syncthreads();
  }
  if (k < n_e) partial[(int64_t)blockIdx.x * n_e + k] = acc;
}

__global__ void dos_sum_kernel(const double* partial, int64_t n_chunks, int n_e, double scale, double* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_e) return;
  double s = 0.0;
  for (int64_t c = 0; c < n_chunks; ++c) s += partial[c * n_e + k];
  out[k] = scale * s;
}

// H's on-site blocks += shift[a] on the diagonal (one thread per atom): the diagonal block of row a found in
// its sorted columns, the stored value decoded, shifted and stored again in its format.
__global__ void onsite_shift_kernel(const int32_t* row_ptr, const int32_t* col, void* valH, int storage,
                                    const double* shift, int64_t n) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < n; a += (int64_t)gridDim.x * blockDim.x) {
    int lo = row_ptr[a], hi = row_ptr[a + 1] - 1, k = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      if (col[mid] == a) { k = mid; break; }
      if (col[mid] < a) lo = mid + 1; else hi = mid - 1;
    }
    if (k < 0) continue;
    for (int o = 0; o < 4; ++o) {
      const int64_t i = (int64_t)k * 16 + 5 * o;
      if (storage == MKA_FP64) reinterpret_cast<double*>(valH)[i] += shift[a];
      else if (storage == MKA_MIXED_FP32) reinterpret_cast<float*>(valH)[i] = (float)((double)reinterpret_cast<float*>(valH)[i] + shift[a]);
      else {
        __nv_bfloat16* v = reinterpret_cast<__nv_bfloat16*>(valH);
        v[i] = __double2bfloat16((double)__bfloat162float(v[i]) + shift[a]);
      }
    }
  }
}

}  // namespace

mka_status launch_onsite_shift(mka_system* sys, const double* shift_host, cudaStream_t st) {
  double* d = nullptr;
  MKA_CUDA_TRY(cudaMallocAsync(&d, sizeof(double) * sys->n_atoms, st));
  cudaError_t e = cudaMemcpyAsync(d, shift_host, sizeof(double) * sys->n_atoms, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((sys->n_atoms + 255) / 256, 4096));
    onsite_shift_kernel<<<(unsigned)blocks, 256, 0, st>>>(sys->d_row_ptr, sys->d_col, sys->d_valH, sys->storage, d,
                                                         sys->n_atoms);
    count_launches();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(d, st);
  if (e != cudaSuccess) return cuda_fail(e, "mka_system_shift_onsite");
  return MKA_OK;
}

mka_status launch_dos(const double* eps, const double* w, int64_t n, const double* energies, int n_e, double eta,
                      cudaStream_t st, double* dos_host) {
  const int64_t n_chunks = std::max<int64_t>(1, (n + kDosChunk - 1) / kDosChunk);
  double* buf = nullptr;
  MKA_CUDA_TRY(cudaMallocAsync(&buf, sizeof(double) * ((size_t)n_chunks * n_e + 2 * (size_t)n_e), st));
  double* d_e = buf + (size_t)n_chunks * n_e;
  double* d_out = d_e + n_e;
  cudaError_t e = cudaMemcpyAsync(d_e, energies, sizeof(double) * n_e, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    const dim3 grid((unsigned)n_chunks, (unsigned)((n_e + kDosThreads - 1) / kDosThreads));
    dos_partial_kernel<<<grid, kDosThreads, 0, st>>>(eps, w, n, d_e, n_e, eta, buf);
    dos_sum_kernel<<<(n_e + 255) / 256, 256, 0, st>>>(buf, n_chunks, n_e, eta / 3.14159265358979323846, d_out);
    count_launches(2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(dos_host, d_out, sizeof(double) * n_e, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(buf, st);
  if (e != cudaSuccess) return cuda_fail(e, "mka_dos");
  return MKA_OK;
}

size_t mu_buffer_bytes() { return sizeof(MuState) + sizeof(double) * 2 * kMaxRedBlocks + 64; }

mka_status find_mu_enqueue(const double* eps, const double* w, int64_t n, double n_electrons, double kT, double tol,
                           int halvings, void* buf, double* mu_dev_out, cudaStream_t st) {
  MuState* S = reinterpret_cast<MuState*>(buf);
  double* partial = reinterpret_cast<double*>(S + 1);
  unsigned* ticket = reinterpret_cast<unsigned*>(partial + 2 * kMaxRedBlocks);
  const int blocks = (int)std::min<int64_t>(red_blocks(), std::max<int64_t>(1, (n + kRedThreads - 1) / kRedThreads));
  mu_init_kernel<<<1, 1, 0, st>>>(S, ticket, n_electrons, kT, tol);
  eps_range_kernel<<<blocks, kRedThreads, 0, st>>>(eps, w, n, partial, ticket, S);
  for (int i = 0; i < halvings; ++i) bisect_kernel<<<blocks, kRedThreads, 0, st>>>(eps, w, n, partial, ticket, S);
  mu_finish_kernel<<<1, 1, 0, st>>>(S, mu_dev_out);
  count_launches(3 + halvings);
  MKA_CUDA_TRY(cudaGetLastError());
  return MKA_OK;
}

mka_status density_enqueue(const mka_system* sys, const int64_t* sel, const int64_t* blk_off, const double* vp,
                           const double* cv, const double* eps, const double* w, int64_t n_sel, int nu,
                           const double* mu_dev, double kT, double* rho_out, double* tmp, cudaStream_t st) {
  density_kernel<<<(unsigned)n_sel, 128, 0, st>>>(vp, cv, eps, blk_off, sel, sys->d_row_ptr, sys->d_valH,
                                                  sys->storage, nu, 0.0, mu_dev, kT, rho_out, tmp);
  sum_kernel<<<1, kRedThreads, 0, st>>>(tmp, n_sel, tmp + n_sel);
  const int rb = red_blocks();
  count_partial_kernel<<<rb, kRedThreads, 0, st>>>(eps, w, 4 * n_sel * nu, 0.0, mu_dev, kT, tmp + n_sel + 2);
  sum_kernel<<<1, kRedThreads, 0, st>>>(tmp + n_sel + 2, rb, tmp + n_sel + 1);
  count_launches(4);
  MKA_CUDA_TRY(cudaGetLastError());
  return MKA_OK;
}

mka_status density_global_enqueue(const mka_system* sys, const int64_t* sel, const int64_t* blk_off, const double* vp,
                                  const double* cv, const double* eps, int64_t n_sel, int nu, double mu, double kT,
                                  double* rho, int64_t out_base, double* e_atom, int64_t e_base, cudaStream_t st) {
  density_kernel<<<(unsigned)n_sel, 128, 0, st>>>(vp, cv, eps, blk_off, sel, sys->d_row_ptr, sys->d_valH, sys->storage,
                                                  nu, mu, nullptr, kT, rho, e_atom, out_base, e_base);
  count_launches();
  MKA_CUDA_TRY(cudaGetLastError());
  return MKA_OK;
}

mka_status launch_find_mu(mka_result* res, double n_electrons, double kT, double tol, double* mu_out) {
  cudaStream_t st = res->stream;
  const int64_t n = res->n_cols * res->nu;
  if (!res->d_mu_state) {
    MKA_CUDA_TRY(cudaMalloc(&res->d_mu_state, mu_buffer_bytes()));
    MKA_CUDA_TRY(cudaMemsetAsync(res->d_mu_state, 0, mu_buffer_bytes(), st));
  }
  MuState* S = reinterpret_cast<MuState*>(res->d_mu_state);
  double* partial = reinterpret_cast<double*>(S + 1);
  unsigned* ticket = reinterpret_cast<unsigned*>(partial + 2 * kMaxRedBlocks);
  MuState h{};
  h.target = n_electrons;
  h.kT = kT;
  h.tol = tol;
  MKA_CUDA_TRY(cudaMemcpyAsync(S, &h, sizeof(MuState), cudaMemcpyHostToDevice, st));
  MKA_CUDA_TRY(cudaMemsetAsync(ticket, 0, sizeof(unsigned), st));
  const int blocks = (int)std::min<int64_t>(red_blocks(), std::max<int64_t>(1, (n + kRedThreads - 1) / kRedThreads));
  eps_range_kernel<<<blocks, kRedThreads, 0, st>>>(res->d_eps, res->d_w, n, partial, ticket, S);
  count_launches();
  MKA_CUDA_TRY(cudaGetLastError());
  MKA_CUDA_TRY(cudaMemcpyAsync(&h, S, sizeof(MuState), cudaMemcpyDeviceToHost, st));
  MKA_CUDA_TRY(cudaStreamSynchronize(st));
  if (!(h.hi > h.lo)) return fail(MKA_ERR_INVALID_ARG, "no level with nonzero weight");
  const int halvings = std::min(200, (int)std::ceil(std::log2((h.hi - h.lo) / tol)) + 2);
  for (int i = 0; i < std::max(halvings, 1); ++i) {
    bisect_kernel<<<blocks, kRedThreads, 0, st>>>(res->d_eps, res->d_w, n, partial, ticket, S);
  }
  count_launches(std::max(halvings, 1));
  MKA_CUDA_TRY(cudaGetLastError());
  MKA_CUDA_TRY(cudaMemcpyAsync(&h, S, sizeof(MuState), cudaMemcpyDeviceToHost, st));
  MKA_CUDA_TRY(cudaStreamSynchronize(st));
  *mu_out = 0.5 * (h.lo + h.hi);
  return MKA_OK;
}

mka_status launch_density(mka_system* sys, mka_result* res, double mu, double kT, double* rho_out, double* e_band,
                          double* n_elec) {
  cudaStream_t st = res->stream;
  double* tmp = nullptr;
  const int rb = red_blocks();
  MKA_CUDA_TRY(cudaMallocAsync(&tmp, sizeof(double) * (res->n_sel + 2 + rb), st));
  density_kernel<<<(unsigned)res->n_sel, 128, 0, st>>>(res->d_vp, res->d_cv, res->d_eps, res->d_blk_off,
                                                       res->d_sel, sys->d_row_ptr, sys->d_valH, sys->storage,
                                                       res->nu, mu, nullptr, kT, rho_out, tmp);
  sum_kernel<<<1, kRedThreads, 0, st>>>(tmp, res->n_sel, tmp + res->n_sel);
  count_partial_kernel<<<rb, kRedThreads, 0, st>>>(res->d_eps, res->d_w, res->n_cols * res->nu, mu, nullptr,
                                                           kT, tmp + res->n_sel + 2);
  sum_kernel<<<1, kRedThreads, 0, st>>>(tmp + res->n_sel + 2, rb, tmp + res->n_sel + 1);
  count_launches(4);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && (e_band || n_elec)) {
    double h[2];
    e = cudaMemcpyAsync(h, tmp + res->n_sel, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
      if (e_band) *e_band = h[0];
      if (n_elec) *n_elec = h[1];
    }
  }
  cudaFreeAsync(tmp, st);
  if (e != cudaSuccess) return cuda_fail(e, "density");
  return MKA_OK;
}

mka_status launch_greens(mka_system* sys, mka_result* res, double z_re, double z_im, double* g_out) {
  greens_kernel<<<(unsigned)res->n_sel, 128, 0, res->stream>>>(res->d_vp, res->d_cv, res->d_eps, res->d_blk_off,
                                                               res->d_sel, sys->d_row_ptr, res->nu, z_re, z_im, g_out);
  count_launches();
  MKA_CUDA_TRY(cudaGetLastError());
  return MKA_OK;
}

mka_status launch_spmv(const mka_system* s, int which, int x_dtype, const void* x, void* y, int k, cudaStream_t st) {
  const void* val = which == 0 ? s->d_valH : s->d_valS;
  switch (s->storage) {
    case MKA_FP64: return spmv_dispatch<double>(s, val, x_dtype, x, y, k, st);
    case MKA_MIXED_FP32: return spmv_dispatch<float>(s, val, x_dtype, x, y, k, st);
    default: return spmv_dispatch<__nv_bfloat16>(s, val, x_dtype, x, y, k, st);
  }
}

}  // namespace mka
