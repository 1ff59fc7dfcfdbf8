// Learned warm start for the inner CG (S s_j = e_j, Sec. 2): input features, the network's
// forward / backward / Adam kernels, and the C entry points.
//
// Features of atom a (one warp per atom): its 32 nearest neighbours within 3 A (minimum
// image, distance order, ties by atom id) as (d, l, m, n) with (l, m, n) the direction
// cosines of r_b - r_a, zeros beyond; the 17-atom output patch is a and its 16 nearest
// neighbours. A column's input row is those 128 numbers and a one-hot of its orbital (132).
//
// Network 132 -> 128 -> 128 -> 68 with SiLU after the hidden layers. Parameters are kept in
// FP32 (Adam master copy) and rounded to BF16 for every product; activations and sums are
// FP32. Loss: mean of (y - t)^2 over the batch and the 68 outputs. Weight gradients are
// batch reductions in a fixed order (one thread per weight), so training is deterministic.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <random>
#include <vector>

#include "mka_internal.h"

namespace mka {
namespace {

constexpr int kIn = 132, kHid = 128, kOut = 68;
constexpr int kNeigh = 32, kPatch = 17;
constexpr int kFeatGather = 256;                   // candidates per atom kept for selection
constexpr int64_t kP = (int64_t)kHid * kIn + kHid + (int64_t)kHid * kHid + kHid + (int64_t)kOut * kHid + kOut;
constexpr int64_t oW1 = 0, ob1 = oW1 + kHid * kIn, oW2 = ob1 + kHid, ob2 = oW2 + kHid * kHid, oW3 = ob2 + kHid,
                  ob3 = oW3 + kOut * kHid;

__device__ __forceinline__ float bf(const __nv_bfloat16* p, int64_t i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ float silu_f(float x) { return x / (1.0f + __expf(-x)); }
__device__ __forceinline__ float dsilu_f(float x) {
  const float s = 1.0f / (1.0f + __expf(-x));
  return s * (1.0f + x * (1.0f - s));
}

// ---- features --------------------------------------------------------------------------
struct FeatArgs {
  const double* pos;
  const float* posf;
  double box[3], inv_box[3];
  float pre_hi;     // FP32 prefilter: candidates beyond pre_hi * r_gather^2 are dropped unseen
  int ncell[3];
  double cell_len[3];
  const int32_t* cell_start;
  const int32_t* cell_atoms;
  const int64_t* sel;
  int64_t n_sel;
  double r_gather2;
  float* X;         // [4 n_sel][132]
  int32_t* patch;   // [n_sel][17] atom ids, -1 where fewer atoms were found
};

__device__ __forceinline__ int cell_coord_f(double x, double len, int n) {
  int v = (int)floor(x / len);
  return v < 0 ? 0 : (v >= n ? n - 1 : v);
}

__device__ __forceinline__ int cell_range_f(int c, int n, int out[3]) {
  if (n < 3) {
    for (int i = 0; i < n; ++i) out[i] = i;
    return n;
  }
  out[0] = (c + n - 1) % n;
  out[1] = c;
  out[2] = (c + 1) % n;
  return 3;
}

// Minimum-image displacement and distance in the operation order of a plain evaluation
// (d = b - a; d -= L k with k = rint(d / L); r^2 = (dx^2 + dy^2) + dz^2), without contraction,
// so that neighbour order and the 3 A cut agree with any IEEE evaluation of the same formula.
// k is taken as rint(d * (1/L)): it differs from rint(d / L) only when d / L is within an ulp of
// +-1/2, i.e. for atoms half a box away, far outside the gather radius.
__device__ __forceinline__ double mi_comp(double pb, double pa, double L, double invL) {
  const double d = __dsub_rn(pb, pa);
  return __dsub_rn(d, __dmul_rn(L, rint(d * invL)));
}

// One warp per atom; per warp kFeatGather (distance, id) candidate slots in shared memory.
__global__ void __launch_bounds__(256) features_kernel(FeatArgs A) {
  __shared__ double rk[8][kFeatGather];
  __shared__ int idk[8][kFeatGather];
  __shared__ int cnt[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t warp = (int64_t)blockIdx.x * 8 + wid, nw = (int64_t)gridDim.x * 8;
  for (int64_t t = warp; t < A.n_sel; t += nw) {
    const int64_t a = A.sel[t];
    const double px = A.pos[3 * a], py = A.pos[3 * a + 1], pz = A.pos[3 * a + 2];
    const float pxf = A.posf[3 * a], pyf = A.posf[3 * a + 1], pzf = A.posf[3 * a + 2];
    const float Lf[3] = {(float)A.box[0], (float)A.box[1], (float)A.box[2]};
    const float iLf[3] = {(float)A.inv_box[0], (float)A.inv_box[1], (float)A.inv_box[2]};
    const float rg2f = (float)A.r_gather2;
    int rx[3], ry[3], rz[3];
    const int nx = cell_range_f(cell_coord_f(px, A.cell_len[0], A.ncell[0]), A.ncell[0], rx);
    const int ny = cell_range_f(cell_coord_f(py, A.cell_len[1], A.ncell[1]), A.ncell[1], ry);
    const int nz = cell_range_f(cell_coord_f(pz, A.cell_len[2], A.ncell[2]), A.ncell[2], rz);
    if (lane == 0) cnt[wid] = 0;
    __syncwarp();
    for (int ci = 0; ci < nx * ny * nz; ++ci) {
      const int ix = ci / (ny * nz), iy = (ci / nz) % ny, iz = ci % nz;
      const int c = (rx[ix] * A.ncell[1] + ry[iy]) * A.ncell[2] + rz[iz];
      for (int k = A.cell_start[c] + lane; k < A.cell_start[c + 1]; k += 32) {
        const int b = A.cell_atoms[k];
        if (b == a) continue;
        float fx = A.posf[3 * b] - pxf, fy = A.posf[3 * b + 1] - pyf, fz = A.posf[3 * b + 2] - pzf;
        fx -= Lf[0] * rintf(fx * iLf[0]);
        fy -= Lf[1] * rintf(fy * iLf[1]);
        fz -= Lf[2] * rintf(fz * iLf[2]);
        if (fx * fx + fy * fy + fz * fz > A.pre_hi * rg2f) continue;
        const double dx = mi_comp(A.pos[3 * b], px, A.box[0], A.inv_box[0]);
        const double dy = mi_comp(A.pos[3 * b + 1], py, A.box[1], A.inv_box[1]);
        const double dz = mi_comp(A.pos[3 * b + 2], pz, A.box[2], A.inv_box[2]);
        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        if (r2 <= A.r_gather2) {
          const int s = atomicAdd(&cnt[wid], 1);
          if (s < kFeatGather) {
            rk[wid][s] = __dsqrt_rn(r2);
            idk[wid][s] = b;
          }
        }
      }
    }
    __syncwarp();
    const int n = min(cnt[wid], kFeatGather);
    float geo[4] = {0, 0, 0, 0};   // lane k < 32 keeps neighbour k's (d, l, m, n)
    int my_id = -1;
    // the 32 nearest by repeated warp minima of (distance, id)
    for (int k = 0; k < kNeigh; ++k) {
      double best = INFINITY;
      int bid = 0x7fffffff, bi = -1;
      for (int s = lane; s < n; s += 32) {
        const double r = rk[wid][s];
        const int id = idk[wid][s];
        if (r < best || (r == best && id < bid)) {
          best = r;
          bid = id;
          bi = s;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oid = __shfl_xor_sync(0xffffffffu, bid, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob < best || (ob == best && oid < bid)) {
          best = ob;
          bid = oid;
          bi = oi;
        }
      }
      if (bi < 0) break;
      if (lane == k) {
        my_id = bid;
        if (best <= 3.0) {
          const double dx = mi_comp(A.pos[3 * bid], px, A.box[0], A.inv_box[0]);
          const double dy = mi_comp(A.pos[3 * bid + 1], py, A.box[1], A.inv_box[1]);
          const double dz = mi_comp(A.pos[3 * bid + 2], pz, A.box[2], A.inv_box[2]);
          geo[0] = (float)best;
          geo[1] = (float)__ddiv_rn(dx, best);
          geo[2] = (float)__ddiv_rn(dy, best);
          geo[3] = (float)__ddiv_rn(dz, best);
        }
      }
      __syncwarp();
      if (lane == 0) rk[wid][bi] = INFINITY;
      __syncwarp();
    }
    for (int o = 0; o < 4; ++o) {
      float* row = A.X + (4 * t + o) * (int64_t)kIn;
      for (int q = 0; q < 4; ++q) row[4 * lane + q] = geo[q];
      if (lane < 4) row[128 + lane] = (lane == o) ? 1.0f : 0.0f;
    }
    if (lane == 0) A.patch[t * kPatch] = (int32_t)a;
    if (lane < kPatch - 1) A.patch[t * kPatch + 1 + lane] = my_id;
    __syncwarp();
  }
}

// ---- network kernels --------------------------------------------------------------------
// Y[b][o] = act(sum_k X[b][k] W[o][k] + bias[o]) (pre-activation into Z when given): a CTA computes
// a 64-row x 64-output tile, each thread 4 x 4, with 32-wide k slices of X and W (W decoded from
// BF16) staged in shared memory.
template <int ACT>
__global__ void __launch_bounds__(256) dense_fwd_tiled(const float* __restrict__ X, int64_t B, int n, int o_dim,
                                                       const __nv_bfloat16* __restrict__ W,
                                                       const __nv_bfloat16* __restrict__ bias, float* __restrict__ Z,
                                                       float* __restrict__ Y) {
  __shared__ float xs[32][68];
  __shared__ float ws[32][68];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t r0 = (int64_t)blockIdx.x * 64;
  const int o0 = blockIdx.y * 64;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
  for (int k0 = 0; k0 < n; k0 += 32) {
    for (int i = threadIdx.x; i < 64 * 32; i += 256) {
      const int r = i >> 5, k = i & 31;
      xs[k][r] = (r0 + r < B && k0 + k < n) ? X[(r0 + r) * n + k0 + k] : 0.0f;
      ws[k][r] = (o0 + r < o_dim && k0 + k < n) ? bf(W, (int64_t)(o0 + r) * n + k0 + k) : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = xs[k][ty * 4 + i];
        b[i] = ws[k][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t r = r0 + ty * 4 + i;
    if (r >= B) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int o = o0 + tx * 4 + j;
      if (o >= o_dim) continue;
      const float z = acc[i][j] + bf(bias, o);
      if (Z) Z[r * o_dim + o] = z;
      Y[r * o_dim + o] = ACT ? silu_f(z) : z;
    }
  }
}

// d_in[b][i] = (sum_o d_out[b][o] W[o][i]) * silu'(z_in[b][i])
__global__ void dense_bwd_data_kernel(const float* __restrict__ dout, int64_t B, int n, int o_dim,
                                      const __nv_bfloat16* __restrict__ W, const float* __restrict__ zin,
                                      float* __restrict__ din) {
  __shared__ float gs[16][kHid + 1];
  const int64_t b0 = (int64_t)blockIdx.x * 16;
  for (int i = threadIdx.x; i < 16 * o_dim; i += blockDim.x) {
    const int r = i / o_dim, c = i % o_dim;
    gs[r][c] = (b0 + r < B) ? dout[(b0 + r) * o_dim + c] : 0.0f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 16 * n; i += blockDim.x) {
    const int r = i / n, k = i % n;
    if (b0 + r >= B) continue;
    float acc = 0.0f;
    for (int o = 0; o < o_dim; ++o) acc += gs[r][o] * bf(W, (int64_t)o * n + k);
    din[(b0 + r) * n + k] = acc * dsilu_f(zin[(b0 + r) * n + k]);
  }
}

// G[o][i] = sum_b d_out[b][o] in[b][i] (i < n), and G_bias[o] = sum_b d_out[b][o]; batch order fixed.
__global__ void dense_bwd_weight_kernel(const float* __restrict__ dout, const float* __restrict__ in, int64_t B,
                                        int n, int o_dim, float* __restrict__ gW, float* __restrict__ gb) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)o_dim * (n + 1);
  if (idx >= total) return;
  const int o = (int)(idx / (n + 1)), i = (int)(idx % (n + 1));
  float acc = 0.0f;
  if (i < n) {
    for (int64_t b = 0; b < B; ++b) acc += dout[b * o_dim + o] * in[b * n + i];
    gW[(int64_t)o * n + i] = acc;
  } else {
    for (int64_t b = 0; b < B; ++b) acc += dout[b * o_dim + o];
    gb[o] = acc;
  }
}

// dY = 2 (Y - T) / (B K); per-block partial sums of (Y - T)^2 / (B K).
__global__ void mse_kernel(const float* Y, const float* T, int64_t n, float inv, float* dY, float* partial) {
  __shared__ float red[8];
  float acc = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = Y[i] - T[i];
    dY[i] = 2.0f * d * inv;
    acc += d * d * inv;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    partial[blockIdx.x] = s;
  }
}

__global__ void sum_f_kernel(const float* x, int n, float* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.0f;
    for (int i = 0; i < n; ++i) s += x[i];
    *out = s;
  }
}

__global__ void adam_kernel(float* theta, __nv_bfloat16* thetab, const float* g, float* m, float* v, int64_t n, float lr,
                            float b1, float b2, float c1, float c2, float eps) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float t = theta[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    theta[i] = t;
    thetab[i] = __float2bfloat16_rn(t);
  }
}

__global__ void to_bf16_kernel(const float* x, __nv_bfloat16* y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

unsigned blocks_for(int64_t n, int per) { return (unsigned)std::max<int64_t>(1, (n + per - 1) / per); }

}  // namespace

// forward through the network for B rows (buffers sized for B)
mka_status mlp_forward_enqueue(const mka_mlp* net, const float* X, int64_t B, float* Z1, float* H1, float* Z2,
                               float* H2, float* Y, cudaStream_t st);

}  // namespace mka

struct mka_mlp {
  float* theta = nullptr;          // FP32 master
  __nv_bfloat16* thetab = nullptr; // BF16 copy used by every product
  float* m = nullptr;
  float* v = nullptr;
  float* g = nullptr;
  float* loss = nullptr;           // [0] loss, [1..] partials
  int64_t t = 0;                   // Adam steps taken
  int64_t cap = 0;                 // batch capacity of the work buffers
  float* work = nullptr;           // Z1, H1, Z2, H2, Y, dY, dZ2, dZ1
};

namespace mka {

mka_status mlp_forward_enqueue(const mka_mlp* net, const float* X, int64_t B, float* Z1, float* H1, float* Z2,
                               float* H2, float* Y, cudaStream_t st) {
  const __nv_bfloat16* P = net->thetab;
  const unsigned nb = blocks_for(B, 64);
  dense_fwd_tiled<1><<<dim3(nb, 2), 256, 0, st>>>(X, B, kIn, kHid, P + oW1, P + ob1, Z1, H1);
  dense_fwd_tiled<1><<<dim3(nb, 2), 256, 0, st>>>(H1, B, kHid, kHid, P + oW2, P + ob2, Z2, H2);
  dense_fwd_tiled<0><<<dim3(nb, 2), 256, 0, st>>>(H2, B, kHid, kOut, P + oW3, P + ob3, nullptr, Y);
  count_launches(3);
  MKA_CUDA_TRY(cudaGetLastError());
  return MKA_OK;
}

mka_status features_enqueue(const mka_system* sys, const int64_t* d_sel, int64_t n, float* X, int32_t* patch,
                            cudaStream_t st) {
  FeatArgs A{};
  A.pos = sys->d_pos;
  A.posf = sys->d_posf;
  const double lmax = std::max(sys->box[0], std::max(sys->box[1], sys->box[2]));
  A.pre_hi = (float)(1.0 + std::max(1e-3, 1e-5 * lmax / 5.5));
  for (int d = 0; d < 3; ++d) {
    A.box[d] = sys->box[d];
    A.inv_box[d] = 1.0 / sys->box[d];
    A.ncell[d] = sys->cells.n[d];
    A.cell_len[d] = sys->cells.len[d];
  }
  A.cell_start = sys->cells.start;
  A.cell_atoms = sys->cells.atoms;
  A.sel = d_sel;
  A.n_sel = n;
  const double rg = std::min(5.5, std::min(sys->cells.len[0], std::min(sys->cells.len[1], sys->cells.len[2])));
  A.r_gather2 = rg * rg;
  A.X = X;
  A.patch = patch;
  features_kernel<<<blocks_for(n, 8), 256, 0, st>>>(A);
  count_launches();
  MKA_CUDA_TRY(cudaGetLastError());
  return MKA_OK;
}

int64_t mlp_work_floats(int64_t B) { return B * (4 * kHid + 2 * kOut + 2 * kHid); }

}  // namespace mka

using namespace mka;

namespace {
mka_status mlp_reserve(mka_mlp* net, int64_t B) {
  if (B <= net->cap) return MKA_OK;
  cudaFree(net->work);
  net->work = nullptr;
  MKA_CUDA_TRY(cudaMalloc(&net->work, sizeof(float) * mlp_work_floats(B)));
  net->cap = B;
  return MKA_OK;
}

// forward + loss + backward into net->g (uses the BF16 weights), loss into net->loss[0]
mka_status mlp_grad_enqueue(mka_mlp* net, const float* X, const float* T, int64_t B, cudaStream_t st) {
  mka_status s = mlp_reserve(net, B);
  if (s) return s;
  float* Z1 = net->work;
  float* H1 = Z1 + B * kHid;
  float* Z2 = H1 + B * kHid;
  float* H2 = Z2 + B * kHid;
  float* Y = H2 + B * kHid;
  float* dY = Y + B * kOut;
  float* dZ2 = dY + B * kOut;
  float* dZ1 = dZ2 + B * kHid;
  s = mlp_forward_enqueue(net, X, B, Z1, H1, Z2, H2, Y, st);
  if (s) return s;
  const __nv_bfloat16* P = net->thetab;
  float* G = net->g;
  const int nred = 64;
  mse_kernel<<<nred, 256, 0, st>>>(Y, T, B * kOut, 1.0f / (float)(B * kOut), dY, net->loss + 1);
  sum_f_kernel<<<1, 32, 0, st>>>(net->loss + 1, nred, net->loss);
  dense_bwd_data_kernel<<<blocks_for(B, 16), 256, 0, st>>>(dY, B, kHid, kOut, P + oW3, Z2, dZ2);
  dense_bwd_data_kernel<<<blocks_for(B, 16), 256, 0, st>>>(dZ2, B, kHid, kHid, P + oW2, Z1, dZ1);
  dense_bwd_weight_kernel<<<blocks_for((int64_t)kOut * (kHid + 1), 128), 128, 0, st>>>(dY, H2, B, kHid, kOut, G + oW3,
                                                                                         G + ob3);
  dense_bwd_weight_kernel<<<blocks_for((int64_t)kHid * (kHid + 1), 128), 128, 0, st>>>(dZ2, H1, B, kHid, kHid, G + oW2,
                                                                                         G + ob2);
  dense_bwd_weight_kernel<<<blocks_for((int64_t)kHid * (kIn + 1), 128), 128, 0, st>>>(dZ1, X, B, kIn, kHid, G + oW1,
                                                                                        G + ob1);
  count_launches(7);
  MKA_CUDA_TRY(cudaGetLastError());
  return MKA_OK;
}
}  // namespace

extern "C" {

int64_t mka_mlp_num_params(void) { return kP; }

void mka_mlp_destroy(mka_mlp* net) {
  if (!net) return;
  cudaFree(net->theta);
  cudaFree(net->thetab);
  cudaFree(net->m);
  cudaFree(net->v);
  cudaFree(net->g);
  cudaFree(net->loss);
  cudaFree(net->work);
  delete net;
}

mka_status mka_mlp_create(uint64_t seed, mka_mlp** out) {
  if (!out) return fail(MKA_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  mka_mlp* net = new mka_mlp();
  cudaError_t e = cudaSuccess;
#define ALLOC(p, bytes) \
  if (e == cudaSuccess) e = cudaMalloc(&(p), (bytes))
  ALLOC(net->theta, sizeof(float) * kP);
  ALLOC(net->thetab, sizeof(__nv_bfloat16) * kP);
  ALLOC(net->m, sizeof(float) * kP);
  ALLOC(net->v, sizeof(float) * kP);
  ALLOC(net->g, sizeof(float) * kP);
  ALLOC(net->loss, sizeof(float) * 80);
#undef ALLOC
  if (e != cudaSuccess) {
    mka_mlp_destroy(net);
    return cuda_fail(e, "mka_mlp_create");
  }
  // He-uniform initialisation (weights U(-sqrt(6/fan_in), +)), zero biases, from a seeded mt19937_64
  std::vector<float> h(kP, 0.0f);
  std::mt19937_64 rng(seed);
  const int fan[3] = {kIn, kHid, kHid}, outd[3] = {kHid, kHid, kOut};
  const int64_t off[3] = {oW1, oW2, oW3};
  for (int l = 0; l < 3; ++l) {
    const double lim = std::sqrt(6.0 / fan[l]);
    std::uniform_real_distribution<double> U(-lim, lim);
    for (int64_t i = 0; i < (int64_t)fan[l] * outd[l]; ++i) h[off[l] + i] = (float)U(rng);
  }
  e = cudaMemcpy(net->theta, h.data(), sizeof(float) * kP, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(net->m, 0, sizeof(float) * kP);
  if (e == cudaSuccess) e = cudaMemset(net->v, 0, sizeof(float) * kP);
  if (e != cudaSuccess) {
    mka_mlp_destroy(net);
    return cuda_fail(e, "mka_mlp_create");
  }
  to_bf16_kernel<<<blocks_for(kP, 256), 256>>>(net->theta, net->thetab, kP);
  count_launches();
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    mka_mlp_destroy(net);
    return cuda_fail(e, "mka_mlp_create");
  }
  *out = net;
  return MKA_OK;
}

mka_status mka_mlp_set_params(mka_mlp* net, const float* host) {
  if (!net || !host) return fail(MKA_ERR_INVALID_ARG, "network and parameters are required");
  MKA_CUDA_TRY(cudaMemcpy(net->theta, host, sizeof(float) * kP, cudaMemcpyHostToDevice));
  MKA_CUDA_TRY(cudaMemset(net->m, 0, sizeof(float) * kP));
  MKA_CUDA_TRY(cudaMemset(net->v, 0, sizeof(float) * kP));
  net->t = 0;
  to_bf16_kernel<<<blocks_for(kP, 256), 256>>>(net->theta, net->thetab, kP);
  count_launches();
  MKA_CUDA_TRY(cudaDeviceSynchronize());
  return MKA_OK;
}

mka_status mka_mlp_get_params(const mka_mlp* net, float* host, int bf16_rounded) {
  if (!net || !host) return fail(MKA_ERR_INVALID_ARG, "network and output are required");
  if (!bf16_rounded) {
    MKA_CUDA_TRY(cudaMemcpy(host, net->theta, sizeof(float) * kP, cudaMemcpyDeviceToHost));
    return MKA_OK;
  }
  std::vector<uint16_t> b(kP);
  MKA_CUDA_TRY(cudaMemcpy(b.data(), net->thetab, sizeof(uint16_t) * kP, cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < kP; ++i) {
    const uint32_t u = (uint32_t)b[i] << 16;
    std::memcpy(&host[i], &u, 4);
  }
  return MKA_OK;
}

mka_status mka_mlp_forward(mka_mlp* net, const float* X, float* Y, int64_t B, void* stream) {
  if (!net || !X || !Y || B < 1) return fail(MKA_ERR_INVALID_ARG, "network, X, Y and B >= 1 are required");
  mka_status s = mlp_reserve(net, B);
  if (s) return s;
  float* Z1 = net->work;
  float* H1 = Z1 + B * kHid;
  float* Z2 = H1 + B * kHid;
  float* H2 = Z2 + B * kHid;
  return mlp_forward_enqueue(net, X, B, Z1, H1, Z2, H2, Y, (cudaStream_t)stream);
}

mka_status mka_mlp_gradients(mka_mlp* net, const float* X, const float* T, int64_t B, float* grad, float* loss,
                             void* stream) {
  if (!net || !X || !T || B < 1) return fail(MKA_ERR_INVALID_ARG, "network, X, T and B >= 1 are required");
  cudaStream_t st = (cudaStream_t)stream;
  mka_status s = mlp_grad_enqueue(net, X, T, B, st);
  if (s) return s;
  if (grad) MKA_CUDA_TRY(cudaMemcpyAsync(grad, net->g, sizeof(float) * kP, cudaMemcpyDeviceToDevice, st));
  if (loss) MKA_CUDA_TRY(cudaMemcpyAsync(loss, net->loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
  return MKA_OK;
}

mka_status mka_mlp_train_step(mka_mlp* net, const float* X, const float* T, int64_t B, float lr, float* loss,
                              void* stream) {
  if (!net || !X || !T || B < 1 || !(lr > 0)) return fail(MKA_ERR_INVALID_ARG, "bad training arguments");
  cudaStream_t st = (cudaStream_t)stream;
  mka_status s = mlp_grad_enqueue(net, X, T, B, st);
  if (s) return s;
  net->t += 1;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - std::pow(b1, (double)net->t)), c2 = (float)(1.0 - std::pow(b2, (double)net->t));
  adam_kernel<<<blocks_for(kP, 256), 256, 0, st>>>(net->theta, net->thetab, net->g, net->m, net->v, kP, lr, (float)b1,
                                                   (float)b2, c1, c2, 1e-8f);
  count_launches();
  MKA_CUDA_TRY(cudaGetLastError());
  if (loss) MKA_CUDA_TRY(cudaMemcpyAsync(loss, net->loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
  return MKA_OK;
}

mka_status mka_warm_start_features(const mka_system* sys, const int64_t* atoms, int64_t n, float* X, int32_t* patch,
                                   void* stream) {
  if (!sys || !atoms || n < 1 || !X || !patch) return fail(MKA_ERR_INVALID_ARG, "bad feature arguments");
  for (int64_t t = 0; t < n; ++t)
    if (atoms[t] < 0 || atoms[t] >= sys->n_atoms) return fail(MKA_ERR_INVALID_ARG, "atom index out of range");
  cudaStream_t st = (cudaStream_t)stream;
  int64_t* d_sel = nullptr;
  MKA_CUDA_TRY(cudaMallocAsync(&d_sel, sizeof(int64_t) * n, st));
  MKA_CUDA_TRY(cudaMemcpyAsync(d_sel, atoms, sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
  mka_status s = features_enqueue(sys, d_sel, n, X, patch, st);
  cudaFreeAsync(d_sel, st);
  return s;
}

mka_status mka_system_set_warm_start(mka_system* sys, mka_mlp* net) {
  if (!sys) return fail(MKA_ERR_INVALID_ARG, "system is NULL");
  sys->warm = net;
  return MKA_OK;
}

}  // extern "C"
