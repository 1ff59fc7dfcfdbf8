// Forces of the multiple Arnoldi method on sm_103a (Sec. 2, Eqs. EQ-FORCE, EQ-FORCE-PART).
//
// With rho_ij (Eq. EQ-DM) and the energy density matrix pi_ij = sum_alpha f eps v_alpha,i v_alpha,j
// on the pattern of column j's row,
//   F_K = -2 sum_j sum_i ( rho_ij dH_ji/dR_K - pi_ij dS_ji/dR_K )
// (two electrons per orbital state; the sign of the pi term is the derivative of the grand
// potential at fixed mu, dOmega = 2 (Tr[rho dH] - Tr[pi dS])). H_ji for j = (b, c) and i = (a, r)
// is entry [c][r] of the Slater-Koster block of d = R_a - R_b, so it moves only with atoms a and b:
// the block contributes g = -2 sum_{c,r} (rho dB_H[c][r]/dd - pi dB_S[c][r]/dd) to F_a and -g to F_b.
// The block derivatives are formed from the positions and the model's FP64 parameters (the
// derivative of the exact model; values may be stored rounded).
//
// force_blocks_kernel: one CTA per selected atom b, thread per pattern entry (k, c, r):
//   rho = U_i . (C diag(f) V_j), pi = U_i . (C diag(f eps) V_j) from the kept data, then the entry's
//   three contributions, summed over the block's 16 entries by a fixed xor tree, one 3-vector per block.
// force_gather_kernel: F_K = sum over K's row blocks k' (neighbour a') of g[block of a' pointing to K]
//   - g[k'], each looked up in a fixed order, so the forces do not depend on timing.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "mka_internal.h"
#include "sk_grad.cuh"

namespace mka {
namespace {

__device__ __forceinline__ double fermi_d(double x, double mu, double kT) {
  const double y = (x - mu) / (2.0 * kT);
  if (y > 20.0) return 0.0;
  if (y < -20.0) return 1.0;
  return 0.5 * (1.0 - tanh(y));
}

}  // namespace

namespace {

struct ForceBlockArgs {
  const double* vp;
  const double* cv;
  const double* eps;
  const int64_t* blk_off;
  const int64_t* sel;
  const int32_t* row_ptr;
  const int32_t* col;
  const double* pos;
  double box[3];
  double Vh[4], Vs[4], d0;
  int nu;
  double mu, kT;
  int64_t out_base;          // < 0: outputs at the batch's blocks; else at row_ptr[atom] - out_base
  double* pi;                // [blocks][16] or NULL
  double* g;                 // [blocks][3]
};

__global__ void __launch_bounds__(128) force_blocks_kernel(const ForceBlockArgs A) {
  __shared__ double f[4 * MKA_MAX_NU], fe[4 * MKA_MAX_NU];
  __shared__ double gr[4 * MKA_MAX_NU], gp[4 * MKA_MAX_NU];
  const int nu = A.nu;
  const int64_t t = blockIdx.x;
  const int64_t atom = A.sel[t];
  const int64_t k0 = A.row_ptr[atom];
  const int nrow = A.row_ptr[atom + 1] - (int)k0;
  const int64_t b0 = A.blk_off[t];
  const int64_t ob = A.out_base < 0 ? b0 : k0 - A.out_base;
  for (int i = threadIdx.x; i < 4 * nu; i += blockDim.x) {
    const double e = A.eps[(4 * t + i / nu) * nu + i % nu];
    f[i] = fermi_d(e, A.mu, A.kT);
    fe[i] = f[i] * e;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * nu; i += blockDim.x) {   // g = C diag(x) V_j for x = f and f eps
    const int c = i / nu, n = i % nu;
    const int64_t colj = 4 * t + c;
    const double* bk = A.cv + (size_t)(colj >> 5) * kept_block_doubles(nu) * 32 + (colj & 31);
    double s1 = 0.0, s2 = 0.0;
    for (int a = 0; a < nu; ++a) {
      const double cv = bk[(size_t)(n * nu + a) * 32] * bk[(size_t)(nu * nu + a) * 32];
      s1 += cv * f[c * nu + a];
      s2 += cv * fe[c * nu + a];
    }
    gr[i] = s1;
    gp[i] = s2;
  }
  __syncthreads();
  const double ax = A.pos[3 * atom], ay = A.pos[3 * atom + 1], az = A.pos[3 * atom + 2];
  for (int base = 0; base < nrow * 16; base += blockDim.x) {   // whole warps iterate together (shuffles below)
    const int i = base + threadIdx.x;
    const bool on = i < nrow * 16;
    const int k = i >> 4, c = (i >> 2) & 3, r = i & 3;
    double e[3] = {0.0, 0.0, 0.0};
    if (on) {
      const double* u = A.vp + ((b0 + k) * 16 + c * 4 + r) * (int64_t)nu;
      double rho = 0.0, pi = 0.0;
      for (int n = 0; n < nu; ++n) {
        rho += u[n] * gr[c * nu + n];
        pi += u[n] * gp[c * nu + n];
      }
      if (A.pi) A.pi[(ob + k) * 16 + c * 4 + r] = pi;
      const int64_t a = A.col[k0 + k];
      if (a != atom) {
        double d[3] = {A.pos[3 * a] - ax, A.pos[3 * a + 1] - ay, A.pos[3 * a + 2] - az};
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
    if (on && (threadIdx.x & 15) == 0)
      for (int q = 0; q < 3; ++q) A.g[(ob + k) * 3 + q] = e[q];
  }
}

// Batch layout: F[a] += g and F[b] -= g for every block (atomic FP64 adds; their order is not fixed).
__global__ void force_scatter_kernel(const double* g, const int64_t* blk_off, const int64_t* sel, const int32_t* row_ptr,
                                     const int32_t* col, int64_t n_sel, double* F) {
  for (int64_t t = blockIdx.x; t < n_sel; t += gridDim.x) {
    const int64_t atom = sel[t];
    const int64_t k0 = row_ptr[atom];
    const int nrow = row_ptr[atom + 1] - (int)k0;
    for (int k = threadIdx.x; k < nrow; k += blockDim.x) {
      const int64_t a = col[k0 + k];
      if (a == atom) continue;
      const double* gk = g + (blk_off[t] + k) * 3;
      for (int q = 0; q < 3; ++q) {
        atomicAdd(&F[3 * a + q], gk[q]);
        atomicAdd(&F[3 * atom + q], -gk[q]);
      }
    }
  }
}

// System layout over the pattern blocks [blk0, blk0 + nblk) of atoms [a0, a1): one thread per atom K of
// the whole system, F_K = sum_{k' in row K, a' = col[k'] != K} ( [a' in range] g[block (a', K)] - [K in range] g[k'] ).
__global__ void force_gather_kernel(const double* g, const int32_t* row_ptr, const int32_t* col, int64_t n_atoms,
                                    int64_t a0, int64_t a1, int64_t blk0, double* F) {
  for (int64_t K = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; K < n_atoms; K += (int64_t)gridDim.x * blockDim.x) {
    double s[3] = {0.0, 0.0, 0.0};
    const bool own = K >= a0 && K < a1;
    for (int64_t k = row_ptr[K]; k < row_ptr[K + 1]; ++k) {
      const int64_t a = col[k];
      if (a == K) continue;
      if (a >= a0 && a < a1) {
        int64_t t = row_ptr[a];
        const int64_t t1 = row_ptr[a + 1];
        while (t < t1 && col[t] != K) ++t;     // the pattern is symmetric: (a, K) exists
        if (t < t1)
          for (int q = 0; q < 3; ++q) s[q] += g[(t - blk0) * 3 + q];
      }
      if (own)
        for (int q = 0; q < 3; ++q) s[q] -= g[(k - blk0) * 3 + q];
    }
    for (int q = 0; q < 3; ++q) F[3 * K + q] = s[q];
  }
}

}  // namespace

mka_status force_blocks_enqueue(const mka_system* sys, const int64_t* sel, const int64_t* blk_off, const double* vp,
                                const double* cv, const double* eps, int64_t n_sel, int nu, double mu, double kT,
                                int64_t out_base, double* pi, double* g, cudaStream_t st) {
  if (!sys->have_sk) return fail(MKA_ERR_INVALID_ARG, "forces need the Slater-Koster model (mka_build_system)");
  ForceBlockArgs A{};
  A.vp = vp;
  A.cv = cv;
  A.eps = eps;
  A.blk_off = blk_off;
  A.sel = sel;
  A.row_ptr = sys->d_row_ptr;
  A.col = sys->d_col;
  A.pos = sys->d_pos;
  for (int q = 0; q < 3; ++q) A.box[q] = sys->box[q];
  for (int q = 0; q < 4; ++q) {
    A.Vh[q] = sys->sk.V[q];
    A.Vs[q] = sys->sk.Sv[q];
  }
  A.d0 = sys->sk.d0;
  A.nu = nu;
  A.mu = mu;
  A.kT = kT;
  A.out_base = out_base;
  A.pi = pi;
  A.g = g;
  force_blocks_kernel<<<(unsigned)n_sel, 128, 0, st>>>(A);
  count_launches();
  MKA_CUDA_TRY(cudaGetLastError());
  return MKA_OK;
}

mka_status force_gather_enqueue(const mka_system* sys, const double* g, int64_t a0, int64_t a1, int64_t blk0, double* F,
                                cudaStream_t st) {
  int dev = 0, sms = 0;
  MKA_CUDA_TRY(cudaGetDevice(&dev));
  MKA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((sys->n_atoms + 255) / 256, (int64_t)sms * 8));
  force_gather_kernel<<<(unsigned)blocks, 256, 0, st>>>(g, sys->d_row_ptr, sys->d_col, sys->n_atoms, a0, a1, blk0, F);
  count_launches();
  MKA_CUDA_TRY(cudaGetLastError());
  return MKA_OK;
}

}  // namespace mka

using namespace mka;

extern "C" mka_status mka_forces(mka_system* sys, mka_result* res, double mu, double kT, double* pi_out, double* forces) {
  if (!sys || !res || res->sys != sys) return fail(MKA_ERR_INVALID_ARG, "result does not belong to this system");
  if (!res->keep) return fail(MKA_ERR_INVALID_ARG, "forces need a result solved with keep_vectors = 1");
  if (!(kT > 0)) return fail(MKA_ERR_INVALID_ARG, "need kT > 0");
  if (!pi_out && !forces) return MKA_OK;
  cudaStream_t st = res->stream;
  double* g = nullptr;
  MKA_CUDA_TRY(cudaMallocAsync(&g, sizeof(double) * 3 * std::max<int64_t>(1, res->n_blocks), st));
  mka_status s = force_blocks_enqueue(sys, res->d_sel, res->d_blk_off, res->d_vp, res->d_cv, res->d_eps, res->n_sel,
                                      res->nu, mu, kT, -1, pi_out, g, st);
  if (!s && forces) {
    force_scatter_kernel<<<(unsigned)std::min<int64_t>(res->n_sel, 4096), 64, 0, st>>>(
        g, res->d_blk_off, res->d_sel, sys->d_row_ptr, sys->d_col, res->n_sel, forces);
    count_launches();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) s = cuda_fail(e, "force_scatter_kernel");
  }
  cudaFreeAsync(g, st);
  return s;
}
