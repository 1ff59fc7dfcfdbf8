// Batched reduced problems of the multiple Arnoldi method on sm_103a.
//
// Every column j ends its basis with the nu x nu projected matrices H_r = U^T H U and
// S_r = U^T S U (formed explicitly, so that a basis that is only nearly S-orthonormal
// still gives the Galerkin pencil of its span) and solves the generalized eigenproblem
// H_r c = eps S_r c (Eq. EQ-SUB-EIG-VEC): Cholesky S_r = L L^T, A = L^{-1} H_r L^{-T},
// Householder tridiagonalisation A = Q T Q^T, implicit-shift QL on T with the rotations
// accumulated into Z = Q, C = L^{-T} Z. The outputs of a column are its levels eps_alpha
// in ascending order, w_alpha = V_{j alpha} (S V)_{j alpha} with V = U C (Eq. EQ-DM's
// weights), and, when vectors are kept, C and the row V_j = (row j of U) C in the same order:
// rho_ij = sum_alpha f_alpha V_i alpha V_j alpha = U_i . (C diag(f) V_j) and G_ij(z) likewise,
// so the kept pattern rows of U never need turning into rows of V.
//
// These solves are short chains of dependent FP64 operations (square roots, divisions,
// the QL recurrence), and the FP64 pipe of an SM issues one warp instruction every 16
// cycles. One lane per column makes every FP64 instruction serve 32 columns: the lane
// runs the textbook sequential algorithm on its own column, its matrices held in a
// lane-interleaved global buffer (element e of the lane's block at e * 32 + lane) so that
// the warp's accesses to the same element coalesce, its vectors in local memory.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mka_internal.h"

namespace mka {
namespace {

enum : int { RS_OK = 0, RS_NOT_SPD = MKA_ERR_NOT_SPD, RS_BREAKDOWN = MKA_ERR_BREAKDOWN };
constexpr int kSmallNu = 64;

struct RedArgs {
  double* blk;               // [groups][red_block_doubles(nu)][32], in place
  int64_t n_cols;
  int nu;
  int32_t* status;           // in: status after the basis; out: final status
  int32_t* nu_eff;           // in: basis size; out: subspace dimension used (0 on failure)
  double* eps;               // [n_cols][nu]
  double* w;                 // [n_cols][nu]
  double* cv;                // kept C and V_j (NULL: not kept), lane-interleaved by column col0 + col
  int64_t col0;
};

// Element (i, j) of the lane's matrices: H_r / Z / C at (i nu + j), S_r / L at nu^2 + (i nu + j).
struct Lane {
  double* b;
  int nu;
  __device__ double& H(int i, int j) const { return b[(size_t)(i * nu + j) * 32]; }
  __device__ double& S(int i, int j) const { return b[(size_t)(nu * nu + i * nu + j) * 32]; }
  __device__ double UJ(int n) const { return b[(size_t)(2 * nu * nu + n) * 32]; }
  __device__ double SUJ(int n) const { return b[(size_t)(2 * nu * nu + nu + n) * 32]; }
};

// S_r = L L^T in the lower triangle of S (right-looking); rdiag[k] = 1 / L_kk.
__device__ bool lane_cholesky(const Lane& M, int n, double* rdiag) {
  for (int k = 0; k < n; ++k) {
    const double akk = M.S(k, k);
    if (!(akk > 0.0)) return false;
    const double lkk = sqrt(akk);
    const double rd = 1.0 / lkk;
    rdiag[k] = rd;
    M.S(k, k) = lkk;
    for (int i = k + 1; i < n; ++i) M.S(i, k) *= rd;
    for (int i = k + 1; i < n; ++i) {
      const double lik = M.S(i, k);
      for (int j = k + 1; j <= i; ++j) M.S(i, j) -= lik * M.S(j, k);
    }
  }
  return true;
}

// H <- L^{-1} H L^{-T} (full storage), symmetrised. `row` (n doubles, lane-local) holds the
// row of L, then of A, that an inner loop reuses.
__device__ void lane_congruence(const Lane& M, int n, const double* rdiag, double* row) {
  for (int i = 0; i < n; ++i) {        // X = L^{-1} H, row i from rows 0..i-1
    for (int k = 0; k < i; ++k) row[k] = M.S(i, k);
    for (int j = 0; j < n; ++j) {
      double v = M.H(i, j);
      for (int k = 0; k < i; ++k) v -= row[k] * M.H(k, j);
      M.H(i, j) = v * rdiag[i];
    }
  }
  for (int i = 0; i < n; ++i)          // A = X L^{-T}, column j from columns 0..j-1
    for (int j = 0; j < n; ++j) {
      double v = M.H(i, j);
      for (int k = 0; k < j; ++k) v -= row[k] * M.S(j, k);
      v *= rdiag[j];
      row[j] = v;
      M.H(i, j) = v;
    }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) {
      const double v = 0.5 * (M.H(i, j) + M.H(j, i));
      M.H(i, j) = v;
      M.H(j, i) = v;
    }
}

// Householder reduction T = Q^T A Q: diagonal d, off-diagonal e (e[k] couples k, k+1;
// e[n-1] = 0); Q accumulated in place of A. v (n doubles, lane-local) holds the current
// Householder vector.
__device__ void lane_tridiag(const Lane& M, int n, double* d, double* e, double* p, double* tau, double* v) {
  for (int k = 0; k + 2 < n; ++k) {
    double s2 = 0.0;
    for (int i = k + 1; i < n; ++i) {
      v[i] = M.H(i, k);
      s2 += v[i] * v[i];
    }
    const double x0 = v[k + 1];
    const double nrm = sqrt(s2);
    const double alpha = x0 >= 0.0 ? -nrm : nrm;
    const double v0 = x0 - alpha;
    const double vtv = s2 - x0 * x0 + v0 * v0;
    const double tk = vtv > 0.0 ? 2.0 / vtv : 0.0;          // H_k = I - tk v v^T
    v[k + 1] = v0;
    M.H(k + 1, k) = v0;                                       // v = A[k+1.., k]
    d[k] = M.H(k, k);
    e[k] = alpha;
    tau[k] = tk;
    double pv = 0.0;
    for (int i = k + 1; i < n; ++i) {                         // p = tk B v
      double acc = 0.0;
      for (int j = k + 1; j < n; ++j) acc += M.H(i, j) * v[j];
      p[i] = tk * acc;
      pv += p[i] * v[i];
    }
    const double kc = 0.5 * tk * pv;
    for (int i = k + 1; i < n; ++i) p[i] -= kc * v[i];        // w = p - kc v
    for (int i = k + 1; i < n; ++i) {                         // B -= v w^T + w v^T
      const double vi = v[i], wi = p[i];
      for (int j = k + 1; j < n; ++j) M.H(i, j) -= vi * p[j] + wi * v[j];
    }
  }
  if (n >= 2) {
    d[n - 2] = M.H(n - 2, n - 2);
    e[n - 2] = M.H(n - 1, n - 2);
  }
  d[n - 1] = M.H(n - 1, n - 1);
  e[n - 1] = 0.0;
  // Q = H_0 H_1 ... H_{n-3}, accumulated backwards in place: before H_k is applied the
  // trailing block [k+1.., k+1..] holds H_{k+1} ... H_{n-3}; v_k sits in column k.
  const int k0 = n >= 2 ? n - 2 : 0;
  for (int i = k0; i < n; ++i)
    for (int j = k0; j < n; ++j) M.H(i, j) = (i == j) ? 1.0 : 0.0;
  for (int k = n - 3; k >= 0; --k) {
    const int b = k + 1;
    for (int j = b; j < n; ++j) {      // grow the block by row / column b, keeping v_k in column k
      M.H(b, j) = (j == b) ? 1.0 : 0.0;
      M.H(j, b) = (j == b) ? 1.0 : 0.0;
    }
    const double tk = tau[k];
    if (tk != 0.0) {
      for (int i = b; i < n; ++i) v[i] = M.H(i, k);
      for (int j = b; j < n; ++j) p[j] = 0.0;
      for (int i = b; i < n; ++i) {    // p_j = tk sum_i v_i Q_ij, row by row
        const double vi = v[i];
        for (int j = b; j < n; ++j) p[j] += vi * M.H(i, j);
      }
      for (int i = b; i < n; ++i) {
        const double vi = tk * v[i];
        for (int j = b; j < n; ++j) M.H(i, j) -= vi * p[j];
      }
    }
  }
  for (int j = 0; j < n; ++j) {        // row / column 0 of Q
    M.H(0, j) = (j == 0) ? 1.0 : 0.0;
    M.H(j, 0) = (j == 0) ? 1.0 : 0.0;
  }
}

// Eigenvalues of the tridiagonal (d, e) by the implicit-shift QL method (Bowdler, Martin,
// Reinsch & Wilkinson, Numer. Math. 11, 1968); each sweep's rotations, recorded in (rc, rs),
// are then applied to the columns of Z (carrying the updated column down the sweep).
// Rotation lengths from rsqrt(f^2 + g^2). False when an eigenvalue needs more than 60 sweeps.
__device__ bool lane_tql(const Lane& M, int n, double* d, double* e, double* rc, double* rs) {
  for (int l = 0; l < n; ++l) {
    for (int iter = 0;; ++iter) {
      int m = l;
      for (; m < n - 1; ++m) {
        const double dd = fabs(d[m]) + fabs(d[m + 1]);
        if (fabs(e[m]) <= 2.2204460492503131e-16 * dd) break;
      }
      if (m == l) break;
      if (iter == 60) return false;
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = sqrt(g * g + 1.0);
      g = d[m] - d[l] + e[l] / (g + (g >= 0.0 ? r : -r));
      double s = 1.0, c = 1.0, p = 0.0;
      bool early = false;
      int i = m - 1;
      for (; i >= l; --i) {
        const double f = s * e[i], b = c * e[i];
        const double t = f * f + g * g;
        if (t == 0.0) {
          e[i + 1] = 0.0;
          d[i + 1] -= p;
          e[m] = 0.0;
          early = true;
          break;
        }
        const double rinv = rsqrt(t);
        e[i + 1] = t * rinv;
        s = f * rinv;
        c = g * rinv;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * b;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - b;
        rc[i] = c;
        rs[i] = s;
      }
      if (!early) {
        d[l] -= p;
        e[l] = g;
        e[m] = 0.0;
      }
      const int i0 = early ? i + 1 : l;
      for (int k = 0; k < n; ++k) {
        double zi1 = M.H(k, m);
        for (int ii = m - 1; ii >= i0; --ii) {
          const double zi = M.H(k, ii);
          M.H(k, ii + 1) = rs[ii] * zi + rc[ii] * zi1;
          zi1 = rc[ii] * zi - rs[ii] * zi1;
        }
        M.H(k, i0) = zi1;
      }
    }
  }
  return true;
}

// NUCAP bounds nu: the lane's vectors live in local memory sized NUCAP, so subspaces up to 64 take
// the small instance and larger ones (up to MKA_MAX_NU) the large one.
template <int NUCAP>
__global__ void __launch_bounds__(128) reduced_kernel(const RedArgs A) {
  const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= A.n_cols) return;
  const int nu = A.nu;
  const Lane M{A.blk + (size_t)(col >> 5) * red_block_doubles(nu) * 32 + (col & 31), nu};
  double d[NUCAP], e[NUCAP], rdiag[NUCAP], p[NUCAP], tau[NUCAP], v[NUCAP];
  int rank[NUCAP];
  const int n = A.nu_eff[col];
  const int st_in = A.status[col];
  bool ok = st_in == RS_OK && n > 0 && n <= nu;
  if (ok) ok = lane_cholesky(M, n, rdiag);
  if (ok) {
    lane_congruence(M, n, rdiag, v);
    lane_tridiag(M, n, d, e, p, tau, v);
    ok = lane_tql(M, n, d, e, p, tau);   // p, tau reused as the rotation record
  }
  if (ok) {
    for (int a = 0; a < n; ++a) {      // C = L^{-T} Z, column a by back substitution (kept in v)
      for (int i = n - 1; i >= 0; --i) {
        double s = M.H(i, a);
        for (int k = i + 1; k < n; ++k) s -= M.S(k, i) * v[k];
        v[i] = s * rdiag[i];
      }
      for (int i = 0; i < n; ++i) M.H(i, a) = v[i];
    }
    for (int a = 0; a < n; ++a) {
      int r = 0;
      for (int k = 0; k < n; ++k) r += (d[k] < d[a]) || (d[k] == d[a] && k < a);
      rank[a] = r;
    }
  }
  int stc = st_in;
  if (stc == RS_OK && n < nu) stc = RS_BREAKDOWN;
  if (!ok && st_in == RS_OK) stc = RS_NOT_SPD;
  A.status[col] = stc;
  A.nu_eff[col] = ok ? n : 0;
  double* epsc = A.eps + col * nu;
  double* wc = A.w + col * nu;
  for (int a = 0; a < nu; ++a) {
    epsc[a] = 0.0;
    wc[a] = 0.0;
  }
  if (ok)
    for (int a = 0; a < n; ++a) {      // w_alpha = V_{j alpha} (S V)_{j alpha}
      double vj = 0.0, svj = 0.0;
      for (int k = 0; k < n; ++k) {
        const double ck = M.H(k, a);
        vj += M.UJ(k) * ck;
        svj += M.SUJ(k) * ck;
      }
      epsc[rank[a]] = d[a];
      wc[rank[a]] = vj * svj;
    }
  if (A.cv) {                           // C and V_j, columns ranked, zero beyond nu_eff
    const int64_t ca = A.col0 + col;
    double* out = A.cv + (size_t)(ca >> 5) * kept_block_doubles(nu) * 32 + (ca & 31);
    const int ne = ok ? n : 0;
    int* inv = reinterpret_cast<int*>(tau);   // tau is free after the solve: rank -> eigenvector
    for (int a = 0; a < ne; ++a) inv[rank[a]] = a;
    if (ok)
      for (int a = 0; a < ne; ++a) {      // V_j alpha = (row j of U) . c_alpha
        double v = 0.0;
        for (int k = 0; k < ne; ++k) v += M.UJ(k) * M.H(k, a);
        e[a] = v;
      }
    for (int r = 0; r < nu; ++r)
      for (int a = 0; a < nu; ++a)
        out[(size_t)(r * nu + a) * 32] = (r < ne && a < ne) ? M.H(r, inv[a]) : 0.0;
    for (int a = 0; a < nu; ++a) out[(size_t)(nu * nu + a) * 32] = a < ne ? e[inv[a]] : 0.0;
  }
}

}  // namespace

mka_status reduced_launch(double* blk, int64_t n_cols, int nu, int32_t* status, int32_t* nu_eff, double* eps,
                          double* w, double* cv, int64_t col0, cudaStream_t st) {
  if (n_cols <= 0) return MKA_OK;
  RedArgs A{};
  A.blk = blk;
  A.n_cols = n_cols;
  A.nu = nu;
  A.status = status;
  A.nu_eff = nu_eff;
  A.eps = eps;
  A.w = w;
  A.cv = cv;
  A.col0 = col0;
  const int threads = 128;
  const unsigned blocks = (unsigned)((n_cols + threads - 1) / threads);
  if (nu <= kSmallNu) reduced_kernel<kSmallNu><<<blocks, threads, 0, st>>>(A);
  else reduced_kernel<MKA_MAX_NU><<<blocks, threads, 0, st>>>(A);
  count_launches();
  MKA_CUDA_TRY(cudaGetLastError());
  return MKA_OK;
}

}  // namespace mka
