// Batched reduced problems of the multiple Arnoldi method on sm_103a.
//
// Every column j ends its basis with the nu x nu projected matrices H_r = U^T H U and
// S_r = U^T S U (formed explicitly, so that a basis that is only nearly S-orthonormal
// still gives the Galerkin pencil of its span) and solves the generalized eigenproblem
// H_r c = eps S_r c (Eq. EQ-SUB-EIG-VEC): Cholesky S_r = L L^T, A = L^{-1} H_r L^{-T} (lower
// triangle), Householder tridiagonalisation A = Q T Q^T, the eigenvalues of T by the
// implicit-shift QL method, the eigenvectors Z of T by inverse iteration (re-orthogonalised
// within clusters of close eigenvalues), C = L^{-T} Q Z with Q applied as its reflectors. The
// outputs of a column are its levels eps_alpha in ascending order, w_alpha = V_{j alpha} (S V)_{j alpha} with V = U C (Eq. EQ-DM's
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
constexpr int kTinyNu = 32, kSmallNu = 64;

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

// Element (i, j) of the lane's matrices: H_r, then X = L^{-1} H_r (upper triangle) and A (lower
// triangle), then Q's reflectors (below the diagonal) at (i nu + j); S_r / L at nu^2 + (i nu + j);
// row j of U and of S U; the eigenvectors Z of T, then C, at 2 nu^2 + 2 nu + (i nu + j).
struct Lane {
  double* b;
  int nu;
  __device__ double& H(int i, int j) const { return b[(size_t)(i * nu + j) * 32]; }
  __device__ double& S(int i, int j) const { return b[(size_t)(nu * nu + i * nu + j) * 32]; }
  __device__ double UJ(int n) const { return b[(size_t)(2 * nu * nu + n) * 32]; }
  __device__ double SUJ(int n) const { return b[(size_t)(2 * nu * nu + nu + n) * 32]; }
  __device__ double& Z(int i, int j) const { return b[(size_t)(2 * nu * nu + 2 * nu + i * nu + j) * 32]; }
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

// The lower triangle of A = L^{-1} H L^{-T} in place of H's, using the symmetry of H and A (n^3 / 2
// FMAs): first the upper triangle of X = L^{-1} H over H's (row j from the rows above it), then A =
// L^{-1} X^T column by column, the entries of column j above the diagonal taken from row j of A. `row`
// and `col` (n doubles each, lane-local) hold the row of L and the column of A an inner loop reuses.
__device__ void lane_congruence(const Lane& M, int n, const double* rdiag, double* row, double* col) {
  for (int j = 0; j < n; ++j) {        // X(j, i), i >= j
    for (int k = 0; k < j; ++k) row[k] = M.S(j, k);
    for (int i = j; i < n; ++i) {
      double v = M.H(j, i);
      for (int k = 0; k < j; ++k) v -= row[k] * M.H(k, i);
      M.H(j, i) = v * rdiag[j];
    }
  }
  for (int j = 0; j < n; ++j) {        // A(i, j), i >= j
    for (int k = 0; k < j; ++k) col[k] = M.H(j, k);
    for (int i = j; i < n; ++i) {
      double v = M.H(j, i);
      for (int k = 0; k < i; ++k) v -= M.S(i, k) * col[k];
      col[i] = v * rdiag[i];
    }
    for (int i = j; i < n; ++i) M.H(i, j) = col[i];
  }
}

// Householder reduction T = Q^T A Q of A given by its lower triangle: diagonal d, off-diagonal e
// (e[k] couples k, k+1; e[n-1] = 0). Q = H_0 H_1 ... H_{n-3} is kept as its reflectors
// H_k = I - tau[k] v_k v_k^T, v_k in column k below the diagonal (rows k+1..n-1). v (n doubles,
// lane-local) holds the current Householder vector.
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
    for (int i = k + 1; i < n; ++i) {                         // p = tk B v, B from its lower triangle
      double acc = 0.0;
      for (int j = k + 1; j <= i; ++j) acc += M.H(i, j) * v[j];
      for (int j = i + 1; j < n; ++j) acc += M.H(j, i) * v[j];
      p[i] = tk * acc;
      pv += p[i] * v[i];
    }
    const double kc = 0.5 * tk * pv;
    for (int i = k + 1; i < n; ++i) p[i] -= kc * v[i];        // w = p - kc v
    for (int i = k + 1; i < n; ++i) {                         // B -= v w^T + w v^T, lower triangle
      const double vi = v[i], wi = p[i];
      for (int j = k + 1; j <= i; ++j) M.H(i, j) -= vi * p[j] + wi * v[j];
    }
  }
  if (n >= 2) {
    d[n - 2] = M.H(n - 2, n - 2);
    e[n - 2] = M.H(n - 1, n - 2);
  }
  d[n - 1] = M.H(n - 1, n - 1);
  e[n - 1] = 0.0;
}

// Eigenvalues of the tridiagonal (d, e) by the implicit-shift QL method (Bowdler, Martin,
// Reinsch & Wilkinson, Numer. Math. 11, 1968), in place on d (e is destroyed); rotation
// lengths from rsqrt(f^2 + g^2). False when an eigenvalue needs more than 60 sweeps.
__device__ bool lane_tql_values(int n, double* d, double* e) {
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
      for (int i = m - 1; i >= l; --i) {
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
      }
      if (!early) {
        d[l] -= p;
        e[l] = g;
        e[m] = 0.0;
      }
    }
  }
  return true;
}

// Gaussian elimination with partial pivoting of the tridiagonal T - lam I (d, e): the multipliers and
// row interchanges in (mlt, swp), U as reciprocal pivots r0 and the two superdiagonals (u1, u2); a
// pivot that vanishes is replaced by `tiny`. One division per row.
__device__ void lane_tri_factor(int n, const double* d, const double* e, double lam, double tiny, double* r0,
                                double* u1, double* u2, double* mlt, int* swp) {
  double a = d[0] - lam, bb = n > 1 ? e[0] : 0.0;   // the working row: a at column k, bb at k + 1
  for (int k = 0; k + 1 < n; ++k) {
    const double sub = e[k], dn = d[k + 1] - lam, sp = k + 2 < n ? e[k + 1] : 0.0;
    if (fabs(a) >= fabs(sub)) {
      const double ra = 1.0 / (a != 0.0 ? a : tiny);
      mlt[k] = sub * ra;
      swp[k] = 0;
      r0[k] = ra;
      u1[k] = bb;
      u2[k] = 0.0;
      a = dn - mlt[k] * bb;
      bb = sp;
    } else {                               // row k + 1 becomes the pivot row
      const double rs = 1.0 / sub;
      mlt[k] = a * rs;
      swp[k] = 1;
      r0[k] = rs;
      u1[k] = dn;
      u2[k] = sp;
      a = bb - mlt[k] * dn;
      bb = -mlt[k] * sp;
    }
  }
  r0[n - 1] = 1.0 / (a != 0.0 ? a : tiny);
}

// x <- (T - lam I)^{-1} x from the factors of lane_tri_factor: the row operations, then back substitution.
__device__ void lane_tri_apply(int n, const double* r0, const double* u1, const double* u2, const double* mlt,
                               const int* swp, double* x) {
  for (int k = 0; k + 1 < n; ++k) {
    if (swp[k]) {
      const double xk = x[k];
      x[k] = x[k + 1];
      x[k + 1] = xk - mlt[k] * x[k + 1];
    } else {
      x[k + 1] -= mlt[k] * x[k];
    }
  }
  x[n - 1] *= r0[n - 1];
  if (n >= 2) x[n - 2] = (x[n - 2] - u1[n - 2] * x[n - 1]) * r0[n - 2];
  for (int k = n - 3; k >= 0; --k) x[k] = (x[k] - u1[k] * x[k + 1] - u2[k] * x[k + 2]) * r0[k];
}

// The eigenvectors of the tridiagonal (d, e) for its eigenvalues lam[0..n) (ascending) by inverse
// iteration (Wilkinson; the scheme of LAPACK's dstein): from a fixed quasi-random start, two solves
// of (T - lam_a I) x = x with one factorisation, each followed by modified Gram-Schmidt against the vectors of the same
// cluster already found (eigenvalues closer than 1e-3 ||T||_1 to their neighbour) and
// normalisation; stored as the columns of Z.
__device__ void lane_tri_vectors(const Lane& M, int n, const double* d, const double* e, const double* lam,
                                 double* x, double* r0, double* u1, double* u2, double* mlt, int* swp) {
  double tn = 0.0;
  for (int k = 0; k < n; ++k)
    tn = fmax(tn, fabs(d[k]) + (k + 1 < n ? fabs(e[k]) : 0.0) + (k > 0 ? fabs(e[k - 1]) : 0.0));
  const double ortol = 1e-3 * tn, tiny = 2.2204460492503131e-16 * (tn > 0.0 ? tn : 1.0);
  int cs = 0;
  for (int a = 0; a < n; ++a) {
    if (a == 0 || lam[a] - lam[a - 1] > ortol) cs = a;
    for (int i = 0; i < n; ++i) {        // start: an additive-recurrence (golden ratio) sequence in [0.5, 1.5)
      const double t = 0.7548776662466927 * (i + 1) + 0.5698402909980532 * (a + 1);
      x[i] = 0.5 + (t - floor(t));
    }
    lane_tri_factor(n, d, e, lam[a], tiny, r0, u1, u2, mlt, swp);
    for (int it = 0; it < 2; ++it) {
      lane_tri_apply(n, r0, u1, u2, mlt, swp, x);
      for (int b = cs; b < a; ++b) {
        double dot = 0.0;
        for (int i = 0; i < n; ++i) dot += M.Z(i, b) * x[i];
        for (int i = 0; i < n; ++i) x[i] -= dot * M.Z(i, b);
      }
      double s2 = 0.0;
      for (int i = 0; i < n; ++i) s2 += x[i] * x[i];
      const double sc = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
      for (int i = 0; i < n; ++i) x[i] *= sc;
    }
    for (int i = 0; i < n; ++i) M.Z(i, a) = x[i];
  }
}

// C = L^{-T} Q Z in place of Z, four columns at a time: the reflectors of Q applied to the block
// (H_{n-3} first), then the back substitution with L^T.
template <int NUCAP>
__device__ void lane_back_transform(const Lane& M, int n, const double* rdiag, const double* tau,
                                    double (*x4)[NUCAP]) {
  for (int a0 = 0; a0 < n; a0 += 4) {
    const int na = min(4, n - a0);
    for (int r = 0; r < 4; ++r)
      for (int k = 0; k < n; ++k) x4[r][k] = r < na ? M.Z(k, a0 + r) : 0.0;
    for (int k = n - 3; k >= 0; --k) {   // x <- (I - tau_k v_k v_k^T) x
      const double tk = tau[k];
      if (tk == 0.0) continue;
      double dot[4] = {0.0, 0.0, 0.0, 0.0};
      for (int i = k + 1; i < n; ++i) {
        const double vi = M.H(i, k);
#pragma unroll
        for (int r = 0; r < 4; ++r) dot[r] += vi * x4[r][i];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) dot[r] *= tk;
      for (int i = k + 1; i < n; ++i) {
        const double vi = M.H(i, k);
#pragma unroll
        for (int r = 0; r < 4; ++r) x4[r][i] -= dot[r] * vi;
      }
    }
    for (int i = n - 1; i >= 0; --i) {   // C = L^{-T} (Q Z)
      double s[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) s[r] = x4[r][i];
      for (int k = i + 1; k < n; ++k) {
        const double l = M.S(k, i);
#pragma unroll
        for (int r = 0; r < 4; ++r) s[r] -= l * x4[r][k];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) x4[r][i] = s[r] * rdiag[i];
    }
    for (int r = 0; r < na; ++r)
      for (int i = 0; i < n; ++i) M.Z(i, a0 + r) = x4[r][i];
  }
}

// NUCAP bounds nu: the lane's vectors live in local memory sized NUCAP, so subspaces up to 32 and 64
// take the small instances and larger ones (up to MKA_MAX_NU) the large one.
template <int NUCAP>
__global__ void __launch_bounds__(128) reduced_kernel(const RedArgs A) {
  const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= A.n_cols) return;
  const int nu = A.nu;
  const Lane M{A.blk + (size_t)(col >> 5) * red_block_doubles(nu) * 32 + (col & 31), nu};
  double d[NUCAP], e[NUCAP], rdiag[NUCAP], p[NUCAP], tau[NUCAP], v[NUCAP];
  double x4[4][NUCAP];
  int rank[NUCAP];
  const int n = A.nu_eff[col];
  const int st_in = A.status[col];
  bool ok = st_in == RS_OK && n > 0 && n <= nu;
  if (ok) ok = lane_cholesky(M, n, rdiag);
  if (ok) {
    lane_congruence(M, n, rdiag, v, p);
    lane_tridiag(M, n, d, e, p, tau, v);
    for (int k = 0; k < n; ++k) {      // the eigenvalues from copies: T stays for the eigenvectors,
      p[k] = d[k];                     // tau for the back-transform
      v[k] = e[k];
    }
    ok = lane_tql_values(n, p, v);
  }
  if (ok) {
    for (int a = 1; a < n; ++a) {      // ascending
      const double t = p[a];
      int b = a - 1;
      for (; b >= 0 && p[b] > t; --b) p[b + 1] = p[b];
      p[b + 1] = t;
    }
    lane_tri_vectors(M, n, d, e, p, v, x4[0], x4[1], x4[2], x4[3], rank);
    lane_back_transform<NUCAP>(M, n, rdiag, tau, x4);
    for (int a = 0; a < n; ++a) {
      d[a] = p[a];
      rank[a] = a;
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
        const double ck = M.Z(k, a);
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
        for (int k = 0; k < ne; ++k) v += M.UJ(k) * M.Z(k, a);
        e[a] = v;
      }
    for (int r = 0; r < nu; ++r)
      for (int a = 0; a < nu; ++a)
        out[(size_t)(r * nu + a) * 32] = (r < ne && a < ne) ? M.Z(r, inv[a]) : 0.0;
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
  if (nu <= kTinyNu) reduced_kernel<kTinyNu><<<blocks, threads, 0, st>>>(A);
  else if (nu <= kSmallNu) reduced_kernel<kSmallNu><<<blocks, threads, 0, st>>>(A);
  else reduced_kernel<MKA_MAX_NU><<<blocks, threads, 0, st>>>(A);
  count_launches();
  MKA_CUDA_TRY(cudaGetLastError());
  return MKA_OK;
}

}  // namespace mka
