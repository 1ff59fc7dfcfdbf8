// Host side of the system build: periodic Slater-Koster sp H and S as 4x4-block CSR,
// storage rounding, device upload, and the cell list of the cluster extraction.
//
// The model (two-centre sp table, on-site diag(Es, Ep, Ep, Ep) for H and I for S,
// exp(-2 (d/d0 - 1)) scaling with a hard cutoff rc) is the tight-binding form the
// paper's method takes as input (Sec. 2: sparse symmetric H, sparse SPD S); the
// cell list serves the real-space projection of Sec. 3. Compiled without FMA
// contraction so that x86 and Arm hosts build bit-identical matrices.
#include <math.h>
#include <omp.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <numeric>
#include <vector>

#include "mka_internal.h"

namespace mka {

static thread_local std::string g_err;
std::atomic<int64_t> g_kernel_launches{0};

void set_error(const std::string& msg) { g_err = msg; }

mka_status fail(mka_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

mka_status cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? MKA_ERR_OOM : MKA_ERR_CUDA;
}

size_t storage_bytes(int storage) { return storage == MKA_FP64 ? 8 : storage == MKA_MIXED_FP32 ? 4 : 2; }

namespace {

inline double min_image(double d, double L) { return d - L * nearbyint(d / L); }

// Round to nearest even FP64 -> FP32 -> BF16 (upper 16 bits of the FP32 pattern).
inline uint16_t to_bf16(double x) {
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

inline double from_bf16(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return (double)f;
}

// 4x4 two-centre block <mu_a|nu_b> for displacement d = r_b - r_a.
void sk_block(const double d[3], double r2, const double V[4], double d0, double out[16]) {
  double dist = sqrt(r2);
  double c[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
  double scale = exp(-2.0 * (dist / d0 - 1.0));
  double ss = V[0] * scale, sp = V[1] * scale, pps = V[2] * scale, ppp = V[3] * scale;
  out[0] = ss;
  for (int k = 0; k < 3; ++k) {
    out[1 + k] = c[k] * sp;
    out[4 * (1 + k)] = -c[k] * sp;
    for (int m = 0; m < 3; ++m) out[4 * (1 + k) + 1 + m] = c[k] * c[m] * (pps - ppp) + (k == m ? ppp : 0.0);
  }
}

struct HostCells {
  int n[3];
  double len[3];
  std::vector<int32_t> start, atoms;
  int cell_of(const double* p) const {
    int c[3];
    for (int d = 0; d < 3; ++d) {
      int v = (int)floor(p[d] / len[d]);
      c[d] = v < 0 ? 0 : (v >= n[d] ? n[d] - 1 : v);
    }
    return (c[0] * n[1] + c[1]) * n[2] + c[2];
  }
};

// Cells of edge >= r (a small margin keeps roundoff at cell faces harmless).
HostCells make_cells(const std::vector<double>& pos, int64_t N, const double box[3], double r) {
  HostCells hc;
  for (int d = 0; d < 3; ++d) {
    int n = (int)floor(box[d] / (r * (1.0 + 1e-9) + 1e-9));
    hc.n[d] = n < 1 ? 1 : n;
    hc.len[d] = box[d] / hc.n[d];
  }
  int64_t nc = (int64_t)hc.n[0] * hc.n[1] * hc.n[2];
  hc.start.assign(nc + 1, 0);
  std::vector<int32_t> cell(N);
  for (int64_t a = 0; a < N; ++a) {
    cell[a] = hc.cell_of(&pos[3 * a]);
    hc.start[cell[a] + 1]++;
  }
  for (int64_t c = 0; c < nc; ++c) hc.start[c + 1] += hc.start[c];
  hc.atoms.resize(N);
  std::vector<int32_t> fill(hc.start.begin(), hc.start.end() - 1);
  for (int64_t a = 0; a < N; ++a) hc.atoms[fill[cell[a]]++] = (int32_t)a;  // ascending within a cell
  return hc;
}

// Neighbour cell coordinates of c along one dimension (all cells when n < 3).
int cell_range(int c, int n, int out[3]) {
  if (n < 3) {
    for (int i = 0; i < n; ++i) out[i] = i;
    return n;
  }
  out[0] = (c + n - 1) % n;
  out[1] = c;
  out[2] = (c + 1) % n;
  return 3;
}

// Sorted neighbours (distance <= rc, minimum image, the atom itself included) of atom a.
void neighbours(const HostCells& hc, const std::vector<double>& pos, const double box[3], double rc2, int64_t a,
                std::vector<std::pair<int32_t, double>>& out) {
  out.clear();
  const double* pa = &pos[3 * a];
  int cc[3];
  for (int d = 0; d < 3; ++d) {
    int v = (int)floor(pa[d] / hc.len[d]);
    cc[d] = v < 0 ? 0 : (v >= hc.n[d] ? hc.n[d] - 1 : v);
  }
  int rx[3], ry[3], rz[3];
  int nx = cell_range(cc[0], hc.n[0], rx), ny = cell_range(cc[1], hc.n[1], ry), nz = cell_range(cc[2], hc.n[2], rz);
  for (int ix = 0; ix < nx; ++ix)
    for (int iy = 0; iy < ny; ++iy)
      for (int iz = 0; iz < nz; ++iz) {
        int c = (rx[ix] * hc.n[1] + ry[iy]) * hc.n[2] + rz[iz];
        for (int32_t k = hc.start[c]; k < hc.start[c + 1]; ++k) {
          int32_t b = hc.atoms[k];
          double dx = min_image(pos[3 * b] - pa[0], box[0]);
          double dy = min_image(pos[3 * b + 1] - pa[1], box[1]);
          double dz = min_image(pos[3 * b + 2] - pa[2], box[2]);
          double r2 = dx * dx + dy * dy + dz * dz;
          if (r2 <= rc2) out.push_back({b, r2});
        }
      }
  std::sort(out.begin(), out.end(), [](const std::pair<int32_t, double>& x, const std::pair<int32_t, double>& y) {
    return x.first < y.first;
  });
}

void convert_store(const double* src, size_t n, int storage, void* dst_host) {
  if (storage == MKA_FP64) {
    memcpy(dst_host, src, n * 8);
  } else if (storage == MKA_MIXED_FP32) {
    float* d = (float*)dst_host;
    for (size_t i = 0; i < n; ++i) d[i] = (float)src[i];
  } else {
    uint16_t* d = (uint16_t*)dst_host;
    for (size_t i = 0; i < n; ++i) d[i] = to_bf16(src[i]);
  }
}

mka_status check_common(const double* pos, int64_t n_atoms, const double box[3], int storage, double R) {
  if (!pos || !box || n_atoms < 1) return fail(MKA_ERR_INVALID_ARG, "positions, box and n_atoms >= 1 are required");
  if (n_atoms > (int64_t)INT32_MAX / 4) return fail(MKA_ERR_INVALID_ARG, "too many atoms for 32-bit indices");
  if (storage < MKA_FP64 || storage > MKA_MIXED_BF16) return fail(MKA_ERR_INVALID_ARG, "unknown storage format");
  for (int d = 0; d < 3; ++d) {
    if (!(box[d] > 0)) return fail(MKA_ERR_INVALID_ARG, "box lengths must be positive");
    if (!(R > 0) || !(2.0 * R < box[d])) return fail(MKA_ERR_INVALID_ARG, "cluster radius must be in (0, box/2)");
  }
  return MKA_OK;
}

std::vector<double> wrap_positions(const double* pos, int64_t N, const double box[3]) {
  std::vector<double> w(3 * N);
  for (int64_t a = 0; a < N; ++a)
    for (int d = 0; d < 3; ++d) {
      double x = fmod(pos[3 * a + d], box[d]);
      if (x < 0) x += box[d];
      if (x >= box[d]) x -= box[d];
      w[3 * a + d] = x;
    }
  return w;
}

// Upload positions, pattern, and the cell list of radius R; allocate value arrays.
mka_status upload_common(mka_system* s, const std::vector<double>& wpos, bool copy_col) {
  int64_t N = s->n_atoms;
  MKA_CUDA_TRY(cudaMalloc(&s->d_pos, sizeof(double) * 3 * N));
  MKA_CUDA_TRY(cudaMemcpy(s->d_pos, wpos.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice));
  {
    std::vector<float> pf(wpos.begin(), wpos.end());
    MKA_CUDA_TRY(cudaMalloc(&s->d_posf, sizeof(float) * 3 * N));
    MKA_CUDA_TRY(cudaMemcpy(s->d_posf, pf.data(), sizeof(float) * 3 * N, cudaMemcpyHostToDevice));
  }
  MKA_CUDA_TRY(cudaMalloc(&s->d_row_ptr, sizeof(int32_t) * (N + 1)));
  MKA_CUDA_TRY(cudaMemcpy(s->d_row_ptr, s->h_row_ptr.data(), sizeof(int32_t) * (N + 1), cudaMemcpyHostToDevice));
  MKA_CUDA_TRY(cudaMalloc(&s->d_col, sizeof(int32_t) * std::max<int64_t>(s->nnzb, 1)));
  if (copy_col)
    MKA_CUDA_TRY(cudaMemcpy(s->d_col, s->h_col.data(), sizeof(int32_t) * s->nnzb, cudaMemcpyHostToDevice));
  size_t vb = storage_bytes(s->storage) * 16 * (size_t)std::max<int64_t>(s->nnzb, 1);
  MKA_CUDA_TRY(cudaMalloc(&s->d_valH, vb));
  MKA_CUDA_TRY(cudaMalloc(&s->d_valS, vb));
  HostCells hc = make_cells(wpos, N, s->box, s->R);
  for (int d = 0; d < 3; ++d) {
    s->cells.n[d] = hc.n[d];
    s->cells.len[d] = hc.len[d];
  }
  MKA_CUDA_TRY(cudaMalloc(&s->cells.start, sizeof(int32_t) * hc.start.size()));
  MKA_CUDA_TRY(cudaMemcpy(s->cells.start, hc.start.data(), sizeof(int32_t) * hc.start.size(), cudaMemcpyHostToDevice));
  MKA_CUDA_TRY(cudaMalloc(&s->cells.atoms, sizeof(int32_t) * N));
  MKA_CUDA_TRY(cudaMemcpy(s->cells.atoms, hc.atoms.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice));
  int mrb = 0;
  for (int64_t a = 0; a < N; ++a) mrb = std::max(mrb, s->h_row_ptr[a + 1] - s->h_row_ptr[a]);
  s->max_row_blocks = mrb;
  return MKA_OK;
}

}  // namespace
}  // namespace mka

using namespace mka;

extern "C" {

const char* mka_last_error(void) { return g_err.c_str(); }

int64_t mka_kernel_launches(void) { return g_kernel_launches.load(); }

const char* mka_status_string(mka_status s) {
  switch (s) {
    case MKA_OK: return "ok";
    case MKA_ERR_INVALID_ARG: return "invalid argument";
    case MKA_ERR_NOT_SPD: return "matrix not positive definite";
    case MKA_ERR_NO_CONVERGENCE: return "inner CG did not converge";
    case MKA_ERR_BREAKDOWN: return "Krylov basis ended early (nu_eff < nu)";
    case MKA_ERR_OOM: return "out of memory";
    case MKA_ERR_CUDA: return "CUDA error";
    case MKA_ERR_TIMEOUT: return "device wait timed out";
    case MKA_ERR_CLUSTER_TOO_LARGE: return "cluster larger than MKA_MAX_CLUSTER_ATOMS";
  }
  return "unknown status";
}

void mka_system_destroy(mka_system* s) {
  if (!s) return;
  cudaFree(s->d_row_ptr);
  cudaFree(s->d_col);
  cudaFree(s->d_valH);
  cudaFree(s->d_valS);
  cudaFree(s->d_pos);
  cudaFree(s->d_posf);
  cudaFree(s->cells.start);
  cudaFree(s->cells.atoms);
  delete s;
}

mka_status mka_build_system(const double* pos, int64_t n_atoms, const double box[3], const mka_sk_params* sk,
                            int storage, double cluster_radius, void* stream, mka_system** out) {
  if (!out) return fail(MKA_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  mka_status st = check_common(pos, n_atoms, box, storage, cluster_radius);
  if (st) return st;
  if (!sk || !(sk->rc > 0) || !(sk->d0 > 0)) return fail(MKA_ERR_INVALID_ARG, "SK parameters need rc > 0, d0 > 0");
  for (int d = 0; d < 3; ++d)
    if (!(2.0 * sk->rc < box[d])) return fail(MKA_ERR_INVALID_ARG, "cutoff rc must be < box/2");
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1)
    return fail(MKA_ERR_CUDA, "no CUDA device available");

  mka_system* s = new mka_system();
  s->n_atoms = n_atoms;
  s->storage = storage;
  s->R = cluster_radius;
  s->stream = (cudaStream_t)stream;
  s->sk = *sk;
  s->have_sk = true;
  for (int d = 0; d < 3; ++d) s->box[d] = box[d];
  std::vector<double> wpos = wrap_positions(pos, n_atoms, box);
  HostCells hc = make_cells(wpos, n_atoms, box, sk->rc);
  const double rc2 = sk->rc * sk->rc;

  // Pass 1: row lengths.
  std::vector<int32_t> cnt(n_atoms);
#pragma omp parallel
  {
    std::vector<std::pair<int32_t, double>> nb;
#pragma omp for schedule(static)
    for (int64_t a = 0; a < n_atoms; ++a) {
      neighbours(hc, wpos, box, rc2, a, nb);
      cnt[a] = (int32_t)nb.size();
    }
  }
  s->h_row_ptr.assign(n_atoms + 1, 0);
  for (int64_t a = 0; a < n_atoms; ++a) {
    if ((int64_t)s->h_row_ptr[a] + cnt[a] > INT32_MAX) {
      delete s;
      return fail(MKA_ERR_INVALID_ARG, "too many blocks for 32-bit offsets");
    }
    s->h_row_ptr[a + 1] = s->h_row_ptr[a] + cnt[a];
  }
  s->nnzb = s->h_row_ptr[n_atoms];
  s->h_col.resize(s->nnzb);
  st = upload_common(s, wpos, false);
  if (st) {
    mka_system_destroy(s);
    return st;
  }

  // Pass 2: columns and values, a chunk of rows at a time (bounded host memory).
  const size_t eb = storage_bytes(storage);
  const int64_t chunk = 1 << 18;
  std::vector<double> h64, s64;
  std::vector<unsigned char> hst, sst;
  for (int64_t a0 = 0; a0 < n_atoms; a0 += chunk) {
    int64_t a1 = std::min(n_atoms, a0 + chunk);
    int64_t k0 = s->h_row_ptr[a0], k1 = s->h_row_ptr[a1];
    h64.assign((k1 - k0) * 16, 0.0);
    s64.assign((k1 - k0) * 16, 0.0);
#pragma omp parallel
    {
      std::vector<std::pair<int32_t, double>> nb;
#pragma omp for schedule(static)
      for (int64_t a = a0; a < a1; ++a) {
        neighbours(hc, wpos, box, rc2, a, nb);
        int64_t k = s->h_row_ptr[a];
        for (auto& e : nb) {
          int32_t b = e.first;
          s->h_col[k] = b;
          double* Hb = &h64[(k - k0) * 16];
          double* Sb = &s64[(k - k0) * 16];
          if (b == a) {
            for (int i = 0; i < 16; ++i) Hb[i] = Sb[i] = 0.0;
            Hb[0] = sk->Es;
            Hb[5] = Hb[10] = Hb[15] = sk->Ep;
            Sb[0] = Sb[5] = Sb[10] = Sb[15] = 1.0;
          } else {
            double d[3];
            for (int x = 0; x < 3; ++x) d[x] = min_image(wpos[3 * b + x] - wpos[3 * a + x], box[x]);
            sk_block(d, e.second, sk->V, sk->d0, Hb);
            sk_block(d, e.second, sk->Sv, sk->d0, Sb);
          }
          ++k;
        }
      }
    }
    hst.resize(h64.size() * eb);
    sst.resize(s64.size() * eb);
    convert_store(h64.data(), h64.size(), storage, hst.data());
    convert_store(s64.data(), s64.size(), storage, sst.data());
    cudaError_t e1 = cudaMemcpy((char*)s->d_valH + k0 * 16 * eb, hst.data(), hst.size(), cudaMemcpyHostToDevice);
    cudaError_t e2 = cudaMemcpy((char*)s->d_valS + k0 * 16 * eb, sst.data(), sst.size(), cudaMemcpyHostToDevice);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      mka_system_destroy(s);
      return cuda_fail(e1 != cudaSuccess ? e1 : e2, "cudaMemcpy(values)");
    }
  }
  cudaError_t e = cudaMemcpy(s->d_col, s->h_col.data(), sizeof(int32_t) * s->nnzb, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    mka_system_destroy(s);
    return cuda_fail(e, "cudaMemcpy(col)");
  }
  *out = s;
  return MKA_OK;
}

mka_status mka_build_system_bsr(const double* pos, int64_t n_atoms, const double box[3], const int32_t* row_ptr,
                                const int32_t* col, int64_t nnzb, const double* valH, const double* valS,
                                int storage, double cluster_radius, void* stream, mka_system** out) {
  if (!out) return fail(MKA_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  mka_status st = check_common(pos, n_atoms, box, storage, cluster_radius);
  if (st) return st;
  if (!row_ptr || !col || !valH || !valS || nnzb < n_atoms || row_ptr[0] != 0 || row_ptr[n_atoms] != nnzb)
    return fail(MKA_ERR_INVALID_ARG, "inconsistent BSR arrays");
  for (int64_t a = 0; a < n_atoms; ++a) {
    if (row_ptr[a + 1] < row_ptr[a]) return fail(MKA_ERR_INVALID_ARG, "row_ptr must be non-decreasing");
    bool diag = false;
    for (int32_t k = row_ptr[a]; k < row_ptr[a + 1]; ++k) {
      if (col[k] < 0 || col[k] >= n_atoms) return fail(MKA_ERR_INVALID_ARG, "column index out of range");
      if (k > row_ptr[a] && col[k] <= col[k - 1]) return fail(MKA_ERR_INVALID_ARG, "columns must ascend in a row");
      diag |= col[k] == a;
    }
    if (!diag) return fail(MKA_ERR_INVALID_ARG, "every row needs its diagonal block");
  }
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1)
    return fail(MKA_ERR_CUDA, "no CUDA device available");
  mka_system* s = new mka_system();
  s->n_atoms = n_atoms;
  s->nnzb = nnzb;
  s->storage = storage;
  s->R = cluster_radius;
  s->stream = (cudaStream_t)stream;
  for (int d = 0; d < 3; ++d) s->box[d] = box[d];
  s->h_row_ptr.assign(row_ptr, row_ptr + n_atoms + 1);
  s->h_col.assign(col, col + nnzb);
  std::vector<double> wpos = wrap_positions(pos, n_atoms, box);
  st = upload_common(s, wpos, true);
  if (st) {
    mka_system_destroy(s);
    return st;
  }
  const size_t eb = storage_bytes(storage);
  std::vector<unsigned char> buf(nnzb * 16 * eb);
  convert_store(valH, nnzb * 16, storage, buf.data());
  cudaError_t e = cudaMemcpy(s->d_valH, buf.data(), buf.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    convert_store(valS, nnzb * 16, storage, buf.data());
    e = cudaMemcpy(s->d_valS, buf.data(), buf.size(), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    mka_system_destroy(s);
    return cuda_fail(e, "cudaMemcpy(values)");
  }
  *out = s;
  return MKA_OK;
}

mka_status mka_system_info(const mka_system* s, int64_t* n_atoms, int64_t* nnzb, int* storage, int* max_row_blocks) {
  if (!s) return fail(MKA_ERR_INVALID_ARG, "system is NULL");
  if (n_atoms) *n_atoms = s->n_atoms;
  if (nnzb) *nnzb = s->nnzb;
  if (storage) *storage = s->storage;
  if (max_row_blocks) *max_row_blocks = s->max_row_blocks;
  return MKA_OK;
}

mka_status mka_system_copy_bsr(const mka_system* s, int32_t* row_ptr, int32_t* col, double* valH, double* valS) {
  if (!s) return fail(MKA_ERR_INVALID_ARG, "system is NULL");
  if (row_ptr) memcpy(row_ptr, s->h_row_ptr.data(), sizeof(int32_t) * (s->n_atoms + 1));
  if (col) memcpy(col, s->h_col.data(), sizeof(int32_t) * s->nnzb);
  const size_t eb = storage_bytes(s->storage);
  std::vector<unsigned char> buf(s->nnzb * 16 * eb);
  double* outs[2] = {valH, valS};
  void* srcs[2] = {s->d_valH, s->d_valS};
  for (int m = 0; m < 2; ++m) {
    if (!outs[m]) continue;
    MKA_CUDA_TRY(cudaMemcpy(buf.data(), srcs[m], buf.size(), cudaMemcpyDeviceToHost));
    size_t n = s->nnzb * 16;
    if (s->storage == MKA_FP64) {
      memcpy(outs[m], buf.data(), n * 8);
    } else if (s->storage == MKA_MIXED_FP32) {
      const float* f = (const float*)buf.data();
      for (size_t i = 0; i < n; ++i) outs[m][i] = f[i];
    } else {
      const uint16_t* h = (const uint16_t*)buf.data();
      for (size_t i = 0; i < n; ++i) outs[m][i] = from_bf16(h[i]);
    }
  }
  return MKA_OK;
}

}  // extern "C"
