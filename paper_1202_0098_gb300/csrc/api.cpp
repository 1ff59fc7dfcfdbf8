// C entry points of the column work flow (Eq. EQ-WORK-FLOW): solve, results, mu,
// density and energy, Green's function, global SpMV, cluster sizes.
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mka_internal.h"

using namespace mka;

namespace {

mka_status copy_selection(const mka_system* sys, const int64_t* atoms, int64_t n_sel, std::vector<int64_t>& sel) {
  if (atoms) {
    if (n_sel < 1) return fail(MKA_ERR_INVALID_ARG, "n_sel must be >= 1");
    sel.assign(atoms, atoms + n_sel);
    for (int64_t a : sel)
      if (a < 0 || a >= sys->n_atoms) return fail(MKA_ERR_INVALID_ARG, "atom index out of range");
  } else {
    sel.resize(sys->n_atoms);
    for (int64_t a = 0; a < sys->n_atoms; ++a) sel[a] = a;
  }
  return MKA_OK;
}

}  // namespace

extern "C" {

mka_status mka_cluster_sizes(const mka_system* sys, const int64_t* atoms, int64_t n_sel, int32_t* sizes) {
  if (!sys || !sizes) return fail(MKA_ERR_INVALID_ARG, "system and sizes are required");
  std::vector<int64_t> sel;
  mka_status s = copy_selection(sys, atoms, atoms ? n_sel : sys->n_atoms, sel);
  if (s) return s;
  const int64_t n = (int64_t)sel.size();
  int64_t* d_sel = nullptr;
  int32_t* d_sizes = nullptr;
  MKA_CUDA_TRY(cudaMalloc(&d_sel, sizeof(int64_t) * n));
  cudaError_t e = cudaMalloc(&d_sizes, sizeof(int32_t) * n);
  if (e == cudaSuccess) e = cudaMemcpy(d_sel, sel.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    s = launch_cluster_sizes(sys, d_sel, n, d_sizes, sys->stream);
    if (s == MKA_OK) e = cudaMemcpy(sizes, d_sizes, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
  }
  cudaFree(d_sel);
  cudaFree(d_sizes);
  if (e != cudaSuccess) return cuda_fail(e, "mka_cluster_sizes");
  return s;
}

void mka_result_destroy(mka_result* r) {
  if (!r) return;
  cudaFree(r->d_sel);
  cudaFree(r->d_blk_off);
  cudaFree(r->d_eps);
  cudaFree(r->d_w);
  cudaFree(r->d_nu_eff);
  cudaFree(r->d_cg_iters);
  cudaFree(r->d_status);
  cudaFree(r->d_vp);
  cudaFree(r->d_cv);
  cudaFree(r->d_mu_state);
  cudaFree(r->d_fallback);
  cudaFree(r->d_s_cl);
  cudaFree(r->d_s);
  delete r;
}

mka_status mka_solve_columns(mka_system* sys, const int64_t* atoms, int64_t n_sel, const mka_solve_params* prm,
                             void* stream, mka_result** out) {
  if (!out) return fail(MKA_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!sys || !prm) return fail(MKA_ERR_INVALID_ARG, "system and params are required");
  if (prm->p < 1 || prm->q < 0 || prm->p + prm->q > MKA_MAX_NU)
    return fail(MKA_ERR_INVALID_ARG, "need p >= 1, q >= 0, p + q <= MKA_MAX_NU");
  if (prm->arith != MKA_FP64 && prm->arith != MKA_MIXED_FP32)
    return fail(MKA_ERR_INVALID_ARG, "arith must be MKA_FP64 or MKA_MIXED_FP32");
  if (!(prm->cg_tol > 0) || prm->cg_maxit < 1) return fail(MKA_ERR_INVALID_ARG, "need cg_tol > 0, cg_maxit >= 1");
  if (prm->subspace != MKA_SUBSPACE_A && prm->subspace != MKA_SUBSPACE_B)
    return fail(MKA_ERR_INVALID_ARG, "subspace must be MKA_SUBSPACE_A or MKA_SUBSPACE_B");
  if (prm->use_warm_start && !sys->warm)
    return fail(MKA_ERR_INVALID_ARG, "use_warm_start needs a network attached with mka_system_set_warm_start");
  if (prm->use_warm_start && prm->s_start)
    return fail(MKA_ERR_INVALID_ARG, "use_warm_start and s_start are exclusive CG starts");
  if (prm->s_start) {
    const mka_result* pr = prm->s_start;
    if (!pr->d_s) return fail(MKA_ERR_INVALID_ARG, "s_start was solved without keep_s");
    if (!pr->sys || pr->sys->n_atoms != sys->n_atoms) return fail(MKA_ERR_INVALID_ARG, "s_start belongs to a system of another size");
    const int64_t n = atoms ? n_sel : sys->n_atoms;
    if (pr->n_sel != n) return fail(MKA_ERR_INVALID_ARG, "s_start has another selection");
    for (int64_t t = 0; t < n; ++t)
      if (pr->h_sel[t] != (atoms ? atoms[t] : t)) return fail(MKA_ERR_INVALID_ARG, "s_start has another selection");
  }
  cudaStream_t st = (cudaStream_t)stream;
  mka_result* r = new mka_result();
  r->sys = sys;
  r->stream = st;
  mka_status s = copy_selection(sys, atoms, atoms ? n_sel : sys->n_atoms, r->h_sel);
  if (s) {
    delete r;
    return s;
  }
  r->n_sel = (int64_t)r->h_sel.size();
  r->n_cols = 4 * r->n_sel;
  r->p = prm->p;
  r->q = prm->q;
  r->nu = prm->p + prm->q;
  r->arith = prm->arith;
  r->keep = prm->keep_vectors ? 1 : 0;
  r->h_blk_off.resize(r->n_sel + 1);
  r->h_blk_off[0] = 0;
  for (int64_t t = 0; t < r->n_sel; ++t) {
    const int64_t a = r->h_sel[t];
    r->h_blk_off[t + 1] = r->h_blk_off[t] + (sys->h_row_ptr[a + 1] - sys->h_row_ptr[a]);
  }
  r->n_blocks = r->h_blk_off[r->n_sel];
  const int64_t nc = r->n_cols, nu = r->nu;
  cudaError_t e = cudaSuccess;
#define ALLOC(ptr, bytes) \
  if (e == cudaSuccess) e = cudaMalloc(&(ptr), (bytes))
  ALLOC(r->d_sel, sizeof(int64_t) * r->n_sel);
  ALLOC(r->d_blk_off, sizeof(int64_t) * (r->n_sel + 1));
  ALLOC(r->d_eps, sizeof(double) * nc * nu);
  ALLOC(r->d_w, sizeof(double) * nc * nu);
  ALLOC(r->d_nu_eff, sizeof(int32_t) * nc);
  ALLOC(r->d_cg_iters, sizeof(int32_t) * nc);
  ALLOC(r->d_status, sizeof(int32_t) * nc);
  if (prm->use_warm_start) ALLOC(r->d_fallback, sizeof(int32_t) * nc);
  if (r->keep) ALLOC(r->d_vp, sizeof(double) * r->n_blocks * 16 * nu);
  if (r->keep) ALLOC(r->d_cv, kept_buffer_bytes(nc, (int)nu));
#undef ALLOC
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r->d_sel, r->h_sel.data(), sizeof(int64_t) * r->n_sel, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r->d_blk_off, r->h_blk_off.data(), sizeof(int64_t) * (r->n_sel + 1), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    mka_result_destroy(r);
    return cuda_fail(e, "mka_solve_columns allocation");
  }
  // largest cluster of the selection sizes the per-CTA scratch
  int32_t* d_sizes = nullptr;
  std::vector<int32_t> sizes(r->n_sel);
  e = cudaMalloc(&d_sizes, sizeof(int32_t) * r->n_sel);
  if (e == cudaSuccess) {
    s = launch_cluster_sizes(sys, r->d_sel, r->n_sel, d_sizes, st);
    if (s == MKA_OK) e = cudaMemcpyAsync(sizes.data(), d_sizes, sizeof(int32_t) * r->n_sel, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFree(d_sizes);
  if (e != cudaSuccess || s != MKA_OK) {
    mka_result_destroy(r);
    return s != MKA_OK ? s : cuda_fail(e, "cluster sizes");
  }
  const int max_cl = *std::max_element(sizes.begin(), sizes.end());
  if (prm->keep_s) {
    r->s_cap = std::max(1, std::min(max_cl, MKA_MAX_CLUSTER_ATOMS));
    e = cudaMalloc(&r->d_s_cl, sizeof(int32_t) * r->n_sel * r->s_cap);
    if (e == cudaSuccess) e = cudaMalloc(&r->d_s, sizeof(double) * 16 * r->n_sel * r->s_cap);
    if (e != cudaSuccess) {
      mka_result_destroy(r);
      return cuda_fail(e, "keep_s allocation");
    }
  }
  s = launch_columns(sys, r, prm, max_cl, st);
  if (s != MKA_OK) {
    mka_result_destroy(r);
    return s;
  }
  *out = r;
  return MKA_OK;
}

mka_status mka_result_info(const mka_result* r, int64_t* n_cols, int* nu, int64_t* n_blocks) {
  if (!r) return fail(MKA_ERR_INVALID_ARG, "result is NULL");
  if (n_cols) *n_cols = r->n_cols;
  if (nu) *nu = r->nu;
  if (n_blocks) *n_blocks = r->n_blocks;
  return MKA_OK;
}

mka_status mka_result_copy_levels(const mka_result* r, double* eps, double* w, int32_t* nu_eff, int32_t* cg_iters,
                                  int32_t* status) {
  if (!r) return fail(MKA_ERR_INVALID_ARG, "result is NULL");
  MKA_CUDA_TRY(cudaStreamSynchronize(r->stream));
  const int64_t nc = r->n_cols, nu = r->nu;
  if (eps) MKA_CUDA_TRY(cudaMemcpy(eps, r->d_eps, sizeof(double) * nc * nu, cudaMemcpyDeviceToHost));
  if (w) MKA_CUDA_TRY(cudaMemcpy(w, r->d_w, sizeof(double) * nc * nu, cudaMemcpyDeviceToHost));
  if (nu_eff) MKA_CUDA_TRY(cudaMemcpy(nu_eff, r->d_nu_eff, sizeof(int32_t) * nc, cudaMemcpyDeviceToHost));
  if (cg_iters) MKA_CUDA_TRY(cudaMemcpy(cg_iters, r->d_cg_iters, sizeof(int32_t) * nc, cudaMemcpyDeviceToHost));
  std::vector<int32_t> stv(nc);
  MKA_CUDA_TRY(cudaMemcpy(stv.data(), r->d_status, sizeof(int32_t) * nc, cudaMemcpyDeviceToHost));
  if (status) memcpy(status, stv.data(), sizeof(int32_t) * nc);
  for (int64_t c = 0; c < nc; ++c) {
    const int32_t v = stv[c];
    if (v != MKA_OK && v != MKA_ERR_BREAKDOWN) {
      return fail((mka_status)v, "column " + std::to_string(c) + ": " + mka_status_string((mka_status)v));
    }
  }
  return MKA_OK;
}

mka_status mka_result_copy_warm_start(const mka_result* r, int32_t* fallback) {
  if (!r || !fallback) return fail(MKA_ERR_INVALID_ARG, "result and fallback are required");
  if (!r->d_fallback) return fail(MKA_ERR_INVALID_ARG, "the result was solved without the learned warm start");
  MKA_CUDA_TRY(cudaStreamSynchronize(r->stream));
  MKA_CUDA_TRY(cudaMemcpy(fallback, r->d_fallback, sizeof(int32_t) * r->n_cols, cudaMemcpyDeviceToHost));
  return MKA_OK;
}

mka_status mka_cg_patch_targets(mka_system* sys, const int64_t* atoms, int64_t n, int arith, double cg_tol,
                                const int32_t* patch, float* Y, int32_t* iters, void* stream) {
  if (!sys || !atoms || n < 1 || !patch || !Y) return fail(MKA_ERR_INVALID_ARG, "bad target arguments");
  if (arith != MKA_FP64 && arith != MKA_MIXED_FP32) return fail(MKA_ERR_INVALID_ARG, "arith must be FP64 or FP32");
  if (!(cg_tol > 0)) return fail(MKA_ERR_INVALID_ARG, "need cg_tol > 0");
  std::vector<int64_t> sel(atoms, atoms + n);
  for (int64_t v : sel)
    if (v < 0 || v >= sys->n_atoms) return fail(MKA_ERR_INVALID_ARG, "atom index out of range");
  std::vector<int32_t> sizes(n);
  mka_status s = mka_cluster_sizes(sys, atoms, n, sizes.data());
  if (s) return s;
  const int max_cl = *std::max_element(sizes.begin(), sizes.end());
  if (max_cl > MKA_MAX_CLUSTER_ATOMS) return fail(MKA_ERR_CLUSTER_TOO_LARGE, "cluster larger than the cap");
  AtomsConfig cf{};
  s = atoms_config(sys, 1, arith, max_cl, 256, 0, &cf);     // basis unused: smallest subspace
  if (s) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t grid = std::min<int64_t>(n, cf.grid_max);
  char* buf = nullptr;
  const size_t scratch_bytes = cf.slot_bytes * grid + 256;
  const size_t extra = sizeof(int64_t) * n + sizeof(int32_t) * 8 * n + 256;
  MKA_CUDA_TRY(cudaMallocAsync(&buf, scratch_bytes + extra, st));
  int64_t* d_sel = reinterpret_cast<int64_t*>(buf + scratch_bytes);
  int32_t* d_status = reinterpret_cast<int32_t*>(d_sel + n);
  int32_t* d_iters = d_status + 4 * n;
  int* counter = reinterpret_cast<int*>(d_iters + 4 * n);
  cudaError_t e = cudaMemcpyAsync(d_sel, sel.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) {
    cudaFreeAsync(buf, st);
    return cuda_fail(e, "mka_cg_patch_targets");
  }
  AtomsLaunchArgs a{};
  a.sel = d_sel;
  a.n_sel = n;
  a.p = 1;
  a.q = 0;
  a.cg_tol = cg_tol;
  a.cg_maxit = 1000;
  a.status = d_status;
  a.cg_iters = iters ? iters : d_iters;
  a.scratch = buf;
  a.counter = counter;
  a.grid = (int)grid;
  a.patch = patch;
  a.cg_only = 1;
  a.cg_target = Y;
  s = atoms_launch(sys, arith, cf, a, st);
  std::vector<int32_t> stv(4 * n);
  if (s == MKA_OK) {
    e = cudaMemcpyAsync(stv.data(), d_status, sizeof(int32_t) * 4 * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFreeAsync(buf, st);
  if (s) return s;
  if (e != cudaSuccess) return cuda_fail(e, "mka_cg_patch_targets");
  for (int64_t i = 0; i < 4 * n; ++i)
    if (stv[i] != MKA_OK) return fail((mka_status)stv[i], "inner CG failed for column " + std::to_string(i));
  return MKA_OK;
}

mka_status mka_result_device_levels(const mka_result* r, const double** eps, const double** w) {
  if (!r) return fail(MKA_ERR_INVALID_ARG, "result is NULL");
  if (eps) *eps = r->d_eps;
  if (w) *w = r->d_w;
  return MKA_OK;
}

mka_status mka_find_mu(mka_result* r, double n_electrons, double kT, double tol, double* mu_out) {
  if (!r || !mu_out) return fail(MKA_ERR_INVALID_ARG, "result and mu_out are required");
  if (!(kT > 0) || !(tol > 0)) return fail(MKA_ERR_INVALID_ARG, "need kT > 0 and tol > 0");
  return launch_find_mu(r, n_electrons, kT, tol, mu_out);
}

mka_status mka_density_energy(mka_system* sys, mka_result* r, double mu, double kT, double* rho_out,
                              double* e_band_out, double* n_elec_out) {
  if (!sys || !r || r->sys != sys) return fail(MKA_ERR_INVALID_ARG, "result does not belong to this system");
  if (!r->keep) return fail(MKA_ERR_INVALID_ARG, "density needs a result solved with keep_vectors = 1");
  if (!(kT > 0)) return fail(MKA_ERR_INVALID_ARG, "need kT > 0");
  return launch_density(sys, r, mu, kT, rho_out, e_band_out, n_elec_out);
}

mka_status mka_greens(mka_system* sys, mka_result* r, double z_re, double z_im, double* g_out) {
  if (!sys || !r || r->sys != sys || !g_out) return fail(MKA_ERR_INVALID_ARG, "system, result and g_out are required");
  if (!r->keep) return fail(MKA_ERR_INVALID_ARG, "greens needs a result solved with keep_vectors = 1");
  return launch_greens(sys, r, z_re, z_im, g_out);
}

mka_status mka_system_shift_onsite(mka_system* sys, const double* shift, void* stream) {
  if (!sys || !shift) return fail(MKA_ERR_INVALID_ARG, "system and shift are required");
  for (int64_t a = 0; a < sys->n_atoms; ++a)
    if (!std::isfinite(shift[a])) return fail(MKA_ERR_INVALID_ARG, "shifts must be finite");
  return launch_onsite_shift(sys, shift, (cudaStream_t)stream);
}

mka_status mka_dos(const double* eps, const double* w, int64_t n_levels, const double* energies, int n_energies,
                   double eta, void* stream, double* dos) {
  if (!eps || !w || !energies || !dos || n_levels < 1 || n_energies < 1)
    return fail(MKA_ERR_INVALID_ARG, "levels, weights, energies and dos are required (n >= 1)");
  if (!(eta > 0)) return fail(MKA_ERR_INVALID_ARG, "need eta > 0");
  return launch_dos(eps, w, n_levels, energies, n_energies, eta, (cudaStream_t)stream, dos);
}

mka_status mka_spmv(const mka_system* sys, int which, int x_dtype, const void* x, void* y, int k, void* stream) {
  if (!sys || !x || !y) return fail(MKA_ERR_INVALID_ARG, "system, x and y are required");
  if (which != 0 && which != 1) return fail(MKA_ERR_INVALID_ARG, "which must be 0 (H) or 1 (S)");
  if (x_dtype != MKA_FP64 && x_dtype != MKA_MIXED_FP32) return fail(MKA_ERR_INVALID_ARG, "x_dtype must be FP64 or FP32");
  if (k != 1 && k != 2 && k != 4) return fail(MKA_ERR_INVALID_ARG, "k must be 1, 2 or 4");
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15)
    return fail(MKA_ERR_INVALID_ARG, "x and y must be 16-byte aligned");
  return launch_spmv(sys, which, x_dtype, x, y, k, (cudaStream_t)stream);
}

}  // extern "C"
