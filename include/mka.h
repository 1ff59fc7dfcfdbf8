/*
 * mka.h - C ABI of the GB300 (sm_103a) multiple Arnoldi library.
 *
 * The method (Hoshi, Yamamoto, Fujiwara, Sogabe, Zhang, arXiv:1202.0098,
 * "An order-N electronic structure theory with generalized eigen-value
 * equations and its application to a ten-million-atom system"): for every
 * basis index j of a non-orthogonal tight-binding model (sparse symmetric H,
 * sparse SPD S, Eq. EQ-ORIG-EQ), independently of every other j,
 *   - solve S s_j = e_j by an inner CG loop (Sec. 2);
 *   - build an S-orthonormal basis u_1..u_nu of the multiple Krylov subspace
 *     L^(j) = K_p(H; e_j) (+) K_q(H; s_j) (Eqs. EQ-SUBSPACE-MULTI-KRY,
 *     EQ-REC-UN, EQ-KN-HUN, EQ-MGram-Schmidt, EQ-CALC-S-INV);
 *   - solve the reduced nu x nu problem (Eq. EQ-SUB-EIG-VEC);
 *   - form the Fermi-weighted density matrix rho_ij (Eq. EQ-DM), the subspace
 *     Green's function G_ij(z) (Eq. EQ-SOLUTION-SUB-GZ) and the band energy
 *     (Eq. EQ-ENE); mu is found by bisection on the electron count (Sec. 2).
 * Every column works on the real-space projection of H and S onto the
 * cluster of atoms within a radius R of j's atom (Sec. 3).
 *
 * Conventions shared by all entry points
 *   - Atoms carry 4 orbitals (s, px, py, pz), M = 4 N; column j = 4 a + o
 *     belongs to atom a, orbital o (composite index, Sec. 1).
 *   - H and S are held as 4x4-block CSR ("BSR"): row_ptr[N+1], col[nnzb]
 *     (ascending within a row, the diagonal block included), values
 *     [nnzb][4][4] row-major; block k of row a is <mu_a | nu_col[k]>.
 *   - Every call returns mka_status. A failing call leaves a message readable
 *     through mka_last_error() (thread-local, valid until the next call on
 *     the same thread).
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the current device. Caller buffers are borrowed for
 *     the duration of the call only. mka_system and mka_result are owned by
 *     the library and freed with their destroy functions.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream). Device
 *     work is ordered on it; calls that return host values synchronise it.
 *   - There is no CPU fallback: without a usable CUDA device every call that
 *     touches the GPU returns MKA_ERR_CUDA.
 */
#ifndef MKA_H
#define MKA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MKA_OK = 0,
  MKA_ERR_INVALID_ARG = 1,      /* bad pointer, size or parameter */
  MKA_ERR_NOT_SPD = 2,          /* S (or a reduced S_r) is not positive definite */
  MKA_ERR_NO_CONVERGENCE = 3,   /* inner CG reached its iteration cap */
  MKA_ERR_BREAKDOWN = 4,        /* a column's basis ended with nu_eff < nu (reported, not fatal) */
  MKA_ERR_OOM = 5,              /* device or host allocation failed */
  MKA_ERR_CUDA = 6,             /* a CUDA runtime call failed (no device, launch error, ...) */
  MKA_ERR_TIMEOUT = 7,          /* a bounded device-side wait gave up */
  MKA_ERR_CLUSTER_TOO_LARGE = 8 /* a cluster exceeds MKA_MAX_CLUSTER_ATOMS */
} mka_status;

/* Storage format of H and S values, and arithmetic of a solve. */
typedef enum {
  MKA_FP64 = 0,        /* values FP64 / all arithmetic FP64 */
  MKA_MIXED_FP32 = 1,  /* values FP32 / FP32 SpMV, CG and basis, FP64 reduced solve */
  MKA_MIXED_BF16 = 2   /* values BF16 (storage only; arithmetic as MKA_MIXED_FP32) */
} mka_precision;

/* Largest cluster a column may have (atoms). m_c = 4 x atoms <= 2048. */
#define MKA_MAX_CLUSTER_ATOMS 512
/* Largest subspace dimension nu = p + q (the density of states, an energy-resolved
 * quantity, wants subspaces of a few hundred: Sec. 3). Subspaces above 64 run the
 * batched reduced problems with larger per-column buffers. */
#define MKA_MAX_NU 320

typedef struct mka_system mka_system; /* device BSR H and S, positions, cell list */
typedef struct mka_result mka_result; /* per-column levels, weights, status, kept vectors */

/* Two-centre Slater-Koster sp parameters of the model Hamiltonian.
 * V, Sv: (ss-sigma, sp-sigma, pp-sigma, pp-pi) for H (eV) and S, given at
 * bond length d0 (A) and scaled by exp(-2 (d/d0 - 1)) for d <= rc.
 * On-site blocks: diag(Es, Ep, Ep, Ep) for H, the unit matrix for S. For the
 * displacement d = r_b - r_a (minimum image) with cosines c = d/|d|:
 *   [s][s] = ss, [s][p_k] = c_k sp, [p_k][s] = -c_k sp,
 *   [p_k][p_m] = c_k c_m (pp_sigma - pp_pi) + delta_km pp_pi. */
typedef struct {
  double Es, Ep;
  double V[4];
  double Sv[4];
  double d0, rc;
} mka_sk_params;

/* Parameters of one mka_solve_columns call. */
typedef struct {
  int p;              /* Krylov dimension of the e_j chain, >= 1 */
  int q;              /* Krylov dimension of the s_j chain, >= 0; nu = p + q <= MKA_MAX_NU */
  int arith;          /* MKA_FP64 or MKA_MIXED_FP32 (mka_precision) */
  int use_warm_start; /* 1: CG starts from the learned guess (see mka_mlp_*), 0: from zero */
  double cg_tol;      /* inner CG stops at ||r||_2 <= cg_tol ||e_j||_2 */
  int cg_maxit;       /* inner CG iteration cap (MKA_ERR_NO_CONVERGENCE beyond it) */
  int keep_vectors;   /* 1: keep what rho and G need to be evaluated later for any mu / z:
                         the basis U on the pattern rows (16 nu doubles per block of the
                         selected rows) and per column the reduced eigenvectors C and
                         the row V_j = (row j of U) C (nu^2 + nu doubles), since
                         sum_alpha x_alpha v_alpha,i v_alpha,j = U_i . (C diag(x) V_j);
                         0: keep only (eps, w) */
  int keep_s;         /* 1: the result keeps every column's s_j = S^{-1} e_j on its cluster (FP64, 16 doubles
                         and 1 int per cluster atom and selected atom) for a later solve's s_start */
  const mka_result* s_start; /* NULL, or an earlier result of mka_solve_columns with keep_s = 1 for the
                         same atoms in the same order, possibly of another system with the same atom
                         numbering (atoms moved by an MD step): the inner CG starts from that s_j,
                         matched by atom id onto the new cluster. With S unchanged (a charge-self-
                         consistent loop changes only H, Sec. 2) CG is already converged. Direct solves
                         only (not plans) */
  int subspace;       /* MKA_SUBSPACE_A (0): the vector after u_p is s_j and H keeps acting on the
                         latest u_n (span K_p(H; e_j) + K_q((I - Pi_p) H; (I - Pi_p) s_j), Pi_p the
                         S-orthogonal projector onto K_p(H; e_j)); MKA_SUBSPACE_B (1): the literal
                         direct sum K_p(H; e_j) + K_q(H; s_j) of Eq. EQ-SUBSPACE-MULTI-KRY, the s_j
                         chain continued from its raw vectors H^k s_j (q more H products) */
} mka_solve_params;

#define MKA_SUBSPACE_A 0
#define MKA_SUBSPACE_B 1

/* ---- system ------------------------------------------------------------ */

/* Build the periodic model H and S (4x4 blocks, SK table above) from atom
 * positions, store their values on the device in `storage` format, and build
 * the cell list the cluster extraction uses (real-space projection, Sec. 3).
 *   pos      host, [n_atoms][3] Cartesian positions (A), any values (wrapped
 *            into the box internally)
 *   box      host, [3] orthorhombic periodic box lengths (A); rc and
 *            cluster_radius must both be < box/2
 *   storage  mka_precision of the stored values (FP64 values are built first,
 *            then rounded to nearest-even: FP64 -> FP32 -> BF16)
 * Returns MKA_ERR_INVALID_ARG for n_atoms < 1, non-positive box, radii that
 * do not fit the box; MKA_ERR_OOM / MKA_ERR_CUDA on allocation failures. */
mka_status mka_build_system(const double* pos, int64_t n_atoms, const double box[3],
                            const mka_sk_params* sk, int storage, double cluster_radius,
                            void* stream, mka_system** out);

/* Same, from a caller's BSR H and S (host arrays, FP64 values, layout above,
 * pattern symmetric, columns ascending, diagonal present). Positions and the
 * box still define the clusters. */
mka_status mka_build_system_bsr(const double* pos, int64_t n_atoms, const double box[3],
                                const int32_t* row_ptr, const int32_t* col, int64_t nnzb,
                                const double* valH, const double* valS, int storage,
                                double cluster_radius, void* stream, mka_system** out);

/* Add shift[a] (host double [n_atoms], eV) to the diagonal of atom a's on-site block of H, in
 * place: the on-site potential a charge-self-consistent loop updates between solves while S and
 * the positions stay fixed (Sec. 2, CSC remark; keep_s / s_start then reuse every s_j). The
 * stored value is decoded, shifted and rounded back to the storage format. Synchronises. */
mka_status mka_system_shift_onsite(mka_system* sys, const double* shift, void* stream);

/* Sizes: atoms, blocks, stored precision. Any output pointer may be NULL. */
mka_status mka_system_info(const mka_system* sys, int64_t* n_atoms, int64_t* nnzb,
                           int* storage, int* max_row_blocks);

/* Copy the BSR pattern and the stored values (decoded to FP64) to host
 * arrays of sizes N+1, nnzb, nnzb*16, nnzb*16. Any output may be NULL. */
mka_status mka_system_copy_bsr(const mka_system* sys, int32_t* row_ptr, int32_t* col,
                               double* valH, double* valS);

/* Cluster sizes (atoms within cluster_radius, minimum image, the atom
 * included) of `n_sel` atoms given as a host list (NULL = all atoms, in
 * order), written to host `sizes`. Computed on the device. */
mka_status mka_cluster_sizes(const mka_system* sys, const int64_t* atoms, int64_t n_sel,
                             int32_t* sizes);

void mka_system_destroy(mka_system* sys);

/* Global block-sparse product y = A x for A = H (which = 0) or S (which = 1),
 * the stored values decoded to FP64 (x_dtype = MKA_FP64: x, y device
 * double[4N][k]) or to FP32 (x_dtype = MKA_MIXED_FP32: float[4N][k]), k in
 * {1, 2, 4} right-hand sides interleaved (row-major [4N][k]); x and y 16-byte
 * aligned (MKA_ERR_INVALID_ARG otherwise). Products and sums in the type of x. */
mka_status mka_spmv(const mka_system* sys, int which, int x_dtype, const void* x, void* y, int k,
                    void* stream);

/* ---- columns ----------------------------------------------------------- */

/* Run the per-column work flow (first brace of Eq. EQ-WORK-FLOW) for the 4
 * columns of each of `n_sel` atoms (host list; NULL = every atom in order):
 * cluster extraction, inner CG for s_j, the S-orthonormal multiple Krylov
 * basis, the projection H_r = U^T H U, S_r = U^T S U, the Cholesky-reduced
 * nu x nu eigensolve, and per column the levels eps_alpha (ascending) and
 * weights w_alpha = v_alpha,j (S v_alpha)_j. Columns are stored in selection
 * order, orbital fastest (column c = 4 t + o for the t-th selected atom).
 * The result's aggregate status is MKA_OK, or the first per-column error
 * (details by mka_result_copy_levels). Device work runs on `stream`; the
 * call returns after enqueueing and the result is valid in stream order. */
mka_status mka_solve_columns(mka_system* sys, const int64_t* atoms, int64_t n_sel,
                             const mka_solve_params* prm, void* stream, mka_result** out);

/* Size of the fixed device scratch array behind mka_solve_columns_static: 64 MiB,
 * reserved on every GPU that loads this library until the process exits. */
#define MKA_STATIC_SCRATCH_BYTES (64ull << 20)

/* mka_solve_columns without any allocation. The paper has no counterpart to
 * this call: it exists for callers that must not allocate device memory, for
 * example code whose device memory is owned by a framework's caching
 * allocator that has already reserved the GPU (a raw cudaMalloc would fail or
 * fragment its pool), or code inside a latency-critical loop where the
 * implicit synchronisation of cudaMalloc/cudaFree is not acceptable.
 *
 * It runs the same per-atom work flow as mka_solve_columns in the FP64 form
 * (values decoded from the system's storage format, FP64 arithmetic), for the
 * 4 columns of each of `n_sel` atoms listed in the HOST array `atoms`, and
 * writes per column, in selection order (column 4 t + o), into the caller's
 * DEVICE buffers:
 *   eps, w      double [4 n_sel][p + q] (entries beyond nu_eff are 0)
 *   nu_eff, cg_iters, status  int32 [4 n_sel] (status: a mka_status value;
 *               MKA_ERR_CLUSTER_TOO_LARGE when an atom's cluster has more
 *               than `max_cluster_atoms` atoms)
 * Nothing for rho / G is kept (keep_vectors = 0 in effect).
 * Work memory (the work-queue counter, the atom list of a chunk, the chunk's
 * reduced problems, 8 (3 nu^2 + 2 nu) bytes per column, and one work slot per
 * CTA of about 8 (2 (p+q) + 2) x 4 max_cluster_atoms x 4 bytes) comes from one
 * file-scope device array of MKA_STATIC_SCRATCH_BYTES; the selection runs in
 * chunks sized to fit. The call returns MKA_ERR_INVALID_ARG, with a message,
 * when one slot and one atom's reduced problems do not fit in it; fewer slots
 * than SMs simply means fewer atoms in flight.
 * The call performs no cudaMalloc, cudaFree or other allocating routine. Each
 * call looks up the array's device address on the current device
 * (cudaGetSymbolAddress, no allocation); the first call on a device may load
 * the library's device code there. Every call on a device shares the one
 * array, so calls whose GPU
 * work overlaps (different streams, or host threads, without ordering between
 * them) race on it and corrupt each other's results; order them on one stream.
 * The work-queue counter is cleared by each call; the rest is overwritten. */
mka_status mka_solve_columns_static(const mka_system* sys, const int64_t* atoms, int64_t n_sel, int p, int q,
                                    double cg_tol, int cg_maxit, int max_cluster_atoms, double* eps, double* w,
                                    int32_t* nu_eff, int32_t* cg_iters, int32_t* status, void* stream);

/* Sizes of a result: columns (= 4 n_sel), nu, and the number of 4x4 output
 * blocks of rho / G (the sum over selected atoms of their H-row lengths). */
mka_status mka_result_info(const mka_result* res, int64_t* n_cols, int* nu, int64_t* n_blocks);

/* Copy per-column data to host arrays: eps, w [n_cols][nu] (entries beyond
 * nu_eff are 0), nu_eff, cg_iters, status [n_cols]. Any output may be NULL.
 * Synchronises the result's stream. */
mka_status mka_result_copy_levels(const mka_result* res, double* eps, double* w, int32_t* nu_eff,
                                  int32_t* cg_iters, int32_t* status);

/* Device pointers of the per-column (eps, w) arrays ([n_cols][nu], FP64). */
mka_status mka_result_device_levels(const mka_result* res, const double** eps, const double** w);

void mka_result_destroy(mka_result* res);

/* ---- global: mu, rho, G, energy --------------------------------------- */

/* Chemical potential by bisection (Sec. 2, after Eq. EQ-DM): the mu with
 * 2 sum_j sum_alpha f(eps_alpha^(j); mu) w_alpha^(j) = n_electrons over the
 * result's columns, f(x) = 1 / (1 + exp((x - mu) / kT)). Bracket
 * [min eps - 40 kT, max eps + 40 kT], halved until narrower than `tol` (eV)
 * or 200 times; returns the midpoint in *mu_out (host). Runs on the device
 * with FP64 sums; synchronises. */
mka_status mka_find_mu(mka_result* res, double n_electrons, double kT, double tol, double* mu_out);

/* Density matrix (Eq. EQ-DM) on the selected rows' pattern, the band energy
 * E = 2 sum_j sum_i rho_ij H_ji (Eq. EQ-ENE, two electrons per orbital state)
 * and the electron count 2 sum_j sum_alpha f w, at chemical potential mu.
 *   rho_out  device double, [n_blocks][4][4] or NULL. Block k of the t-th
 *            selected atom b (its H-row blocks in order, neighbour a = col[k])
 *            holds rho_out[k][c][r] = rho_{(a,r),(b,c)}: the part of column
 *            j = 4b + c on atom a's orbitals.
 *   e_band_out, n_elec_out  host, may be NULL.
 * Needs a result solved with keep_vectors = 1; otherwise MKA_ERR_INVALID_ARG.
 * Synchronises when a host output is requested. */
mka_status mka_density_energy(mka_system* sys, mka_result* res, double mu, double kT,
                              double* rho_out, double* e_band_out, double* n_elec_out);

/* Subspace Green's function G_ij(z) = sum_alpha v_alpha,i v_alpha,j / (z - eps_alpha)
 * (Eq. EQ-SOLUTION-SUB-GZ) at complex z = z_re + i z_im, same pattern and
 * layout as rho, complex128 interleaved (re, im): device double
 * [n_blocks][4][4][2]. Needs keep_vectors = 1. */
mka_status mka_greens(mka_system* sys, mka_result* res, double z_re, double z_im, double* g_out);

/* Energy density matrix pi_ij = sum_alpha f(eps_alpha; mu) eps_alpha v_alpha,i v_alpha,j
 * (Sec. 2, after Eq. EQ-DM) on the selected rows' pattern, layout as rho in
 * mka_density_energy (device double [n_blocks][4][4], may be NULL), and the
 * forces of Eqs. EQ-FORCE / EQ-FORCE-PART from the result's columns, ADDED to
 * the caller's device double [n_atoms][3] (may be NULL): F_K += -2 sum_j sum_i
 * (rho_ij dH_ji/dR_K - pi_ij dS_ji/dR_K) (sign as for mka_sweep_forces). The adds
 * are atomic, so the last bits may differ between runs. Needs keep_vectors = 1
 * and a system built by mka_build_system (MKA_ERR_INVALID_ARG otherwise). */
mka_status mka_forces(mka_system* sys, mka_result* res, double mu, double kT, double* pi_out, double* forces);

/* Density of states from the subspace Green's function (Sec. 3):
 *   D(E) = -(1/pi) Im sum_j (G(E + i eta) S)_jj = (eta / pi) sum_j sum_alpha w_alpha / ((E - eps_alpha)^2 + eta^2),
 * since sum_i G_ji(z) S_ij = sum_alpha w_alpha / (z - eps_alpha) for each column's Galerkin pairs.
 *   eps, w    device double [n_levels]: any columns' levels and weights, flattened (for example a
 *             result's or a sweep's [n_cols][nu] arrays; entries with w = 0 add nothing)
 *   energies  host double [n_energies]; eta > 0 the broadening (eV)
 *   dos       host double [n_energies] out, states per eV (one per state, no spin factor)
 * FP64, fixed summation order; synchronises `stream`. */
mka_status mka_dos(const double* eps, const double* w, int64_t n_levels, const double* energies, int n_energies,
                   double eta, void* stream, double* dos);

/* ---- learned warm start for the inner CG ---------------------------------- */
/* The inner CG for s_j = S^{-1} e_j (Sec. 2) may start from any x0. A small
 * network predicts x0 on the 17-atom patch around j's atom (the atom and its 16
 * nearest neighbours by minimum-image distance, ties by atom id; 4 orbitals
 * each = 68 values, patch order then s, px, py, pz). Its 132 inputs per column:
 * the 32 nearest neighbours within 3 A as (d, l, m, n), (l, m, n) the direction
 * cosines of r_b - r_a, zeros beyond, then a one-hot of the column's orbital.
 * Network 132 -> 128 -> 128 -> 68, SiLU after the hidden layers; parameters
 * packed W1 [128][132], b1, W2 [128][128], b2, W3 [68][128], b3 (FP32 master,
 * BF16 for every product, FP32 sums); loss = mean squared error over the batch
 * and the 68 outputs; Adam (beta 0.9 / 0.999, eps 1e-8, bias-corrected).
 * CG from the prediction always runs to the solve's tolerance; where the
 * prediction's residual is no smaller than ||e_j|| the column starts from zero
 * instead (counted as a fallback). */
typedef struct mka_mlp mka_mlp;

int64_t mka_mlp_num_params(void);
/* New network, He-uniform weights and zero biases from a seeded generator. */
mka_status mka_mlp_create(uint64_t seed, mka_mlp** out);
void mka_mlp_destroy(mka_mlp* net);
/* Host FP32 parameters in the packed order (set resets the Adam state). get with
 * bf16_rounded = 1 returns the BF16 values the products use. */
mka_status mka_mlp_set_params(mka_mlp* net, const float* params);
mka_status mka_mlp_get_params(const mka_mlp* net, float* params, int bf16_rounded);
/* Y = net(X): device X [B][132], device Y [B][68], FP32. */
mka_status mka_mlp_forward(mka_mlp* net, const float* X, float* Y, int64_t B, void* stream);
/* Loss and its gradient with respect to the (BF16) parameters for device X, targets T
 * [B][68]: grad (device, num_params floats) and loss (device, 1 float); either may be NULL. */
mka_status mka_mlp_gradients(mka_mlp* net, const float* X, const float* T, int64_t B, float* grad,
                             float* loss, void* stream);
/* One Adam step on the batch (gradient as above); loss before the step into device `loss`
 * (may be NULL). */
mka_status mka_mlp_train_step(mka_mlp* net, const float* X, const float* T, int64_t B, float lr,
                              float* loss, void* stream);
/* Inputs of the 4 columns of each of n atoms (host list): device X [4n][132] and the
 * patch atoms, device int32 [n][17] (-1 where fewer atoms lie within min(5.5 A, cell edge)). */
mka_status mka_warm_start_features(const mka_system* sys, const int64_t* atoms, int64_t n, float* X,
                                   int32_t* patch, void* stream);
/* Training targets: the inner CG alone (x0 = 0, `arith`, tolerance cg_tol) for the 4
 * columns of each atom, s_j written on the given patch: device Y [4n][68] (FP32), device
 * iterations [4n] (may be NULL). */
mka_status mka_cg_patch_targets(mka_system* sys, const int64_t* atoms, int64_t n, int arith, double cg_tol,
                                const int32_t* patch, float* Y, int32_t* iters, void* stream);
/* Network used by solves with use_warm_start = 1 (NULL detaches; not owned). */
mka_status mka_system_set_warm_start(mka_system* sys, mka_mlp* net);
/* Per-column warm-start fallback flags (1 = started from zero) of a solve made with
 * use_warm_start = 1, into host int32 [n_cols]. */
mka_status mka_result_copy_warm_start(const mka_result* res, int32_t* fallback);

/* ---- persistent, graph-captured batches ---------------------------------- */

/* Launch shape of the per-atom kernel. */
typedef struct {
  int threads;        /* CTA size: 128, 256 or 512 (0 = 256) */
  int ctas_per_sm;    /* cap on resident CTAs per SM (0 = as many as fit) */
  int order_by_size;  /* 1: the work queue takes atoms by descending cluster size */
} mka_tuning;

typedef struct mka_plan mka_plan; /* every buffer of one batch of the work flow, plus its CUDA graphs */

/* A plan for batches of up to `max_atoms` atoms of `sys` (4 columns each): the
 * whole work flow of Eq. EQ-WORK-FLOW for one batch (the per-column brace with
 * kept data as for keep_vectors, mu by bisection over the batch's columns, rho and the band
 * energy) with every buffer allocated here, once. `tune` may be NULL (defaults,
 * or pass the result of mka_autotune). The plan computes the largest cluster of
 * the whole system once, to size its work slots. Work runs on `stream`. */
mka_status mka_plan_create(mka_system* sys, int64_t max_atoms, const mka_solve_params* prm,
                           const mka_tuning* tune, void* stream, mka_plan** out);

/* Run one batch: `atoms` (host, n_sel <= max_atoms) are staged in pinned memory
 * and the batch is enqueued as one CUDA graph (captured the first time this
 * (n_sel, n_electrons, kT, rho_out) combination is seen, replayed afterwards):
 * copy-in, optional ordering by cluster size, the persistent per-atom kernel,
 * 64 device bisection steps for mu (bracket as mka_find_mu, tolerance 1e-12 eV),
 * rho into `rho_out` (device, [n_blocks][4][4] as in mka_density_energy, may be
 * NULL) and the band energy. Returns without waiting for the GPU; the call waits
 * only for the previous batch to have read the staging buffer. */
mka_status mka_plan_run(mka_plan* plan, const int64_t* atoms, int64_t n_sel, double n_electrons, double kT,
                        double* rho_out);

/* mu, band energy 2 sum_j sum_i rho_ij H_ji and electron count 2 sum f w of the
 * last batch (host outputs, any may be NULL); synchronises the plan's stream. */
mka_status mka_plan_scalars(mka_plan* plan, double* mu, double* e_band, double* n_elec);

/* Device times (ms) of the last batch's two column kernels, from events the
 * graph records around them: the per-atom kernel (cluster, CG, basis,
 * projection) and the batched reduced problems (one lane per column). Either
 * output may be NULL; waits for that batch's reduced problems to finish. */
mka_status mka_plan_kernel_ms(mka_plan* plan, float* atoms_ms, float* reduced_ms);

/* The plan's result object (levels, weights, status and kept rows of the last
 * batch), borrowed: valid until the next run or mka_plan_destroy, never
 * destroyed by the caller. Usable with mka_result_copy_levels, mka_greens and
 * mka_density_energy (another mu). */
mka_status mka_plan_result(mka_plan* plan, mka_result** res);

/* The plan's launch shape, grid size and resident CTAs per SM in use. */
mka_status mka_plan_info(const mka_plan* plan, mka_tuning* tune, int* grid, int* ctas_per_sm_used);

void mka_plan_destroy(mka_plan* plan);

/* Choose a launch shape for `prm` on this GPU: each candidate (threads 128/256/
 * 512, resident CTAs per SM max/1/2, ordering by cluster size off/on) that fits
 * runs the sample batch (host atoms) three times through a plan, the fastest of
 * the last two timings wins. With `cache_path` (a JSON file, NULL = none) the
 * choice is looked up first under a key of GPU name, storage, arithmetic, p+q,
 * the sample's largest cluster (rounded down to 16) and the sample size, and
 * stored there after a search. */
mka_status mka_autotune(mka_system* sys, const mka_solve_params* prm, const int64_t* sample, int64_t n_sample,
                        double n_electrons, double kT, const char* cache_path, void* stream, mka_tuning* out);

/* Choose the batch size of plans for `prm` and launch shape `tune` (NULL = defaults): each candidate
 * (host array, atoms per batch) that fits runs a batch of consecutive atoms from first_atom through a
 * plan twice; the highest columns/s of the second run wins, into *out_batch. With `cache_path` the
 * choice is looked up first and stored after a search (key: GPU, storage, arithmetic, p + q, subspace,
 * system size, launch shape, candidates). MKA_ERR_OOM when no candidate fits. */
mka_status mka_autotune_batch(mka_system* sys, const mka_solve_params* prm, const mka_tuning* tune,
                              const int64_t* candidates, int n_candidates, int64_t first_atom,
                              double electrons_per_atom, double kT, const char* cache_path, void* stream,
                              int64_t* out_batch);

/* ---- whole-system sweep: every column, one mu, then rho ------------------ */

/* The work flow of Eq. EQ-WORK-FLOW over a whole system (or one contiguous range
 * of its atoms, for a process that owns that range): first every column's
 * levels (eps_alpha, w_alpha), then one chemical potential from the total
 * electron count of all of them (Sec. 2, bisection), then rho_ij (Eq. EQ-DM) and
 * the band energy (Eq. EQ-ENE) at that mu.
 *
 * A sweep keeps, in device memory, for every column of its range: the levels and
 * weights (FP64 [4 n][nu]); and for every entry (i, j) of the pattern, the two
 * pieces rho_ij needs at any mu inside the sweep's window [win_lo, win_hi]:
 *   occupied part  sum over levels below win_lo of v_alpha,i v_alpha,j  (FP64)
 *   products       v_alpha,i v_alpha,j of the levels inside the window, at most
 *                  kp per column, in ascending order (FP64 [kp])
 * so that rho_ij(mu) = occupied + sum_window f(eps_alpha; mu) v_alpha,i v_alpha,j
 * holds exactly (up to the rounding of the sums) whenever every level below
 * win_lo has f = 1 and every level above win_hi has f = 0 at mu, that is for
 * win_lo + 40 kT <= mu <= win_hi - 40 kT (f(x) = (1 - tanh((x - mu) / 2kT)) / 2
 * is 0 or 1 in FP64 beyond 40 kT). Columns with more than kp levels in the
 * window ("overflow" atoms, all 4 columns of the atom) and, when mu falls
 * outside that range, every atom, are solved again at mu by a plan.
 * Memory: 16 (kp + 1) x 8 bytes per pattern block of the range, plus
 * 16 nu bytes and 2 bytes per column.
 *
 * Deterministic sums: the electron count, the band energy and the
 * level-energy are summed per chunk of `chunk_atoms` consecutive atoms (chunk g
 * = atoms [g chunk_atoms, (g+1) chunk_atoms) of the whole system) in a fixed
 * order, and the chunk sums are added in chunk order. Processes whose ranges
 * start on chunk boundaries therefore produce the very chunk sums a single
 * process over the whole system produces, and a root finder that adds them in
 * chunk order and takes the same steps (mka_sweep_find_mu here, or a host
 * driver over all processes' mka_sweep_chunk_sums) finds the same mu, bit for
 * bit. */
typedef struct mka_sweep mka_sweep;

/* A sweep over atoms [atom_begin, atom_end) of `sys` for subspaces of size nu
 * (= p + q of the plans that feed it). win_lo < win_hi (eV); 1 <= kp <= nu;
 * chunk_atoms >= 1. with_forces = 1 also keeps the occupied part of the energy
 * density matrix pi (16 more doubles per pattern block) and 3 doubles per block
 * for mka_sweep_forces (needs a system built by mka_build_system). Allocates
 * its device arrays (MKA_ERR_OOM when they do not fit); work runs on `stream`. */
mka_status mka_sweep_create(mka_system* sys, int64_t atom_begin, int64_t atom_end, int nu, double win_lo,
                            double win_hi, int kp, int64_t chunk_atoms, int with_forces, void* stream,
                            mka_sweep** out);

/* Chunks of the sweep's range (global index of the first one, count), pattern
 * blocks of the range, and device bytes the sweep holds. Any output may be NULL. */
mka_status mka_sweep_info(const mka_sweep* sw, int64_t* chunk0, int64_t* n_chunks, int64_t* n_blocks,
                          int64_t* bytes);

/* Solve a batch of atoms (host list, all inside the sweep's range, n_sel <=
 * the plan's max_atoms) with `plan` (whose nu and system must match the
 * sweep's) and store their levels and rho pieces in the sweep: one CUDA graph
 * per batch size (copy-in, the column kernels, the packing kernel). Returns
 * without waiting for the GPU, as mka_plan_run. An atom swept again is
 * overwritten. */
mka_status mka_plan_run_sweep(mka_plan* plan, mka_sweep* sw, const int64_t* atoms, int64_t n_sel);

/* Atoms of the range stored so far, and how many of them overflowed the
 * window (host outputs, either may be NULL); synchronises. */
mka_status mka_sweep_status(mka_sweep* sw, int64_t* n_stored, int64_t* n_overflow);

/* Smallest and largest level with nonzero weight over the stored columns
 * (host outputs); synchronises. MKA_ERR_INVALID_ARG when there is none. */
mka_status mka_sweep_level_range(mka_sweep* sw, double* lo, double* hi);

/* mu with 2 sum_j sum_alpha f(eps; mu) w = n_electrons over every column of
 * the range, all on the device, by a bracketing root finder: the bracket
 * [lo - 40 kT, hi + 40 kT] from mka_sweep_level_range (the count is 0 at its
 * lower end); its upper end evaluated first; bisection while the bracket is
 * wider than 16 kT, then the secant through the bracket's ends (regula falsi
 * with the Illinois rule), the midpoint when the secant leaves the bracket;
 * a point where the count equals n_electrons exactly closes the bracket on
 * it; until the bracket is no wider than `tol` (eV), at most 200 steps; mu =
 * the bracket's midpoint. The count at each point is the chunk-ordered sum above,
 * and every step uses IEEE-rounded operations only. Every atom of the range
 * must have been stored (MKA_ERR_INVALID_ARG otherwise). */
mka_status mka_sweep_find_mu(mka_sweep* sw, double n_electrons, double kT, double tol, double* mu);

/* rho at mu into the caller's device buffer `rho` (double [n_blocks][4][4],
 * the system's pattern blocks of the range in order: block k of atom b's row,
 * neighbour a = col[k], rho[k][c][r] = rho_{(a,r),(b,c)}), and the per-atom band
 * energies that mka_sweep_chunk_sums adds up. Atoms that overflowed the window,
 * and every atom when mu lies outside [win_lo + 40 kT, win_hi - 40 kT], are
 * solved again with `plan` (may be NULL only when there are none:
 * MKA_ERR_INVALID_ARG otherwise); their count goes to *n_resolved (may be
 * NULL). Returns after enqueueing the work. */
mka_status mka_sweep_density(mka_sweep* sw, mka_plan* plan, double mu, double kT, double* rho, int64_t* n_resolved);

/* Forces on every atom of the system from the sweep's columns (Eqs. EQ-FORCE,
 * EQ-FORCE-PART) at mu: F_K = -2 sum_j sum_i (rho_ij dH_ji/dR_K - pi_ij dS_ji/dR_K)
 * over the range's columns j and their pattern entries i, with pi_ij =
 * sum_alpha f eps_alpha v_alpha,i v_alpha,j the energy density matrix (Sec. 2)
 * and the Slater-Koster block derivatives of the model at the current
 * positions. The sign of the pi term is that of the derivative of the grand
 * potential at fixed mu (dOmega = 2 (Tr[rho dH] - Tr[pi dS])). Output: device
 * double [n_atoms][3] (eV/A), overwritten; atoms outside the range get the
 * contributions of the range's columns only (a process's share, to be summed
 * over processes). The sums run in a fixed order. Overflowed atoms (or all,
 * when mu is outside the window's range, as for mka_sweep_density) are solved
 * again with `plan`; their count goes to *n_resolved (may be NULL). Needs a
 * sweep created with with_forces = 1. */
mka_status mka_sweep_forces(mka_sweep* sw, mka_plan* plan, double mu, double kT, double* forces, int64_t* n_resolved);

/* Chunk sums over the range at mu, into host arrays of n_chunks doubles (any
 * may be NULL): count[g] = 2 sum f w, e_levels[g] = 2 sum f eps w, and
 * e_rho[g] = 2 sum_j sum_i rho_ij H_ji from the last mka_sweep_density (whose
 * mu must be the same: MKA_ERR_INVALID_ARG otherwise). Adding a vector in
 * chunk order gives the electron count, the band energy from the levels, and
 * the band energy of Eq. EQ-ENE; the last two agree because e_j lies in every
 * column's subspace. Synchronises. */
mka_status mka_sweep_chunk_sums(mka_sweep* sw, double mu, double kT, double* count, double* e_levels,
                                double* e_rho);

/* Device pointers of the levels and weights of the range ([4 n][nu], FP64,
 * column 4 (a - atom_begin) + o). */
mka_status mka_sweep_device_levels(const mka_sweep* sw, const double** eps, const double** w);

void mka_sweep_destroy(mka_sweep* sw);

/* ---- accounting ---------------------------------------------------------- */

/* Number of CUDA kernels this library has launched since it was loaded (all
 * threads, all devices). Lets a caller count the device launches of a timed
 * region: read it before and after. */
int64_t mka_kernel_launches(void);

/* ---- errors -------------------------------------------------------------- */

const char* mka_last_error(void);
const char* mka_status_string(mka_status s);

#ifdef __cplusplus
}
#endif

#endif /* MKA_H */
