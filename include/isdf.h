/*
 * isdf.h -- C ABI of the GB300 (sm_103a) multigrid ISDF / THC exchange library.
 *
 * Method: Smyser, White & Sharma, "Use of multigrids to reduce the cost of
 * performing interpolative separable density fitting" (arXiv:2404.09373).
 *
 * The library factorises the electron-repulsion integrals of a periodic,
 * uncontracted Cartesian Gaussian basis into tensor-hypercontraction form by
 * interpolative separable density fitting (ISDF) on a hierarchy of real-space
 * grids, and builds the exact-exchange matrix from the factors:
 *
 *   isdf_plan           set-up: basis, grid levels, device buffers (no math)
 *   isdf_select_points  interpolation points by pivoted Cholesky on M (Eq. 2)
 *   isdf_fit            interpolation vectors xi(R) by least squares (Eq. 3)
 *   isdf_coulomb        two-centre Coulomb matrix (xi|xi') by FFT (Eq. 1)
 *   isdf_exchange       exchange matrix K from the four-term THC form (Eq. 8)
 *
 * Conventions shared by every call
 *   - Units: bohr and hartree.  All floating point arguments are FP64.
 *   - Pointers: every array argument may be host memory or device memory of
 *     the plan's device; the library tells them apart with
 *     cudaPointerGetAttributes.  The caller owns all inputs and outputs; the
 *     plan owns every device buffer it allocates and frees them in
 *     isdf_destroy.
 *   - Stream: all device work is enqueued on the stream given to isdf_plan.
 *     Calls return after the results they write to HOST memory are complete;
 *     results written to DEVICE memory are valid once that stream reaches
 *     the point where the call returned.
 *   - Errors: every call returns an isdf_status; nothing throws or exits
 *     across the ABI.  isdf_last_error(plan) gives a message.  After a failed
 *     call the plan can always be destroyed.  Calls must come in the order
 *     plan -> select_points -> fit -> coulomb -> exchange (exchange may be
 *     repeated, e.g. once per SCF iteration); a call out of order returns
 *     ISDF_ERR_STATE and changes nothing.
 *   - Basis function order: shells in the order given; an s shell gives one
 *     function, a p shell three (x, y, z).  Function mu has level
 *     l(mu) = #{e in level_min_exp : exponent < e} (level 0 = finest grid).
 *   - Grid point g of a level with (nx, ny, nz) points is r_g = (i Lx/nx,
 *     j Ly/ny, k Lz/nz) with g = i + nx (j + ny k).
 *   - Pivot code: (level << 40) | g  (int64).
 */
#ifndef ISDF_H
#define ISDF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ISDF_MAX_LEVELS 4

typedef struct isdf_plan_s* isdf_plan_t;

typedef enum {
  ISDF_OK = 0,
  ISDF_ERR_ARG = 1,     /* invalid argument (nothing was changed)          */
  ISDF_ERR_OOM = 2,     /* device allocation failed                        */
  ISDF_ERR_NOT_PD = 3,  /* Cholesky of C C^T broke down (non-positive pivot)*/
  ISDF_ERR_CUDA = 4,    /* a CUDA runtime call or kernel launch failed     */
  ISDF_ERR_CUFFT = 5,   /* a cuFFT call failed                             */
  ISDF_ERR_TIMEOUT = 6, /* the selection loop exceeded options.timeout_ms  */
  ISDF_ERR_STATE = 7    /* call out of order                               */
} isdf_status;

/* The periodic system.  Read once by isdf_plan (copied; not referenced
 * afterwards).  All pointers here are HOST pointers.
 *   lattice        row-major 3x3 lattice vectors a1, a2, a3 (bohr); must be
 *                  diagonal (orthorhombic cell), else ISDF_ERR_ARG
 *   xyz            natom x 3 Cartesian atom positions (any image)
 *   shell_*        nshell uncontracted shells: atom index, angular momentum
 *                  l in {0, 1}, Gaussian exponent alpha > 0
 *   grid           nlevel x 3 points per axis (nx, ny, nz); level 0 finest;
 *                  every count even, and per axis strictly decreasing from
 *                  one level to the next (so a coarser level's mode set is
 *                  inside every finer one)
 *   level_min_exp  nlevel-1 strictly decreasing exponent edges
 *   image_tol      image-sum truncation: on each axis a lattice translation
 *                  t is kept when the shifted centre A + t L lies within
 *                  r_cut = sqrt(ln(1/image_tol)/alpha) of [0, L]            */
typedef struct {
  double lattice[9];
  int natom;
  const double* xyz;
  int nshell;
  const int* shell_atom;
  const int* shell_l;
  const double* shell_exp;
  int nlevel;
  const int* grid;
  const double* level_min_exp;
  double image_tol;
} isdf_system;

/* Options.  Fill with isdf_options_default, then override.
 *   precision   0: every contraction in FP64 on the SIMT pipes ("plain");
 *               1: the dense contractions of the fit, the Coulomb matrix and
 *                  the exchange build on the tensor cores with FP64-accurate
 *                  sliced BF16 products (FP64 pivot decisions, Cholesky and
 *                  energy reduction are unchanged); the fit is kept in the
 *                  factored form Xi = ZC (CC^T)^-1 and the Coulomb matrix is
 *                  built as W (ZC^T v ZC) W with W = (CC^T)^-1, so the
 *                  interpolation vectors and the fit residual are computed
 *                  only when isdf_get asks for them
 *   tie_rel, tie_abs  pivot tie rule: among points whose residual is at
 *               least d_max - max(tie_rel d_max, tie_abs d_0) the smallest
 *               (level, g) wins (defaults 1e-9, 1e-13)
 *   reg_rel     fit regularisation lambda = reg_rel tr(CC^T)/k per level
 *               (default 0)
 *   col_batch   interpolation vectors per cuFFT batch (0 = automatic)
 *   timeout_ms  wall-clock budget of the selection loop, measured on the
 *               device (0 = none); exceeding it ends the loop early with
 *               ISDF_ERR_TIMEOUT
 *   prefilter   0: every grid point is a candidate.  1: exact prefilter --
 *               points whose initial residual is below a threshold tau are
 *               dropped; the call verifies that the last pivot value stays
 *               above tau plus the tie margin (then the result equals the
 *               full greedy one, residuals never grow) and otherwise repeats
 *               the selection with a lower tau (1e-5, 1e-6, 1e-9 d_0, then
 *               none; the step-by-step form starts at 1e-6).  With
 *               select_block > 0, candidates whose residual falls below tau
 *               are dropped between blocks (same pivots, fewer candidates),
 *               and an attempt stops as soon as a pivot value breaks the
 *               certificate
 *   profile     1: time every kernel family with CUDA events on the plan's
 *               stream and count its algorithmic work (isdf_profile_json)
 *   select_block  0: the selection takes one step at a time (FP64 column of
 *               M and factor-row products per step).  s in [1, 256]:
 *               speculative blocks -- the s largest local maxima of the
 *               residual on the grids form a set S, the columns that S would
 *               produce are computed for all candidates by FP64-grade
 *               tensor-core products (8 BF16 digits, exact level sums), and
 *               greedy steps finish them until a pivot falls outside S.  The
 *               pivots are the same greedy ones (every decision is the argmax
 *               over all candidates' residuals with the same tie rule); only
 *               the rounding of the factor columns differs.  Default 0.
 *   coarse_sinc 1: the coarsest level is the paper's sparse universal grid
 *               (Section III; Section III.A after Eq. 8): every one of its
 *               points is an interpolation point with the grid's sinc
 *               function as fitting function (Xi = I there), so the selection
 *               and the fit run on the finer levels only and nip counts their
 *               points; isdf_coulomb forms V over the fitted points plus
 *               V_FU = (xi_P | sinc_g) (the fitted functions' potentials on
 *               the coarse grid), and the coarse-coarse block (R_U|R_U') is
 *               never formed: isdf_exchange applies it in Fourier space
 *               (occ-RI over the coarse grid).  Needs nlevel >= 2; candidates
 *               on the coarsest level are refused.  Not with isdf_save or
 *               isdf_exchange_graph.  Default 0.
 *   local_grids 1: the finest level on atom-centred local dense grids
 *               (Section III, Eq. 5, Fig. Grids).  Atom A's grid is the
 *               finest grid's points within r_max = sqrt(-ln(local_eps_r) /
 *               alpha_min) of A, alpha_min = level_min_exp[0] (every
 *               finest-level function has alpha >= alpha_min), taken from a
 *               box of (2 r + 1)^3 points, r = floor(r_max / h) + 1 per axis,
 *               centred on A's nearest grid index floor(x / h + 1/2); box
 *               point (i, j, k), i fastest, is the parent point
 *               (c - r + i) mod n per axis.  On it L_A = the finest-level
 *               functions of A and N_A = the finest-level functions of atoms
 *               with a larger index plus every coarser function (a sharp
 *               product of two atoms lives on the lower-index atom's grid).
 *               Each atom runs its own greedy selection (Eq. 2 on w M_A, w the
 *               finest volume element; at most local_cap pivots, stopping
 *               once the largest residual is below local_tol times the atom's
 *               largest initial residual) and its own fit (Eq. 3, lambda per
 *               atom); the xi_A, zero off the sphere, are placed on the full
 *               finest grid for the Coulomb matrix.  isdf_select_points then
 *               runs the usual greedy on the coarser levels (nip and tol count
 *               those; with coarse_sinc the coarsest is the sinc grid) and
 *               returns the local pivots first, atom by atom: piv_out and
 *               dval_out must hold nip + natom * local_cap values.  Local
 *               pivot code: level 0, (atom << 24) | box index.  Needs
 *               nlevel >= 2, a box no wider than the cell, at most 255 box
 *               points per axis and 65535 atoms.  Not with isdf_save or the
 *               learned proposal.  Default 0.
 *   local_eps_r, local_tol, local_cap   defaults 1e-5 (the paper's eps_r),
 *               1e-6, 64 */
typedef struct {
  int precision;
  double tie_rel;
  double tie_abs;
  double reg_rel;
  int col_batch;
  int timeout_ms;
  int prefilter;
  int profile;
  int select_block;
  int coarse_sinc;
  int local_grids;
  double local_eps_r;
  double local_tol;
  int local_cap;
} isdf_options;

void isdf_options_default(isdf_options* opt);

/* Create a plan for one system (Section III, Fig. Grids: basis split by
 * exponent, one grid per level).  Validates the system, expands the shells,
 * assigns levels, allocates the basis tables and evaluates the basis on
 * every level.  stream: a cudaStream_t (NULL = legacy default stream).
 * On success *out receives the plan; on failure *out is NULL. */
isdf_status isdf_plan(const isdf_system* sys, const isdf_options* opt, void* stream, isdf_plan_t* out);

/* Plans for a batch of independent cells (cells of uneven size, each with
 * its own grids; the paper treats one cell at a time, so batching is an
 * extension of this library, and every plan is exactly what isdf_plan makes
 * for its cell: levels by exponent, Section II.B): isdf_plan for every systems[i] (plan i on streams[i]; a
 * NULL `streams` puts every plan on the legacy default stream), except that
 * the basis values of all cells and all levels are evaluated by one launch
 * of each basis kernel (1-D image-sum factors, then their outer products) on
 * streams[0], after which the call returns.  out: ncells plan handles.  On
 * any failure every plan already made is destroyed, out[] is all NULL and
 * isdf_last_error(NULL) names the cell.  The plans are independent
 * afterwards (select, fit, Coulomb, exchange per plan, on their streams). */
isdf_status isdf_plan_batch(const isdf_system* systems, int ncells, const isdf_options* opt, void* const* streams,
                            isdf_plan_t* out);

/* Select up to nip interpolation points (Section II.A, Eq. 2): greedy
 * pivoted Cholesky on the block-diagonal matrix (+)_l w_l M_l, with
 * M_l = A_L o A_L + 2 A_L o A_N, A_X(g,g') = sum_{mu in X} phi_mu(g)phi_mu(g'),
 * L_l = functions of level l, N_l = functions of coarser levels, and
 * w_l = Omega / N_g,l.  Stops after nip pivots or once the largest residual
 * falls below tol * d_0 (tol = 0: never).
 *   cand, ncand   optional candidate pivot codes (NULL / 0 = all points)
 *   piv_out       nip int64 pivot codes in selection order (host or device)
 *   dval_out      nip FP64 pivot values d_k (nullable)
 *   nip_out       number of pivots actually selected (host int)
 * The factor columns are freed when the call returns.  Returns
 * ISDF_ERR_TIMEOUT when the loop ran out of options.timeout_ms (the pivots
 * found so far are valid and are returned). */
isdf_status isdf_select_points(isdf_plan_t plan, int nip, double tol, const int64_t* cand, int64_t ncand,
                               int64_t* piv_out, double* dval_out, int* nip_out);

/* Fit the interpolation vectors (Section II.A, Eq. 3) for the given pivots
 * (any pivot set, e.g. the one returned by isdf_select_points):
 * Xi_l = (ZC^T)_l ((CC^T)_l + lambda I)^-1 with (ZC^T)_l = M_l[:, P_l],
 * (CC^T)_l = M_l[P_l, P_l], via an FP64 Cholesky.  Also forms X^L and X^N,
 * the basis values at the pivots.  piv: nip pivot codes (host or device);
 * duplicates or out-of-range codes give ISDF_ERR_ARG.  Internally pivots are
 * ordered level by level (selection order kept within a level); that order
 * is used by every matrix the library returns (see isdf_get). */
isdf_status isdf_fit(isdf_plan_t plan, const int64_t* piv, int nip);

/* Two-centre Coulomb matrix V_PQ = (xi_P|xi_Q) (Section II, Eq. 1) by
 * batched 3-D FFTs of the interpolation vectors: every grid function stands
 * for its trigonometric interpolant (a mode at +-n/2 on an axis is split
 * evenly between the two), the G = 0 term is dropped, and pairs on two
 * levels are summed over the coarser level's mode set.  V_out: nullable,
 * nip x nip row-major FP64 in level-ordered pivot order (host or device). */
isdf_status isdf_coulomb(isdf_plan_t plan, double* V_out);

/* Exchange matrix (Section III.A, Eq. 8) for the density D = C C^T:
 *   K_{mu nu} = sum_{lam sig} D_{lam sig} (mu lam|sig nu),
 *   (mu lam|sig nu) = sum_PQ c_{mu lam}(P) V_PQ c_{sig nu}(Q),
 *   c_{mu lam}(P) = X^L_{mu P} X^G_{lam P} + X^N_{mu P} X^L_{lam P},
 * and E_x = -Tr(D K).
 *   C      N x n row-major FP64 occupied-orbital coefficients (host/device)
 *   K_out  nullable N x N row-major FP64 (host or device)
 *   Ex_out nullable host double                                            */
isdf_status isdf_exchange(isdf_plan_t plan, const double* C, int n, double* K_out, double* Ex_out);

/* occ-RI output of the exchange build (Section III.A: only the occupied
 * block of the exchange matrix is needed; Section II.A: K_ip with real
 * orbitals):
 *   KC_{mu i} = sum_nu K_{mu nu} C_{nu i} = sum_j (mu j | j i),
 * with (mu lam|sig nu) from Eq. 8 as in isdf_exchange, and E_x =
 * -sum_{mu i} C_{mu i} KC_{mu i} = -Tr(D K).  K itself is never formed: with
 * Y_A = X^A^T C and W as in isdf_exchange, KC = [X^L X^N] (W [Y_L; Y_N]),
 * contracted over the nonzero (function level x pivot level) blocks of X^L
 * and X^N only (the block structure of (mu|xi) in the paper's figure).
 *   C       N x n row-major FP64 occupied-orbital coefficients (host/device)
 *   KC_out  nullable N x n row-major FP64 (host or device)
 *   Ex_out  nullable host double
 * Same call order and errors as isdf_exchange; may be repeated. */
isdf_status isdf_exchange_occ(isdf_plan_t plan, const double* C, int n, double* KC_out, double* Ex_out);

/* Captured exchange builds of many cells (the batched workload: the exchange
 * is the per-SCF-iteration part, with shapes fixed once the ISDF is done).
 * isdf_exchange_graph runs one exchange build per plan (each after
 * isdf_coulomb; n_occ[i] orbitals), then captures them on `stream` into one
 * CUDA graph in which every plan's build is an independent branch: isdf_exchange
 * (occ = 0, K outputs N x N) or isdf_exchange_occ (occ = 1, K C outputs N x n).
 * The graph owns device buffers for every plan's C, output and E_x.
 * isdf_exchange_graph_run copies C[i] (host or device, N_i x n_i row-major)
 * into them, launches the graph once, copies the outputs to out[i] (host or
 * device, nullable entries or NULL array) and E_x to Ex_out[i] (host,
 * nullable), and returns when `stream` is idle.  Replays may repeat with new
 * orbitals.  The plans must not be used elsewhere while a replay runs and must
 * outlive the graph; destroy the graph with isdf_exchange_graph_destroy.  A
 * tensor-core pipeline wait that expired during a replay returns
 * ISDF_ERR_TIMEOUT.  (The selection, fit and Coulomb stages are host-driven
 * loops with data-dependent shapes and are not captured.) */
typedef struct isdf_exchange_graph_s* isdf_exchange_graph_t;
isdf_status isdf_exchange_graph(isdf_plan_t* plans, int nplans, const int* n_occ, int occ, void* stream,
                                isdf_exchange_graph_t* out);
isdf_status isdf_exchange_graph_run(isdf_exchange_graph_t graph, const double* const* C, double* const* out,
                                    double* Ex_out);
void isdf_exchange_graph_destroy(isdf_exchange_graph_t graph);

/* Split-K autotuner of the tensor-core products (the launch shape the
 * library picks by measurement; not in the paper): the first product of a
 * shape outside any graph capture times every admissible split-K factor on
 * its own operands (CUDA events) and keeps the fastest for the process
 * (setting ISDF_NO_AUTOTUNE in the environment keeps the built-in
 * heuristic).  This returns the table so far as JSON text, one object per
 * shape {M, N, k_tiles, digits, sym, splits, ms}; valid until the next call
 * on this thread. */
const char* isdf_autotune_table(void);

/* Checkpoint and resume.  The ISDF runs once, before the SCF iterations
 * (Section II.B: the fit is charged once, the exchange every iteration); the
 * exchange build needs only the pivots, X^L, X^N and V.
 * isdf_save writes them to `path` (after isdf_coulomb, else ISDF_ERR_STATE):
 * "ISDFCKP1", int32 nfun, nlevel, nip, int32 grid[nlevel][3], double cell
 * edges[3], int64 pivot codes [nip] (level order), double X^L [nfun][nip],
 * X^N [nfun][nip], V [nip][nip], native byte order.
 * isdf_load reads such a file into a plan made for the same system (same
 * basis size, levels, grids and cell, else ISDF_ERR_ARG and the plan is
 * unchanged); afterwards isdf_exchange and isdf_exchange_occ run as after
 * isdf_coulomb, and the interpolation vectors are not available.  A missing,
 * truncated or malformed file gives ISDF_ERR_ARG.  `path` is a host string;
 * both calls return after the data are written / on the device. */
isdf_status isdf_save(isdf_plan_t plan, const char* path);

/* Free every buffer of a plan that the exchange build does not read (needs
 * isdf_coulomb first): the basis values and their 1-D factors (except the
 * coarsest level's with options.coarse_sinc, whose exchange reads them), the
 * fit's ZC^T, R^-1 and interpolation vectors, the spectra, residuals and
 * selection leftovers, and the local grids' per-atom buffers.  The pivots,
 * X^L, X^N and V stay: isdf_exchange, isdf_exchange_occ, isdf_exchange_graph,
 * isdf_save and isdf_get of those keep working; isdf_select_points, isdf_fit,
 * isdf_coulomb and the learned proposal return ISDF_ERR_STATE afterwards.
 * For batches of cells whose ISDF runs once before many exchange builds
 * (the paper runs the ISDF once, before the SCF iterations). */
isdf_status isdf_release_fit(isdf_plan_t plan);
isdf_status isdf_load(isdf_plan_t plan, const char* path);

/* Copy plan data out (host or device destination) for tests and tools.
 * isdf_get_size returns the number of elements (0 if not available yet). */
enum {
  ISDF_GET_NBASIS = 0,     /* int32[1]                                     */
  ISDF_GET_NIP_LEVEL = 1,  /* int32[nlevel] pivots per level               */
  ISDF_GET_PIVOTS = 2,     /* int64[nip] pivot codes, level-ordered        */
  ISDF_GET_XL = 3,         /* double[N x nip] X^L (level-ordered columns)  */
  ISDF_GET_XN = 4,         /* double[N x nip] X^N                          */
  ISDF_GET_V = 5,          /* double[nip x nip]                            */
  ISDF_GET_XI_LEVEL0 = 6,  /* double[k_l x N_g,l] Xi^T of level 0; add the
                              level index for the others (precision 1:
                              computed on the first request)               */
  ISDF_GET_NPOINTS = 4 + 16,  /* int64[1]: grid points of all levels       */
  ISDF_GET_FIT_RESIDUAL = 5 + 16, /* double[2 nlevel]: per level the largest
                              and the summed residual w (M(g,g) - M(g,P)
                              M_PP^-1 M(P,g)) over all grid points after
                              isdf_fit, i.e. the Schur complement left by the
                              pivots (sum = weighted fit error^2); on a level
                              without pivots, of w M(g,g) (precision 1:
                              computed on the first request)               */
  ISDF_GET_PHI_LEVEL0 = 10, /* double[|G_l| x N_g,l] basis values of level
                              0 (rows: functions of the level in index order,
                              then coarser ones); add the level index      */
  ISDF_GET_V_COARSE = 7 + 16,     /* double[nip x N_g,coarsest]: V_FU of
                                    options.coarse_sinc (after isdf_coulomb) */
  ISDF_GET_SELECT_STATS = 6 + 16, /* int64[3]: speculative blocks, single
                              steps and candidate compactions of the last
                              selection (0, 0, 0 when options.select_block
                              = 0)                                         */
  ISDF_GET_LOCAL_BOX = 8 + 16,  /* double[4]: options.local_grids r_max and
                              the box's points per axis                    */
  ISDF_GET_LOCAL_NIP = 9 + 16   /* int32[natom]: local pivots per atom of
                              the last fit (options.local_grids)           */
};
int64_t isdf_get_size(isdf_plan_t plan, int what);
isdf_status isdf_get(isdf_plan_t plan, int what, void* dst);

/* Kernel timing report of a plan created with options.profile = 1: a JSON
 * object {"kernels": {name: {"launches": L, "ms": T, "work": W, "unit": U}}}
 * accumulated over all calls so far (U is "flop" or "byte": the algorithmic
 * work the method needs, not what the kernel executes).  Synchronises the
 * plan's stream.  The string stays valid until the next call on the plan. */
const char* isdf_profile_json(isdf_plan_t plan);

/* Number of kernels this library has launched in this process so far (its
 * own kernels; cuFFT's are not counted).  Host-side counter; instrumentation
 * of this library with no counterpart in the paper. */
int64_t isdf_kernel_launches(void);

/* ---- Learned point proposer (not in the paper: an extension of this
 * library).  A small network (8 inputs, two hidden layers of 64 with ReLU,
 * one logistic output; 4801 FP32 parameters in the order W1 8x64, b1, W2
 * 64x64, b2, W3 64, b3) scores grid points so that isdf_select_points can
 * run on a short candidate list: the greedy of Section II.A, Eq. 2 then
 * runs over those candidates only.  The full selection stays the reference. */

int isdf_mlp_num_params(void);

/* Eight FP32 features per grid point, all levels concatenated (level 0
 * first, grid order g within a level; isdf_get_size(plan, ISDF_GET_NPOINTS)
 * points): log10 of the initial residual relative to the largest, log10 of
 * sum_L phi^2 and of sum_N phi^2, log10 |grad (sum_G phi^2)|, distances to
 * the nearest and second-nearest atom (bohr / 4), the L share of the basis
 * weight, level / (nlevel-1).  feat_out: host or device, npoints x 8. */
isdf_status isdf_features(isdf_plan_t plan, float* feat_out);

/* One training step on n samples (DEVICE pointers): class-weighted binary
 * cross entropy L = -sum_i w_i [y_i log p_i + (1-y_i) log(1-p_i)] / sum_i w_i,
 * gradient by the library's fused forward/backward kernel, then an Adam
 * update (step counts from 1; lr = 0 skips the update).  adam_m/adam_v are
 * the moment vectors (nullable when lr = 0).  loss_out: host float of the
 * loss before the update (nullable); grad_out: device copy of the gradient
 * (nullable).  X is n x 8 row-major, y and w length n. */
isdf_status isdf_mlp_train_step(float* params, float* adam_m, float* adam_v, int step, float lr, const float* X,
                                const float* y, const float* w, int64_t n, float* loss_out, float* grad_out,
                                void* stream);

/* Logits of n samples with BF16 weights and activations (FP32 sums);
 * DEVICE pointers. */
isdf_status isdf_mlp_score(const float* params, const float* X, int64_t n, float* scores, void* stream);

/* Candidate list for isdf_select_points: on every level l the quota[l]
 * highest-scoring grid points of that level (ties to the smallest g), as
 * pivot codes in ascending (level, g) order.  quota: host, nlevel entries,
 * 0 <= quota[l] <= N_g,l.  params: device.  cand_out: host or device, sum of
 * the quotas int64. */
isdf_status isdf_propose(isdf_plan_t plan, const float* params, const int64_t* quota, int64_t* cand_out);

/* After isdf_fit: on every level l the quota[l] grid points with the largest
 * fit residual w (M(g,g) - M(g,P) M_PP^-1 M(P,g)) -- the diagonal of the
 * Schur complement the pivots leave (Section II.A, Eq. 2 and 3), i.e. the
 * points the current pivots represent worst -- as pivot codes in ascending
 * (level, g) order, ties to the smallest g.  Used to repair a candidate list
 * that missed important points.  quota: host, nlevel entries, 0 <= quota[l]
 * <= N_g,l.  cand_out: host or device, sum of the quotas int64.  Before
 * isdf_fit: ISDF_ERR_STATE. */
isdf_status isdf_propose_residual(isdf_plan_t plan, const int64_t* quota, int64_t* cand_out);

/* FP64-accurate matrix product on the tensor cores -- the contraction
 * kernel behind options.precision = 1, exposed for verification and reuse
 * (the paper has no counterpart; it is this library's building block):
 *   C[m*ldc + n] = alpha * sum_k A[m*lda + k] * B[n*ldb + k]
 * A, B, C are DEVICE pointers (row-major FP64).  Each operand row is scaled
 * by a power of two and split into `slices` BF16 digit planes (5 to 8,
 * about 7 bits each).  With 5 or 6, digit-pair products accumulate in FP32
 * tensor memory per 1024-wide k chunk and are summed in double-float
 * registers; the error is below 2^-(7*slices-2) * K * max_k|A[m,k]| *
 * max_k|B[n,k]| per element.  With 7 or 8, the six leading digit levels are
 * summed exactly (512-wide chunks, integer accumulation) and the rest, below
 * 2^-42 of the result, in FP32: with 7 the error is below 2^-47 * K *
 * max_k|A[m,k]| * max_k|B[n,k]|, with 8 (FP64-grade) below 2^-52 * K *
 * max_k|A[m,k]| * max_k|B[n,k]| + 2^-53 |C[m,n]|.
 * splits > 1 divides K over that many CTAs (needs splits*M*N*8 bytes of
 * scratch, allocated by the call).  Enqueued on `stream`; returns after the
 * stream is idle.  A pipeline wait that exceeds its bound returns
 * ISDF_ERR_TIMEOUT (no fault or trap). */
isdf_status isdf_gemm_f64(const double* A, const double* B, double* C, int64_t M, int64_t N, int64_t K, int64_t lda,
                          int64_t ldb, int64_t ldc, double alpha, int slices, int splits, void* stream);

/* The same product as isdf_gemm_f64 for callers that cannot allocate device
 * memory: code inside a framework whose caching allocator owns the device's
 * memory (a cudaMalloc there can fail or fragment the pool), and paths that
 * cannot take the implicit device synchronisation of cudaMalloc/cudaFree
 * (a solver loop that must not stall other streams).  (The paper has no
 * counterpart; this is an interface of this library only.)
 * All scratch -- the BF16 digit planes of both operands, their row scales and
 * an error word -- lives in one static device array of
 * isdf_gemm_f64_noalloc_capacity() bytes (32 MiB), which every GPU that loads
 * the library holds until the process exits.  The call allocates nothing: no
 * cudaMalloc, no cudaFree, no allocating library routine.  Operands whose
 * digit planes need more than the array (about 10 (M + N) K bytes plus
 * padding) are rejected with ISDF_ERR_ARG and a message giving both sizes;
 * there is no k splitting here.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current) and
 * caches it; make that first call before any stream capture starts.  Every
 * call on a device shares the one array, so calls whose GPU work overlaps
 * (different streams or host threads) race and corrupt each other: serialise
 * them.  A, B, C must be device pointers (a host pointer is refused with
 * ISDF_ERR_ARG before anything is launched); same layout, slices and error
 * behaviour as isdf_gemm_f64, and a launch that cannot start returns
 * ISDF_ERR_CUDA.  Returns after `stream` is idle. */
isdf_status isdf_gemm_f64_noalloc(const double* A, const double* B, double* C, int64_t M, int64_t N, int64_t K,
                                  int64_t lda, int64_t ldb, int64_t ldc, double alpha, int slices, void* stream);
int64_t isdf_gemm_f64_noalloc_capacity(void);

/* Threshold-driven grids (Section III, Eq. 6; the paper's eps_K of its
 * threshold table).  A Gaussian exp(-a r^2) has the Fourier transform
 * exp(-G^2 / 4a), which falls to eps_K at G_max = sqrt(-4 a ln eps_K); a
 * grid of n points over an edge L carries wave numbers up to pi n / L.  For
 * every level l this writes, per axis, the smallest even 2^i 3^j count with
 * pi n / L >= G_max, a being the largest exponent among the functions of
 * level l (or, if it has none, among the coarser ones); then, from the
 * coarsest level up, a finer level's count is raised to the next admissible
 * size where it does not exceed the coarser level's (isdf_plan needs the
 * counts to fall from level to level).  Reads sys->lattice (diagonal),
 * nlevel, nshell, shell_exp and level_min_exp only (sys->grid may be NULL);
 * grid_out: HOST int array of nlevel x 3.  0 < eps_K < 1, else
 * ISDF_ERR_ARG; more than 4096 points per axis gives ISDF_ERR_ARG.  Host
 * computation only.  The number of interpolation points then follows the
 * paper's eps_ISDF through isdf_select_points' tol (stop once the largest
 * residual falls below tol * d_0). */
isdf_status isdf_grids_for_threshold(const isdf_system* sys, double eps_K, int* grid_out);

/* Batched 3-D real-to-half-complex DFT -- the transform behind the Coulomb
 * integrals of Section II, Eq. 1 (the half spectra that isdf_coulomb builds
 * with options.precision = 1), exposed for verification:
 *   S[b][qz][qy][qx] = sum_{z,y,x} f[b][z][y][x] exp(-2 pi i (qx x/nx + qy y/ny + qz z/nz)),
 * qx in [0, nx/2] (the unnormalised D2Z layout), computed in double-float
 * arithmetic (pairs of FP32 values, about 48 significant bits) on the FP32
 * pipes.  f: batch x nz x ny x nx FP64; S: batch x nz x ny x (nx/2+1) complex
 * FP64 (interleaved re, im); DEVICE pointers, S must not overlap f.  Every axis
 * must be 2^a 3^b <= 128, else ISDF_ERR_ARG (isdf_coulomb then uses cuFFT).
 * Enqueued on `stream`; returns after the stream is idle. */
isdf_status isdf_rfft3(const double* f, int nx, int ny, int nz, int64_t batch, double* S, void* stream);

/* Message of the last failed call on this plan (or of the last failed
 * isdf_plan when plan is NULL).  Valid until the next call. */
const char* isdf_last_error(isdf_plan_t plan);

/* Free every device buffer and the plan (resource management of this
 * library; no counterpart in the paper).  NULL is ignored. */
void isdf_destroy(isdf_plan_t plan);

#ifdef __cplusplus
}
#endif
#endif /* ISDF_H */
