// Internal declarations of the multigrid ISDF library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "isdf.h"

namespace isdf {

constexpr int kPivShift = 40;
constexpr int64_t kPivMask = (int64_t(1) << kPivShift) - 1;

// One real-space grid level (Section III, Fig. Grids).
struct Level {
  int n[3] = {0, 0, 0};  // points per axis
  int64_t ng = 0;        // points
  double w = 0.0;        // volume element Omega / ng (selection weight)
  std::vector<int> L;    // functions of this level
  std::vector<int> N;    // functions of coarser levels
  int nL = 0, nN = 0, nG = 0;
  // a box of a finer full grid (an atom's local grid): point (i, j, k) is the
  // parent point ((o + i) mod pn) per axis; pn[0] == 0 for a full-cell grid.
  // Basis values are zero outside the sphere |(o + i) h - mc| <= r (mr2 = r^2,
  // h = edge / pn); mr2 < 0: no sphere
  int o[3] = {0, 0, 0};
  int pn[3] = {0, 0, 0};
  double mc[3] = {0.0, 0.0, 0.0};
  double mr2 = -1.0;
  double* tab[3] = {nullptr, nullptr, nullptr};  // 1-D factors [nG][n[a]]
  double* phi = nullptr;                         // basis values [nG][ng]
  // selection factor columns [fac_cap][ng]
  double* fac = nullptr;
  int64_t fac_cap = 0;
  // fit
  int k = 0;                 // pivots on this level
  std::vector<int64_t> pg;   // pivot grid indices (selection order)
  int64_t* d_pg = nullptr;
  double* xiT = nullptr;     // Xi^T [k][ng] (precision 1: made on request from zct and rinv)
  float* resid = nullptr;    // fit residual per grid point (FP32 copy, for proposals)
  // precision 1 keeps the fit in factored form, Xi = ZC W with W = R^-T R^-1:
  double* zct = nullptr;     // ZC^T [k][ng]
  double* rinv = nullptr;    // R^-1 [k][k], lower triangular (CC^T = R R^T)
  // Coulomb
  int nh[3] = {0, 0, 0};     // half-spectrum dims (nx/2+1, ny, nz)
  int64_t nq = 0;            // half-spectrum modes
  double2* spec = nullptr;   // [k][nq]
};

// Kernel timing (options.profile): CUDA events around launch groups.
struct ProfEvent {
  std::string name;
  cudaEvent_t a = nullptr, b = nullptr;
  double work = 0.0;
  const char* unit = "flop";
  int64_t launches = 0;
  double flop = 0.0;  // FP64-equivalent flops of a byte-counted tensor-core family (else 0)
};
struct KStat {
  int64_t launches = 0;
  double ms = 0.0, work = 0.0, flop = 0.0;
  std::string unit;
};

extern std::atomic<long long> g_launches;
extern thread_local long long t_launches;  // this host thread's share of g_launches
inline void count_launches(long long n) {
  g_launches.fetch_add(n, std::memory_order_relaxed);
  t_launches += n;
}

struct Plan {
  cudaStream_t stream = nullptr;
  isdf_options opt{};
  double edge[3] = {0, 0, 0};
  double omega = 0.0;
  double image_tol = 1e-10;
  int natom = 0;
  std::vector<double> xyz;
  int nfun = 0;
  std::vector<int> f_atom, f_l[3], f_level;
  std::vector<double> f_alpha, f_norm;
  int nlev = 0;
  Level lev[ISDF_MAX_LEVELS];
  int state = 0;  // 0 planned, 1 selected, 2 fitted, 3 Coulomb done
  bool released = false;  // isdf_release_fit: only the exchange's inputs remain
  // selection (all levels concatenated)
  int64_t ntot = 0;
  int64_t off[ISDF_MAX_LEVELS + 1] = {0};
  double* d_diag = nullptr;    // residual diagonal [ntot]
  void* d_selstate = nullptr;
  int64_t* d_piv = nullptr;    // selection-order pivot codes
  double* d_dval = nullptr;
  int sel_cap = 0;
  int64_t sel_blocks = 0, sel_plain_steps = 0;  // speculative-block statistics of the last selection
  int64_t sel_compactions = 0;                   // candidate compactions of the last selection
  // fit results, level-ordered pivots
  int nip = 0;
  int poff[ISDF_MAX_LEVELS + 1] = {0};
  std::vector<int64_t> piv_lo;  // level-ordered pivot codes
  double* XL = nullptr;         // [N][nip]
  double* XN = nullptr;
  double* V = nullptr;          // [nip][nip]
  int* d_err = nullptr;         // device error word (Cholesky breakdown etc.)
  int* d_ozerr = nullptr;       // tensor-core pipeline error word
  double fit_resid[2 * ISDF_MAX_LEVELS] = {0};  // per level: max and sum of the fit residual
  bool resid_ready = false;     // fit_resid / lev[].resid computed for the current fit
  std::string err;
  std::string fault;            // host fault injection (ISDF_FAULT)
  // exchange build: function level order on the device (made by the first
  // exchange), and the capture mode of isdf_exchange_graph (no host
  // synchronisation, no pageable copies, E_x written to *d_ex_slot)
  int* d_perm = nullptr;
  double* VFU = nullptr;  // options.coarse_sinc: (xi_P | sinc_g) [nip][N_g of the coarsest level]
  bool capturing = false;
  double* d_ex_slot = nullptr;
  // options.local_grids: level 0 on atom-centred local grids (Section III,
  // Eq. 5).  One single-level sub-plan per atom holds its box, basis values,
  // selection and fit; level 0 of this plan holds no basis values, only the
  // assembled fit on the full finest grid (for the Coulomb matrix).
  std::vector<Plan*> sub;
  double r_max = 0.0;
  int sel_lo = 0;  // first level of this plan's own greedy selection
  // BF16 digits of the fit's tensor-core products: 5 for the full-cell levels;
  // 8 (FP64-grade) on an atom's local grid, where a threshold-driven
  // selection can leave CC^T conditioned beyond 1e9
  int fit_slices = 5;
  // profiling
  std::vector<ProfEvent> pend;
  std::map<std::string, KStat> stats;
  std::string prof_json;
};

// RAII timer of one launch group on the plan's stream (no-op unless profiling).
// launches >= 0: the group's launches, counted here; kLaunchesInside: the
// group's kernels count themselves and the timer records how many ran.
constexpr int64_t kLaunchesInside = -1;
struct Prof {
  Plan* p;
  ProfEvent e;
  long long t0 = 0;
  Prof(Plan* p_, const char* name, double work, const char* unit, int64_t launches);
  ~Prof();
};
void prof_flush(Plan* p);  // resolve pending events (stream must be idle)
isdf_status oz_check(Plan* p);  // sync; ISDF_ERR_TIMEOUT if a tensor-core wait expired

// ---- helpers (api.cu) ----
isdf_status fail(Plan* p, isdf_status s, const std::string& msg);
isdf_status cuda_check(Plan* p, cudaError_t e, const char* what);
isdf_status dalloc(Plan* p, void** ptr, size_t bytes, const char* what);
template <class T>
inline isdf_status dalloc_t(Plan* p, T** ptr, size_t n, const char* what) {
  return dalloc(p, reinterpret_cast<void**>(ptr), n * sizeof(T), what);
}
void dfree(void* ptr);
bool is_device_ptr(const void* ptr);

// ---- kernels / stages ----
isdf_status basis_build(Plan* p);                                    // basis.cu
isdf_status basis_alloc(Plan* p);                                    // basis.cu
isdf_status basis_eval(Plan* const* plans, int nplans, cudaStream_t s);  // basis.cu: one launch per kernel
isdf_status select_run(Plan* p, int nip, double tol, const std::vector<int64_t>* cand, int* nfound);  // select.cu
isdf_status fit_run(Plan* p);                                        // fit.cu
isdf_status fit_residual_run(Plan* p);  // fit.cu: residual statistics on request (precision 1)
isdf_status fit_xi_run(Plan* p, int level);  // fit.cu: Xi^T of a level on request (precision 1)
isdf_status coulomb_run(Plan* p);                                    // coulomb.cu
// the coarsest level as the universal sinc grid (sinc.cu)
isdf_status sinc_coulomb(Plan* p);
isdf_status sinc_exchange(Plan* p, const double* dC, const double* yl, const double* yg, int n, double* dK);
// coulomb.cu helpers shared with sinc.cu
void fold_spectra(int k, const double2* spf, int fx, int fy, int fz, double2* H, int cx, int cy, int cz,
                  cudaStream_t s);
isdf_status transform_real(Plan* p, const double* f, int nx, int ny, int nz, int64_t batch, double2* spec);
// the exchange build's tensor-core product C = A B^T over strided operands (exchange.cu)
isdf_status tc_product_ex(Plan* p, const double* a, int64_t M, int64_t sar, int64_t sak, const double* b, int64_t N,
                        int64_t sbr, int64_t sbk, int64_t K, double* C, int64_t ldc);
// dK (N x N) and dKC (N x n, K C) are nullable; exchange.cu
isdf_status exchange_run(Plan* p, const double* dC, int n, double* dK, double* dKC, double* Ex);
isdf_status gather_pivot_factors(Plan* p);                           // basis.cu
// local grids (local.cu)
constexpr int kLocalAtomShift = 24;  // local pivot code on level 0: (atom << 24) | box index
isdf_status local_setup(Plan* p, double alpha_min);  // alpha_min: the finest level's edge
bool local_inside(const Plan* q, int64_t b);  // box point b of sub-plan q inside its sphere
isdf_status local_select(Plan* p, std::vector<int64_t>& piv, std::vector<double>& dval);
isdf_status local_fit(Plan* p, const std::vector<std::vector<int64_t>>& per_atom);  // sub-plan fits
isdf_status local_assemble(Plan* p);  // level 0 of p from the sub-plans' fits (after fit_run(p))

// FP64 SIMT GEMM (dgemm.cu):
//   C[m][n] = alpha * sum_k opA(m,k) w(k) opB(k,n) + beta * C[m][n]
//   opA(m,k) = ta ? A[k*lda+m] : A[m*lda+k];  opB(k,n) = tb ? B[n*ldb+k] : B[k*ldb+n]
//   tri: 0 dense, 1 opA lower triangular (k <= m), 2 opA upper triangular (k >= m)
//   sym: only output tiles on or below the diagonal are computed
struct GemmArgs {
  int ta = 0, tb = 0;
  int64_t M = 0, N = 0, K = 0;
  double alpha = 1.0, beta = 0.0;
  const double* A = nullptr;
  int64_t lda = 0;
  const double* B = nullptr;
  int64_t ldb = 0;
  double* C = nullptr;
  int64_t ldc = 0;
  const double* kw = nullptr;
  int tri = 0;
  int sym = 0;
};
void dgemm(const GemmArgs& g, cudaStream_t s);
// ZC^T = A_L o (A_L + 2 A_N) with A_X = PhiP_X^T Phi_X (fit.cu uses it)
void zc_gemm(int64_t k, int64_t ng, int nL, int nG, const double* phiP, const double* phi, double* out,
             cudaStream_t s);
// lower Cholesky in place (row-major n x n, lda); breakdown column -> *err
void dpotrf_lower(double* A, int64_t n, int64_t lda, int* err, double* scratch, cudaStream_t s);
// inverse of a lower-triangular matrix: Li (n x n, zero-initialised by callee);
// with a plan (tensor-core precision) the large off-diagonal products run as
// FP64-grade 8-digit tensor-core products, their error flag the plan's
struct Plan;
void dtrtri_lower(const double* Lm, double* Li, int64_t n, double* scratch, cudaStream_t s, Plan* tc = nullptr);

// FP64-accurate GEMM from sliced BF16 products on tcgen05 (ozgemm.cu).
// An operand is rows x K, pre-sliced into S BF16 digit planes (S = 5 or 6)
// and pre-tiled for the tensor cores; A operands use row tiles of 128, B
// operands row tiles of oz_bn(S).
// Two-level index map i -> (i / in) so + (i % in) si (in = 0: i si) of
// operand rows / k values and result rows / columns (plain strides today).
struct OzMap {
  int64_t in = 0, so = 0, si = 1;
};
inline OzMap oz_stride(int64_t st) {
  OzMap m;
  m.si = st;
  return m;
}
constexpr int kOzBK = 32;  // k values per digit tile (two K = 16 tcgen05.mma steps, one pipeline stage)
struct OzOperand {
  void* tiles = nullptr;  // __nv_bfloat16 slices
  int* exps = nullptr;    // per-row power-of-two scale
  int64_t rows = 0, K = 0, nrt = 0, nkt = 0;
  int64_t kst = 0;        // k-tile stride of the tile array (capacity in k tiles)
  int rt = 0, S = 0;
};
int oz_bn(int S);
isdf_status oz_alloc(Plan* p, OzOperand& op, int64_t rows, int64_t K, int rt, int S, const char* what);
int64_t oz_tile_bytes(const OzOperand& op);  // bytes of the whole tile array
void oz_free(OzOperand& op);
// X(r, k) = mul * kw[k] * src[r*sr + k*sk]  (kw nullable)
void oz_slice(const double* src, int64_t sr, int64_t sk, const double* kw, double mul, OzOperand& op, cudaStream_t s);
// Gathered rows (row r = source row ridx[r], ridx nullable) and a window
// [kg0, kg1) of 8-wide k groups of an operand allocated for op.kst k tiles;
// op.K is the current K (entries at k >= op.K are written as zero).
// exps_ready: the row scales are already in op.exps (they must bound every
// |x| the operand will ever hold).  Groups outside the window are untouched.
// the same digits in another row-tile height (same rows, K, S and k tiles);
// copies lines of 8 rows instead of slicing the FP64 source again
void oz_retile(const OzOperand& from, OzOperand& to, cudaStream_t s);
void oz_slice_ex(const double* src, int64_t sr, int64_t sk, const int* ridx, OzOperand& op, int64_t kg0, int64_t kg1,
                 bool exps_ready, cudaStream_t s);
// C = alpha * A B^T (A: M x K as the 128-row side, B: N x K); trans: C[n*ldc+m];
// tri 1/2: B-side lower/upper triangular in (n, k); sym: lower-triangle tiles only;
// splits > 1 needs work of splits*M*N doubles.  Error codes go to *err.
void oz_gemm(const OzOperand& A, const OzOperand& B, double* C, int64_t ldc, int trans, double alpha, int tri, int sym,
             int splits, double* work, int* err, cudaStream_t s);
int64_t oz_tile_elems(int64_t rows, int64_t K, int rt, int S);
// the same product with its scratch in a fixed static device array (no allocation)
// split-K factor of a product shape: cached, else timed on these operands
// (outside graph capture; ISDF_NO_AUTOTUNE keeps the heuristic)
int oz_tuned_splits(Plan* p, const OzOperand& A, const OzOperand& B, double* C, int64_t ldc, int trans, int sym,
                    int heuristic, cudaStream_t s);
std::string oz_tune_json();
size_t gemm_noalloc_capacity();
isdf_status gemm_noalloc(const double* A, const double* B, double* C, int64_t M, int64_t N, int64_t K, int64_t lda,
                         int64_t ldb, int64_t ldc, double alpha, int slices, cudaStream_t s, std::string& why);

// batched 3-D real-to-half-complex transform in double-float arithmetic (fft.cu):
// f batch x (nz ny nx) FP64 -> S batch x (nz ny (nx/2+1)) double2, D2Z layout;
// every axis 2^a 3^b <= 128 (rfft3_df_supported), else ISDF_ERR_ARG
bool rfft3_df_supported(int nx, int ny, int nz);
isdf_status rfft3_df(Plan* p, const double* f, int nx, int ny, int nz, int64_t batch, double2* S, cudaStream_t s);

// learned point proposer (learn.cu)
int mlp_num_params();
isdf_status learn_features(Plan* p, float* dfeat);
isdf_status learn_propose_residual(Plan* p, const int64_t* quota, int64_t* dcand);
isdf_status mlp_grad_step(float* params, float* m, float* v, int step, float lr, const float* X, const float* y,
                          const float* w, int64_t n, float* loss_host, float* grad_dev, cudaStream_t s,
                          std::string& why);
void mlp_score(const float* params, const float* X, int64_t n, float* out, cudaStream_t s);
isdf_status learn_propose(Plan* p, const float* params, const int64_t* quota, int64_t* dcand);

}  // namespace isdf
