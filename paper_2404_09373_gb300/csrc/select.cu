// Interpolation-point selection (kernel family (b)): greedy pivoted Cholesky on
// the block-diagonal matrix (+)_l w_l M_l (Section II.A, Eq. 2).
//
// The loop stays on the device: each step is four kernels that read and write
// a small state record, so the pivot index never travels to the host.
//   k_sel_max    d_max = max residual (atomicMax on the bit pattern, d >= 0)
//   k_sel_first  tie rule: smallest global index with d >= thr (atomicMin)
//   k_sel_pick   one thread: records the pivot, advances counters, checks the
//                stop rules and the device-clock time budget
//   k_sel_col    new factor column on the pivot's level and residual update:
//                L[g,k] = (w M(g,p) - sum_j L[g,j] L[p,j]) / sqrt(d_p),
//                d(g) -= L[g,k]^2,  L[p,k] = sqrt(d_p), d(p) = 0
// Steps are captured once into a CUDA graph and replayed.  No kernel waits on
// another; there is no spin anywhere.
#include <climits>

#include "internal.cuh"

namespace isdf {
namespace {

struct SelState {
  unsigned long long dmax_bits;
  unsigned long long first;
  double d0;
  double dp;
  long long gp;
  int lev;
  int col;
  int k;
  int done;  // no further steps
  int skip;  // this step has no pivot
  int err;
  int kl[ISDF_MAX_LEVELS];
  unsigned long long t0;
};

struct SelParams {
  double* d;
  const unsigned char* active;
  int64_t ntot;
  int nlev;
  int64_t off[ISDF_MAX_LEVELS + 1];
  double* fac[ISDF_MAX_LEVELS];
  const double* phi[ISDF_MAX_LEVELS];
  int64_t ng[ISDF_MAX_LEVELS];
  int nL[ISDF_MAX_LEVELS];
  int nG[ISDF_MAX_LEVELS];
  double w[ISDF_MAX_LEVELS];
  int64_t* piv;
  double* dval;
  int nip;
  double tol, tie_rel, tie_abs;
  unsigned long long timeout_ns;
};

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <class T, class Op>
__device__ __forceinline__ T block_reduce(T v, Op op, T* sh) {
  for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (wid == 0) {
    v = (lane < nw) ? sh[lane] : sh[0];
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;
}

struct MaxOp {
  __device__ double operator()(double a, double b) const { return fmax(a, b); }
};
struct MinOp {
  __device__ unsigned long long operator()(unsigned long long a, unsigned long long b) const { return a < b ? a : b; }
};

// w_l M_l(g, g) = w (aL^2 + 2 aL aN), aX = sum_{mu in X} phi_mu(g)^2
__global__ void k_sel_diag(const double* __restrict__ phi, int64_t ng, int nL, int nG, double w,
                           const unsigned char* __restrict__ act, double* __restrict__ d) {
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < ng; g += int64_t(gridDim.x) * blockDim.x) {
    double aL = 0.0, aN = 0.0;
    for (int r = 0; r < nL; ++r) {
      const double v = phi[int64_t(r) * ng + g];
      aL = fma(v, v, aL);
    }
    for (int r = nL; r < nG; ++r) {
      const double v = phi[int64_t(r) * ng + g];
      aN = fma(v, v, aN);
    }
    const double m = w * (aL * (aL + 2.0 * aN));
    d[g] = (act && !act[g]) ? 0.0 : m;
  }
}

__global__ void k_sel_max(SelParams P, SelState* st) {
  if (st->done) return;
  __shared__ double sh[32];
  double m = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < P.ntot; i += int64_t(gridDim.x) * blockDim.x)
    m = fmax(m, P.d[i]);
  m = block_reduce(m, MaxOp(), sh);
  if (threadIdx.x == 0) atomicMax(&st->dmax_bits, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_sel_first(SelParams P, SelState* st) {
  if (st->done) return;
  __shared__ unsigned long long sh[32];
  const double dmax = __longlong_as_double((long long)st->dmax_bits);
  const int k = st->k;
  const double d0 = (k == 0) ? dmax : st->d0;
  const bool stop = (k >= P.nip) || !(dmax > 0.0) || (dmax < P.tol * d0);
  if (stop) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->done = 1;
      st->skip = 1;
    }
    return;
  }
  const double thr = dmax - fmax(P.tie_rel * dmax, P.tie_abs * d0);
  unsigned long long best = ULLONG_MAX;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < P.ntot; i += int64_t(gridDim.x) * blockDim.x) {
    const double v = P.d[i];
    if (v >= thr && v > 0.0) {
      best = (unsigned long long)i;
      break;  // grid-stride order: the first hit is this thread's smallest
    }
  }
  best = block_reduce(best, MinOp(), sh);
  if (threadIdx.x == 0 && best != ULLONG_MAX) atomicMin(&st->first, best);
}

__global__ void k_sel_pick(SelParams P, SelState* st) {
  if (threadIdx.x != 0 || st->done) return;
  const unsigned long long idx = st->first;
  if (idx == ULLONG_MAX) {  // nothing qualified (cannot happen with dmax > 0)
    st->done = 1;
    st->skip = 1;
    return;
  }
  int l = 0;
  while (l + 1 < P.nlev && (long long)idx >= P.off[l + 1]) ++l;
  const long long g = (long long)idx - P.off[l];
  const double dp = P.d[idx];
  const int k = st->k;
  if (k == 0) st->d0 = __longlong_as_double((long long)st->dmax_bits);
  st->lev = l;
  st->gp = g;
  st->dp = dp;
  st->col = st->kl[l];
  P.piv[k] = ((long long)l << kPivShift) | g;
  P.dval[k] = dp;
  st->kl[l] += 1;
  st->k = k + 1;
  st->skip = 0;
  st->dmax_bits = 0ull;
  st->first = ULLONG_MAX;
  if (P.timeout_ns) {
    const unsigned long long now = globaltimer();
    if (k == 0) {
      st->t0 = now;
    } else if (now - st->t0 > P.timeout_ns) {
      st->err = ISDF_ERR_TIMEOUT;
      st->done = 1;  // this step's column is still computed
    }
  }
}

__global__ __launch_bounds__(256) void k_sel_col(SelParams P, const SelState* st) {
  if (st->skip) return;
  extern __shared__ double cp[];  // phi_G(p)
  const int l = st->lev;
  const int64_t gp = st->gp;
  const int col = st->col;
  const double dp = st->dp;
  const int64_t ng = P.ng[l];
  const int nL = P.nL[l], nG = P.nG[l];
  const double* __restrict__ phi = P.phi[l];
  double* __restrict__ fac = P.fac[l];
  double* __restrict__ d = P.d + P.off[l];
  const unsigned char* act = P.active ? P.active + P.off[l] : nullptr;
  for (int r = threadIdx.x; r < nG; r += blockDim.x) cp[r] = phi[int64_t(r) * ng + gp];
  __syncthreads();
  const double sq = sqrt(dp);
  const double w = P.w[l];
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < ng; g += int64_t(gridDim.x) * blockDim.x) {
    double aL = 0.0, aN = 0.0;
    for (int r = 0; r < nL; ++r) aL = fma(phi[int64_t(r) * ng + g], cp[r], aL);
    for (int r = nL; r < nG; ++r) aN = fma(phi[int64_t(r) * ng + g], cp[r], aN);
    const double m = w * (aL * (aL + 2.0 * aN));
    double s = 0.0;
    for (int j = 0; j < col; ++j) s = fma(fac[int64_t(j) * ng + g], __ldg(&fac[int64_t(j) * ng + gp]), s);
    double v = (m - s) / sq;
    const bool inactive = act && !act[g];
    if (g == gp) v = sq;
    if (inactive) v = 0.0;
    fac[int64_t(col) * ng + g] = v;
    if (g == gp)
      d[g] = 0.0;
    else if (!inactive)
      d[g] = d[g] - v * v;
  }
}

}  // namespace

isdf_status select_run(Plan* p, int nip, double tol, const std::vector<int64_t>* cand, int* nfound) {
  cudaStream_t s = p->stream;
  isdf_status st;
  // (re)allocate selection buffers
  dfree(p->d_diag);
  p->d_diag = nullptr;
  dfree(p->d_active);
  p->d_active = nullptr;
  dfree(p->d_piv);
  p->d_piv = nullptr;
  dfree(p->d_dval);
  p->d_dval = nullptr;
  if (!p->d_selstate) {
    st = dalloc(p, &p->d_selstate, sizeof(SelState), "selection state");
    if (st) return st;
  }
  if ((st = dalloc_t(p, &p->d_diag, size_t(p->ntot), "residual diagonal"))) return st;
  if ((st = dalloc_t(p, &p->d_piv, size_t(nip), "pivots"))) return st;
  if ((st = dalloc_t(p, &p->d_dval, size_t(nip), "pivot values"))) return st;
  if (cand) {
    std::vector<unsigned char> act(size_t(p->ntot), 0);
    for (int64_t c : *cand) {
      const int l = int(c >> kPivShift);
      const int64_t g = c & kPivMask;
      act[size_t(p->off[l] + g)] = 1;
    }
    if ((st = dalloc_t(p, &p->d_active, size_t(p->ntot), "candidate mask"))) return st;
    if ((st = cuda_check(p, cudaMemcpyAsync(p->d_active, act.data(), act.size(), cudaMemcpyHostToDevice, s), "copy")))
      return st;
    if ((st = cuda_check(p, cudaStreamSynchronize(s), "copy candidates"))) return st;
  }
  for (int l = 0; l < p->nlev; ++l) {
    Level& lv = p->lev[l];
    dfree(lv.fac);
    lv.fac = nullptr;
    lv.fac_cap = std::min<int64_t>(nip, lv.ng);
    if ((st = dalloc_t(p, &lv.fac, size_t(lv.fac_cap) * size_t(lv.ng), "selection factor columns"))) return st;
  }
  SelParams P{};
  P.d = p->d_diag;
  P.active = p->d_active;
  P.ntot = p->ntot;
  P.nlev = p->nlev;
  for (int l = 0; l <= p->nlev; ++l) P.off[l] = p->off[l];
  int nGmax = 1;
  for (int l = 0; l < p->nlev; ++l) {
    Level& lv = p->lev[l];
    P.fac[l] = lv.fac;
    P.phi[l] = lv.phi;
    P.ng[l] = lv.ng;
    P.nL[l] = lv.nL;
    P.nG[l] = lv.nG;
    P.w[l] = lv.w;
    nGmax = std::max(nGmax, lv.nG);
    Prof pr(p, "select_diag", 2.0 * double(lv.nG) * double(lv.ng), "flop", 1);
    k_sel_diag<<<152 * 8, 256, 0, s>>>(lv.phi, lv.ng, lv.nL, lv.nG, lv.w,
                                       p->d_active ? p->d_active + p->off[l] : nullptr, p->d_diag + p->off[l]);
  }
  P.piv = p->d_piv;
  P.dval = p->d_dval;
  P.nip = nip;
  P.tol = tol;
  P.tie_rel = p->opt.tie_rel;
  P.tie_abs = p->opt.tie_abs;
  P.timeout_ns = (unsigned long long)p->opt.timeout_ms * 1000000ull;
  SelState h{};
  h.dmax_bits = 0;
  h.first = ULLONG_MAX;
  h.skip = 1;
  if ((st = cuda_check(p, cudaMemcpyAsync(p->d_selstate, &h, sizeof(h), cudaMemcpyHostToDevice, s), "state init")))
    return st;
  SelState* dst = static_cast<SelState*>(p->d_selstate);
  const size_t smem = sizeof(double) * size_t(nGmax);
  if (smem > 48 * 1024) {
    if ((st = cuda_check(p, cudaFuncSetAttribute(k_sel_col, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)),
                         "smem attribute")))
      return st;
  }
  const unsigned red_blocks = 152 * 4, col_blocks = 152 * 8;
  auto one_step = [&]() {
    k_sel_max<<<red_blocks, 256, 0, s>>>(P, dst);
    k_sel_first<<<red_blocks, 256, 0, s>>>(P, dst);
    k_sel_pick<<<1, 32, 0, s>>>(P, dst);
    k_sel_col<<<col_blocks, 256, smem, s>>>(P, dst);
  };
  // Capture a chunk of steps into a graph (not possible on the legacy stream).
  const int chunk = 32;
  bool graphed = false;
  Prof* loop_prof = new Prof(p, "select_loop", 0.0, "flop", 4ll * nip);
  if (s != nullptr && nip >= chunk) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      for (int i = 0; i < chunk; ++i) one_step();
      if (cudaStreamEndCapture(s, &graph) == cudaSuccess && graph &&
          cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
        graphed = true;
        const int full = nip / chunk;
        for (int c = 0; c < full; ++c) cudaGraphLaunch(exec, s);
        for (int i = full * chunk; i < nip; ++i) one_step();
      }
      if (exec) {
        cudaStreamSynchronize(s);
        cudaGraphExecDestroy(exec);
      }
      if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();  // a failed capture leaves a sticky-free error; clear it
  }
  if (!graphed)
    for (int i = 0; i < nip; ++i) one_step();
  delete loop_prof;  // records the end event; work is filled in below
  if ((st = cuda_check(p, cudaGetLastError(), "selection kernels"))) return st;
  if ((st = cuda_check(p, cudaMemcpyAsync(&h, p->d_selstate, sizeof(h), cudaMemcpyDeviceToHost, s), "state copy")))
    return st;
  if ((st = cuda_check(p, cudaStreamSynchronize(s), "selection"))) return st;
  *nfound = h.k;
  if (p->opt.profile && !p->pend.empty() && p->pend.back().name == "select_loop") {
    // algorithmic flops: step c on level l costs 2 (nG + c) ng (M column and
    // the factor-row dot product)
    double work = 0.0;
    for (int l = 0; l < p->nlev; ++l) {
      const double k = h.kl[l], ng = double(p->lev[l].ng), nG = p->lev[l].nG;
      work += 2.0 * ng * (nG * k + 0.5 * k * (k - 1.0));
    }
    p->pend.back().work = work;
  }
  // the factor columns are not needed after selection
  for (int l = 0; l < p->nlev; ++l) {
    dfree(p->lev[l].fac);
    p->lev[l].fac = nullptr;
  }
  if (h.err == ISDF_ERR_TIMEOUT) return fail(p, ISDF_ERR_TIMEOUT, "selection loop exceeded options.timeout_ms");
  return ISDF_OK;
}

}  // namespace isdf
