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
//
// Candidates.  Every level works on a compacted, ascending list of candidate
// grid points (all points, a caller-given list, or the exact prefilter), so
// the factor columns, the residual and every step scale with the number of
// candidates.  Exact prefilter: a point whose initial residual is below tau
// can never be picked while every pivot value stays above tau plus the tie
// margin, because residuals only shrink; the host checks that certificate on
// the returned pivot values and otherwise repeats with a lower tau.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace isdf {
namespace {

struct SelState {
  unsigned long long dmax_bits;
  unsigned long long first;
  double d0;
  double dp;
  long long gp;  // grid index of this step's pivot
  long long tp;  // its position in the level's candidate list
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
  double* d;  // residual over all levels' candidates (concatenated)
  int64_t ntot;
  int nlev;
  int64_t coff[ISDF_MAX_LEVELS + 1];  // candidate offsets per level
  const int* cidx[ISDF_MAX_LEVELS];   // candidate grid indices (nullptr: all points)
  int64_t nc[ISDF_MAX_LEVELS];
  double* fac[ISDF_MAX_LEVELS];       // factor columns [col][nc]
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

// w_l M_l(g, g) = w (aL^2 + 2 aL aN), aX = sum_{mu in X} phi_mu(g)^2, every grid point
__global__ void k_sel_diag(const double* __restrict__ phi, int64_t ng, int nL, int nG, double w,
                           double* __restrict__ d) {
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
    d[g] = w * (aL * (aL + 2.0 * aN));
  }
}

// max of a vector into a scalar slot (slot preset to 0; values >= 0 compare as bits)
__global__ void k_vec_max(const double* __restrict__ v, int64_t n, unsigned long long* out) {
  __shared__ double sh[32];
  double m = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    m = fmax(m, v[i]);
  m = block_reduce(m, MaxOp(), sh);
  if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// ordered compaction of {g : d0[g] >= tau}: per-block counts, then scatter
constexpr int kCompactBlock = 1024;
__global__ void k_flag_count(const double* __restrict__ d0, int64_t ng, double tau, int* __restrict__ counts) {
  __shared__ int sh[32];
  const int64_t g = int64_t(blockIdx.x) * kCompactBlock + threadIdx.x;
  const int f = (g < ng && d0[g] >= tau) ? 1 : 0;
  const unsigned b = __ballot_sync(0xffffffffu, f);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    int c = 0;
    for (int i = 0; i < kCompactBlock / 32; ++i) c += sh[i];
    counts[blockIdx.x] = c;
  }
}

__global__ void k_compact(const double* __restrict__ d0, int64_t ng, double tau, const int* __restrict__ block_off,
                          int* __restrict__ cidx) {
  __shared__ int warp_off[32];
  const int64_t g = int64_t(blockIdx.x) * kCompactBlock + threadIdx.x;
  const int f = (g < ng && d0[g] >= tau) ? 1 : 0;
  const unsigned b = __ballot_sync(0xffffffffu, f);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) warp_off[wid] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int i = 0; i < kCompactBlock / 32; ++i) {
      const int c = warp_off[i];
      warp_off[i] = acc;
      acc += c;
    }
  }
  __syncthreads();
  if (f) cidx[block_off[blockIdx.x] + warp_off[wid] + __popc(b & ((1u << lane) - 1u))] = int(g);
}

// residual over the candidates of one level
__global__ void k_gather_diag(const double* __restrict__ d0, const int* __restrict__ cidx, int64_t nc,
                              double* __restrict__ d) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < nc) d[t] = d0[cidx ? cidx[t] : t];
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
  while (l + 1 < P.nlev && (long long)idx >= P.coff[l + 1]) ++l;
  const long long t = (long long)idx - P.coff[l];
  const long long g = P.cidx[l] ? P.cidx[l][t] : t;
  const double dp = P.d[idx];
  const int k = st->k;
  if (k == 0) st->d0 = __longlong_as_double((long long)st->dmax_bits);
  st->lev = l;
  st->gp = g;
  st->tp = t;
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

// One block works on 32 candidate points at a time (one point per lane, so
// every load is a coalesced row segment); its 8 warps split the basis
// functions and factor columns 8 ways and the partial dot products are added
// in shared memory in a fixed order.  Grid-striding over 32-point groups keeps
// every SM equally busy whatever the number of candidates.
constexpr int kColWarps = 8;
__global__ __launch_bounds__(32 * kColWarps) void k_sel_col(SelParams P, const SelState* st) {
  if (st->skip) return;
  extern __shared__ double sm[];
  const int l = st->lev;
  const int nL = P.nL[l], nG = P.nG[l];
  double* cp = sm;                                 // phi_G(p)
  double* part = sm + ((nG + 1) & ~1);             // [3][kColWarps][32]
  const int64_t gp = st->gp, tp = st->tp;
  const int col = st->col;
  const double dp = st->dp;
  const int64_t ng = P.ng[l], nc = P.nc[l];
  const int* __restrict__ cidx = P.cidx[l];
  const double* __restrict__ phi = P.phi[l];
  double* __restrict__ fac = P.fac[l];
  double* __restrict__ d = P.d + P.coff[l];
  for (int r = threadIdx.x; r < nG; r += blockDim.x) cp[r] = phi[int64_t(r) * ng + gp];
  __syncthreads();
  const double sq = sqrt(dp);
  const double w = P.w[l];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ngroups = (nc + 31) / 32;
  for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int64_t t = grp * 32 + lane;
    const bool valid = t < nc;
    double aL = 0.0, aN = 0.0, s = 0.0;
    if (valid) {
      const int64_t g = cidx ? cidx[t] : t;
      // independent partial sums keep several loads and FMAs in flight
      double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
      int r = warp;
      for (; r + kColWarps < nL; r += 2 * kColWarps) {
        a0 = fma(phi[int64_t(r) * ng + g], cp[r], a0);
        a1 = fma(phi[int64_t(r + kColWarps) * ng + g], cp[r + kColWarps], a1);
      }
      if (r < nL) a0 = fma(phi[int64_t(r) * ng + g], cp[r], a0);
      r = nL + warp;
      for (; r + kColWarps < nG; r += 2 * kColWarps) {
        b0 = fma(phi[int64_t(r) * ng + g], cp[r], b0);
        b1 = fma(phi[int64_t(r + kColWarps) * ng + g], cp[r + kColWarps], b1);
      }
      if (r < nG) b0 = fma(phi[int64_t(r) * ng + g], cp[r], b0);
      aL = a0 + a1;
      aN = b0 + b1;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      const double* fp = fac + tp;
      const double* ft = fac + t;
      int j = warp;
      for (; j + 3 * kColWarps < col; j += 4 * kColWarps) {
        s0 = fma(ft[int64_t(j) * nc], fp[int64_t(j) * nc], s0);
        s1 = fma(ft[int64_t(j + kColWarps) * nc], fp[int64_t(j + kColWarps) * nc], s1);
        s2 = fma(ft[int64_t(j + 2 * kColWarps) * nc], fp[int64_t(j + 2 * kColWarps) * nc], s2);
        s3 = fma(ft[int64_t(j + 3 * kColWarps) * nc], fp[int64_t(j + 3 * kColWarps) * nc], s3);
      }
      for (; j < col; j += kColWarps) s0 = fma(ft[int64_t(j) * nc], fp[int64_t(j) * nc], s0);
      s = (s0 + s1) + (s2 + s3);
    }
    part[(0 * kColWarps + warp) * 32 + lane] = aL;
    part[(1 * kColWarps + warp) * 32 + lane] = aN;
    part[(2 * kColWarps + warp) * 32 + lane] = s;
    __syncthreads();
    if (warp == 0 && valid) {
      aL = aN = s = 0.0;
      for (int q = 0; q < kColWarps; ++q) {
        aL += part[(0 * kColWarps + q) * 32 + lane];
        aN += part[(1 * kColWarps + q) * 32 + lane];
        s += part[(2 * kColWarps + q) * 32 + lane];
      }
      const double m = w * (aL * (aL + 2.0 * aN));
      double v = (m - s) / sq;
      if (t == tp) v = sq;
      fac[int64_t(col) * nc + t] = v;
      d[t] = (t == tp) ? 0.0 : d[t] - v * v;
    }
    __syncthreads();
  }
}

}  // namespace

namespace {

constexpr unsigned kColBlocks = 152 * 6;  // fallback grid if the occupancy query fails

// One greedy run over the given candidates (cidx[l] == nullptr: all points).
isdf_status select_loop(Plan* p, int nip, double tol, const double* d0full, int* const* cidx, const int64_t* nc,
                        int* nfound, int* kl_out) {
  cudaStream_t s = p->stream;
  isdf_status st;
  SelParams P{};
  P.nlev = p->nlev;
  P.coff[0] = 0;
  int nGmax = 1;
  for (int l = 0; l < p->nlev; ++l) {
    P.coff[l + 1] = P.coff[l] + nc[l];
    P.cidx[l] = cidx[l];
    P.nc[l] = nc[l];
  }
  P.ntot = P.coff[p->nlev];
  dfree(p->d_diag);
  p->d_diag = nullptr;
  if ((st = dalloc_t(p, &p->d_diag, size_t(std::max<int64_t>(P.ntot, 1)), "residual diagonal"))) return st;
  P.d = p->d_diag;
  for (int l = 0; l < p->nlev; ++l) {
    Level& lv = p->lev[l];
    dfree(lv.fac);
    lv.fac = nullptr;
    lv.fac_cap = std::min<int64_t>(nip, nc[l]);
    if ((st = dalloc_t(p, &lv.fac, size_t(std::max<int64_t>(lv.fac_cap * nc[l], 1)), "selection factor columns")))
      return st;
    P.fac[l] = lv.fac;
    P.phi[l] = lv.phi;
    P.ng[l] = lv.ng;
    P.nL[l] = lv.nL;
    P.nG[l] = lv.nG;
    P.w[l] = lv.w;
    nGmax = std::max(nGmax, lv.nG);
    if (nc[l]) {
      k_gather_diag<<<unsigned((nc[l] + 255) / 256), 256, 0, s>>>(d0full + p->off[l], cidx[l], nc[l],
                                                                  p->d_diag + P.coff[l]);
      count_launches(1);
    }
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
  const size_t smem = sizeof(double) * (size_t((nGmax + 1) & ~1) + 3 * kColWarps * 32);
  if (smem > 48 * 1024) {
    if ((st = cuda_check(p, cudaFuncSetAttribute(k_sel_col, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)),
                         "smem attribute")))
      return st;
  }
  // one wave of resident blocks: grid-striding then splits the groups evenly
  int dev = 0, nsm = 152, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sel_col, 32 * kColWarps, smem);
  const unsigned red_blocks = unsigned(nsm) * 4;
  const unsigned col_blocks = per_sm > 0 ? unsigned(per_sm * nsm) : kColBlocks;
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
  for (int l = 0; l < p->nlev; ++l) kl_out[l] = h.kl[l];
  if (p->opt.profile && !p->pend.empty() && p->pend.back().name == "select_loop") {
    // algorithmic flops: step c on level l costs 2 (nG + c) n_cand (M column
    // and the factor-row dot product)
    double work = 0.0;
    for (int l = 0; l < p->nlev; ++l) {
      const double k = h.kl[l], n = double(nc[l]), nG = p->lev[l].nG;
      work += 2.0 * n * (nG * k + 0.5 * k * (k - 1.0));
    }
    p->pend.back().work = work;
  }
  for (int l = 0; l < p->nlev; ++l) {  // factor columns are not needed after selection
    dfree(p->lev[l].fac);
    p->lev[l].fac = nullptr;
  }
  if (h.err == ISDF_ERR_TIMEOUT) return fail(p, ISDF_ERR_TIMEOUT, "selection loop exceeded options.timeout_ms");
  return ISDF_OK;
}

}  // namespace

isdf_status select_run(Plan* p, int nip, double tol, const std::vector<int64_t>* cand, int* nfound) {
  cudaStream_t s = p->stream;
  isdf_status st;
  dfree(p->d_piv);
  p->d_piv = nullptr;
  dfree(p->d_dval);
  p->d_dval = nullptr;
  if (!p->d_selstate && (st = dalloc(p, &p->d_selstate, sizeof(SelState), "selection state"))) return st;
  if ((st = dalloc_t(p, &p->d_piv, size_t(nip), "pivots"))) return st;
  if ((st = dalloc_t(p, &p->d_dval, size_t(nip), "pivot values"))) return st;
  // initial residual diagonal on every point of every level
  double* d0 = nullptr;
  if ((st = dalloc_t(p, &d0, size_t(p->ntot), "initial diagonal"))) return st;
  for (int l = 0; l < p->nlev; ++l) {
    Level& lv = p->lev[l];
    Prof pr(p, "select_diag", 2.0 * double(lv.nG) * double(lv.ng), "flop", 1);
    k_sel_diag<<<152 * 8, 256, 0, s>>>(lv.phi, lv.ng, lv.nL, lv.nG, lv.w, d0 + p->off[l]);
  }
  int* cidx[ISDF_MAX_LEVELS] = {nullptr, nullptr, nullptr, nullptr};
  int64_t nc[ISDF_MAX_LEVELS] = {0, 0, 0, 0};
  auto free_cidx = [&]() {
    for (int l = 0; l < p->nlev; ++l) {
      dfree(cidx[l]);
      cidx[l] = nullptr;
    }
  };
  auto done = [&](isdf_status r) {
    free_cidx();
    dfree(d0);
    return r;
  };
  int kl[ISDF_MAX_LEVELS];
  if (cand) {
    // caller-given candidates: ascending, unique per level
    std::vector<std::vector<int>> per(p->nlev);
    for (int64_t c : *cand) per[c >> kPivShift].push_back(int(c & kPivMask));
    for (int l = 0; l < p->nlev; ++l) {
      std::sort(per[l].begin(), per[l].end());
      per[l].erase(std::unique(per[l].begin(), per[l].end()), per[l].end());
      nc[l] = int64_t(per[l].size());
      if (!nc[l]) continue;
      if ((st = dalloc_t(p, &cidx[l], size_t(nc[l]), "candidates"))) return done(st);
      if ((st = cuda_check(p, cudaMemcpyAsync(cidx[l], per[l].data(), sizeof(int) * nc[l], cudaMemcpyHostToDevice, s),
                           "copy candidates")))
        return done(st);
    }
    if ((st = cuda_check(p, cudaStreamSynchronize(s), "copy candidates"))) return done(st);
    return done(select_loop(p, nip, tol, d0, cidx, nc, nfound, kl));
  }
  if (!p->opt.prefilter) {
    for (int l = 0; l < p->nlev; ++l) nc[l] = p->lev[l].ng;
    return done(select_loop(p, nip, tol, d0, cidx, nc, nfound, kl));
  }
  // exact prefilter: tau relative to the largest initial residual d_0
  unsigned long long* dmax_slot = nullptr;
  if ((st = dalloc_t(p, &dmax_slot, 1, "max slot"))) return done(st);
  cudaMemsetAsync(dmax_slot, 0, sizeof(unsigned long long), s);
  k_vec_max<<<152 * 4, 256, 0, s>>>(d0, p->ntot, dmax_slot);
  count_launches(1);
  unsigned long long bits = 0;
  cudaMemcpyAsync(&bits, dmax_slot, sizeof(bits), cudaMemcpyDeviceToHost, s);
  st = cuda_check(p, cudaStreamSynchronize(s), "prefilter max");
  dfree(dmax_slot);
  if (st) return done(st);
  double dmax0;
  std::memcpy(&dmax0, &bits, sizeof(dmax0));
  const double taus[3] = {1e-6, 1e-9, 0.0};
  for (int attempt = 0; attempt < 3; ++attempt) {
    const double tau = taus[attempt] * dmax0;
    free_cidx();
    for (int l = 0; l < p->nlev; ++l) {
      Level& lv = p->lev[l];
      if (tau <= 0.0) {
        nc[l] = lv.ng;
        continue;
      }
      const int64_t nb = (lv.ng + kCompactBlock - 1) / kCompactBlock;
      int* counts = nullptr;
      if ((st = dalloc_t(p, &counts, size_t(nb), "compaction counts"))) return done(st);
      k_flag_count<<<unsigned(nb), kCompactBlock, 0, s>>>(d0 + p->off[l], lv.ng, tau, counts);
      std::vector<int> hc(nb);
      cudaMemcpyAsync(hc.data(), counts, sizeof(int) * nb, cudaMemcpyDeviceToHost, s);
      if ((st = cuda_check(p, cudaStreamSynchronize(s), "compaction counts"))) {
        dfree(counts);
        return done(st);
      }
      int64_t acc = 0;
      for (int64_t b = 0; b < nb; ++b) {
        const int c = hc[b];
        hc[b] = int(acc);
        acc += c;
      }
      nc[l] = acc;
      if (acc) {
        if ((st = dalloc_t(p, &cidx[l], size_t(acc), "candidates"))) {
          dfree(counts);
          return done(st);
        }
        cudaMemcpyAsync(counts, hc.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, s);
        k_compact<<<unsigned(nb), kCompactBlock, 0, s>>>(d0 + p->off[l], lv.ng, tau, counts, cidx[l]);
      }
      count_launches(acc ? 2 : 1);
      st = cuda_check(p, cudaStreamSynchronize(s), "compaction");
      dfree(counts);
      if (st) return done(st);
    }
    bool all_kept = true;
    for (int l = 0; l < p->nlev; ++l) all_kept = all_kept && nc[l] == p->lev[l].ng;
    if (all_kept) {  // nothing dropped: this is the full greedy run
      free_cidx();
      return done(select_loop(p, nip, tol, d0, cidx, nc, nfound, kl));
    }
    st = select_loop(p, nip, tol, d0, cidx, nc, nfound, kl);
    if (st || tau <= 0.0) return done(st);
    // certificate: every step's tie threshold stayed above tau
    std::vector<double> dv(*nfound);
    cudaMemcpyAsync(dv.data(), p->d_dval, sizeof(double) * dv.size(), cudaMemcpyDeviceToHost, s);
    if ((st = cuda_check(p, cudaStreamSynchronize(s), "pivot values"))) return done(st);
    bool ok = *nfound == nip || (tol > 0.0 && tau <= tol * dmax0);
    for (double v : dv) ok = ok && (v * (1.0 - 2.0 * p->opt.tie_rel) - 2.0 * p->opt.tie_abs * dmax0 >= tau);
    if (ok) return done(ISDF_OK);
  }
  return done(ISDF_OK);
}

}  // namespace isdf
