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

#include "dfloat.cuh"
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
  // speculative blocks
  int final_;                // a stop rule ended the selection
  int jpos;                  // this step's pivot: its position in the block's set S
  int bsteps;                // steps taken in the current block
  int kb[ISDF_MAX_LEVELS];   // factor columns per level when the block began
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
struct MaxU64 {
  __device__ unsigned long long operator()(unsigned long long a, unsigned long long b) const { return a > b ? a : b; }
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
      st->final_ = 1;
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

// ---------------------------------------------------------------- speculative blocks
//
// A block of the greedy loop first guesses a set S of up to s points that are
// likely to be the next pivots (the largest local maxima of the residual on
// the grids), computes the factor columns they would produce with
// tensor-core products over all candidates,
//   B[j][t] = w M(t, S_j) - sum_{k < kb} L[t,k] L[S_j,k]        (kb = columns so far)
// and then takes ordinary greedy steps, each finishing its column from B with
// the few columns added inside the block:
//   L[t,col] = (B[pos(p)][t] - sum_{kb <= k < col} L[t,k] L[p,k]) / sqrt(d_p).
// The pivot of every step is still the argmax over ALL candidates' exact
// residuals (same tie rule); the block ends at the first pivot outside S.  S
// only decides how many steps one block covers, never which point is chosen.

struct BlkParams {
  SelParams P;
  const int* spos;                      // [ntot] position of a candidate in S's range of its level, -1 if not in S
  const double* bm[ISDF_MAX_LEVELS];    // [s_l][nc_l]
  float2* bdf[ISDF_MAX_LEVELS];         // [s][nc_l] the block's columns so far, double-float
};

// Order-preserving key of a residual value: its bits when positive, else 0
// (integer operations only).
__device__ __forceinline__ unsigned long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 ? (unsigned long long)b : 0ull;
}

// Column entry of a block step for one candidate:
//   v = (b - sum_q F_q lp_q) / sqrt(d_p),
// F_q the block's earlier columns at this candidate (stride nc) and lp_q at
// the pivot, all double-float; the products' errors and the partial sums'
// rounding errors are gathered in one FP32 word.  FP32 pipes only.
__device__ __forceinline__ DF blk_col_df(const float2* __restrict__ fq, int64_t nc, int nbk, const DF* lpd, double b,
                                         DF inv_sq) {
  float ah = 0.0f, al = 0.0f;
  int q = 0;
  for (; q + 4 <= nbk; q += 4) {
    float2 c[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) c[u] = __ldcg(fq + int64_t(q + u) * nc);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const DF l = lpd[q + u];
      const float pr = __fmul_rn(c[u].x, l.hi);
      float e = __fmaf_rn(c[u].x, l.hi, -pr);
      e = __fmaf_rn(c[u].x, l.lo, e);
      e = __fmaf_rn(c[u].y, l.hi, e);
      const DF t = two_sum(ah, pr);
      ah = t.hi;
      al = __fadd_rn(al, __fadd_rn(t.lo, e));
    }
  }
  for (; q < nbk; ++q) {
    const float2 c = __ldcg(fq + int64_t(q) * nc);
    const DF l = lpd[q];
    const float pr = __fmul_rn(c.x, l.hi);
    float e = __fmaf_rn(c.x, l.hi, -pr);
    e = __fmaf_rn(c.x, l.lo, e);
    e = __fmaf_rn(c.y, l.hi, e);
    const DF t = two_sum(ah, pr);
    ah = t.hi;
    al = __fadd_rn(al, __fadd_rn(t.lo, e));
  }
  return df_mul(df_sub(df_from_double(b), two_sum(ah, al)), inv_sq);
}

struct LmParams {
  const double* d;
  int64_t ntot;
  int nlev;
  int64_t coff[ISDF_MAX_LEVELS + 1];
  const int* cidx[ISDF_MAX_LEVELS];  // candidate -> grid index (nullptr: identity)
  const int* gpos[ISDF_MAX_LEVELS];  // grid index -> candidate (-1: none; nullptr: identity)
  int n[ISDF_MAX_LEVELS][3];
};

// d at the 6 periodic grid neighbours of candidate i (non-candidates count 0)
__device__ __forceinline__ bool is_local_max(const LmParams& Q, int64_t i) {
  const double v = Q.d[i];
  if (!(v > 0.0)) return false;
  int l = 0;
  while (l + 1 < Q.nlev && i >= Q.coff[l + 1]) ++l;
  const int64_t t = i - Q.coff[l];
  const int64_t g = Q.cidx[l] ? Q.cidx[l][t] : t;
  const int nx = Q.n[l][0], ny = Q.n[l][1], nz = Q.n[l][2];
  const int x = int(g % nx), y = int((g / nx) % ny), z = int(g / (int64_t(nx) * ny));
  const double* dl = Q.d + Q.coff[l];
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    int xx = x, yy = y, zz = z;
    if (a == 0) xx = x + 1 == nx ? 0 : x + 1;
    if (a == 1) xx = x == 0 ? nx - 1 : x - 1;
    if (a == 2) yy = y + 1 == ny ? 0 : y + 1;
    if (a == 3) yy = y == 0 ? ny - 1 : y - 1;
    if (a == 4) zz = z + 1 == nz ? 0 : z + 1;
    if (a == 5) zz = z == 0 ? nz - 1 : z - 1;
    const int64_t gg = xx + int64_t(nx) * (yy + int64_t(ny) * zz);
    const int64_t tt = Q.gpos[l] ? int64_t(Q.gpos[l][gg]) : gg;
    if (tt >= 0 && dl[tt] > v) return false;
  }
  return true;
}

// ordered compaction of the local maxima: per-block counts, one-block scan, scatter
__global__ void k_lm_count(LmParams Q, int* __restrict__ counts) {
  __shared__ int sh[32];
  const int64_t i = int64_t(blockIdx.x) * kCompactBlock + threadIdx.x;
  const int f = (i < Q.ntot && is_local_max(Q, i)) ? 1 : 0;
  const unsigned b = __ballot_sync(0xffffffffu, f);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    int c = 0;
    for (int w = 0; w < kCompactBlock / 32; ++w) c += sh[w];
    counts[blockIdx.x] = c;
  }
}

// exclusive scan of nb counts in place; total into *total (one block of 1024)
__global__ void k_scan_counts(int* __restrict__ counts, int64_t nb, int* __restrict__ total) {
  __shared__ int sh[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
    const int64_t b = b0 + threadIdx.x;
    const int v = b < nb ? counts[b] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const int add = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += add;
      __syncthreads();
    }
    if (b < nb) counts[b] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += sh[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_lm_write(LmParams Q, const int* __restrict__ offs, int* __restrict__ list) {
  __shared__ int woff[32];
  const int64_t i = int64_t(blockIdx.x) * kCompactBlock + threadIdx.x;
  const int f = (i < Q.ntot && is_local_max(Q, i)) ? 1 : 0;
  const unsigned b = __ballot_sync(0xffffffffu, f);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) woff[wid] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0;
    for (int w = 0; w < kCompactBlock / 32; ++w) {
      const int c = woff[w];
      woff[w] = a;
      a += c;
    }
  }
  __syncthreads();
  if (f) list[offs[blockIdx.x] + woff[wid] + __popc(b & ((1u << lane) - 1u))] = int(i);
}

// The s largest residuals of the list (ties to the smallest index), by an
// 8-bit radix select on the bit patterns (d > 0 orders like its bits).
// Writes S in ascending candidate order: sidx (concatenated index), sg (grid
// index), st (position in its level), per-level counts and offsets, spos.
struct TopSOut {
  int* sidx;
  int* sg;
  int* st;
  int* scount;  // [ISDF_MAX_LEVELS + 1]: per-level counts, then the total
  int* spos;    // [ntot]
};
__global__ void __launch_bounds__(1024) k_top_s(LmParams Q, const int* __restrict__ list, const int* __restrict__ nlist,
                                                int smax, TopSOut O) {
  __shared__ int hist[256];
  __shared__ unsigned long long prefix, pmask;
  __shared__ int need, take_gt;
  __shared__ int wsum[32];
  __shared__ int base;
  __shared__ int lcount[ISDF_MAX_LEVELS];
  const int n = *nlist;
  const int tid = threadIdx.x;
  if (tid == 0) {
    prefix = 0ull;
    pmask = 0ull;
    need = n < smax ? n : smax;
    take_gt = 0;
    base = 0;
  }
  if (tid < ISDF_MAX_LEVELS) lcount[tid] = 0;
  __syncthreads();
  const int want = need;
  // find the threshold key T: count(key > T) < want <= count(key >= T)
  if (want > 0 && want < n) {
    int above = 0;  // keys above the current prefix range (already counted)
    for (int shift = 56; shift >= 0; shift -= 8) {
      for (int b = tid; b < 256; b += blockDim.x) hist[b] = 0;
      __syncthreads();
      for (int i = tid; i < n; i += blockDim.x) {
        const unsigned long long key = (unsigned long long)__double_as_longlong(Q.d[list[i]]);
        if ((key & pmask) == prefix) atomicAdd(&hist[(key >> shift) & 255], 1);
      }
      __syncthreads();
      if (tid == 0) {
        int acc = above, b = 255;
        for (; b > 0; --b) {
          if (acc + hist[b] >= want) break;
          acc += hist[b];
        }
        above = acc;
        prefix |= (unsigned long long)b << shift;
        pmask |= 255ull << shift;
        take_gt = acc;
      }
      __syncthreads();
      above = take_gt;
    }
  }
  const unsigned long long T = prefix;
  const bool all = !(want > 0 && want < n);
  const int n_eq_needed = all ? 0 : want - take_gt;
  // ordered pass: keep key > T, and key == T while the equal quota lasts
  __shared__ int eq_base;
  if (tid == 0) eq_base = 0;
  __syncthreads();
  for (int i0 = 0; i0 < n; i0 += blockDim.x) {
    const int i = i0 + tid;
    bool gt = false, eq = false;
    int idx = 0;
    if (i < n) {
      idx = list[i];
      const unsigned long long key = (unsigned long long)__double_as_longlong(Q.d[idx]);
      gt = all || key > T;
      eq = !all && key == T;
    }
    // rank of the equals in list order
    const unsigned be = __ballot_sync(0xffffffffu, eq);
    const int lane = tid & 31, wid = tid >> 5;
    if (lane == 0) wsum[wid] = __popc(be);
    __syncthreads();
    if (tid == 0) {
      int a = eq_base;
      for (int w = 0; w < 32; ++w) {
        const int c = wsum[w];
        wsum[w] = a;
        a += c;
      }
      eq_base = a;
    }
    __syncthreads();
    const int eq_rank = wsum[wid] + __popc(be & ((1u << lane) - 1u));
    const bool sel = gt || (eq && eq_rank < n_eq_needed);
    __syncthreads();
    const unsigned bs = __ballot_sync(0xffffffffu, sel);
    if (lane == 0) wsum[wid] = __popc(bs);
    __syncthreads();
    if (tid == 0) {
      int a = base;
      for (int w = 0; w < 32; ++w) {
        const int c = wsum[w];
        wsum[w] = a;
        a += c;
      }
      base = a;
    }
    __syncthreads();
    if (sel) {
      const int pos = wsum[wid] + __popc(bs & ((1u << lane) - 1u));
      int l = 0;
      while (l + 1 < Q.nlev && idx >= Q.coff[l + 1]) ++l;
      const int64_t t = idx - Q.coff[l];
      O.sidx[pos] = idx;
      O.st[pos] = int(t);
      O.sg[pos] = Q.cidx[l] ? Q.cidx[l][t] : int(t);
      atomicAdd(&lcount[l], 1);
    }
    __syncthreads();
  }
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int l = 0; l < Q.nlev; ++l) {
      O.scount[l] = lcount[l];
      acc += lcount[l];
    }
    O.scount[ISDF_MAX_LEVELS] = acc;
  }
  __syncthreads();
  // positions within each level's range
  const int total = base;
  for (int j = tid; j < total; j += blockDim.x) {
    const int idx = O.sidx[j];
    int l = 0;
    while (l + 1 < Q.nlev && idx >= Q.coff[l + 1]) ++l;
    int first = 0;
    for (int q = 0; q < l; ++q) first += lcount[q];
    O.spos[idx] = j - first;
  }
}

__global__ void k_spos_clear(const int* __restrict__ sidx, const int* __restrict__ scount, int* __restrict__ spos) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < scount[ISDF_MAX_LEVELS]) spos[sidx[j]] = -1;
}

// B = w * aL (aL + 2 aN) - F over [s_l][nc]; in place in aL
__global__ void k_blk_combine(double* __restrict__ aL, const double* __restrict__ aN, const double* __restrict__ F,
                              int64_t n, double w) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    const double a = aL[e];
    const double b = aN ? aN[e] : 0.0;
    double v = w * (a * (a + 2.0 * b));
    if (F) v -= F[e];
    aL[e] = v;
  }
}

// per-candidate power-of-two bound of the factor rows: sum_k L[t,k]^2 <= d0(t)
// Row scales of the speculative set's basis-value rows: those of the same
// candidates' rows on the candidate side (the same rows, the same exact max)
__global__ void k_gather_exps(const int* __restrict__ pos, int n, const int* __restrict__ src, int* __restrict__ dst) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) dst[r] = src[pos[r]];
}

// Fixed row scales of the factor columns: |L[c][k]| <= sqrt(d0_c)
__global__ void k_fac_exps(const double* __restrict__ d0c, int64_t nc, int64_t npad, int* __restrict__ exps) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= npad) return;
  int e = 0;
  if (t < nc && d0c[t] > 0.0) frexp(sqrt(d0c[t]) * (1.0 + 0x1p-20), &e);
  exps[t] = e;
}

__global__ void k_blk_begin(SelState* st) {
  if (threadIdx.x != 0) return;
  st->done = st->final_ ? 1 : 0;
  st->skip = 1;
  st->bsteps = 0;
  st->dmax_bits = 0ull;
  st->first = ULLONG_MAX;
  for (int l = 0; l < ISDF_MAX_LEVELS; ++l) st->kb[l] = st->kl[l];
}

__global__ void k_blk_pick(BlkParams B, SelState* st) {
  const SelParams& P = B.P;
  if (threadIdx.x != 0 || st->done) return;
  const unsigned long long idx = st->first;
  if (idx == ULLONG_MAX) {
    st->done = 1;
    st->skip = 1;
    st->final_ = 1;
    return;
  }
  const int pos = B.spos[idx];
  if (pos < 0) {  // the greedy pivot is outside S: the block ends here
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
  st->jpos = pos;
  st->col = st->kl[l];
  P.piv[k] = ((long long)l << kPivShift) | g;
  P.dval[k] = dp;
  st->kl[l] += 1;
  st->k = k + 1;
  st->bsteps += 1;
  st->skip = 0;
  st->dmax_bits = 0ull;
  st->first = ULLONG_MAX;
  if (P.timeout_ns) {
    const unsigned long long now = globaltimer();
    if (k == 0) {
      st->t0 = now;
    } else if (now - st->t0 > P.timeout_ns) {
      st->err = ISDF_ERR_TIMEOUT;
      st->done = 1;
      st->final_ = 1;
    }
  }
}

// column of this step from B and the block's earlier columns; residual update
__global__ void __launch_bounds__(256) k_blk_col(BlkParams B, const SelState* st) {
  if (st->skip) return;
  __shared__ DF lp[256];  // L[p, kb..col) (a block has at most 256 steps)
  const SelParams& P = B.P;
  const int l = st->lev;
  const int col = st->col, kb = st->kb[l];
  const int nb = col - kb;
  const int64_t nc = P.nc[l], tp = st->tp;
  float2* __restrict__ bdf = B.bdf[l];
  __shared__ double sq_sh;
  __shared__ DF inv_sh;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    const float2 c = bdf[int64_t(i) * nc + tp];
    lp[i] = {c.x, c.y};
  }
  if (threadIdx.x == 0) {
    sq_sh = sqrt(st->dp);
    inv_sh = df_from_double(1.0 / sq_sh);
  }
  __syncthreads();
  const double sq = sq_sh;
  const DF inv = inv_sh;
  const double* __restrict__ bcol = B.bm[l] + int64_t(st->jpos) * nc;
  double* __restrict__ facw = P.fac[l];
  double* __restrict__ d = P.d + P.coff[l];
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < nc; t += int64_t(gridDim.x) * blockDim.x) {
    const DF v = (t == tp) ? df_from_double(sq) : blk_col_df(bdf + t, nc, nb, lp, bcol[t], inv);
    const double vd = (t == tp) ? sq : df_to_double(v);
    facw[int64_t(col) * nc + t] = vd;
    bdf[int64_t(nb) * nc + t] = make_float2(v.hi, v.lo);
    d[t] = (t == tp) ? 0.0 : fma(-vd, vd, d[t]);
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

// ---------------------------------------------------------------- persistent block steps
//
// All greedy steps of one speculative block in one cooperative launch (every
// CTA resident).  Each step is two phases separated by grid barriers:
//   B: tie rule on d_max (computed in the previous phase A): smallest index
//      with d >= thr, atomicMin;
//   A: every CTA derives the same pivot from the shared slots, keeps its own
//      copy of the counters, writes its share of the new column and residual
//      and reduces the residual's maximum for the next step; CTA 0 records
//      the pivot.
// The pivot's own residual is zeroed in the next phase B (other CTAs read it
// during phase A), and that phase's search skips it.  Barriers are bounded:
// after ~1 s of device time a CTA records an error and leaves; every CTA
// leaves at the next barrier it reaches, so the launch always ends.

struct StepSync {
  unsigned int count;
  unsigned int gen;
  int abort;
  int pad;
  unsigned long long dmax[2];
  unsigned long long first[2];
};

constexpr unsigned long long kBarrierNs = 1000000000ull;

__device__ bool grid_sync(StepSync* sy, unsigned int nblocks) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int* gen = &sy->gen;
    const unsigned int g = *gen;
    __threadfence();
    if (atomicAdd(&sy->count, 1u) == nblocks - 1) {
      sy->count = 0;
      __threadfence();
      atomicAdd(&sy->gen, 1u);
    } else {
      const unsigned long long t0 = globaltimer();
      long long i = 0;
      while (*gen == g) {
        if (*(volatile int*)&sy->abort) { ok = 0; break; }
        if ((++i & 1023) == 0 && globaltimer() - t0 > kBarrierNs) {
          atomicExch(&sy->abort, 1);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    if (*(volatile int*)&sy->abort) ok = 0;
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

__global__ void k_sync_init(StepSync* sy) {
  if (threadIdx.x != 0) return;
  sy->count = 0;
  sy->gen = 0;
  sy->abort = 0;
  sy->dmax[0] = sy->dmax[1] = 0ull;
  sy->first[0] = sy->first[1] = ULLONG_MAX;
}

__global__ void __launch_bounds__(512) k_blk_steps(BlkParams B, SelState* st, StepSync* sy, int smax) {
  const SelParams& P = B.P;
  __shared__ DF lpd[256];  // the pivot's entries in the block's earlier columns
  __shared__ int kl_sh[ISDF_MAX_LEVELS];
  __shared__ unsigned long long red[32];
  __shared__ int stop_sh;
  __shared__ unsigned long long thr_sh;
  __shared__ double sq_sh;
  __shared__ DF inv_sh;
  const unsigned int nb = gridDim.x;
  const int tid = threadIdx.x;
  const int64_t gtid = int64_t(blockIdx.x) * blockDim.x + tid, gstride = int64_t(gridDim.x) * blockDim.x;
  // private copies of the counters (identical in every CTA)
  int k = st->k;
  double d0 = st->d0;
  __shared__ int kb[ISDF_MAX_LEVELS];  // columns per level when the block began
  if (tid < ISDF_MAX_LEVELS) kl_sh[tid] = kb[tid] = st->kl[tid];
  __syncthreads();
  long long last = -1;  // global index of the previous step's pivot (its residual is zeroed next phase B)
  double last_dp = st->dp;  // value of the last pivot taken (written back with the counters)
  int bsteps = 0, reason = 0;  // reason: 0 running, 1 block end, 2 final, 3 timeout, 4 barrier failure
  // Residual comparisons use the order-preserving integer keys of the values,
  // and the per-step scalars are formed by one thread per CTA: the FP64 unit
  // is left to the two operations per candidate that need it.
  // phase 0: d_max of the current residual into slot 0
  {
    unsigned long long mk = 0ull;
    for (int64_t i = gtid; i < P.ntot; i += gstride) mk = max(mk, dkey(__ldcg(P.d + i)));
    mk = block_reduce(mk, MaxU64(), red);
    if (tid == 0) atomicMax(&sy->dmax[0], mk);
  }
  if (!grid_sync(sy, nb)) reason = 4;
  for (int j = 0; reason == 0; ++j) {
    const int par = j & 1;
    // ---------------- phase B
    if (last >= 0 && gtid == 0) P.d[last] = 0.0;  // visible after the barrier
    const double dmax = __longlong_as_double((long long)*(volatile unsigned long long*)&sy->dmax[par]);
    if (tid == 0) {
      const double dz = (k == 0) ? dmax : d0;
      int stop = 0;
      if (j >= smax)
        stop = 1;
      else if (k >= P.nip || !(dmax > 0.0) || dmax < P.tol * dz)
        stop = 2;
      stop_sh = stop;
      // d >= thr and d > 0  <=>  key(d) >= max(key(thr), 1)
      thr_sh = max(dkey(dmax - fmax(P.tie_rel * dmax, P.tie_abs * dz)), 1ull);
    }
    __syncthreads();
    if (stop_sh) {
      reason = stop_sh;
      break;
    }
    const unsigned long long tk = thr_sh;
    unsigned long long best = ULLONG_MAX;
    for (int64_t i = gtid; i < P.ntot; i += gstride) {
      if (i == last) continue;
      if (dkey(__ldcg(P.d + i)) >= tk) {
        best = (unsigned long long)i;
        break;
      }
    }
    best = block_reduce(best, MinOp(), red);
    if (tid == 0 && best != ULLONG_MAX) atomicMin(&sy->first[par], best);
    if (gtid == 0) {  // slots of the next step
      sy->dmax[par ^ 1] = 0ull;
      sy->first[par ^ 1] = ULLONG_MAX;
    }
    if (!grid_sync(sy, nb)) { reason = 4; break; }
    // ---------------- phase A
    const unsigned long long idx = *(volatile unsigned long long*)&sy->first[par];
    if (idx == ULLONG_MAX) { reason = 2; break; }
    const int pos = __ldcg(B.spos + idx);
    if (pos < 0) { reason = 1; break; }  // greedy pivot outside S: block ends
    int l = 0;
    while (l + 1 < P.nlev && (long long)idx >= P.coff[l + 1]) ++l;
    const long long tp = (long long)idx - P.coff[l];
    const double dp = __ldcg(P.d + idx);
    const int col = kl_sh[l];
    const int nbk = col - kb[l];
    const int64_t nc = P.nc[l];
    float2* __restrict__ bdf = B.bdf[l];
    __syncthreads();
    for (int i = tid; i < nbk; i += blockDim.x) {
      const float2 c = __ldcg(bdf + int64_t(i) * nc + tp);
      lpd[i] = {c.x, c.y};
    }
    if (tid == 0) {
      sq_sh = sqrt(dp);
      inv_sh = df_from_double(1.0 / sq_sh);
    }
    __syncthreads();
    if (k == 0) d0 = dmax;
    last_dp = dp;
    if (gtid == 0) {
      const long long g = P.cidx[l] ? P.cidx[l][tp] : tp;
      P.piv[k] = ((long long)l << kPivShift) | g;
      P.dval[k] = dp;
      if (k == 0) {
        st->d0 = dmax;
        st->t0 = globaltimer();
      }
    }
    const double sq = sq_sh;
    const DF inv = inv_sh;
    const double* __restrict__ bcol = B.bm[l] + int64_t(pos) * nc;
    double* __restrict__ facw = P.fac[l];
    const int64_t lo = P.coff[l], hi = P.coff[l + 1];
    unsigned long long mk = 0ull;
    for (int64_t i = gtid; i < P.ntot; i += gstride) {
      unsigned long long key;
      if (i >= lo && i < hi) {
        const int64_t t = i - lo;
        const double di = __ldcg(P.d + i);
        const DF v = (t == tp) ? df_from_double(sq) : blk_col_df(bdf + t, nc, nbk, lpd, bcol[t], inv);
        const double vd = (t == tp) ? sq : df_to_double(v);
        facw[int64_t(col) * nc + t] = vd;
        bdf[int64_t(nbk) * nc + t] = make_float2(v.hi, v.lo);
        if (t == tp) {
          key = 0ull;  // written as 0 in the next phase B
        } else {
          const double dn = fma(-vd, vd, di);
          P.d[i] = dn;
          key = dkey(dn);
        }
      } else {
        key = (i == (long long)idx) ? 0ull : dkey(__ldcg(P.d + i));
      }
      mk = max(mk, key);
    }
    mk = block_reduce(mk, MaxU64(), red);
    if (tid == 0) atomicMax(&sy->dmax[par ^ 1], mk);
    // counters advance identically in every CTA
    __syncthreads();
    if (tid == 0) kl_sh[l] = col + 1;
    __syncthreads();
    ++k;
    ++bsteps;
    last = (long long)idx;
    // time budget: CTA 0's clock decides for everyone and publishes the decision
    // before the barrier (this step's column is complete)
    if (gtid == 0 && P.timeout_ns && globaltimer() - st->t0 > P.timeout_ns) atomicExch(&sy->abort, 2);
    if (!grid_sync(sy, nb)) {
      reason = (*(volatile int*)&sy->abort == 2) ? 3 : 4;
      break;
    }
  }
  // the last pivot's residual is zeroed here if no phase B followed it
  if (last >= 0 && gtid == 0) P.d[last] = 0.0;
  if (gtid == 0) {
    st->k = k;
    st->dp = last_dp;
    for (int l = 0; l < ISDF_MAX_LEVELS; ++l) st->kl[l] = kl_sh[l];
    st->bsteps = bsteps;
    st->done = 1;
    st->skip = 1;
    if (reason == 2) st->final_ = 1;
    if (reason == 3) {
      st->err = ISDF_ERR_TIMEOUT;
      st->final_ = 1;
    }
    if (reason == 4) {
      st->err = ISDF_ERR_CUDA;
      st->final_ = 1;
    }
  }
}

__global__ void k_scatter_pos(const int* __restrict__ cidx, int64_t nc, int* __restrict__ gpos) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < nc) gpos[cidx[t]] = int(t);
}

// out[j] = in ? in[keep[j]] : keep[j]  (candidate grid indices after compaction)
__global__ void k_map_idx(const int* __restrict__ in, const int* __restrict__ keep, int64_t n, int* __restrict__ out) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n) out[t] = in ? in[keep[t]] : keep[t];
}

// fac_new[c][j] = fac_old[c][keep[j]] for the first ncol columns
__global__ void k_gather_cols(const double* __restrict__ fo, int64_t no, const int* __restrict__ keep, int64_t nn,
                              int64_t ncol, double* __restrict__ fn) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= nn * ncol) return;
  const int64_t c = e / nn, j = e % nn;
  fn[e] = fo[c * no + keep[j]];
}

constexpr int kSlices = 8;  // FP64-grade sliced products for the selection

// Speculative-block form of select_loop (same result: every pivot is the
// greedy one).  Per block: S from the residual's local maxima, three
// tensor-core products per level for the columns of S, then up to s greedy
// steps replayed from a CUDA graph; a step whose pivot lies outside S ends the
// block (if it was the block's first step, one ordinary step is taken).
// tau > 0: the candidates are the points with initial residual >= tau (the
// exact prefilter).  Residuals only shrink, so a candidate whose residual
// falls below tau can never be picked while every pivot value stays above
// tau plus the tie margin (the certificate select_run checks): between
// blocks such candidates are dropped and every candidate-side array is
// rebuilt for the rest, which changes no pivot and no column entry (rows
// are computed independently, ties go to the smallest grid index either
// way).  As soon as a pivot value breaks the certificate the attempt stops
// (*aborted) so that select_run can retry with a lower tau.
isdf_status select_loop_blocked(Plan* p, int nip, double tol, const double* d0full, int* const* cidx,
                                const int64_t* nc_in, int* nfound, int* kl_out, double tau, bool* aborted) {
  cudaStream_t s = p->stream;
  isdf_status st = ISDF_OK;
  const int smax = p->opt.select_block;
  const int nlev = p->nlev;
  *aborted = false;
  int64_t nc[ISDF_MAX_LEVELS] = {0, 0, 0, 0};
  for (int l = 0; l < nlev; ++l) nc[l] = nc_in[l];
  // with the cooperative block steps the factor storage of a level starts at
  // a quarter of nip and grows between blocks (a level rarely takes more);
  // the captured graph of the other form holds fixed arrays: full capacity
  bool growable = false;
  {
    int d = 0, coop_attr = 0, spsm = 0;
    cudaGetDevice(&d);
    cudaDeviceGetAttribute(&coop_attr, cudaDevAttrCooperativeLaunch, d);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&spsm, k_blk_steps, 512, 0);
    cudaGetLastError();
    growable = coop_attr && spsm > 0;
  }
  int* cur_cidx[ISDF_MAX_LEVELS] = {nullptr, nullptr, nullptr, nullptr};  // after compaction: owned here
  for (int l = 0; l < nlev; ++l) cur_cidx[l] = cidx[l];
  std::vector<int*> own_cidx;
  SelParams P{};
  P.nlev = nlev;
  P.coff[0] = 0;
  int nGmax = 1;
  for (int l = 0; l < nlev; ++l) {
    P.coff[l + 1] = P.coff[l] + nc[l];
    P.cidx[l] = cidx[l];
    P.nc[l] = nc[l];
  }
  P.ntot = P.coff[nlev];
  dfree(p->d_diag);
  p->d_diag = nullptr;
  if ((st = dalloc_t(p, &p->d_diag, size_t(std::max<int64_t>(P.ntot, 1)), "residual diagonal"))) return st;
  P.d = p->d_diag;

  struct LevBuf {
    OzOperand aL, aN, aF, bL, bN, bF;
    double *cL = nullptr, *cN = nullptr, *cF = nullptr;
    int* gpos = nullptr;
    int sliced = 0;
  } lb[ISDF_MAX_LEVELS];
  int *counts = nullptr, *nlist = nullptr, *list = nullptr, *sidx = nullptr, *sg = nullptr, *stp = nullptr,
      *scount = nullptr, *spos = nullptr;
  cudaGraphExec_t exec = nullptr;
  void* sync_mem = nullptr;
  auto cleanup = [&]() {
    for (int* q : own_cidx) dfree(q);
    own_cidx.clear();
    for (int l = 0; l < nlev; ++l) {
      oz_free(lb[l].aL), oz_free(lb[l].aN), oz_free(lb[l].aF);
      oz_free(lb[l].bL), oz_free(lb[l].bN), oz_free(lb[l].bF);
      dfree(lb[l].cL), dfree(lb[l].cN), dfree(lb[l].cF), dfree(lb[l].gpos);
      dfree(p->lev[l].fac);
      p->lev[l].fac = nullptr;
    }
    dfree(counts), dfree(nlist), dfree(list), dfree(sidx), dfree(sg), dfree(stp), dfree(scount), dfree(spos);
    dfree(sync_mem);
    if (exec) cudaGraphExecDestroy(exec);
  };
  auto bail = [&](isdf_status r) {
    cleanup();
    return r;
  };

  // ---- set-up: residual, factor storage, candidate-side operands
  LmParams Q{};
  Q.d = P.d;
  Q.nlev = nlev;
  Q.ntot = P.ntot;
  for (int l = 0; l <= nlev; ++l) Q.coff[l] = P.coff[l];
  for (int l = 0; l < nlev; ++l) {
    Level& lv = p->lev[l];
    LevBuf& b = lb[l];
    dfree(lv.fac);
    lv.fac = nullptr;
    lv.fac_cap = std::min<int64_t>(nip, nc[l]);
    if (growable)
      lv.fac_cap = std::min<int64_t>(lv.fac_cap, std::max<int64_t>(4 * int64_t(smax) + 1, nip / 4));
    if ((st = dalloc_t(p, &lv.fac, size_t(std::max<int64_t>(lv.fac_cap * nc[l], 1)), "selection factor columns")))
      return bail(st);
    P.fac[l] = lv.fac;
    P.phi[l] = lv.phi;
    P.ng[l] = lv.ng;
    P.nL[l] = lv.nL;
    P.nG[l] = lv.nG;
    P.w[l] = lv.w;
    nGmax = std::max(nGmax, lv.nG);
    Q.cidx[l] = cidx[l];
    for (int a = 0; a < 3; ++a) Q.n[l][a] = lv.n[a];
    if (!nc[l]) continue;
    k_gather_diag<<<unsigned((nc[l] + 255) / 256), 256, 0, s>>>(d0full + p->off[l], cidx[l], nc[l], p->d_diag + P.coff[l]);
    count_launches(1);
    if (cidx[l]) {
      if ((st = dalloc_t(p, &b.gpos, size_t(lv.ng), "grid-to-candidate map"))) return bail(st);
      cudaMemsetAsync(b.gpos, 0xFF, sizeof(int) * size_t(lv.ng), s);
      k_scatter_pos<<<unsigned((nc[l] + 255) / 256), 256, 0, s>>>(cidx[l], nc[l], b.gpos);
      count_launches(1);
    }
    Q.gpos[l] = b.gpos;
    const int bn = oz_bn(kSlices);
    if ((st = oz_alloc(p, b.aL, nc[l], std::max(lv.nL, 1), 128, kSlices, "selection slices")) ||
        (st = oz_alloc(p, b.bL, smax, std::max(lv.nL, 1), bn, kSlices, "selection slices")) ||
        (st = oz_alloc(p, b.aF, nc[l], lv.fac_cap, 128, kSlices, "selection slices")) ||
        (st = oz_alloc(p, b.bF, smax, lv.fac_cap, bn, kSlices, "selection slices")) ||
        (st = dalloc_t(p, &b.cL, size_t(smax) * nc[l], "selection columns")) ||
        (st = dalloc_t(p, &b.cF, size_t(smax) * nc[l], "selection columns")))
      return bail(st);
    if (lv.nN > 0 && ((st = oz_alloc(p, b.aN, nc[l], lv.nN, 128, kSlices, "selection slices")) ||
                      (st = oz_alloc(p, b.bN, smax, lv.nN, bn, kSlices, "selection slices")) ||
                      (st = dalloc_t(p, &b.cN, size_t(smax) * nc[l], "selection columns"))))
      return bail(st);
    {
      Prof pr(p, "select_slice", 8.0 * double(nc[l]) * lv.nG, "byte", 4);
      if (lv.nL > 0) oz_slice_ex(lv.phi, 1, lv.ng, cidx[l], b.aL, 0, b.aL.nkt * (kOzBK / 8), false, s);
      if (lv.nN > 0)
        oz_slice_ex(lv.phi + int64_t(lv.nL) * lv.ng, 1, lv.ng, cidx[l], b.aN, 0, b.aN.nkt * (kOzBK / 8), false, s);
      // factor-column digits are written group by group as columns appear:
      // groups not yet written must read as zero
      cudaMemsetAsync(b.aF.tiles, 0, size_t(oz_tile_bytes(b.aF)), s);
      // factor rows are bounded by sqrt(d0): fixed scales, columns appended in place
      k_fac_exps<<<unsigned((b.aF.nrt * 128 + 255) / 256), 256, 0, s>>>(p->d_diag + P.coff[l], nc[l], b.aF.nrt * 128,
                                                                         b.aF.exps);
      count_launches(1);
    }
    b.aF.K = 0;
    b.aF.nkt = 0;
  }
  P.piv = p->d_piv;
  P.dval = p->d_dval;
  P.nip = nip;
  P.tol = tol;
  P.tie_rel = p->opt.tie_rel;
  P.tie_abs = p->opt.tie_abs;
  P.timeout_ns = (unsigned long long)p->opt.timeout_ms * 1000000ull;
  int64_t nbk = (P.ntot + kCompactBlock - 1) / kCompactBlock;
  if ((st = dalloc_t(p, &counts, size_t(std::max<int64_t>(nbk, 1)), "block counts")) ||
      (st = dalloc_t(p, &nlist, 1, "list size")) ||
      (st = dalloc_t(p, &list, size_t(std::max<int64_t>(P.ntot, 1)), "local maxima")) ||
      (st = dalloc_t(p, &sidx, size_t(smax), "speculative set")) || (st = dalloc_t(p, &sg, size_t(smax), "speculative set")) ||
      (st = dalloc_t(p, &stp, size_t(smax), "speculative set")) ||
      (st = dalloc_t(p, &scount, size_t(ISDF_MAX_LEVELS + 1), "speculative set")) ||
      (st = dalloc_t(p, &spos, size_t(std::max<int64_t>(P.ntot, 1)), "speculative positions")))
    return bail(st);
  cudaMemsetAsync(spos, 0xFF, sizeof(int) * size_t(std::max<int64_t>(P.ntot, 1)), s);
  BlkParams BP{};
  BP.P = P;
  BP.spos = spos;
  for (int l = 0; l < nlev; ++l) {
    BP.bm[l] = lb[l].cL;
    // the factor product's output is free during the steps: it holds the
    // double-float copy of the block's columns (s x nc values of 8 bytes)
    BP.bdf[l] = reinterpret_cast<float2*>(lb[l].cF);
  }
  TopSOut O{sidx, sg, stp, scount, spos};

  SelState h{};
  h.dmax_bits = 0;
  h.first = ULLONG_MAX;
  h.skip = 1;
  if ((st = cuda_check(p, cudaMemcpyAsync(p->d_selstate, &h, sizeof(h), cudaMemcpyHostToDevice, s), "state init")))
    return bail(st);
  SelState* dst = static_cast<SelState*>(p->d_selstate);
  const size_t smem = sizeof(double) * (size_t((nGmax + 1) & ~1) + 3 * kColWarps * 32);
  if (smem > 48 * 1024 &&
      (st = cuda_check(p, cudaFuncSetAttribute(k_sel_col, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)),
                       "smem attribute")))
    return bail(st);
  int dev = 0, nsm = 152, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sel_col, 32 * kColWarps, smem);
  const unsigned red_blocks = unsigned(nsm) * 4;
  const unsigned col_blocks = per_sm > 0 ? unsigned(per_sm * nsm) : kColBlocks;
  auto block_step = [&]() {
    k_sel_max<<<red_blocks, 256, 0, s>>>(P, dst);
    k_sel_first<<<red_blocks, 256, 0, s>>>(P, dst);
    k_blk_pick<<<1, 32, 0, s>>>(BP, dst);
    k_blk_col<<<unsigned(nsm) * 8, 256, 0, s>>>(BP, dst);
  };
  // persistent steps: one cooperative launch per block (every CTA resident)
  StepSync* sync = nullptr;
  int coop_dev = 0, steps_per_sm = 0;
  cudaDeviceGetAttribute(&coop_dev, cudaDevAttrCooperativeLaunch, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&steps_per_sm, k_blk_steps, 512, 0);
  cudaGetLastError();
  const unsigned steps_blocks = unsigned(nsm) * unsigned(std::min(steps_per_sm, 2));
  const bool coop = coop_dev && steps_per_sm > 0;
  if (coop && (st = dalloc_t(p, &sync, 1, "step barrier"))) return bail(st);
  sync_mem = sync;
  if (!coop && s != nullptr) {
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      for (int i = 0; i < smax; ++i) block_step();
      if (cudaStreamEndCapture(s, &graph) != cudaSuccess || !graph || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
        exec = nullptr;
      if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();
  }

  // ---- exact compaction of the candidates below tau (see above)
  int64_t since_compact = 0;
  auto compact = [&]() -> isdf_status {
    isdf_status cst;
    // survivors per level (ordered compaction of {t : d[t] >= tau})
    int64_t keep_n[ISDF_MAX_LEVELS] = {0, 0, 0, 0}, tot_old = 0, tot_new = 0;
    std::vector<std::vector<int>> offs(nlev);
    for (int l = 0; l < nlev; ++l) {
      tot_old += nc[l];
      if (!nc[l]) continue;
      const int64_t nb = (nc[l] + kCompactBlock - 1) / kCompactBlock;
      k_flag_count<<<unsigned(nb), kCompactBlock, 0, s>>>(P.d + P.coff[l], nc[l], tau, counts);
      offs[l].resize(nb);
      cudaMemcpyAsync(offs[l].data(), counts, sizeof(int) * nb, cudaMemcpyDeviceToHost, s);
      if ((cst = cuda_check(p, cudaStreamSynchronize(s), "compaction counts"))) return cst;
      int64_t acc = 0;
      for (int64_t b = 0; b < nb; ++b) {
        const int c = offs[l][b];
        offs[l][b] = int(acc);
        acc += c;
      }
      keep_n[l] = acc;
      tot_new += acc;
      count_launches(1);
    }
    // rebuild only when at least a third of the candidates would go (the
    // rebuild re-slices the survivors' basis values; a third, checked every
    // other block, measured best: 0.418 s with a fifth, 0.401 s with a third,
    // 0.410 s with a half for the selection of the 2x2x2 diamond workload)
    if (tot_new == 0 || 3 * tot_new > 2 * tot_old) return ISDF_OK;
    double* dnew = nullptr;
    if ((cst = dalloc_t(p, &dnew, size_t(tot_new), "residual diagonal"))) return cst;
    int64_t coff_new[ISDF_MAX_LEVELS + 1] = {0};
    for (int l = 0; l < nlev; ++l) coff_new[l + 1] = coff_new[l] + keep_n[l];
    for (int l = 0; l < nlev; ++l) {
      if (!nc[l]) continue;
      Level& lv = p->lev[l];
      LevBuf& b = lb[l];
      const int64_t nn = keep_n[l], no = nc[l];
      const int64_t nb = (no + kCompactBlock - 1) / kCompactBlock;
      int *keep = nullptr, *ci = nullptr;
      double *fnew = nullptr, *d0c = nullptr;
      if (nn && ((cst = dalloc_t(p, &keep, size_t(nn), "compaction")) || (cst = dalloc_t(p, &ci, size_t(nn), "candidates")) ||
                 (cst = dalloc_t(p, &fnew, size_t(std::max<int64_t>(lv.fac_cap * nn, 1)), "selection factor columns")) ||
                 (cst = dalloc_t(p, &d0c, size_t(nn), "initial residuals")))) {
        dfree(keep), dfree(ci), dfree(fnew), dfree(d0c), dfree(dnew);
        return cst;
      }
      if (nn) {
        cudaMemcpyAsync(counts, offs[l].data(), sizeof(int) * nb, cudaMemcpyHostToDevice, s);
        k_compact<<<unsigned(nb), kCompactBlock, 0, s>>>(P.d + P.coff[l], no, tau, counts, keep);
        k_map_idx<<<unsigned((nn + 255) / 256), 256, 0, s>>>(cur_cidx[l], keep, nn, ci);
        k_gather_diag<<<unsigned((nn + 255) / 256), 256, 0, s>>>(P.d + P.coff[l], keep, nn, dnew + coff_new[l]);
        if (h.kl[l] > 0)
          k_gather_cols<<<unsigned((nn * h.kl[l] + 255) / 256), 256, 0, s>>>(lv.fac, no, keep, nn, h.kl[l], fnew);
        k_gather_diag<<<unsigned((nn + 255) / 256), 256, 0, s>>>(d0full + p->off[l], ci, nn, d0c);
        count_launches(5);
      }
      // grid -> candidate map
      if (!b.gpos && (cst = dalloc_t(p, &b.gpos, size_t(lv.ng), "grid-to-candidate map"))) {
        dfree(keep), dfree(ci), dfree(fnew), dfree(d0c), dfree(dnew);
        return cst;
      }
      cudaMemsetAsync(b.gpos, 0xFF, sizeof(int) * size_t(lv.ng), s);
      if (nn) {
        k_scatter_pos<<<unsigned((nn + 255) / 256), 256, 0, s>>>(ci, nn, b.gpos);
        count_launches(1);
      }
      // candidate-side digit planes for the survivors: basis values, then the
      // factor columns so far (fixed scales from sqrt(d0), as at set-up)
      auto setrows = [&](OzOperand& op, int64_t rows) {
        op.rows = rows;
        op.nrt = (rows + op.rt - 1) / op.rt;
      };
      setrows(b.aL, nn);
      if (lv.nN > 0) setrows(b.aN, nn);
      setrows(b.aF, nn);
      if (nn) {
        Prof pr(p, "select_slice", 8.0 * double(nn) * (lv.nG + h.kl[l]), "byte", 0);
        if (lv.nL > 0) oz_slice_ex(lv.phi, 1, lv.ng, ci, b.aL, 0, b.aL.nkt * (kOzBK / 8), false, s);
        if (lv.nN > 0)
          oz_slice_ex(lv.phi + int64_t(lv.nL) * lv.ng, 1, lv.ng, ci, b.aN, 0, b.aN.nkt * (kOzBK / 8), false, s);
        const int64_t kst_keep = b.aF.kst;
        cudaMemsetAsync(b.aF.tiles, 0, size_t(b.aF.nrt) * size_t(kst_keep) * kSlices * 128 * kOzBK * 2, s);
        k_fac_exps<<<unsigned((b.aF.nrt * 128 + 255) / 256), 256, 0, s>>>(d0c, nn, b.aF.nrt * 128, b.aF.exps);
        count_launches(1);
        if (h.kl[l] > 0) oz_slice_ex(fnew, 1, nn, nullptr, b.aF, 0, (h.kl[l] + 7) / 8, true, s);
      }
      dfree(lv.fac);
      lv.fac = fnew;
      P.fac[l] = fnew;
      cur_cidx[l] = ci;
      if (ci) own_cidx.push_back(ci);
      P.cidx[l] = ci;
      Q.cidx[l] = ci;
      Q.gpos[l] = b.gpos;
      nc[l] = nn;
      P.nc[l] = nn;
      if ((cst = cuda_check(p, cudaStreamSynchronize(s), "compaction"))) {
        dfree(keep), dfree(d0c), dfree(dnew);
        return cst;
      }
      dfree(keep);
      dfree(d0c);
    }
    dfree(p->d_diag);
    p->d_diag = dnew;
    P.d = dnew;
    Q.d = dnew;
    for (int l = 0; l <= nlev; ++l) P.coff[l] = Q.coff[l] = coff_new[l];
    P.ntot = Q.ntot = coff_new[nlev];
    BP.P = P;
    since_compact = 0;
    ++p->sel_compactions;
    return ISDF_OK;
  };
  // ---- factor capacity: before a block that could fill a level (at most
  // smax block steps and one single step), that level's factor columns move
  // to twice the storage and their digits are sliced again (fixed scales
  // from sqrt(d0), as at set-up)
  auto grow = [&]() -> isdf_status {
    isdf_status gst;
    for (int l = 0; l < nlev; ++l) {
      Level& lv = p->lev[l];
      LevBuf& b = lb[l];
      if (!nc[l]) continue;
      const int64_t full = std::min<int64_t>(nip, nc[l]);
      const int64_t need = std::min<int64_t>(full, int64_t(h.kl[l]) + smax + 1);
      if (need <= lv.fac_cap) continue;
      const int64_t cap = std::min<int64_t>(full, std::max<int64_t>(2 * lv.fac_cap, need));
      const int kl = h.kl[l];
      double *fnew = nullptr, *d0c = nullptr;
      if ((gst = dalloc_t(p, &fnew, size_t(cap * nc[l]), "selection factor columns"))) return gst;
      if (kl > 0)
        cudaMemcpyAsync(fnew, lv.fac, sizeof(double) * size_t(kl) * size_t(nc[l]), cudaMemcpyDeviceToDevice, s);
      const double* d0src = d0full + p->off[l];
      if (cur_cidx[l]) {
        if ((gst = dalloc_t(p, &d0c, size_t(nc[l]), "initial residuals"))) {
          dfree(fnew);
          return gst;
        }
        k_gather_diag<<<unsigned((nc[l] + 255) / 256), 256, 0, s>>>(d0full + p->off[l], cur_cidx[l], nc[l], d0c);
        count_launches(1);
        d0src = d0c;
      }
      oz_free(b.aF);
      oz_free(b.bF);
      if ((gst = oz_alloc(p, b.aF, nc[l], cap, 128, kSlices, "selection slices")) ||
          (gst = oz_alloc(p, b.bF, smax, cap, oz_bn(kSlices), kSlices, "selection slices"))) {
        dfree(fnew), dfree(d0c);
        return gst;
      }
      cudaMemsetAsync(b.aF.tiles, 0, size_t(oz_tile_bytes(b.aF)), s);
      k_fac_exps<<<unsigned((b.aF.nrt * 128 + 255) / 256), 256, 0, s>>>(d0src, nc[l], b.aF.nrt * 128, b.aF.exps);
      count_launches(1);
      b.aF.K = kl;
      if (kl > 0) oz_slice_ex(fnew, 1, nc[l], nullptr, b.aF, 0, (kl + 7) / 8, true, s);
      b.sliced = kl;
      gst = cuda_check(p, cudaStreamSynchronize(s), "factor capacity");
      dfree(lv.fac);
      dfree(d0c);
      lv.fac = fnew;
      lv.fac_cap = cap;
      P.fac[l] = fnew;
      if (gst) return gst;
    }
    BP.P = P;
    return ISDF_OK;
  };
  int64_t nblocks = 0, nplain = 0;
  std::vector<int> hcount(ISDF_MAX_LEVELS + 1);
  while (true) {
    if (growable && (st = grow())) return bail(st);
    // ---- 1. the speculative set S
    {
      Prof pr(p, "select_spec", double(P.ntot) * 8.0, "byte", 4);
      k_lm_count<<<unsigned(std::max<int64_t>(nbk, 1)), kCompactBlock, 0, s>>>(Q, counts);
      k_scan_counts<<<1, 1024, 0, s>>>(counts, nbk, nlist);
      k_lm_write<<<unsigned(std::max<int64_t>(nbk, 1)), kCompactBlock, 0, s>>>(Q, counts, list);
      k_top_s<<<1, 1024, 0, s>>>(Q, list, nlist, smax, O);
      count_launches(4);
    }
    cudaMemcpyAsync(hcount.data(), scount, sizeof(int) * hcount.size(), cudaMemcpyDeviceToHost, s);
    if ((st = cuda_check(p, cudaStreamSynchronize(s), "speculative set"))) return bail(st);
    // ---- 2. columns of S: three products per level, then B = w M - F
    int soff = 0;
    for (int l = 0; l < nlev; ++l) {
      const int sl = hcount[l];
      if (!sl) continue;
      Level& lv = p->lev[l];
      LevBuf& b = lb[l];
      const int kb = h.kl[l];
      auto setrows = [&](OzOperand& op, int rows) {
        op.rows = rows;
        op.nrt = (rows + op.rt - 1) / op.rt;
      };
      {
        // digits of S's rows: basis values and factor rows of the set
        Prof pb(p, "select_sslice", 8.0 * sl * (lv.nL + lv.nN + kb), "byte", kLaunchesInside);
        const unsigned gb = unsigned((sl + 127) / 128);
        setrows(b.bL, sl);
        if (lv.nL > 0) {
          k_gather_exps<<<gb, 128, 0, s>>>(stp + soff, sl, b.aL.exps, b.bL.exps);
          count_launches(1);
        }
        oz_slice_ex(lv.phi, 1, lv.ng, sg + soff, b.bL, 0, b.bL.nkt * (kOzBK / 8), lv.nL > 0, s);
        if (lv.nN > 0) {
          setrows(b.bN, sl);
          k_gather_exps<<<gb, 128, 0, s>>>(stp + soff, sl, b.aN.exps, b.bN.exps);
          count_launches(1);
          oz_slice_ex(lv.phi + int64_t(lv.nL) * lv.ng, 1, lv.ng, sg + soff, b.bN, 0, b.bN.nkt * (kOzBK / 8), true, s);
        }
        if (kb > 0) {
          setrows(b.bF, sl);
          b.bF.K = kb;
          b.bF.nkt = (kb + kOzBK - 1) / kOzBK;
          oz_slice_ex(lv.fac, 1, nc[l], stp + soff, b.bF, 0, b.bF.nkt * (kOzBK / 8), false, s);
        }
      }
      // algorithmic traffic: the candidates' FP64 basis values and factor rows, read once per block
      Prof pr(p, "select_gemm", 8.0 * double(nc[l]) * (lv.nL + lv.nN + kb), "byte", 3);
      pr.e.flop = 2.0 * double(nc[l]) * double(sl) * double(lv.nL + lv.nN + kb);
      oz_gemm(b.aL, b.bL, b.cL, nc[l], 1, 1.0, 0, 0, 1, nullptr, p->d_ozerr, s);
      if (lv.nN > 0) oz_gemm(b.aN, b.bN, b.cN, nc[l], 1, 1.0, 0, 0, 1, nullptr, p->d_ozerr, s);
      if (kb > 0) {
        b.aF.K = kb;
        b.aF.nkt = (kb + kOzBK - 1) / kOzBK;
        oz_gemm(b.aF, b.bF, b.cF, nc[l], 1, 1.0, 0, 0, 1, nullptr, p->d_ozerr, s);
      }
      const int64_t n = int64_t(sl) * nc[l];
      k_blk_combine<<<unsigned(std::min<int64_t>((n + 255) / 256, int64_t(nsm) * 16)), 256, 0, s>>>(
          b.cL, lv.nN > 0 ? b.cN : nullptr, kb > 0 ? b.cF : nullptr, n, lv.w);
      count_launches(1);
      soff += sl;
    }
    // ---- 3. greedy steps of this block
    {
      Prof pr(p, "select_steps", 0.0, "byte", coop ? 1 : 4ll * smax);
      k_blk_begin<<<1, 32, 0, s>>>(dst);
      if (coop) {
        k_sync_init<<<1, 32, 0, s>>>(sync);
        int smax_arg = smax;
        void* args[] = {&BP, &dst, &sync, &smax_arg};
        if ((st = cuda_check(p, cudaLaunchCooperativeKernel((const void*)k_blk_steps, dim3(steps_blocks), dim3(512), args,
                                                            0, s),
                             "block steps launch")))
          return bail(st);
        count_launches(2);
      } else if (exec) {
        cudaGraphLaunch(exec, s);
        count_launches(4ll * smax);
      } else {
        for (int i = 0; i < smax; ++i) block_step();
        count_launches(4ll * smax);
      }
      k_spos_clear<<<unsigned((smax + 255) / 256), 256, 0, s>>>(sidx, scount, spos);
      count_launches(2);
    }
    ++nblocks;
    if ((st = cuda_check(p, cudaGetLastError(), "selection kernels"))) return bail(st);
    int kl_before[ISDF_MAX_LEVELS];
    for (int l = 0; l < nlev; ++l) kl_before[l] = h.kl[l];
    cudaMemcpyAsync(&h, dst, sizeof(h), cudaMemcpyDeviceToHost, s);
    if ((st = cuda_check(p, cudaStreamSynchronize(s), "block state"))) return bail(st);
    if (p->opt.profile && !p->pend.empty() && p->pend.back().name == "select_steps") {
      // algorithmic bytes of the block's steps: two passes over the residual
      // (max, tie rule), then per candidate of the pivot's level the column of
      // B, the block's earlier columns, the new column and the residual
      double bytes = 0.0;
      for (int l = 0; l < nlev; ++l) {
        const double dk = h.kl[l] - kl_before[l], n = double(nc[l]);
        bytes += dk * (16.0 * double(P.ntot) + 32.0 * n) + 8.0 * n * dk * (dk - 1.0) / 2.0;
      }
      p->pend.back().work = bytes;
    }
    if (h.err || h.final_ || h.k >= nip) break;
    if (tau > 0.0 && h.dp * (1.0 - 2.0 * p->opt.tie_rel) - 2.0 * p->opt.tie_abs * h.d0 < tau) {
      *aborted = true;  // a pivot value broke the certificate: retry with a lower tau
      break;
    }
    if (h.bsteps == 0) {
      // the greedy pivot was not in S: one ordinary step
      Prof pr(p, "select_loop", 0.0, "flop", 4);
      k_blk_begin<<<1, 32, 0, s>>>(dst);
      k_sel_max<<<red_blocks, 256, 0, s>>>(P, dst);
      k_sel_first<<<red_blocks, 256, 0, s>>>(P, dst);
      k_sel_pick<<<1, 32, 0, s>>>(P, dst);
      k_sel_col<<<col_blocks, 256, smem, s>>>(P, dst);
      count_launches(5);
      ++nplain;
      cudaMemcpyAsync(&h, dst, sizeof(h), cudaMemcpyDeviceToHost, s);
      if ((st = cuda_check(p, cudaStreamSynchronize(s), "plain step"))) return bail(st);
      if (h.err || h.final_ || h.k >= nip) break;
    }
    if (tau > 0.0 && h.dp * (1.0 - 2.0 * p->opt.tie_rel) - 2.0 * p->opt.tie_abs * h.d0 < tau) {
      *aborted = true;
      break;
    }
    // ---- 4. digits of the new factor columns (whole k tiles from the first changed one)
    {
      Prof pr(p, "select_slice", 0.0, "byte", nlev);
      for (int l = 0; l < nlev; ++l) {
        LevBuf& b = lb[l];
        if (h.kl[l] <= b.sliced) continue;
        b.aF.K = h.kl[l];
        oz_slice_ex(p->lev[l].fac, 1, nc[l], nullptr, b.aF, b.sliced / 8, (h.kl[l] + 7) / 8, true, s);
        b.sliced = h.kl[l];
      }
    }
    // ---- 5. drop the candidates whose residual fell below tau (checked every
    // other block; the graph of the non-cooperative form holds the old arrays)
    if (tau > 0.0 && !exec && ++since_compact >= 2) {
      if ((st = compact())) return bail(st);
      nbk = (P.ntot + kCompactBlock - 1) / kCompactBlock;
    }
  }
  if ((st = oz_check(p))) return bail(st);
  *nfound = h.k;
  for (int l = 0; l < nlev; ++l) kl_out[l] = h.kl[l];
  p->sel_blocks = nblocks;
  p->sel_plain_steps = nplain;
  cleanup();
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
    if (lv.nG == 0) {  // a level without basis values of its own (local grids' level 0)
      cudaMemsetAsync(d0 + p->off[l], 0, sizeof(double) * size_t(lv.ng), s);
      continue;
    }
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
  // with the coarsest level as the universal sinc grid it takes no part in
  // the selection: no candidates there, and d_0 is the finer levels' largest;
  // levels below sel_lo (local grids' level 0) have their own selections
  const int nsel = p->opt.coarse_sinc ? p->nlev - 1 : p->nlev;
  const int lo = p->sel_lo;
  int kl[ISDF_MAX_LEVELS];
  bool aborted = false;
  p->sel_compactions = 0;
  auto loop = [&](int* const* ci, const int64_t* n, double tau = 0.0) {
    aborted = false;
    return p->opt.select_block > 0 ? select_loop_blocked(p, nip, tol, d0, ci, n, nfound, kl, tau, &aborted)
                                   : select_loop(p, nip, tol, d0, ci, n, nfound, kl);
  };
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
    return done(loop(cidx, nc));
  }
  if (!p->opt.prefilter) {
    for (int l = 0; l < p->nlev; ++l) nc[l] = (l >= lo && l < nsel) ? p->lev[l].ng : 0;
    return done(loop(cidx, nc));
  }
  // exact prefilter: tau relative to the largest initial residual d_0
  unsigned long long* dmax_slot = nullptr;
  if ((st = dalloc_t(p, &dmax_slot, 1, "max slot"))) return done(st);
  cudaMemsetAsync(dmax_slot, 0, sizeof(unsigned long long), s);
  k_vec_max<<<152 * 4, 256, 0, s>>>(d0, p->off[nsel], dmax_slot);
  count_launches(1);
  unsigned long long bits = 0;
  cudaMemcpyAsync(&bits, dmax_slot, sizeof(bits), cudaMemcpyDeviceToHost, s);
  st = cuda_check(p, cudaStreamSynchronize(s), "prefilter max");
  dfree(dmax_slot);
  if (st) return done(st);
  double dmax0;
  std::memcpy(&dmax0, &bits, sizeof(dmax0));
  // attempts: the blocked form starts at 1e-5 d_0 (its candidates shrink as
  // the residuals fall below tau, and an attempt whose pivot values break the
  // certificate stops at once); the step-by-step form at 1e-6 d_0
  const bool blocked = p->opt.select_block > 0;
  const double taus[4] = {blocked ? 1e-5 : 1e-6, 1e-6, 1e-9, 0.0};
  for (int attempt = blocked ? 0 : 1; attempt < 4; ++attempt) {
    const double tau = (attempt == 0 ? taus[0] : taus[attempt]) * dmax0;
    free_cidx();
    for (int l = 0; l < p->nlev; ++l) {
      Level& lv = p->lev[l];
      if (l >= nsel || l < lo) {
        nc[l] = 0;
        continue;
      }
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
    for (int l = lo; l < nsel; ++l) all_kept = all_kept && nc[l] == p->lev[l].ng;
    if (all_kept) {  // nothing dropped: this is the full greedy run
      free_cidx();
      return done(loop(cidx, nc));
    }
    st = loop(cidx, nc, tau);
    if (st || tau <= 0.0) return done(st);
    if (aborted) continue;
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
