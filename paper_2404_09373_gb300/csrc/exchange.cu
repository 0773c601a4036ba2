// Exchange build from the four-term multigrid THC form (Section III.A, Eq. 8).
//
// With c_{mu lam}(P) = X^L_{mu P} X^G_{lam P} + X^N_{mu P} X^L_{lam P} and
// D = C C^T, K = sum_PQ V_PQ c(P) D c(Q) factorises through the occupied
// space:  c(P) C = x_L(P) y_G(P)^T + x_N(P) y_L(P)^T  with  Y_A = X^A^T C, so
//   K = [X^L X^N] W [X^L X^N]^T,
//   W = [[V o R_GG, V o R_GL], [V o R_LG, V o R_LL]],  R_AB = Y_A Y_B^T.
// E_x = -Tr(D K) = -sum_{mu i} C_{mu i} (K C)_{mu i}, reduced in FP64.
//
// Block structure of (mu|xi) (Section III.A, figure of (mu|xi)^L,N,G): a
// pivot of level l carries X^L only on the functions of level l and X^N only
// on the coarser ones.  With the functions ordered by level (a permutation)
// and the pivots level by level, every nonzero block is a contiguous
// sub-matrix, so the projections Y_A and the occupied-space product below
// run over the nonzero blocks only.
//
// occ-RI output (Section III.A, last paragraphs; Section II.A, the K_ip of
// the occ-RI remedy): K_ip = sum_j (mu j|j i) = (K C)_{mu i}
//   = [X^L X^N] W [Y_L; Y_N],
// formed without K: U = W [Y_L; Y_N] (2 nip x n), then per function level m
// (K C)[F_m] = X^L[F_m, P_m] U_L[P_m] + X^N[F_m, P_<m] U_N[P_<m].
#include <algorithm>
#include <numeric>
#include <vector>

#include "internal.cuh"

namespace isdf {
namespace {

__global__ void k_add(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ c) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e < n) c[e] = a[e] + b[e];
}

// R_GG and R_LL hold their lower triangles only (symmetric GEMMs).
__global__ void k_build_w(int64_t nip, const double* __restrict__ V, const double* __restrict__ rgg,
                          const double* __restrict__ rgl, const double* __restrict__ rll, double* __restrict__ W) {
  const int64_t n2 = 2 * nip;
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n2 * n2) return;
  const int64_t P = e / n2, Q = e % n2;
  const int bp = P >= nip, bq = Q >= nip;
  const int64_t p = P - bp * nip, q = Q - bq * nip;
  const int64_t hi = p > q ? p : q, lo = p > q ? q : p;
  double r;
  if (!bp && !bq)
    r = rgg[hi * nip + lo];
  else if (!bp && bq)
    r = rgl[p * nip + q];
  else if (bp && !bq)
    r = rgl[q * nip + p];
  else
    r = rll[hi * nip + lo];
  W[e] = V[p * nip + q] * r;
}

// [X^L | X^N] as one N x 2nip matrix
__global__ void k_concat(int64_t nfun, int64_t nip, const double* __restrict__ xl, const double* __restrict__ xn,
                         double* __restrict__ x2) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= nfun * 2 * nip) return;
  const int64_t mu = e / (2 * nip), c = e % (2 * nip);
  x2[e] = c < nip ? xl[mu * nip + c] : xn[mu * nip + c - nip];
}

// C[r][c] += t[r][c]  (C with leading dimension ldc, t dense M x N)
__global__ void k_add2d(int64_t M, int64_t N, const double* __restrict__ t, double* __restrict__ C, int64_t ldc) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= M * N) return;
  C[(e / N) * ldc + e % N] += t[e];
}

// out[i][c] = in[perm[i]][c]  (rows gathered by the level order)
__global__ void k_gather_rows(int64_t rows, int64_t cols, const int* __restrict__ perm, const double* __restrict__ in,
                              double* __restrict__ out) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const int64_t i = e / cols, c = e % cols;
  out[e] = in[int64_t(perm[i]) * cols + c];
}

// out[perm[i]][c] = in[i][c]
__global__ void k_scatter_rows(int64_t rows, int64_t cols, const int* __restrict__ perm, const double* __restrict__ in,
                               double* __restrict__ out) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const int64_t i = e / cols, c = e % cols;
  out[int64_t(perm[i]) * cols + c] = in[e];
}

// partial[b] = sum over this block's slice of C o KC (FP64)
__global__ void k_dot_partial(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                              double* __restrict__ part) {
  __shared__ double sh[256];
  double t = 0.0;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
    t = fma(a[e], b[e], t);
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_final(int nb, const double* __restrict__ part, double scale, double* __restrict__ out) {
  __shared__ double sh[256];
  double t = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) t += part[i];
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = scale * sh[0];
}

GemmArgs gemm(int ta, int tb, int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, const double* B,
              int64_t ldb, double* C, int64_t ldc, int sym = 0) {
  GemmArgs g;
  g.ta = ta;
  g.tb = tb;
  g.M = M;
  g.N = N;
  g.K = K;
  g.A = A;
  g.lda = lda;
  g.B = B;
  g.ldb = ldb;
  g.C = C;
  g.ldc = ldc;
  g.sym = sym;
  return g;
}

// C (M x N) = A_rows B_rows^T on the tensor cores; A given as rows x K with
// element (r, k) at a[r*sar + k*sak], B likewise.
isdf_status tc_product(Plan* p, const double* a, int64_t M, int64_t sar, int64_t sak, const double* b, int64_t N,
                       int64_t sbr, int64_t sbk, int64_t K, double* C, int64_t ldc, int sym) {
  cudaStream_t s = p->stream;
  const int S = 5;
  OzOperand A, B;
  double* work = nullptr;
  isdf_status st;
  if ((st = oz_alloc(p, A, M, K, 128, S, "exchange slices")) || (st = oz_alloc(p, B, N, K, oz_bn(S), S, "exchange slices")))
    return oz_free(A), oz_free(B), st;
  oz_slice(a, sar, sak, nullptr, 1.0, A, s);
  oz_slice(b, sbr, sbk, nullptr, 1.0, B, s);
  int64_t tiles = A.nrt * B.nrt;
  int64_t splits = std::max<int64_t>(1, std::min<int64_t>((2 * 152 + tiles - 1) / tiles, A.nkt / 32 + 1));
  splits = std::min<int64_t>(splits, 16);
  splits = oz_tuned_splits(p, A, B, C, ldc, 0, sym, int(splits), s);
  if (splits > 1 && (st = dalloc_t(p, &work, size_t(splits) * M * N, "split-k partials")))
    return oz_free(A), oz_free(B), st;
  oz_gemm(A, B, C, ldc, 0, 1.0, 0, sym, int(splits), work, p->d_ozerr, s);
  // under graph capture the error word is read after the graph has run
  st = p->capturing ? cuda_check(p, cudaGetLastError(), "tensor-core launch") : oz_check(p);
  oz_free(A);
  oz_free(B);
  dfree(work);
  return st;
}

}  // namespace

isdf_status tc_product_ex(Plan* p, const double* a, int64_t M, int64_t sar, int64_t sak, const double* b, int64_t N,
                        int64_t sbr, int64_t sbk, int64_t K, double* C, int64_t ldc) {
  return tc_product(p, a, M, sar, sak, b, N, sbr, sbk, K, C, ldc, 0);
}

namespace {

// C (M x N, ldc) = A B^T over sub-blocks, FP64 SIMT (precision 0) or
// tensor cores (precision 1); A element (r, k) at a[r sar + k sak], B
// element (c, k) at b[c sbr + k sbk].  accumulate: C += A B^T (through
// `tmp`, M x N, on the tensor-core path).
isdf_status block_product(Plan* p, const double* a, int64_t M, int64_t sar, int64_t sak, const double* b, int64_t N,
                          int64_t sbr, int64_t sbk, int64_t K, double* C, int64_t ldc, bool accumulate, double* tmp) {
  cudaStream_t s = p->stream;
  if (M == 0 || N == 0) return ISDF_OK;
  if (K == 0) {
    if (!accumulate) cudaMemset2DAsync(C, sizeof(double) * size_t(ldc), 0, sizeof(double) * size_t(N), size_t(M), s);
    return ISDF_OK;
  }
  if (p->opt.precision == 1) {
    if (!accumulate) return tc_product(p, a, M, sar, sak, b, N, sbr, sbk, K, C, ldc, 0);
    isdf_status st = tc_product(p, a, M, sar, sak, b, N, sbr, sbk, K, tmp, N, 0);
    if (st) return st;
    k_add2d<<<unsigned((M * N + 255) / 256), 256, 0, s>>>(M, N, tmp, C, ldc);
    count_launches(1);
    return ISDF_OK;
  }
  // SIMT FP64: express the strided operands through the transpose flags
  GemmArgs g;
  g.M = M, g.N = N, g.K = K;
  if (sak == 1) g.ta = 0, g.A = a, g.lda = sar;  // A row-major M x K
  else g.ta = 1, g.A = a, g.lda = sak;           // A^T stored row-major (K x M), sar == 1
  if (sbk == 1) g.tb = 1, g.B = b, g.ldb = sbr;  // B rows are k-contiguous: op(B) = B^T
  else g.tb = 0, g.B = b, g.ldb = sbk;           // B stored as K x N row-major, sbr == 1
  g.C = C, g.ldc = ldc;
  g.beta = accumulate ? 1.0 : 0.0;
  dgemm(g, s);
  return ISDF_OK;
}

struct LevelOrder {
  std::vector<int> perm;             // permuted position -> function
  int fb[ISDF_MAX_LEVELS + 1] = {0};  // function-level ranges in permuted order
};

LevelOrder level_order(const Plan* p) {
  LevelOrder o;
  o.perm.resize(p->nfun);
  std::iota(o.perm.begin(), o.perm.end(), 0);
  std::stable_sort(o.perm.begin(), o.perm.end(), [&](int a, int b) { return p->f_level[a] < p->f_level[b]; });
  for (int l = 0; l < p->nlev; ++l) {
    int c = 0;
    for (int mu = 0; mu < p->nfun; ++mu) c += p->f_level[mu] == l;
    o.fb[l + 1] = o.fb[l] + c;
  }
  return o;
}

}  // namespace

// dK: N x N exchange matrix (nullable); dKC: N x n occ-RI output K C (nullable).
isdf_status exchange_run(Plan* p, const double* dC, int n, double* dK, double* dKC, double* Ex) {
  if (p->opt.coarse_sinc && !dK) {
    // the coarse-grid terms are built into K: the occ-RI output is K C
    double* tk = nullptr;
    isdf_status st = dalloc_t(p, &tk, size_t(p->nfun) * p->nfun, "K");
    if (!st) st = exchange_run(p, dC, n, tk, dKC, Ex);
    dfree(tk);
    return st;
  }
  cudaStream_t s = p->stream;
  const int64_t nip = p->nip, N = p->nfun, n2 = 2 * nip;
  const LevelOrder lo = level_order(p);
  const int nlev = p->nlev;
  double *y2 = nullptr, *yg = nullptr, *rgg = nullptr, *rgl = nullptr, *rll = nullptr, *W = nullptr, *x2 = nullptr,
         *T = nullptr, *kc = nullptr, *kcp = nullptr, *cp = nullptr, *xlp = nullptr, *xnp = nullptr, *u = nullptr,
         *tmp = nullptr, *part = nullptr, *dex = nullptr;
  auto cleanup = [&]() {
    for (double* q : {y2, yg, rgg, rgl, rll, W, x2, T, kc, kcp, cp, xlp, xnp, u, tmp, part, dex}) dfree(q);
  };
  isdf_status st;
  if (!p->d_perm) {
    // the level order lives with the plan (uploaded once, outside any capture)
    if (p->capturing) return fail(p, ISDF_ERR_STATE, "exchange under capture before a first exchange");
    if ((st = dalloc_t(p, &p->d_perm, size_t(N), "level order"))) return st;
    if ((st = cuda_check(p, cudaMemcpyAsync(p->d_perm, lo.perm.data(), sizeof(int) * size_t(N), cudaMemcpyHostToDevice,
                                            s),
                         "level order")) ||
        (st = cuda_check(p, cudaStreamSynchronize(s), "level order")))
      return st;
  }
  const int* dperm = p->d_perm;
  if ((st = dalloc_t(p, &y2, size_t(n2) * n, "Y_L, Y_N")) || (st = dalloc_t(p, &yg, size_t(nip) * n, "Y_G")) ||
      (st = dalloc_t(p, &rgg, size_t(nip) * nip, "R_GG")) || (st = dalloc_t(p, &rgl, size_t(nip) * nip, "R_GL")) ||
      (st = dalloc_t(p, &rll, size_t(nip) * nip, "R_LL")) || (st = dalloc_t(p, &W, size_t(n2) * n2, "W")) ||
      (st = dalloc_t(p, &cp, size_t(N) * n, "C by level")) || (st = dalloc_t(p, &xlp, size_t(N) * nip, "X^L by level")) ||
      (st = dalloc_t(p, &xnp, size_t(N) * nip, "X^N by level")) || (st = dalloc_t(p, &kc, size_t(N) * n, "K C")) ||
      (st = dalloc_t(p, &tmp, size_t(N) * std::max<int64_t>(n, nip), "block partials")) ||
      (st = dalloc_t(p, &part, 1024, "reduction")) ||
      (st = dalloc_t(p, &dex, 1, "E_x"))) {
    cleanup();
    return st;
  }
  if (dK && ((st = dalloc_t(p, &x2, size_t(N) * n2, "[X^L X^N]")) || (st = dalloc_t(p, &T, size_t(n2) * N, "W X^T")))) {
    cleanup();
    return st;
  }
  if (!dK && ((st = dalloc_t(p, &u, size_t(n2) * n, "W Y")) || (st = dalloc_t(p, &kcp, size_t(N) * n, "K C by level")))) {
    cleanup();
    return st;
  }
  double* yl = y2;
  double* yn = y2 + nip * n;
  // nonzero (function level x pivot level) blocks: X^L on (F_l, P_l), X^N on (F_>l, P_l)
  double fl_y = 0.0, fl_kc = 0.0;
  for (int l = 0; l < nlev; ++l) {
    const double k = p->lev[l].k, fL = lo.fb[l + 1] - lo.fb[l], fN = lo.fb[nlev] - lo.fb[l + 1];
    fl_y += 2.0 * k * n * (fL + fN);
    fl_kc += 2.0 * fL * n * (k + p->poff[l]);
  }
  const double fl_r = 2.0 * nip * (nip + 1) * n * 2.0 + 2.0 * nip * nip * n;
  const double fl = fl_y + fl_r + (dK ? 2.0 * n2 * n2 * N + 2.0 * N * N * n2 + 2.0 * N * N * n : 2.0 * n2 * n2 * n + fl_kc);
  {
    Prof pr(p, "exchange", fl, "flop", kLaunchesInside);
    k_gather_rows<<<unsigned((N * n + 255) / 256), 256, 0, s>>>(N, n, dperm, dC, cp);
    k_gather_rows<<<unsigned((N * nip + 255) / 256), 256, 0, s>>>(N, nip, dperm, p->XL, xlp);
    k_gather_rows<<<unsigned((N * nip + 255) / 256), 256, 0, s>>>(N, nip, dperm, p->XN, xnp);
    count_launches(3);
    // Y_A[P_l][i] = sum over the block's functions mu of X^A[mu][P] C[mu][i]
    for (int l = 0; l < nlev; ++l) {
      const int64_t k = p->lev[l].k, q0 = p->poff[l], f0 = lo.fb[l], f1 = lo.fb[l + 1], f2 = lo.fb[nlev];
      if (!k) continue;
      // local grids: X^N of a level-0 pivot also holds the finest-level
      // functions of higher-index atoms
      const int64_t fn = (l == 0 && p->opt.local_grids) ? f0 : f1;
      if ((st = block_product(p, xlp + f0 * nip + q0, k, 1, nip, cp + f0 * n, n, 1, n, f1 - f0, yl + q0 * n, n, false,
                              tmp)) ||
          (st = block_product(p, xnp + fn * nip + q0, k, 1, nip, cp + fn * n, n, 1, n, f2 - fn, yn + q0 * n, n, false,
                              tmp))) {
        cleanup();
        return st;
      }
    }
    k_add<<<unsigned((nip * n + 255) / 256), 256, 0, s>>>(nip * n, yl, yn, yg);
    count_launches(1);
    if (p->opt.precision == 1) {
      if ((st = tc_product(p, yg, nip, n, 1, yg, nip, n, 1, n, rgg, nip, 1)) ||
          (st = tc_product(p, yg, nip, n, 1, yl, nip, n, 1, n, rgl, nip, 0)) ||
          (st = tc_product(p, yl, nip, n, 1, yl, nip, n, 1, n, rll, nip, 1))) {
        cleanup();
        return st;
      }
    } else {
      dgemm(gemm(0, 1, nip, nip, n, yg, n, yg, n, rgg, nip, 1), s);
      dgemm(gemm(0, 1, nip, nip, n, yg, n, yl, n, rgl, nip), s);
      dgemm(gemm(0, 1, nip, nip, n, yl, n, yl, n, rll, nip, 1), s);
    }
    k_build_w<<<unsigned((n2 * n2 + 255) / 256), 256, 0, s>>>(nip, p->V, rgg, rgl, rll, W);
    count_launches(1);
    if (dK) {
      k_concat<<<unsigned((N * n2 + 255) / 256), 256, 0, s>>>(N, nip, p->XL, p->XN, x2);
      count_launches(1);
      if (p->opt.precision == 1) {
        // T = W X2^T (rows of W against rows of X2), K = X2 T (rows of X2 against columns of T)
        if ((st = tc_product(p, W, n2, n2, 1, x2, N, n2, 1, n2, T, N, 0)) ||
            (st = tc_product(p, x2, N, n2, 1, T, N, 1, N, n2, dK, N, 0))) {
          cleanup();
          return st;
        }
      } else {
        dgemm(gemm(0, 1, n2, N, n2, W, n2, x2, n2, T, N), s);  // T = W X2^T
        dgemm(gemm(0, 0, N, N, n2, x2, n2, T, N, dK, N), s);   // K = X2 T
      }
      // the universal sinc grid's terms: K_FU + K_FU^T + K_UU
      if (p->opt.coarse_sinc && (st = sinc_exchange(p, dC, yl, yg, n, dK))) {
        cleanup();
        return st;
      }
      if (p->opt.precision == 1) {
        if ((st = tc_product(p, dK, N, N, 1, dC, n, 1, n, N, kc, n, 0))) {  // (K C)[mu][i]
          cleanup();
          return st;
        }
      } else {
        dgemm(gemm(0, 0, N, n, N, dK, N, dC, n, kc, n), s);  // K C
      }
      if (dKC) cudaMemcpyAsync(dKC, kc, sizeof(double) * size_t(N) * n, cudaMemcpyDeviceToDevice, s);
    } else {
      // U = W [Y_L; Y_N]: rows of W against the columns i of Y2
      if ((st = block_product(p, W, n2, n2, 1, y2, n, 1, n, n2, u, n, false, tmp))) {
        cleanup();
        return st;
      }
      // (K C)[F_m] = X^L[F_m, P_m] U_L[P_m] + X^N[F_m, P_<m] U_N[P_<m], in level order
      for (int m = 0; m < nlev; ++m) {
        const int64_t f0 = lo.fb[m], fm = lo.fb[m + 1] - lo.fb[m], q0 = p->poff[m], k = p->lev[m].k;
        if (!fm) continue;
        // local grids: the finest-level functions also have X^N on level-0 pivots
        const int64_t qn = (m == 0 && p->opt.local_grids) ? p->poff[1] : q0;
        if ((st = block_product(p, xlp + f0 * nip + q0, fm, nip, 1, u + q0 * n, n, 1, n, k, kcp + f0 * n, n, false,
                                tmp)) ||
            (st = block_product(p, xnp + f0 * nip, fm, nip, 1, u + nip * n, n, 1, n, qn, kcp + f0 * n, n, true, tmp))) {
          cleanup();
          return st;
        }
      }
      k_scatter_rows<<<unsigned((N * n + 255) / 256), 256, 0, s>>>(N, n, dperm, kcp, kc);
      count_launches(1);
      if (dKC) cudaMemcpyAsync(dKC, kc, sizeof(double) * size_t(N) * n, cudaMemcpyDeviceToDevice, s);
    }
    const int nb = 512;  // partial sums of the E_x reduction
    k_dot_partial<<<nb, 256, 0, s>>>(N * n, dC, kc, part);
    k_sum_final<<<1, 256, 0, s>>>(nb, part, -1.0, dex);
    count_launches(2);
  }
  if (p->capturing) {
    st = cuda_check(p, cudaMemcpyAsync(p->d_ex_slot, dex, sizeof(double), cudaMemcpyDeviceToDevice, s), "E_x copy");
    cleanup();
    return st;
  }
  st = cuda_check(p, cudaMemcpyAsync(Ex, dex, sizeof(double), cudaMemcpyDeviceToHost, s), "E_x copy");
  if (!st) st = cuda_check(p, cudaStreamSynchronize(s), "exchange");
  if (!st) st = oz_check(p);
  cleanup();
  return st;
}

}  // namespace isdf
