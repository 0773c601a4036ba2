// Exchange build from the four-term multigrid THC form (Section III.A, Eq. 8).
//
// With c_{mu lam}(P) = X^L_{mu P} X^G_{lam P} + X^N_{mu P} X^L_{lam P} and
// D = C C^T, K = sum_PQ V_PQ c(P) D c(Q) factorises through the occupied
// space:  c(P) C = x_L(P) y_G(P)^T + x_N(P) y_L(P)^T  with  Y_A = X^A^T C, so
//   K = [X^L X^N] W [X^L X^N]^T,
//   W = [[V o R_GG, V o R_GL], [V o R_LG, V o R_LL]],  R_AB = Y_A Y_B^T.
// E_x = -Tr(D K) = -sum_{mu i} C_{mu i} (K C)_{mu i}, reduced in FP64.
#include <algorithm>

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
  if (splits > 1 && (st = dalloc_t(p, &work, size_t(splits) * M * N, "split-k partials")))
    return oz_free(A), oz_free(B), st;
  oz_gemm(A, B, C, ldc, 0, 1.0, 0, sym, int(splits), work, p->d_ozerr, s);
  st = oz_check(p);
  oz_free(A);
  oz_free(B);
  dfree(work);
  return st;
}

}  // namespace

isdf_status exchange_run(Plan* p, const double* dC, int n, double* dK, double* Ex) {
  cudaStream_t s = p->stream;
  const int64_t nip = p->nip, N = p->nfun, n2 = 2 * nip;
  double *yl = nullptr, *yn = nullptr, *yg = nullptr, *rgg = nullptr, *rgl = nullptr, *rll = nullptr, *W = nullptr,
         *x2 = nullptr, *T = nullptr, *kc = nullptr, *part = nullptr, *dex = nullptr;
  auto cleanup = [&]() {
    for (double* q : {yl, yn, yg, rgg, rgl, rll, W, x2, T, kc, part, dex}) dfree(q);
  };
  isdf_status st;
  if ((st = dalloc_t(p, &yl, size_t(nip) * n, "Y_L")) || (st = dalloc_t(p, &yn, size_t(nip) * n, "Y_N")) ||
      (st = dalloc_t(p, &yg, size_t(nip) * n, "Y_G")) || (st = dalloc_t(p, &rgg, size_t(nip) * nip, "R_GG")) ||
      (st = dalloc_t(p, &rgl, size_t(nip) * nip, "R_GL")) || (st = dalloc_t(p, &rll, size_t(nip) * nip, "R_LL")) ||
      (st = dalloc_t(p, &W, size_t(n2) * n2, "W")) || (st = dalloc_t(p, &x2, size_t(N) * n2, "[X^L X^N]")) ||
      (st = dalloc_t(p, &T, size_t(n2) * N, "W X^T")) || (st = dalloc_t(p, &kc, size_t(N) * n, "K C")) ||
      (st = dalloc_t(p, &part, 1024, "reduction")) || (st = dalloc_t(p, &dex, 1, "E_x"))) {
    cleanup();
    return st;
  }
  const double fl = 2.0 * 2.0 * nip * n * N + 2.0 * nip * (nip + 1) * n * 2.0 + 2.0 * nip * nip * n +
                    2.0 * n2 * n2 * N + 2.0 * N * N * n2 + 2.0 * N * N * n;
  {
  Prof pr(p, "exchange", fl, "flop", 13);
  if (p->opt.precision == 1) {
    // Y_A[P][i] = sum_mu X^A[mu][P] C[mu][i]: rows P (stride 1, k stride nip) against rows i of C^T
    if ((st = tc_product(p, p->XL, nip, 1, nip, dC, n, 1, n, N, yl, n, 0)) ||
        (st = tc_product(p, p->XN, nip, 1, nip, dC, n, 1, n, N, yn, n, 0))) {
      cleanup();
      return st;
    }
  } else {
    dgemm(gemm(1, 0, nip, n, N, p->XL, nip, dC, n, yl, n), s);  // Y_L = X^L^T C
    dgemm(gemm(1, 0, nip, n, N, p->XN, nip, dC, n, yn, n), s);  // Y_N = X^N^T C
  }
  k_add<<<unsigned((nip * n + 255) / 256), 256, 0, s>>>(nip * n, yl, yn, yg);
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
  k_concat<<<unsigned((N * n2 + 255) / 256), 256, 0, s>>>(N, nip, p->XL, p->XN, x2);
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
  if (p->opt.precision == 1) {
    // (K C)[mu][i] = sum_nu K[mu][nu] C[nu][i]
    if ((st = tc_product(p, dK, N, N, 1, dC, n, 1, n, N, kc, n, 0))) {
      cleanup();
      return st;
    }
  } else {
    dgemm(gemm(0, 0, N, n, N, dK, N, dC, n, kc, n), s);  // K C
  }
  const int nb = 512;  // partial sums of the E_x reduction
  k_dot_partial<<<nb, 256, 0, s>>>(N * n, dC, kc, part);
  k_sum_final<<<1, 256, 0, s>>>(nb, part, -1.0, dex);
  }
  st = cuda_check(p, cudaMemcpyAsync(Ex, dex, sizeof(double), cudaMemcpyDeviceToHost, s), "E_x copy");
  if (!st) st = cuda_check(p, cudaStreamSynchronize(s), "exchange");
  cleanup();
  return st;
}

}  // namespace isdf
