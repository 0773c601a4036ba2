// FP64 SIMT dense kernels: tiled GEMM, the fused Hadamard GEMM of the fit,
// blocked Cholesky and triangular inverse.  These are the "plain FP64" form of
// the contractions (options.precision = 0).
#include "internal.cuh"

namespace isdf {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

struct Tiles {
  double a[BK][BM + 1];
  double b[BK][BN + 1];
};

// Accumulate acc[i][j] += sum_{k in [kbeg,kend)} opA(m0+ty+16i, k) w(k) opB(k, n0+tx+16j).
template <int TA, int TB>
__device__ __forceinline__ void tile_accumulate(double (&acc)[4][4], Tiles& t, const double* __restrict__ A,
                                                int64_t lda, const double* __restrict__ B, int64_t ldb,
                                                const double* __restrict__ kw, int64_t M, int64_t N, int64_t m0,
                                                int64_t n0, int64_t kbeg, int64_t kend) {
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + NT * q;
      int kk, mm;
      if (TA) {
        kk = e / BM;
        mm = e % BM;
      } else {
        mm = e / BK;
        kk = e % BK;
      }
      const int64_t gk = k0 + kk, gm = m0 + mm;
      double v = 0.0;
      if (gk < kend && gm < M) {
        v = TA ? A[gk * lda + gm] : A[gm * lda + gk];
        if (kw) v *= kw[gk];
      }
      t.a[kk][mm] = v;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + NT * q;
      int kk, nn;
      if (TB) {
        nn = e / BK;
        kk = e % BK;
      } else {
        kk = e / BN;
        nn = e % BN;
      }
      const int64_t gk = k0 + kk, gn = n0 + nn;
      double v = 0.0;
      if (gk < kend && gn < N) v = TB ? B[gn * ldb + gk] : B[gk * ldb + gn];
      t.b[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = t.a[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = t.b[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
}

template <int TA, int TB>
__global__ __launch_bounds__(NT) void k_dgemm(GemmArgs g) {
  const int64_t m0 = int64_t(blockIdx.y) * BM, n0 = int64_t(blockIdx.x) * BN;
  if (g.sym && n0 > m0 + BM - 1) return;
  __shared__ Tiles t;
  double acc[4][4] = {};
  int64_t kbeg = 0, kend = g.K;
  if (g.tri == 1) kend = (m0 + BM < g.K) ? m0 + BM : g.K;
  if (g.tri == 2) kbeg = m0;
  tile_accumulate<TA, TB>(acc, t, g.A, g.lda, g.B, g.ldb, g.kw, g.M, g.N, m0, n0, kbeg, kend);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t m = m0 + ty + 16 * i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t n = n0 + tx + 16 * j;
      if (n >= g.N) continue;
      double* c = g.C + m * g.ldc + n;
      const double v = g.alpha * acc[i][j];
      *c = (g.beta == 0.0) ? v : fma(g.beta, *c, v);
    }
  }
}

// (ZC^T)^T[j][g] = aL (aL + 2 aN), aL = sum_{r<nL} phiP[r][j] phi[r][g],
// aN = sum_{nL<=r<nG} phiP[r][j] phi[r][g]   (M_l[:, P], Eq. 2 / Eq. 3)
__global__ __launch_bounds__(NT) void k_zc(int64_t k, int64_t ng, int nL, int nG, const double* __restrict__ phiP,
                                           const double* __restrict__ phi, double* __restrict__ out) {
  const int64_t m0 = int64_t(blockIdx.y) * BM, n0 = int64_t(blockIdx.x) * BN;
  __shared__ Tiles t;
  double aL[4][4] = {}, aN[4][4] = {};
  tile_accumulate<1, 0>(aL, t, phiP, k, phi, ng, nullptr, k, ng, m0, n0, 0, nL);
  tile_accumulate<1, 0>(aN, t, phiP, k, phi, ng, nullptr, k, ng, m0, n0, nL, nG);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t m = m0 + ty + 16 * i;
    if (m >= k) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t n = n0 + tx + 16 * j;
      if (n >= ng) continue;
      const double l = aL[i][j];
      out[m * ng + n] = l * (l + 2.0 * aN[i][j]);
    }
  }
}

// ---- Cholesky (right-looking, 64-column blocks) ----
constexpr int CB = 64;

// Factor the b x b diagonal block at (kb, kb) in shared memory.
__global__ void k_potrf_diag(double* A, int64_t lda, int64_t kb, int b, int* err) {
  __shared__ double s[CB][CB + 1];
  const int tid = threadIdx.x;
  for (int e = tid; e < b * b; e += blockDim.x) s[e / b][e % b] = A[(kb + e / b) * lda + kb + e % b];
  __syncthreads();
  __shared__ double rpiv;
  for (int j = 0; j < b; ++j) {
    if (tid == 0) {
      double d = s[j][j];
      if (!(d > 0.0) || !isfinite(d)) {
        atomicMin(err, int(kb + j));
        d = 1.0;
      }
      s[j][j] = sqrt(d);
      rpiv = 1.0 / s[j][j];  // one division per column; the column is scaled by the reciprocal
    }
    __syncthreads();
    const double rp = rpiv;
    for (int i = j + 1 + tid; i < b; i += blockDim.x) s[i][j] *= rp;
    __syncthreads();
    for (int e = tid; e < (b - j - 1) * (b - j - 1); e += blockDim.x) {
      const int i = j + 1 + e / (b - j - 1), c = j + 1 + e % (b - j - 1);
      if (c <= i) s[i][c] -= s[i][j] * s[c][j];
    }
    __syncthreads();
  }
  for (int e = tid; e < b * b; e += blockDim.x) {
    const int i = e / b, c = e % b;
    A[(kb + i) * lda + kb + c] = (c <= i) ? s[i][c] : 0.0;
  }
}

// Rows i >= r0 of the panel: x L_kk^T = a  (forward substitution per row).
__global__ __launch_bounds__(64) void k_trsm_panel(double* A, int64_t lda, int64_t n, int64_t kb, int b, int64_t r0) {
  __shared__ double l[CB][CB + 1];
  __shared__ double rdiag[CB];
  for (int e = threadIdx.x; e < CB * CB; e += blockDim.x) {
    const int i = e / CB, c = e % CB;
    double v = (i == c) ? 1.0 : 0.0;
    if (i < b && c < b) v = A[(kb + i) * lda + kb + c];
    l[i][c] = v;
  }
  __syncthreads();
  // reciprocals of the diagonal once per CTA: the rows then multiply
  for (int c = threadIdx.x; c < CB; c += blockDim.x) rdiag[c] = 1.0 / l[c][c];
  __syncthreads();
  const int64_t row = r0 + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (row >= n) return;
  double x[CB];
#pragma unroll
  for (int c = 0; c < CB; ++c) x[c] = (c < b) ? A[row * lda + kb + c] : 0.0;
#pragma unroll
  for (int c = 0; c < CB; ++c) {
    double v = x[c];
#pragma unroll
    for (int p = 0; p < c; ++p) v -= x[p] * l[c][p];
    x[c] = v * rdiag[c];
  }
#pragma unroll
  for (int c = 0; c < CB; ++c)
    if (c < b) A[row * lda + kb + c] = x[c];
}

// Inverse of each b x b lower-triangular diagonal block (one CTA per block).
__global__ __launch_bounds__(64) void k_trtri_diag(const double* Lm, double* Li, int64_t n, int64_t ld) {
  __shared__ double l[CB][CB + 1];
  __shared__ double v[CB][CB + 1];
  const int64_t kb = int64_t(blockIdx.x) * CB;
  const int b = int((n - kb < CB) ? n - kb : CB);
  for (int e = threadIdx.x; e < CB * CB; e += blockDim.x) {
    const int i = e / CB, c = e % CB;
    l[i][c] = (i < b && c < b) ? Lm[(kb + i) * ld + kb + c] : 0.0;
    v[i][c] = 0.0;
  }
  __syncthreads();
  const int c = threadIdx.x;  // column of the inverse owned by this thread
  if (c < b) {
    v[c][c] = 1.0 / l[c][c];
    for (int i = c + 1; i < b; ++i) {
      double s = 0.0;
      for (int p = c; p < i; ++p) s += l[i][p] * v[p][c];
      v[i][c] = -s / l[i][i];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, cc = e % b;
    Li[(kb + i) * ld + kb + cc] = v[i][cc];
  }
}

}  // namespace

void dgemm(const GemmArgs& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return;
  dim3 grid(unsigned((g.N + BN - 1) / BN), unsigned((g.M + BM - 1) / BM));
  if (g.ta == 0 && g.tb == 0) k_dgemm<0, 0><<<grid, NT, 0, s>>>(g);
  if (g.ta == 1 && g.tb == 0) k_dgemm<1, 0><<<grid, NT, 0, s>>>(g);
  if (g.ta == 0 && g.tb == 1) k_dgemm<0, 1><<<grid, NT, 0, s>>>(g);
  if (g.ta == 1 && g.tb == 1) k_dgemm<1, 1><<<grid, NT, 0, s>>>(g);
}

void zc_gemm(int64_t k, int64_t ng, int nL, int nG, const double* phiP, const double* phi, double* out,
             cudaStream_t s) {
  if (k <= 0 || ng <= 0) return;
  dim3 grid(unsigned((ng + BN - 1) / BN), unsigned((k + BM - 1) / BM));
  k_zc<<<grid, NT, 0, s>>>(k, ng, nL, nG, phiP, phi, out);
}

void dpotrf_lower(double* A, int64_t n, int64_t lda, int* err, double* /*scratch*/, cudaStream_t s) {
  for (int64_t kb = 0; kb < n; kb += CB) {
    const int b = int((n - kb < CB) ? n - kb : CB);
    k_potrf_diag<<<1, 256, 0, s>>>(A, lda, kb, b, err);
    const int64_t r0 = kb + b;
    if (r0 >= n) break;
    const int64_t rows = n - r0;
    k_trsm_panel<<<unsigned((rows + 63) / 64), 64, 0, s>>>(A, lda, n, kb, b, r0);
    GemmArgs g;
    g.ta = 0;
    g.tb = 1;
    g.M = rows;
    g.N = rows;
    g.K = b;
    g.alpha = -1.0;
    g.beta = 1.0;
    g.A = A + r0 * lda + kb;
    g.lda = lda;
    g.B = A + r0 * lda + kb;
    g.ldb = lda;
    g.C = A + r0 * lda + r0;
    g.ldc = lda;
    g.sym = 1;
    dgemm(g, s);
  }
}

namespace {

// Off-diagonal blocks of the inverse, top-down on [r0, r0 + n):
//   inv([A 0; C B]) = [A^-1 0; -B^-1 C A^-1  B^-1],  A: n1 x n1, B: n2 x n2,
// with n1 a multiple of the 64-row diagonal blocks (already inverted).
// T = C A^-1 goes to the scratch (n2 x n1), then Li[C] = -B^-1 T.
// C (M x N, ldc) = alpha A B, A row-major (M x K, lda), B row-major (K x N,
// ldb), as an 8-digit tensor-core product; false if its buffers could not be
// allocated (the caller then takes the FP64 product)
bool tc_product(Plan* p, const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int64_t M,
                int64_t N, int64_t K, double alpha, cudaStream_t s) {
  OzOperand a, b;
  const bool ok = oz_alloc(p, a, M, K, 128, 8, "triangular inverse slices") == ISDF_OK &&
                  oz_alloc(p, b, N, K, oz_bn(8), 8, "triangular inverse slices") == ISDF_OK;
  if (ok) {
    oz_slice(A, lda, 1, nullptr, 1.0, a, s);
    oz_slice(B, 1, ldb, nullptr, 1.0, b, s);  // row j of the B operand: column j of B
    oz_gemm(a, b, C, ldc, 0, alpha, 0, 0, 1, nullptr, p->d_ozerr, s);
  }
  oz_free(a);
  oz_free(b);
  return ok;
}

constexpr int64_t kTcMin = 256;  // products with halves at least this large go to the tensor cores

void trtri_rec(const double* Lm, double* Li, int64_t ld, int64_t r0, int64_t n, double* scratch, cudaStream_t s,
               Plan* tc) {
  if (n <= CB) return;
  const int64_t n1 = ((n / 2 + CB - 1) / CB) * CB, n2 = n - n1;
  trtri_rec(Lm, Li, ld, r0, n1, scratch, s, tc);
  trtri_rec(Lm, Li, ld, r0 + n1, n2, scratch, s, tc);
  if (tc && n2 >= kTcMin &&
      tc_product(tc, Lm + (r0 + n1) * ld + r0, ld, Li + r0 * ld + r0, ld, scratch, n1, n2, n1, n1, 1.0, s) &&
      tc_product(tc, Li + (r0 + n1) * ld + r0 + n1, ld, scratch, n1, Li + (r0 + n1) * ld + r0, ld, n2, n1, n2, -1.0,
                 s))
    return;
  GemmArgs g;  // T = C A^-1
  g.M = n2;
  g.N = n1;
  g.K = n1;
  g.A = Lm + (r0 + n1) * ld + r0;
  g.lda = ld;
  g.B = Li + r0 * ld + r0;
  g.ldb = ld;
  g.C = scratch;
  g.ldc = n1;
  dgemm(g, s);
  GemmArgs h;  // Li[C] = -B^-1 T (B^-1 lower triangular: opA(m, k) nonzero for k <= m)
  h.M = n2;
  h.N = n1;
  h.K = n2;
  h.alpha = -1.0;
  h.A = Li + (r0 + n1) * ld + r0 + n1;
  h.lda = ld;
  h.B = scratch;
  h.ldb = n1;
  h.C = Li + (r0 + n1) * ld + r0;
  h.ldc = ld;
  h.tri = 1;
  dgemm(h, s);
}

}  // namespace

// Inverse of a lower-triangular n x n matrix: every 64 x 64 diagonal block in
// one launch, then the off-diagonal blocks by recursive halving (products of
// the size of the halves instead of 64-row strips).
// scratch: (n / 2 + 64) * n doubles.
void dtrtri_lower(const double* Lm, double* Li, int64_t n, double* scratch, cudaStream_t s, Plan* tc) {
  cudaMemsetAsync(Li, 0, sizeof(double) * n * n, s);
  const int64_t nb = (n + CB - 1) / CB;
  k_trtri_diag<<<unsigned(nb), 64, 0, s>>>(Lm, Li, n, n);
  trtri_rec(Lm, Li, n, 0, n, scratch, s, tc);
}

}  // namespace isdf
