// The coarsest level as the paper's sparse universal grid U (Section III,
// grids figure; Section III.A, the paragraphs after Eq. 8).
//
// Every point g of U is an interpolation point whose fitting function is the
// sinc function of the grid (Xi = I on U), so U carries no selection and no
// fit.  With F the fitted interpolation points of the finer levels:
//
//   V_FU[P][g] = (xi_P | sinc_g)  -- the potential of xi_P sampled on U: the
//                fine half spectrum folded onto U's modes (the Nyquist split of
//                the trigonometric interpolant), weighted by 4 pi Omega /
//                (|G|^2 N_g,P N_U), and one inverse 3-D transform on U
//                (cuFFT Z2D, batched);
//   V_UU       -- (R_U | R_U'), a circulant: never formed, only applied in
//                Fourier space.
//
// Exchange (Eq. 8 over F and U; reading R6 of the four terms), D = C C^T:
//   K = K_FF + K_FU + K_FU^T + K_UU,
//   K_FU = X^L_F (V_FU o R^GU) Phi_U^T + X^N_F (V_FU o R^LU) Phi_U^T,
//          R^AU = Y_A Psi,  Psi[i][g] = sum_{lam in L_U} C[lam][i] phi_lam(g),
//   K_UU[mu][nu] = sum_i (rho_mu,i | rho_nu,i),  rho_mu,i(g) = phi_mu(g) psi_i(g)
// (occ-RI on U: one transform per function and orbital, then the Coulomb
// integrals as one weighted product over the half spectra).  Phi_U: the
// values of the functions of U's level L_U at the points of U (the plan's
// basis matrix of that level).
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace isdf {
namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

// H[P][q] *= pref / |G_q|^2 (0 at G = 0), on U's half grid (cx, cy, cz).
__global__ void k_pot_weights(int64_t k, double2* __restrict__ H, int cx, int cy, int cz, double Lx, double Ly,
                              double Lz, double pref) {
  const int cxh = cx / 2 + 1;
  const int64_t nq = int64_t(cxh) * cy * cz;
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= k * nq) return;
  const int64_t q = e % nq;
  const int qx = int(q % cxh), qy = int((q / cxh) % cy), qz = int(q / (int64_t(cxh) * cy));
  const int sy = (2 * qy < cy) ? qy : qy - cy, sz = (2 * qz < cz) ? qz : qz - cz;
  const double gx = kTwoPi * qx / Lx, gy = kTwoPi * sy / Ly, gz = kTwoPi * sz / Lz;
  const double G2 = gx * gx + gy * gy + gz * gz;
  const double w = G2 > 0.0 ? pref / G2 : 0.0;
  H[e].x *= w;
  H[e].y *= w;
}

// Same-level Coulomb weights of U's half spectrum, as square roots (the
// product A A^T then carries the weight once):
//   wt(q) = mult(q_x) 2^-(#Nyquist axes) 4 pi Omega / (|G_q|^2 N_U^2).
__global__ void k_sqrt_weights(int cx, int cy, int cz, double Lx, double Ly, double Lz, double pref,
                               double* __restrict__ w2) {
  const int cxh = cx / 2 + 1;
  const int64_t nq = int64_t(cxh) * cy * cz;
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const int qx = int(q % cxh), qy = int((q / cxh) % cy), qz = int(q / (int64_t(cxh) * cy));
  const int sy = (2 * qy < cy) ? qy : qy - cy, sz = (2 * qz < cz) ? qz : qz - cz;
  const double gx = kTwoPi * qx / Lx, gy = kTwoPi * sy / Ly, gz = kTwoPi * sz / Lz;
  const double G2 = gx * gx + gy * gy + gz * gz;
  double w = 0.0;
  if (G2 > 0.0) {
    const double mult = (qx == 0 || 2 * qx == cx) ? 1.0 : 2.0;
    const int nyq = (2 * qx == cx) + (2 * qy == cy) + (2 * qz == cz);
    w = std::sqrt(ldexp(pref * mult / G2, -nyq));
  }
  w2[2 * q] = w;
  w2[2 * q + 1] = w;
}

// S[v][j] *= w2[j] for every vector v (interleaved re, im of the half spectrum)
__global__ void k_scale_rows(int64_t nv, int64_t len, double* __restrict__ S, const double* __restrict__ w2) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= nv * len) return;
  S[e] *= w2[e % len];
}

// a[e] *= v[e], b[e] *= v[e]
__global__ void k_hadamard2(int64_t n, const double* __restrict__ v, double* __restrict__ a, double* __restrict__ b) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n) return;
  a[e] *= v[e];
  b[e] *= v[e];
}

// rho[(mu nb + ii) ng + g] = phi[mu][g] psiT[g][i0 + ii]
__global__ void k_rho(int nL, int nb, int64_t ng, const double* __restrict__ phi, const double* __restrict__ psiT,
                      int n, int i0, double* __restrict__ rho) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= int64_t(nL) * nb * ng) return;
  const int64_t g = e % ng, v = e / ng;
  const int mu = int(v / nb), ii = int(v % nb);
  rho[e] = phi[int64_t(mu) * ng + g] * psiT[g * n + i0 + ii];
}

// out[j][c] = C[fun[j]][c]
__global__ void k_gather_c(int nL, int n, const int* __restrict__ fun, const double* __restrict__ C,
                           double* __restrict__ out) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= int64_t(nL) * n) return;
  out[e] = C[int64_t(fun[e / n]) * n + e % n];
}

// K[mu][fun[j]] += A[mu][j]  (targets distinct within one launch)
__global__ void k_add_cols(int64_t N, int nL, const int* __restrict__ fun, const double* __restrict__ A,
                           double* __restrict__ K) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= N * nL) return;
  const int64_t mu = e / nL;
  const int j = int(e % nL);
  K[mu * N + fun[j]] += A[e];
}

// K[fun[j]][mu] += A[mu][j]
__global__ void k_add_rows(int64_t N, int nL, const int* __restrict__ fun, const double* __restrict__ A,
                           double* __restrict__ K) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= N * nL) return;
  const int64_t mu = e / nL;
  const int j = int(e % nL);
  K[int64_t(fun[j]) * N + mu] += A[e];
}

// K[fun[i]][fun[j]] += A[i][j]
__global__ void k_add_block(int nL, int64_t N, const int* __restrict__ fun, const double* __restrict__ A,
                            double* __restrict__ K) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= int64_t(nL) * nL) return;
  K[int64_t(fun[e / nL]) * N + fun[e % nL]] += A[e];
}

// acc[e] += a[e]
__global__ void k_accumulate(int64_t n, const double* __restrict__ a, double* __restrict__ acc) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e < n) acc[e] += a[e];
}

inline unsigned blocks(int64_t n) { return unsigned((n + 255) / 256); }

// C = A B^T (A rows M with strides sar, sak; B rows N with sbr, sbk): FP64
// SIMT at precision 0, FP64-grade 8-digit tensor-core products otherwise
isdf_status product(Plan* p, const double* a, int64_t M, int64_t sar, int64_t sak, const double* b, int64_t N,
                    int64_t sbr, int64_t sbk, int64_t K, double* C, int64_t ldc, int S) {
  cudaStream_t s = p->stream;
  if (p->opt.precision == 1) {
    OzOperand A, B;
    isdf_status st;
    if ((st = oz_alloc(p, A, M, K, 128, S, "sinc products")) || (st = oz_alloc(p, B, N, K, oz_bn(S), S, "sinc products")))
      return oz_free(A), oz_free(B), st;
    oz_slice(a, sar, sak, nullptr, 1.0, A, s);
    oz_slice(b, sbr, sbk, nullptr, 1.0, B, s);
    oz_gemm(A, B, C, ldc, 0, 1.0, 0, 0, 1, nullptr, p->d_ozerr, s);
    st = oz_check(p);
    oz_free(A);
    oz_free(B);
    return st;
  }
  GemmArgs g;
  g.M = M, g.N = N, g.K = K;
  if (sak == 1) g.ta = 0, g.A = a, g.lda = sar;
  else g.ta = 1, g.A = a, g.lda = sak;
  if (sbk == 1) g.tb = 1, g.B = b, g.ldb = sbr;
  else g.tb = 0, g.B = b, g.ldb = sbk;
  g.C = C, g.ldc = ldc;
  dgemm(g, s);
  return cuda_check(p, cudaGetLastError(), "sinc product");
}

}  // namespace

isdf_status sinc_coulomb(Plan* p) {
  cudaStream_t s = p->stream;
  Level& lu = p->lev[p->nlev - 1];
  const int64_t nu = lu.ng, nqu = int64_t(lu.n[0] / 2 + 1) * lu.n[1] * lu.n[2];
  const int64_t nip = p->nip;
  dfree(p->VFU);
  p->VFU = nullptr;
  isdf_status st;
  if ((st = dalloc_t(p, &p->VFU, size_t(std::max<int64_t>(nip, 1)) * nu, "V_FU"))) return st;
  if (nip == 0) return ISDF_OK;
  const double four_pi_omega = 4.0 * 3.14159265358979323846 * p->omega;
  int dev = 0;
  cudaGetDevice(&dev);
  cufftHandle plan = 0;
  int dims[3] = {lu.n[2], lu.n[1], lu.n[0]};
  Prof pr(p, "coulomb_sinc", double(nip) * (16.0 * double(nqu) + 8.0 * double(nu)), "byte", kLaunchesInside);
  for (int l = 0; l + 1 < p->nlev; ++l) {
    Level& lv = p->lev[l];
    if (!lv.k) continue;
    double2* H = nullptr;
    if ((st = dalloc_t(p, &H, size_t(lv.k) * nqu, "folded spectra"))) return st;
    const int64_t tot = int64_t(lv.k) * nqu;
    fold_spectra(lv.k, lv.spec, lv.n[0], lv.n[1], lv.n[2], H, lu.n[0], lu.n[1], lu.n[2], s);
    k_pot_weights<<<blocks(tot), 256, 0, s>>>(lv.k, H, lu.n[0], lu.n[1], lu.n[2], p->edge[0], p->edge[1], p->edge[2],
                                              four_pi_omega / (double(lv.ng) * double(nu)));
    count_launches(2);
    // potentials on U: one batched inverse transform (real output)
    cufftResult r = cufftPlanMany(&plan, 3, dims, nullptr, 1, int(nqu), nullptr, 1, int(nu), CUFFT_Z2D, lv.k);
    if (r == CUFFT_SUCCESS) r = cufftSetStream(plan, s);
    if (r == CUFFT_SUCCESS)
      r = cufftExecZ2D(plan, reinterpret_cast<cufftDoubleComplex*>(H), p->VFU + int64_t(p->poff[l]) * nu);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (plan) cufftDestroy(plan);
    plan = 0;
    dfree(H);
    if (r != CUFFT_SUCCESS) return fail(p, ISDF_ERR_CUFFT, "sinc potentials: cuFFT Z2D failed (" + std::to_string(int(r)) + ")");
    if ((st = cuda_check(p, e, "sinc potentials"))) return st;
    if (lv.zct) {
      // factored fit: these were the potentials of ZC; Xi = ZC W, W = R^-T R^-1
      double *W = nullptr, *T = nullptr;
      const int k = lv.k;
      if ((st = dalloc_t(p, &W, size_t(k) * k, "W")) || (st = dalloc_t(p, &T, size_t(k) * nu, "W V_FU"))) {
        dfree(W);
        return st;
      }
      double* rows = p->VFU + int64_t(p->poff[l]) * nu;
      // W[m][n] = sum_kk R^-1[kk][m] R^-1[kk][n];  T[m][g] = sum_i W[m][i] rows[i][g]
      if (!(st = product(p, lv.rinv, k, 1, k, lv.rinv, k, 1, k, k, W, k, 8)) &&
          !(st = product(p, W, k, k, 1, rows, nu, 1, nu, k, T, nu, 8)))
        st = cuda_check(p, cudaMemcpyAsync(rows, T, sizeof(double) * size_t(k) * nu, cudaMemcpyDeviceToDevice, s),
                        "copy V_FU");
      if (!st) st = cuda_check(p, cudaStreamSynchronize(s), "V_FU");
      dfree(W);
      dfree(T);
      if (st) return st;
    }
  }
  return ISDF_OK;
}

isdf_status sinc_exchange(Plan* p, const double* dC, const double* yl, const double* yg, int n, double* dK) {
  cudaStream_t s = p->stream;
  const Level& lu = p->lev[p->nlev - 1];
  const int64_t nu = lu.ng, N = p->nfun, nip = p->nip;
  const int nL = lu.nL;
  if (nL == 0) return ISDF_OK;
  const int64_t nqu = int64_t(lu.n[0] / 2 + 1) * lu.n[1] * lu.n[2];
  int* fun = nullptr;
  double *cu = nullptr, *psiT = nullptr, *rg = nullptr, *rl = nullptr, *tu = nullptr, *tl = nullptr, *kfl = nullptr,
         *kfn = nullptr, *w2 = nullptr, *rho = nullptr, *kuu = nullptr, *part = nullptr;
  double2* spec = nullptr;
  auto cleanup = [&]() {
    dfree(fun);
    for (double* q : {cu, psiT, rg, rl, tu, tl, kfl, kfn, w2, rho, kuu, part}) dfree(q);
    dfree(spec);
  };
  // exchange products: 5 digits on the tensor cores, as the rest of the
  // exchange build; FP64 SIMT at precision 0
  auto prod = [&](const double* a, int64_t M, int64_t sar, int64_t sak, const double* b, int64_t Nn, int64_t sbr,
                  int64_t sbk, int64_t K, double* C, int64_t ldc) {
    return p->opt.precision == 1 ? tc_product_ex(p, a, M, sar, sak, b, Nn, sbr, sbk, K, C, ldc)
                                 : product(p, a, M, sar, sak, b, Nn, sbr, sbk, K, C, ldc, 5);
  };
  isdf_status st;
  // orbitals per batch of the K_UU transforms: about 512 MB of rho
  const int nb = int(std::max<int64_t>(1, std::min<int64_t>(n, (int64_t(512) << 20) / (8 * nu * nL))));
  if ((st = dalloc_t(p, &fun, size_t(nL), "U functions")) || (st = dalloc_t(p, &cu, size_t(nL) * n, "C of U")) ||
      (st = dalloc_t(p, &psiT, size_t(nu) * n, "Psi")) || (st = dalloc_t(p, &w2, size_t(2) * nqu, "weights")) ||
      (st = dalloc_t(p, &rho, size_t(nL) * nb * nu, "rho")) ||
      (st = dalloc_t(p, &spec, size_t(nL) * nb * nqu, "rho spectra")) ||
      (st = dalloc_t(p, &kuu, size_t(nL) * nL, "K_UU")) || (st = dalloc_t(p, &part, size_t(nL) * nL, "K_UU part"))) {
    cleanup();
    return st;
  }
  const double four_pi_omega = 4.0 * 3.14159265358979323846 * p->omega;
  Prof pr(p, "exchange_sinc",
          2.0 * double(nu) * n * nL + 2.0 * 2.0 * nip * nu * (n + nL) + 4.0 * N * nip * nL + 2.0 * double(n) * nL * nL * 2.0 * nqu,
          "flop", kLaunchesInside);
  if ((st = cuda_check(p, cudaMemcpyAsync(fun, lu.L.data(), sizeof(int) * size_t(nL), cudaMemcpyHostToDevice, s),
                       "U functions")) ||
      (st = cuda_check(p, cudaStreamSynchronize(s), "U functions"))) {
    cleanup();
    return st;
  }
  k_gather_c<<<blocks(int64_t(nL) * n), 256, 0, s>>>(nL, n, fun, dC, cu);
  count_launches(1);
  // Psi^T[g][i] = sum_lam Phi_U[lam][g] C[lam][i]
  if ((st = prod(lu.phi, nu, 1, nu, cu, n, 1, n, nL, psiT, n))) {
    cleanup();
    return st;
  }
  // ---- K_FU + K_FU^T
  if (nip > 0) {
    if ((st = dalloc_t(p, &rg, size_t(nip) * nu, "R^GU")) || (st = dalloc_t(p, &rl, size_t(nip) * nu, "R^LU")) ||
        (st = dalloc_t(p, &tu, size_t(nip) * nL, "T_U")) || (st = dalloc_t(p, &tl, size_t(nip) * nL, "T'_U")) ||
        (st = dalloc_t(p, &kfl, size_t(N) * nL, "K_FU")) || (st = dalloc_t(p, &kfn, size_t(N) * nL, "K_FU"))) {
      cleanup();
      return st;
    }
    // R^AU[P][g] = sum_i Y_A[P][i] Psi^T[g][i], then V_FU o R^AU in place
    if ((st = prod(yg, nip, n, 1, psiT, nu, n, 1, n, rg, nu)) || (st = prod(yl, nip, n, 1, psiT, nu, n, 1, n, rl, nu))) {
      cleanup();
      return st;
    }
    k_hadamard2<<<blocks(nip * nu), 256, 0, s>>>(nip * nu, p->VFU, rg, rl);
    count_launches(1);
    // T[P][lam] = sum_g (V o R)[P][g] Phi_U[lam][g]
    if ((st = prod(rg, nip, nu, 1, lu.phi, nL, nu, 1, nu, tu, nL)) ||
        (st = prod(rl, nip, nu, 1, lu.phi, nL, nu, 1, nu, tl, nL))) {
      cleanup();
      return st;
    }
    // K_FU[mu][lam] = sum_P X^L[mu][P] T_U[P][lam] + X^N[mu][P] T'_U[P][lam]
    if ((st = prod(p->XL, N, nip, 1, tu, nL, 1, nL, nip, kfl, nL)) ||
        (st = prod(p->XN, N, nip, 1, tl, nL, 1, nL, nip, kfn, nL))) {
      cleanup();
      return st;
    }
    for (double* kf : {kfl, kfn}) {
      k_add_cols<<<blocks(N * nL), 256, 0, s>>>(N, nL, fun, kf, dK);
      k_add_rows<<<blocks(N * nL), 256, 0, s>>>(N, nL, fun, kf, dK);
    }
    count_launches(4);
  }
  // ---- K_UU = sum_i (rho_mu,i | rho_nu,i): transforms of rho on U, then one
  // product of the weighted half spectra per batch of orbitals
  k_sqrt_weights<<<blocks(nqu), 256, 0, s>>>(lu.n[0], lu.n[1], lu.n[2], p->edge[0], p->edge[1], p->edge[2],
                                             four_pi_omega / (double(nu) * double(nu)), w2);
  count_launches(1);
  cudaMemsetAsync(kuu, 0, sizeof(double) * size_t(nL) * nL, s);
  for (int i0 = 0; i0 < n; i0 += nb) {
    const int b = std::min(nb, n - i0);
    const int64_t nv = int64_t(nL) * b;
    k_rho<<<blocks(nv * nu), 256, 0, s>>>(nL, b, nu, lu.phi, psiT, n, i0, rho);
    count_launches(1);
    if ((st = transform_real(p, rho, lu.n[0], lu.n[1], lu.n[2], nv, spec))) {
      cleanup();
      return st;
    }
    k_scale_rows<<<blocks(nv * 2 * nqu), 256, 0, s>>>(nv, 2 * nqu, reinterpret_cast<double*>(spec), w2);
    count_launches(1);
    // part[mu][nu] = sum over (i, q, re/im) of A[mu][.] A[nu][.]: row mu holds b x 2 nqu values
    const double* A = reinterpret_cast<const double*>(spec);
    const int64_t K2 = int64_t(b) * 2 * nqu;
    if ((st = prod(A, nL, K2, 1, A, nL, K2, 1, K2, part, nL))) {
      cleanup();
      return st;
    }
    k_accumulate<<<blocks(int64_t(nL) * nL), 256, 0, s>>>(int64_t(nL) * nL, part, kuu);
    count_launches(1);
  }
  k_add_block<<<blocks(int64_t(nL) * nL), 256, 0, s>>>(nL, N, fun, kuu, dK);
  count_launches(1);
  st = cuda_check(p, cudaStreamSynchronize(s), "sinc exchange");
  cleanup();
  return st;
}

}  // namespace isdf
