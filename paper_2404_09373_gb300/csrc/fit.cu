// Least-squares fit of the interpolation vectors (kernel families (c), (d)),
// Section II.A, Eq. 3:  Xi_l = (ZC^T)_l ((CC^T)_l + lambda I)^-1 with
// (ZC^T)_l = M_l[:, P_l] and (CC^T)_l = M_l[P_l, P_l].
//
// Per level: gather the basis at the pivots, form (ZC^T)^T = A_L o (A_L + 2A_N)
// as one fused GEMM ([k][ng], g contiguous so every row is one interpolation
// vector ready for the FFT), pick CC^T out of its pivot columns, factor it
// with an FP64 Cholesky R R^T, invert R, and apply Xi^T = R^-T (R^-1 ZC^T^T)
// as two triangular GEMMs.
#include "internal.cuh"

namespace isdf {
namespace {

__global__ void k_gather_phiP(int nG, int k, const double* __restrict__ phi, int64_t ng,
                              const int64_t* __restrict__ pg, double* __restrict__ out) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= int64_t(nG) * k) return;
  const int r = int(e / k), j = int(e % k);
  out[e] = phi[int64_t(r) * ng + pg[j]];
}

// CC[i][j] = M(P_i, P_j) = zct[j][P_i] on and below the diagonal, 0 above
__global__ void k_gather_cc(int k, const double* __restrict__ zct, int64_t ng, const int64_t* __restrict__ pg,
                            double* __restrict__ cc) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= int64_t(k) * k) return;
  const int i = int(e / k), j = int(e % k);
  cc[e] = (j <= i) ? zct[int64_t(j) * ng + pg[i]] : 0.0;
}

// lambda = reg_rel tr(CC)/k added on the diagonal (single block)
__global__ void k_regularise(int k, double reg_rel, double* cc) {
  __shared__ double sh[256];
  double t = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) t += cc[int64_t(i) * k + i];
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double lam = reg_rel * sh[0] / double(k);
  for (int i = threadIdx.x; i < k; i += blockDim.x) cc[int64_t(i) * k + i] += lam;
}

// zct = t1 o t2 (elementwise), both [k][ng]
__global__ void k_hadamard(int64_t n, const double* __restrict__ t1, double* __restrict__ t2_out, double* zct) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e < n) zct[e] = t1[e] * t2_out[e];
}

__global__ void k_fill_kw(int nL, int nG, double* kw) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nG) kw[r] = r < nL ? 1.0 : 2.0;
}

// Tensor-core form of the fit contractions (options.precision = 1): the same
// three products as the FP64 path, each an FP64-accurate sliced-BF16 GEMM
// with the grid points on the 128-lane side so every store is coalesced.
isdf_status fit_products_tc(Plan* p, Level& lv, int k, const double* phiP, double* zct, double* y, const double* li,
                            int64_t ng) {
  cudaStream_t s = p->stream;
  const int S = p->fit_slices;
  OzOperand aL, aG, bL, bG, az, bli;
  double* kw = nullptr;
  isdf_status st = ISDF_OK;
  auto cleanup = [&]() {
    oz_free(aL), oz_free(aG), oz_free(bL), oz_free(bG), oz_free(az), oz_free(bli);
    dfree(kw);
  };
  (void)li;
  // (ZC^T)^T = T1 o T2, T1 = A_L B_L^T, T2 = [A_L A_N] [B_L 2 B_N]^T
  if ((st = oz_alloc(p, aL, ng, lv.nL, 128, S, "fit slices")) || (st = oz_alloc(p, bL, k, lv.nL, oz_bn(S), S, "fit slices")))
    return cleanup(), st;
  oz_slice(lv.phi, 1, ng, nullptr, 1.0, aL, s);
  oz_slice(phiP, 1, k, nullptr, 1.0, bL, s);
  {
    Prof pr(p, "fit_zc", 2.0 * double(k) * double(ng) * double(lv.nL), "flop", kLaunchesInside);
    oz_gemm(aL, bL, zct, ng, 1, 1.0, 0, 0, 1, nullptr, p->d_ozerr, s);
  }
  oz_free(aL);
  oz_free(bL);
  if (lv.nN > 0) {
    if ((st = dalloc_t(p, &kw, size_t(lv.nG), "fit weights")) || (st = oz_alloc(p, aG, ng, lv.nG, 128, S, "fit slices")) ||
        (st = oz_alloc(p, bG, k, lv.nG, oz_bn(S), S, "fit slices")))
      return cleanup(), st;
    k_fill_kw<<<unsigned((lv.nG + 255) / 256), 256, 0, s>>>(lv.nL, lv.nG, kw);
    count_launches(1);
    oz_slice(lv.phi, 1, ng, nullptr, 1.0, aG, s);
    oz_slice(phiP, 1, k, kw, 1.0, bG, s);
    Prof pr(p, "fit_zc", 2.0 * double(k) * double(ng) * double(lv.nG), "flop", kLaunchesInside);
    oz_gemm(aG, bG, y, ng, 1, 1.0, 0, 0, 1, nullptr, p->d_ozerr, s);
    oz_free(aG);
    oz_free(bG);
  } else {
    cudaMemcpyAsync(y, zct, sizeof(double) * size_t(k) * ng, cudaMemcpyDeviceToDevice, s);
  }
  const int64_t tot = int64_t(k) * ng;
  k_hadamard<<<unsigned((tot + 255) / 256), 256, 0, s>>>(tot, zct, y, zct);
  count_launches(1);
  cleanup();
  return ISDF_OK;
}

// Y = R^-1 ZC^T^T ([k][ng]); then, if xi_out, Xi^T = R^-T Y into xi_out
// (which may be zct itself).
isdf_status fit_solve_tc(Plan* p, int k, const double* zct, double* y, const double* li, int64_t ng, double* xi_out) {
  cudaStream_t s = p->stream;
  const int S = p->fit_slices;
  OzOperand a, b;
  isdf_status st;
  Prof pr(p, "fit_solve", (xi_out ? 2.0 : 1.0) * double(k) * double(k + 1) * double(ng), "flop", kLaunchesInside);
  // Y^T[g][j] = sum_kk Z^T[g][kk] R^-1[j][kk]   (R^-1 lower: kk <= j)
  if ((st = oz_alloc(p, a, ng, k, 128, S, "solve slices")) || (st = oz_alloc(p, b, k, k, oz_bn(S), S, "solve slices")))
    return oz_free(a), oz_free(b), st;
  oz_slice(zct, 1, ng, nullptr, 1.0, a, s);
  oz_slice(li, k, 1, nullptr, 1.0, b, s);
  oz_gemm(a, b, y, ng, 1, 1.0, 1, 0, 1, nullptr, p->d_ozerr, s);
  if (xi_out) {
    // Xi^T[j][g] = sum_kk Y[kk][g] R^-1[kk][j]   (R^-T upper: kk >= j)
    oz_slice(y, 1, ng, nullptr, 1.0, a, s);
    oz_slice(li, 1, k, nullptr, 1.0, b, s);
    oz_gemm(a, b, xi_out, ng, 1, 1.0, 2, 0, 1, nullptr, p->d_ozerr, s);
  }
  oz_free(a);
  oz_free(b);
  return ISDF_OK;
}

// residual of the pair fit at every grid point, r(g) = w (M(g,g) - |Y[:,g]|^2)
// with Y = R^-1 (ZC^T)^T: the Schur complement left after the pivots; max and
// sum (= the weighted Frobenius fit error^2) go to out[0], out[1]
__global__ void k_fit_residual(const double* __restrict__ phi, int64_t ng, int nL, int nG, double w,
                               const double* __restrict__ y, int k, unsigned long long* out_max, double* out_sum,
                               float* __restrict__ rpt) {
  double mx = 0.0, sm = 0.0;
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < ng; g += int64_t(gridDim.x) * blockDim.x) {
    double aL = 0.0, aN = 0.0, q = 0.0;
    for (int r = 0; r < nL; ++r) aL = fma(phi[int64_t(r) * ng + g], phi[int64_t(r) * ng + g], aL);
    for (int r = nL; r < nG; ++r) aN = fma(phi[int64_t(r) * ng + g], phi[int64_t(r) * ng + g], aN);
    for (int j = 0; j < k; ++j) q = fma(y[int64_t(j) * ng + g], y[int64_t(j) * ng + g], q);
    const double res = w * (aL * (aL + 2.0 * aN) - q);
    if (rpt) rpt[g] = float(res);
    mx = fmax(mx, res);
    sm += res;
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    sm += __shfl_xor_sync(0xffffffffu, sm, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out_max, (unsigned long long)__double_as_longlong(fmax(mx, 0.0)));
    atomicAdd(out_sum, sm);
  }
}

}  // namespace

isdf_status fit_run(Plan* p) {
  cudaStream_t s = p->stream;
  isdf_status st;
  p->resid_ready = false;
  for (int l = 0; l < p->nlev; ++l) {
    Level& lv = p->lev[l];
    dfree(lv.xiT);
    lv.xiT = nullptr;
    dfree(lv.resid);
    lv.resid = nullptr;
    dfree(lv.zct);
    lv.zct = nullptr;
    dfree(lv.rinv);
    lv.rinv = nullptr;
    if (l < p->sel_lo) continue;  // local grids' level 0: fitted atom by atom (local.cu)
    if ((st = dalloc_t(p, &lv.resid, size_t(lv.ng), "fit residual"))) return st;
    if (lv.k == 0) {
      // no pivots: the residual is the whole diagonal w M(g,g)
      double* scr = nullptr;
      if ((st = dalloc_t(p, &scr, 2, "residual statistics"))) return st;
      cudaMemsetAsync(scr, 0, 2 * sizeof(double), s);
      k_fit_residual<<<152 * 4, 256, 0, s>>>(lv.phi, lv.ng, lv.nL, lv.nG, lv.w, nullptr, 0,
                                             reinterpret_cast<unsigned long long*>(scr), scr + 1, lv.resid);
      count_launches(1);
      cudaMemcpyAsync(&p->fit_resid[2 * l], scr, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
      st = cuda_check(p, cudaStreamSynchronize(s), "fit residual");
      dfree(scr);
      if (st) return st;
      continue;
    }
    const int k = lv.k;
    const int64_t ng = lv.ng;
    double *phiP = nullptr, *zct = nullptr, *y = nullptr, *cc = nullptr, *li = nullptr, *scr = nullptr;
    auto cleanup = [&]() {
      dfree(phiP);
      dfree(y);
      dfree(cc);
      dfree(li);
      dfree(scr);
    };
    if ((st = dalloc_t(p, &phiP, size_t(lv.nG) * k, "phi at pivots")) ||
        (st = dalloc_t(p, &zct, size_t(k) * ng, "ZC^T / Xi")) || (st = dalloc_t(p, &y, size_t(k) * ng, "fit scratch")) ||
        (st = dalloc_t(p, &cc, size_t(k) * k, "CC^T")) || (st = dalloc_t(p, &li, size_t(k) * k, "R^-1")) ||
        (st = dalloc_t(p, &scr, size_t(k / 2 + 64) * k + 64, "trtri scratch"))) {
      cleanup();
      dfree(zct);
      return st;
    }
    const bool factored = p->opt.precision == 1;  // keep ZC^T and R^-1; Xi only on request
    if (factored)
      lv.zct = zct;
    else
      lv.xiT = zct;
    const int64_t np = int64_t(lv.nG) * k;
    count_launches(2 + (p->opt.reg_rel > 0.0));
    k_gather_phiP<<<unsigned((np + 255) / 256), 256, 0, s>>>(lv.nG, k, lv.phi, ng, lv.d_pg, phiP);
    if (p->opt.precision == 1) {
      if ((st = fit_products_tc(p, lv, k, phiP, zct, y, li, ng))) {
        cleanup();
        return st;
      }
    } else {
      Prof pr(p, "fit_zc", 2.0 * double(k) * double(ng) * double(lv.nG), "flop", 1);
      zc_gemm(k, ng, lv.nL, lv.nG, phiP, lv.phi, zct, s);
    }
    k_gather_cc<<<unsigned((int64_t(k) * k + 255) / 256), 256, 0, s>>>(k, zct, ng, lv.d_pg, cc);
    if (p->opt.reg_rel > 0.0) k_regularise<<<1, 256, 0, s>>>(k, p->opt.reg_rel, cc);
    const int big = 0x7fffffff;
    cudaMemcpyAsync(p->d_err, &big, sizeof(int), cudaMemcpyHostToDevice, s);
    {
      const int64_t nb = (k + 63) / 64;
      Prof pr(p, "fit_cholesky", double(k) * k * k / 3.0, "flop", 3 * nb - 2);
      dpotrf_lower(cc, k, k, p->d_err, nullptr, s);
    }
    int herr = big;
    cudaMemcpyAsync(&herr, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if ((st = cuda_check(p, cudaStreamSynchronize(s), "Cholesky of CC^T"))) {
      cleanup();
      return st;
    }
    if (herr != big || p->fault == "not_pd") {
      cleanup();
      return fail(p, ISDF_ERR_NOT_PD,
                  "Cholesky of CC^T broke down at column " + std::to_string(herr == big ? 0 : herr) + " of level " +
                      std::to_string(l));
    }
    {
      const int64_t nb = (k + 63) / 64;
      Prof pr(p, "fit_trtri", double(k) * k * k / 3.0, "flop", 1 + 2 * (nb - 1));
      dtrtri_lower(cc, li, k, scr, s, p->opt.precision == 1 ? p : nullptr);
    }
    if (factored) {
      // Coulomb and exchange need Xi only through V = W (ZC^T v ZC) W with
      // W = R^-T R^-1 (see coulomb.cu): no solve over the grid here
      lv.rinv = li;
      li = nullptr;
      st = cuda_check(p, cudaStreamSynchronize(s), "fit");
      if (!st) st = oz_check(p);
      cleanup();
      if (st) return st;
      continue;
    } else {
    Prof pr_solve(p, "fit_solve", 2.0 * double(k) * double(k + 1) * double(ng), "flop", 2);
    GemmArgs g1;  // Y = R^-1 ZC^T^T (R^-1 lower triangular)
    g1.M = k;
    g1.N = ng;
    g1.K = k;
    g1.A = li;
    g1.lda = k;
    g1.B = zct;
    g1.ldb = ng;
    g1.C = y;
    g1.ldc = ng;
    g1.tri = 1;
    dgemm(g1, s);
    GemmArgs g2;  // Xi^T = R^-T Y (opA upper triangular)
    g2.ta = 1;
    g2.M = k;
    g2.N = ng;
    g2.K = k;
    g2.A = li;
    g2.lda = k;
    g2.B = y;
    g2.ldb = ng;
    g2.C = zct;
    g2.ldc = ng;
    g2.tri = 2;
    dgemm(g2, s);
    }
    {
      // y still holds R^-1 (ZC^T)^T: residual statistics of this level
      unsigned long long* rmax = reinterpret_cast<unsigned long long*>(scr);
      double* rsum = scr + 1;
      cudaMemsetAsync(scr, 0, 2 * sizeof(double), s);
      k_fit_residual<<<152 * 4, 256, 0, s>>>(lv.phi, ng, lv.nL, lv.nG, lv.w, y, k, rmax, rsum, lv.resid);
      count_launches(1);
      cudaMemcpyAsync(&p->fit_resid[2 * l], scr, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    }
    st = cuda_check(p, cudaStreamSynchronize(s), "fit");
    cleanup();
    if (st) return st;
  }
  p->resid_ready = p->opt.precision != 1;
  return gather_pivot_factors(p);
}

// Residual statistics of a factored fit: Y = R^-1 ZC^T^T, then w (M(g,g) - |Y[:,g]|^2).
isdf_status fit_residual_run(Plan* p) {
  if (p->resid_ready) return ISDF_OK;
  cudaStream_t s = p->stream;
  isdf_status st;
  for (int l = 0; l < p->nlev; ++l) {
    Level& lv = p->lev[l];
    if (lv.k == 0 || !lv.zct || lv.nG == 0) continue;  // done by the fit; local grids' level 0: not kept
    double *y = nullptr, *scr = nullptr;
    if ((st = dalloc_t(p, &y, size_t(lv.k) * lv.ng, "fit scratch")) || (st = dalloc_t(p, &scr, 2, "residual statistics"))) {
      dfree(y);
      return st;
    }
    st = fit_solve_tc(p, lv.k, lv.zct, y, lv.rinv, lv.ng, nullptr);
    if (!st) {
      cudaMemsetAsync(scr, 0, 2 * sizeof(double), s);
      k_fit_residual<<<152 * 4, 256, 0, s>>>(lv.phi, lv.ng, lv.nL, lv.nG, lv.w, y, lv.k,
                                             reinterpret_cast<unsigned long long*>(scr), scr + 1, lv.resid);
      count_launches(1);
      cudaMemcpyAsync(&p->fit_resid[2 * l], scr, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
      st = cuda_check(p, cudaStreamSynchronize(s), "fit residual");
      if (!st) st = oz_check(p);
    }
    dfree(y);
    dfree(scr);
    if (st) return st;
  }
  p->resid_ready = true;
  return ISDF_OK;
}

// Xi^T of one level of a factored fit: Xi^T = R^-T R^-1 ZC^T^T.
isdf_status fit_xi_run(Plan* p, int l) {
  Level& lv = p->lev[l];
  if (lv.xiT || lv.k == 0 || !lv.zct) return ISDF_OK;
  isdf_status st;
  double *y = nullptr, *xi = nullptr;
  if ((st = dalloc_t(p, &y, size_t(lv.k) * lv.ng, "fit scratch")) ||
      (st = dalloc_t(p, &xi, size_t(lv.k) * lv.ng, "interpolation vectors"))) {
    dfree(y);
    return st;
  }
  st = fit_solve_tc(p, lv.k, lv.zct, y, lv.rinv, lv.ng, xi);
  if (!st) st = cuda_check(p, cudaStreamSynchronize(p->stream), "interpolation vectors");
  if (!st) st = oz_check(p);
  dfree(y);
  if (st) {
    dfree(xi);
    return st;
  }
  lv.xiT = xi;
  return ISDF_OK;
}

}  // namespace isdf
