// Two-centre Coulomb matrix (kernel family (e)), Section II Eq. 1 and the
// cross-grid integrals of Section III:
//   V_PQ = 4 pi Omega sum_{G != 0} Re[conj c_P(G) c_Q(G)] / |G|^2,
// where c(G) are the Fourier coefficients of the trigonometric interpolant
// of a grid function (a coefficient whose mode index is n/2 on an axis is
// split evenly between +n/2 and -n/2).  For two levels the sum runs over the
// coarser level's mode set.
//
// Every interpolation vector goes through one cuFFT D2Z transform (batched).
// With the half spectrum S(q) (q_x in [0, nx/2]) the sums collapse to
//   same level : V_PQ = sum_q wt_s(q) Re[conj S_P(q) S_Q(q)],
//                wt_s = mult(q_x) 2^{-#Nyquist axes} 4 pi Omega / (|G_q|^2 N_g^2)
//   two levels : V_PQ = sum_q wt_c(q) Re[conj H_P(q) S_Q(q)],
//                H_P(q) = sum over the (up to 8) signed preimages m of q of
//                2^{-#Nyquist axes} S^fine_P(m),
//                wt_c = mult(q_x) 4 pi Omega / (|G_q|^2 N_g,fine N_g,coarse)
// with mult = 1 for q_x in {0, nx/2}, else 2 (Hermitian partner).  Each sum is
// one real GEMM over interleaved (Re, Im) with a per-k weight.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include "internal.cuh"

namespace isdf {
namespace {

// Process-wide pool of cuFFT plans keyed by (device, nz, ny, nx, batch):
// creating a plan allocates its work area and synchronises the device, so a
// plan is created once and checked out by one caller at a time (concurrent
// library plans on other streams get their own handles).  Handles live until
// the process exits.
using FftKey = std::tuple<int, int, int, int, int>;
std::mutex g_fft_mu;
std::multimap<FftKey, cufftHandle> g_fft_free;

cufftResult fft_acquire(const FftKey& key, cufftHandle* h) {
  {
    std::lock_guard<std::mutex> lock(g_fft_mu);
    auto it = g_fft_free.find(key);
    if (it != g_fft_free.end()) {
      *h = it->second;
      g_fft_free.erase(it);
      return CUFFT_SUCCESS;
    }
  }
  int dims[3] = {std::get<1>(key), std::get<2>(key), std::get<3>(key)};
  const int ng = dims[0] * dims[1] * dims[2];
  const int nq = dims[0] * dims[1] * (dims[2] / 2 + 1);
  return cufftPlanMany(h, 3, dims, nullptr, 1, ng, nullptr, 1, nq, CUFFT_D2Z, std::get<4>(key));
}

void fft_release(const FftKey& key, cufftHandle h) {
  std::lock_guard<std::mutex> lock(g_fft_mu);
  g_fft_free.emplace(key, h);
}

__global__ void k_coul_weights(int nx, int ny, int nz, double Lx, double Ly, double Lz, double pref, int same,
                               double* __restrict__ wt2) {
  const int nxh = nx / 2 + 1;
  const int64_t nq = int64_t(nxh) * ny * nz;
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const int qx = int(q % nxh);
  const int qy = int((q / nxh) % ny);
  const int qz = int(q / (int64_t(nxh) * ny));
  const int sx = qx;
  const int sy = (2 * qy < ny) ? qy : qy - ny;
  const int sz = (2 * qz < nz) ? qz : qz - nz;
  const double two_pi = 6.283185307179586476925286766559;
  const double gx = two_pi * sx / Lx, gy = two_pi * sy / Ly, gz = two_pi * sz / Lz;
  const double G2 = gx * gx + gy * gy + gz * gz;
  double w = 0.0;
  if (G2 > 0.0) {
    const double mult = (qx == 0 || 2 * qx == nx) ? 1.0 : 2.0;
    w = pref * mult / G2;
    if (same) {
      const int nyq = (2 * qx == nx) + (2 * qy == ny) + (2 * qz == nz);
      w = ldexp(w, -nyq);
    }
  }
  wt2[2 * q] = w;
  wt2[2 * q + 1] = w;
}

// H_P(q) on the coarse half grid (cx, cy, cz) from the fine half spectrum.
__global__ void k_fold(int k, const double2* __restrict__ spf, int fx, int fy, int fz, double2* __restrict__ H, int cx,
                       int cy, int cz) {
  const int cxh = cx / 2 + 1, fxh = fx / 2 + 1;
  const int64_t nqc = int64_t(cxh) * cy * cz;
  const int64_t nqf = int64_t(fxh) * fy * fz;
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= nqc * k) return;
  const int64_t P = e / nqc, q = e % nqc;
  const int qx = int(q % cxh);
  const int qy = int((q / cxh) % cy);
  const int qz = int(q / (int64_t(cxh) * cy));
  int mx[2], my[2], mz[2], nx_ = 1, ny_ = 1, nz_ = 1;
  if (2 * qx == cx) { mx[0] = cx / 2; mx[1] = -cx / 2; nx_ = 2; } else { mx[0] = qx; }
  if (2 * qy == cy) { my[0] = cy / 2; my[1] = -cy / 2; ny_ = 2; } else { my[0] = (2 * qy < cy) ? qy : qy - cy; }
  if (2 * qz == cz) { mz[0] = cz / 2; mz[1] = -cz / 2; nz_ = 2; } else { mz[0] = (2 * qz < cz) ? qz : qz - cz; }
  const double wgt = 1.0 / double(nx_ * ny_ * nz_);
  const double2* sp = spf + P * nqf;
  double re = 0.0, im = 0.0;
  for (int a = 0; a < nx_; ++a)
    for (int b = 0; b < ny_; ++b)
      for (int c = 0; c < nz_; ++c) {
        int sx = mx[a], sy = my[b], sz = mz[c];
        bool conj = false;
        if (sx < 0) {  // Hermitian partner
          sx = -sx;
          sy = -sy;
          sz = -sz;
          conj = true;
        }
        const int iy = ((sy % fy) + fy) % fy, iz = ((sz % fz) + fz) % fz;
        const double2 v = sp[(int64_t(iz) * fy + iy) * fxh + sx];
        re += v.x;
        im += conj ? -v.y : v.y;
      }
  H[e] = make_double2(wgt * re, wgt * im);
}

// V[off_b + j][off_a + i] = V[off_a + i][off_b + j]
__global__ void k_mirror(double* V, int64_t ld, int64_t offa, int64_t offb, int64_t ka, int64_t kb, int lower_only) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= ka * kb) return;
  const int64_t i = e / kb, j = e % kb;
  if (lower_only && j >= i) return;  // within one block: copy lower to upper
  if (lower_only)
    V[(offa + j) * ld + offb + i] = V[(offa + i) * ld + offb + j];
  else
    V[(offb + j) * ld + offa + i] = V[(offa + i) * ld + offb + j];
}

__global__ void k_sqrt_inplace(int64_t n, double* w) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e < n) w[e] = sqrt(w[e]);
}

// V block on the tensor cores: weights split as sqrt(w) on both operands
// (w >= 0), sliced-BF16 FP64-accurate product, split over k.
isdf_status coulomb_block_tc(Plan* p, const double2* left, const Level& la, const Level& lb, double* wt2, bool same,
                             double* Cblk) {
  cudaStream_t s = p->stream;
  // 7 digits (49 fraction bits, exact level sums) when the blocks are those of
  // ZC: W = (CC^T)^-1 applied afterwards amplifies their error by up to
  // cond(CC^T) (5 digits missed the 1e-6 Ha bar on the undisplaced cell by
  // 600x, 7 digits take 2^14 off that); else 5
  const int S = (la.zct || lb.zct) ? 7 : 5;
  const int64_t K2 = 2 * lb.nq;
  k_sqrt_inplace<<<unsigned((K2 + 255) / 256), 256, 0, s>>>(K2, wt2);
  count_launches(1);
  OzOperand a, b;
  double* work = nullptr;
  isdf_status st;
  if ((st = oz_alloc(p, a, la.k, K2, 128, S, "Coulomb slices")) ||
      (st = oz_alloc(p, b, lb.k, K2, oz_bn(S), S, "Coulomb slices"))) {
    oz_free(a), oz_free(b);
    return st;
  }
  {
    // FP64 read twice (row scales, digits), S BF16 digits written per value
    Prof pr(p, "coulomb_slice", double(la.k + lb.k) * double(K2) * (16.0 + 2.0 * S), "byte", 4);
    oz_slice(reinterpret_cast<const double*>(left), K2, 1, wt2, 1.0, a, s);
    if (same)
      oz_retile(a, b, s);  // same spectra and weights: B's digits are A's, re-tiled
    else
      oz_slice(reinterpret_cast<const double*>(lb.spec), K2, 1, wt2, 1.0, b, s);
  }
  int64_t tiles = a.nrt * b.nrt;
  if (same) tiles = (tiles + a.nrt) / 2;
  int64_t splits = (4 * 152 + tiles - 1) / tiles;
  splits = std::max<int64_t>(1, std::min<int64_t>(splits, std::min<int64_t>(64, a.nkt / 64 + 1)));
  splits = oz_tuned_splits(p, a, b, Cblk, p->nip, 0, same ? 1 : 0, int(splits), s);
  if (splits > 1 && (st = dalloc_t(p, &work, size_t(splits) * la.k * lb.k, "split-k partials"))) {
    oz_free(a), oz_free(b);
    return st;
  }
  {
    const double work_fl = same ? double(la.k) * double(la.k + 1) * double(K2) : 2.0 * la.k * double(lb.k) * K2;
    Prof pr(p, "coulomb_V", work_fl, "flop", kLaunchesInside);
    oz_gemm(a, b, Cblk, p->nip, 0, 1.0, 0, same ? 1 : 0, int(splits), work, p->d_ozerr, s);
  }
  st = oz_check(p);
  oz_free(a);
  oz_free(b);
  dfree(work);
  return st;
}

}  // namespace

namespace {

// V_ab <- W_a V_ab W_b for every block of levels a <= b (then mirrored), with
// W_a = R_a^-T R_a^-1 = (C C^T)_a^-1, all in FP64-grade 8-digit products:
// the blocks computed from the spectra of ZC are those of Xi = ZC W.
isdf_status apply_w(Plan* p) {
  cudaStream_t s = p->stream;
  const int S = 8, bn = oz_bn(S);
  const int64_t nip = p->nip;
  double* W[ISDF_MAX_LEVELS] = {nullptr, nullptr, nullptr, nullptr};
  double* T = nullptr;
  OzOperand a, b;
  auto cleanup = [&]() {
    for (int l = 0; l < p->nlev; ++l) dfree(W[l]);
    dfree(T);
    oz_free(a);
    oz_free(b);
  };
  isdf_status st;
  int kmax = 1;
  for (int l = 0; l < p->nlev; ++l) kmax = std::max(kmax, p->lev[l].k);
  if ((st = dalloc_t(p, &T, size_t(kmax) * kmax, "Coulomb transform")) ||
      (st = oz_alloc(p, a, kmax, kmax, 128, S, "Coulomb transform")) ||
      (st = oz_alloc(p, b, kmax, kmax, bn, S, "Coulomb transform")))
    return cleanup(), st;
  auto view = [&](OzOperand& op, int64_t rows, int64_t K) {
    op.rows = rows;
    op.K = K;
    op.nrt = (rows + op.rt - 1) / op.rt;
    op.nkt = (K + kOzBK - 1) / kOzBK;
    op.kst = op.nkt;
  };
  double flop = 0.0;
  for (int l = 0; l < p->nlev; ++l) flop += 2.0 * std::pow(double(p->lev[l].k), 3.0);
  for (int x = 0; x < p->nlev; ++x)
    for (int y = x; y < p->nlev; ++y) flop += 2.0 * 2.0 * double(p->lev[x].k) * p->lev[y].k * (p->lev[x].k + p->lev[y].k) / 2.0;
  Prof pr(p, "coulomb_w", flop, "flop", kLaunchesInside);
  // W_l[m][n] = sum_kk R^-1[kk][m] R^-1[kk][n]; a level that holds Xi itself
  // (no R^-1: local grids' level 0) has W = I
  for (int l = 0; l < p->nlev; ++l) {
    const int k = p->lev[l].k;
    if (!k || !p->lev[l].rinv) continue;
    if ((st = dalloc_t(p, &W[l], size_t(k) * k, "W"))) return cleanup(), st;
    view(a, k, k);
    view(b, k, k);
    oz_slice(p->lev[l].rinv, 1, k, nullptr, 1.0, a, s);
    oz_slice(p->lev[l].rinv, 1, k, nullptr, 1.0, b, s);
    oz_gemm(a, b, W[l], k, 0, 1.0, 0, 0, 1, nullptr, p->d_ozerr, s);
  }
  for (int x = 0; x < p->nlev; ++x) {
    const int ka = p->lev[x].k;
    if (!ka) continue;
    for (int y = x; y < p->nlev; ++y) {
      const int kb = p->lev[y].k;
      if (!kb) continue;
      double* blk = p->V + int64_t(p->poff[x]) * nip + p->poff[y];
      if (!W[x] && !W[y]) continue;  // both levels hold Xi: the block is V already
      // T = V_Z,ab W_b   (T[m][n] = sum_j V[m][j] W_b[n][j], W_b symmetric)
      if (W[y]) {
        view(a, ka, kb);
        view(b, kb, kb);
        oz_slice(blk, nip, 1, nullptr, 1.0, a, s);
        oz_slice(W[y], kb, 1, nullptr, 1.0, b, s);
        oz_gemm(a, b, T, kb, 0, 1.0, 0, 0, 1, nullptr, p->d_ozerr, s);
      } else {
        cudaMemcpy2DAsync(T, sizeof(double) * kb, blk, sizeof(double) * nip, sizeof(double) * kb, ka,
                          cudaMemcpyDeviceToDevice, s);
      }
      // V_ab = W_a T   (V[m][n] = sum_i W_a[m][i] T[i][n])
      if (W[x]) {
        view(a, ka, ka);
        view(b, kb, ka);
        oz_slice(W[x], ka, 1, nullptr, 1.0, a, s);
        oz_slice(T, 1, kb, nullptr, 1.0, b, s);
        oz_gemm(a, b, blk, nip, 0, 1.0, 0, 0, 1, nullptr, p->d_ozerr, s);
      } else {
        cudaMemcpy2DAsync(blk, sizeof(double) * nip, T, sizeof(double) * kb, sizeof(double) * kb, ka,
                          cudaMemcpyDeviceToDevice, s);
      }
      if (x != y) {
        const int64_t tot = int64_t(ka) * kb;
        k_mirror<<<unsigned((tot + 255) / 256), 256, 0, s>>>(p->V, nip, p->poff[x], p->poff[y], ka, kb, 0);
        count_launches(1);
      }
    }
  }
  st = oz_check(p);
  cleanup();
  return st;
}

}  // namespace

void fold_spectra(int k, const double2* spf, int fx, int fy, int fz, double2* H, int cx, int cy, int cz,
                  cudaStream_t s) {
  const int64_t tot = int64_t(k) * (cx / 2 + 1) * cy * cz;
  if (tot > 0) k_fold<<<unsigned((tot + 255) / 256), 256, 0, s>>>(k, spf, fx, fy, fz, H, cx, cy, cz);
}

isdf_status transform_real(Plan* p, const double* f, int nx, int ny, int nz, int64_t batch, double2* spec) {
  cudaStream_t s = p->stream;
  if (p->opt.precision == 1 && rfft3_df_supported(nx, ny, nz)) return rfft3_df(p, f, nx, ny, nz, batch, spec, s);
  const int64_t ng = int64_t(nx) * ny * nz, nq = int64_t(nx / 2 + 1) * ny * nz;
  int dev = 0;
  cudaGetDevice(&dev);
  for (int64_t b0 = 0; b0 < batch;) {
    const int nb = int(std::min<int64_t>(batch - b0, 4096));
    const FftKey key{dev, nz, ny, nx, nb};
    cufftHandle h = 0;
    cufftResult r = fft_acquire(key, &h);
    if (r != CUFFT_SUCCESS) return fail(p, ISDF_ERR_CUFFT, "cufftPlanMany failed (" + std::to_string(int(r)) + ")");
    r = cufftSetStream(h, s);
    if (r == CUFFT_SUCCESS)
      r = cufftExecD2Z(h, const_cast<double*>(f) + b0 * ng, reinterpret_cast<cufftDoubleComplex*>(spec + b0 * nq));
    const cudaError_t e = cudaStreamSynchronize(s);
    fft_release(key, h);
    if (r != CUFFT_SUCCESS) return fail(p, ISDF_ERR_CUFFT, "cufftExecD2Z failed (" + std::to_string(int(r)) + ")");
    isdf_status st = cuda_check(p, e, "FFT");
    if (st) return st;
    b0 += nb;
  }
  return ISDF_OK;
}

isdf_status coulomb_run(Plan* p) {
  cudaStream_t s = p->stream;
  isdf_status st;
  const double four_pi_omega = 4.0 * 3.14159265358979323846 * p->omega;
  // 1. half spectra of every interpolation vector
  for (int l = 0; l < p->nlev; ++l) {
    Level& lv = p->lev[l];
    dfree(lv.spec);
    lv.spec = nullptr;
    lv.nh[0] = lv.n[0] / 2 + 1;
    lv.nh[1] = lv.n[1];
    lv.nh[2] = lv.n[2];
    lv.nq = int64_t(lv.nh[0]) * lv.nh[1] * lv.nh[2];
    if (lv.k == 0) continue;
    if ((st = dalloc_t(p, &lv.spec, size_t(lv.k) * lv.nq, "spectra"))) return st;
    if (p->opt.precision == 1 && p->fault != "fft_plan" && rfft3_df_supported(lv.n[0], lv.n[1], lv.n[2])) {
      // double-float transform on the FP32 pipes (the FP64 one is bound by the FP64 rate)
      Prof pr(p, "coulomb_fft", double(lv.k) * (8.0 * double(lv.ng) + 16.0 * double(lv.nq)), "byte", 3);
      if ((st = rfft3_df(p, lv.zct ? lv.zct : lv.xiT, lv.n[0], lv.n[1], lv.n[2], lv.k, lv.spec, s))) return st;
      continue;
    }
    // batches of about 256 MB of input (at least one vector, at most 64)
    int batch = p->opt.col_batch > 0 ? p->opt.col_batch
                                     : int(std::max<int64_t>(1, std::min<int64_t>(64, (int64_t(256) << 20) / (8 * lv.ng))));
    if (batch > lv.k) batch = lv.k;
    if (p->fault == "fft_plan") return fail(p, ISDF_ERR_CUFFT, "cufftPlanMany failed (injected)");
    int dev = 0;
    cudaGetDevice(&dev);
    Prof pr(p, "coulomb_fft", double(lv.k) * (8.0 * double(lv.ng) + 16.0 * double(lv.nq)), "byte", 0);
    for (int b0 = 0; b0 < lv.k;) {
      const int nb = (lv.k - b0 >= batch) ? batch : lv.k - b0;
      const FftKey key{dev, lv.n[2], lv.n[1], lv.n[0], nb};
      cufftHandle h = 0;
      cufftResult r = fft_acquire(key, &h);
      if (r != CUFFT_SUCCESS) return fail(p, ISDF_ERR_CUFFT, "cufftPlanMany failed (" + std::to_string(int(r)) + ")");
      r = cufftSetStream(h, s);
      // every full batch with this plan, then the remainder with its own
      const int nfull = (lv.k - b0) / nb;
      for (int c = 0; c < nfull && r == CUFFT_SUCCESS; ++c) {
        r = cufftExecD2Z(h, (lv.zct ? lv.zct : lv.xiT) + int64_t(b0) * lv.ng,
                         reinterpret_cast<cufftDoubleComplex*>(lv.spec + int64_t(b0) * lv.nq));
        b0 += nb;
      }
      // the handle goes back to the pool only once its work on this stream is done
      const cudaError_t e = cudaStreamSynchronize(s);
      fft_release(key, h);
      if (r != CUFFT_SUCCESS) return fail(p, ISDF_ERR_CUFFT, "cufftExecD2Z failed (" + std::to_string(int(r)) + ")");
      if ((st = cuda_check(p, e, "FFT"))) return st;
    }
  }
  // 2. V blocks
  const int64_t nip = p->nip;
  dfree(p->V);
  p->V = nullptr;
  if ((st = dalloc_t(p, &p->V, size_t(nip) * nip, "V"))) return st;
  for (int a = 0; a < p->nlev; ++a) {
    Level& la = p->lev[a];
    if (la.k == 0) continue;
    for (int b = a; b < p->nlev; ++b) {
      Level& lb = p->lev[b];
      if (lb.k == 0) continue;
      double* wt2 = nullptr;
      double2* H = nullptr;
      if ((st = dalloc_t(p, &wt2, size_t(2) * lb.nq, "Coulomb weights"))) return st;
      const bool same = (a == b);
      const double scale = same ? 1.0 / (double(lb.ng) * double(lb.ng)) : 1.0 / (double(la.ng) * double(lb.ng));
      count_launches(2 + (same ? 0 : 1));
      k_coul_weights<<<unsigned((lb.nq + 255) / 256), 256, 0, s>>>(lb.n[0], lb.n[1], lb.n[2], p->edge[0], p->edge[1],
                                                                   p->edge[2], four_pi_omega * scale, same ? 1 : 0, wt2);
      const double2* left = la.spec;
      if (!same) {
        if ((st = dalloc_t(p, &H, size_t(la.k) * lb.nq, "folded spectra"))) {
          dfree(wt2);
          return st;
        }
        const int64_t tot = int64_t(la.k) * lb.nq;
        k_fold<<<unsigned((tot + 255) / 256), 256, 0, s>>>(la.k, la.spec, la.n[0], la.n[1], la.n[2], H, lb.n[0],
                                                           lb.n[1], lb.n[2]);
        left = H;
      }
      GemmArgs g;
      g.ta = 0;
      g.tb = 1;
      g.M = la.k;
      g.N = lb.k;
      g.K = 2 * lb.nq;
      g.A = reinterpret_cast<const double*>(left);
      g.lda = 2 * lb.nq;
      g.B = reinterpret_cast<const double*>(lb.spec);
      g.ldb = 2 * lb.nq;
      g.C = p->V + int64_t(p->poff[a]) * nip + p->poff[b];
      g.ldc = nip;
      g.kw = wt2;
      g.sym = same ? 1 : 0;
      if (p->opt.precision == 1) {
        if ((st = coulomb_block_tc(p, left, la, lb, wt2, same, g.C))) {
          dfree(wt2);
          dfree(H);
          return st;
        }
      } else {
        const double K2 = 2.0 * double(lb.nq);
        const double work = same ? double(la.k) * double(la.k + 1) * K2 : 2.0 * double(la.k) * double(lb.k) * K2;
        Prof pr(p, "coulomb_V", work, "flop", 1);
        dgemm(g, s);
      }
      const int64_t tot = int64_t(la.k) * lb.k;
      k_mirror<<<unsigned((tot + 255) / 256), 256, 0, s>>>(p->V, nip, p->poff[a], p->poff[b], la.k, lb.k, same ? 1 : 0);
      st = cuda_check(p, cudaStreamSynchronize(s), "Coulomb block");
      dfree(wt2);
      dfree(H);
      if (st) return st;
    }
  }
  // A factored fit (Xi = ZC W, W = R^-T R^-1) transformed ZC: V = W V_Z W
  bool factored = false;
  for (int l = 0; l < p->nlev; ++l) factored = factored || p->lev[l].zct != nullptr;
  if (factored && (st = apply_w(p))) return st;
  // the coarsest level as the universal sinc grid: V_FU (V_UU is never formed)
  return p->opt.coarse_sinc ? sinc_coulomb(p) : ISDF_OK;
}

}  // namespace isdf
