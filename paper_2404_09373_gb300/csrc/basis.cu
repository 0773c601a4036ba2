// Basis evaluation on the grid levels (kernel family (a)).
//
// A periodic uncontracted Cartesian Gaussian on an orthorhombic cell is the
// product of three 1-D image sums (the Gaussian and the monomial both
// separate over x, y, z, and the kept lattice translations form a box), so
//   phi_mu(i, j, k) = N_mu T^x_mu(i) T^y_mu(j) T^z_mu(k).
// k_tab1d evaluates the 1-D factors (the only exp work); k_phi expands them
// into the basis matrix Phi[f][g] of a level, an HBM-write-bound outer product.
#include <cmath>

#include "internal.cuh"

namespace isdf {
namespace {

// tab[r * n + i] = scale[r] * sum_{t = tlo[r]}^{thi[r]} u^l exp(-alpha u^2),
// u = i L / n - A[r] - t L
__global__ void k_tab1d(int nG, int n, double Lax, const double* __restrict__ A, const double* __restrict__ alpha,
                        const int* __restrict__ lpow, const int* __restrict__ tlo, const int* __restrict__ thi,
                        const double* __restrict__ scale, double* __restrict__ tab) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= int64_t(nG) * n) return;
  const int r = int(e / n), i = int(e % n);
  const double x = double(i) * (Lax / double(n));
  const double a = alpha[r];
  double s = 0.0;
  for (int t = tlo[r]; t <= thi[r]; ++t) {
    const double u = x - A[r] - double(t) * Lax;
    const double g = exp(-a * u * u);
    s += (lpow[r] ? u * g : g);
  }
  tab[e] = scale[r] * s;
}

// Phi[r][g] = tx[r][i] ty[r][j] tz[r][k], g = i + nx (j + ny k)
// One warp per grid line (function r, y index j, z index k): the line's
// factor ty * tz is formed once, the lanes walk x with coalesced stores, so
// every value costs one FP64 multiply and no 64-bit division.
__global__ void k_phi(int nG, int nx, int ny, int nz, const double* __restrict__ tx, const double* __restrict__ ty,
                      const double* __restrict__ tz, double* __restrict__ phi) {
  const int lane = threadIdx.x & 31;
  const int64_t nyz = int64_t(ny) * nz, nlines = nyz * nG;
  const int64_t ng = nyz * nx;
  const int64_t wstride = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t line = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); line < nlines; line += wstride) {
    const int64_t r = line / nyz;
    const int rem = int(line - r * nyz);
    const int k = rem / ny, j = rem - k * ny;
    const double yz = ty[r * ny + j] * tz[r * nz + k];
    const double* __restrict__ xr = tx + r * nx;
    double* __restrict__ out = phi + r * ng + (int64_t(k) * ny + j) * nx;
    for (int i = lane; i < nx; i += 32) out[i] = xr[i] * yz;
  }
}

// X^L / X^N: out[mu][c] = phi_level(row(mu), g_c) for the functions of one
// set; zero elsewhere (the caller clears the matrices first).
__global__ void k_gather_pivots(int nrows, const int* __restrict__ rows_phi, const int* __restrict__ fun,
                                int kcols, const int64_t* __restrict__ pg, const double* __restrict__ phi, int64_t ng,
                                double* __restrict__ out, int64_t ldo, int64_t col0) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= int64_t(nrows) * kcols) return;
  const int r = int(e / kcols), c = int(e % kcols);
  out[int64_t(fun[r]) * ldo + col0 + c] = phi[int64_t(rows_phi[r]) * ng + pg[c]];
}

// Image translations kept on one axis: t with dist(A + t L, [0, L]) <= r_cut.
void image_range(double A, double L, double alpha, double tol, int* lo, int* hi) {
  const double rcut = std::sqrt(std::log(1.0 / tol) / alpha);
  const int tmax = int(std::ceil((rcut + L) / L)) + 1;
  *lo = 1;
  *hi = 0;
  for (int t = -tmax; t <= tmax; ++t) {
    const double c = A + t * L;
    const double dist = (c >= 0.0 && c <= L) ? 0.0 : std::fmin(std::fabs(c), std::fabs(c - L));
    if (dist <= rcut) {
      if (*lo > *hi) *lo = t;
      *hi = t;
    }
  }
}

}  // namespace

isdf_status basis_build(Plan* p) {
  cudaStream_t s = p->stream;
  for (int l = 0; l < p->nlev; ++l) {
    Level& lv = p->lev[l];
    std::vector<int> rows(lv.L);  // rows of Phi: L then N
    rows.insert(rows.end(), lv.N.begin(), lv.N.end());
    const int nG = lv.nG;
    if (nG == 0) continue;
    for (int a = 0; a < 3; ++a) {
      std::vector<double> A(nG), al(nG), sc(nG);
      std::vector<int> lp(nG), lo(nG), hi(nG);
      for (int r = 0; r < nG; ++r) {
        const int mu = rows[r];
        A[r] = p->xyz[3 * p->f_atom[mu] + a];
        al[r] = p->f_alpha[mu];
        lp[r] = p->f_l[a][mu];
        sc[r] = (a == 0) ? p->f_norm[mu] : 1.0;
        image_range(A[r], p->edge[a], al[r], p->image_tol, &lo[r], &hi[r]);
      }
      // one staging buffer: A, alpha, scale (double) then lpow, tlo, thi (int)
      double* dd = nullptr;
      isdf_status st = dalloc_t(p, &dd, size_t(3) * nG + size_t(3) * nG, "basis staging");
      if (st) return st;
      int* di = reinterpret_cast<int*>(dd + 3 * nG);
      std::vector<double> hd(3 * nG);
      std::vector<int> hi3(3 * nG);
      for (int r = 0; r < nG; ++r) {
        hd[r] = A[r];
        hd[nG + r] = al[r];
        hd[2 * nG + r] = sc[r];
        hi3[r] = lp[r];
        hi3[nG + r] = lo[r];
        hi3[2 * nG + r] = hi[r];
      }
      st = cuda_check(p, cudaMemcpyAsync(dd, hd.data(), sizeof(double) * 3 * nG, cudaMemcpyHostToDevice, s), "copy");
      if (st) return st;
      st = cuda_check(p, cudaMemcpyAsync(di, hi3.data(), sizeof(int) * 3 * nG, cudaMemcpyHostToDevice, s), "copy");
      if (st) return st;
      st = dalloc_t(p, &lv.tab[a], size_t(nG) * lv.n[a], "basis 1-D tables");
      if (st) return st;
      const int64_t tot = int64_t(nG) * lv.n[a];
      Prof pr(p, "basis_tab1d", 8.0 * double(tot), "byte", 1);
      k_tab1d<<<unsigned((tot + 255) / 256), 256, 0, s>>>(nG, lv.n[a], p->edge[a], dd, dd + nG, di, di + nG,
                                                          di + 2 * nG, dd + 2 * nG, lv.tab[a]);
      st = cuda_check(p, cudaGetLastError(), "k_tab1d");
      if (st) return st;
      // the staging buffer must outlive the kernel: synchronise before freeing
      st = cuda_check(p, cudaStreamSynchronize(s), "basis tables");
      dfree(dd);
      if (st) return st;
    }
    isdf_status st = dalloc_t(p, &lv.phi, size_t(nG) * lv.ng, "basis values Phi");
    if (st) return st;
    Prof pr(p, "basis_phi", 8.0 * double(nG) * double(lv.ng), "byte", 1);
    k_phi<<<152 * 16, 256, 0, s>>>(nG, lv.n[0], lv.n[1], lv.n[2], lv.tab[0], lv.tab[1], lv.tab[2], lv.phi);
    st = cuda_check(p, cudaGetLastError(), "k_phi");
    if (st) return st;
  }
  return ISDF_OK;
}

// X^L and X^N (N x nip, level-ordered pivot columns) from Phi at the pivots.
isdf_status gather_pivot_factors(Plan* p) {
  cudaStream_t s = p->stream;
  const int64_t nip = p->nip;
  isdf_status st = cuda_check(p, cudaMemsetAsync(p->XL, 0, sizeof(double) * p->nfun * nip, s), "memset XL");
  if (st) return st;
  st = cuda_check(p, cudaMemsetAsync(p->XN, 0, sizeof(double) * p->nfun * nip, s), "memset XN");
  if (st) return st;
  for (int l = 0; l < p->nlev; ++l) {
    Level& lv = p->lev[l];
    if (lv.k == 0) continue;
    for (int set = 0; set < 2; ++set) {
      const std::vector<int>& fun = set == 0 ? lv.L : lv.N;
      const int nr = int(fun.size());
      if (nr == 0) continue;
      std::vector<int> h(2 * nr);
      for (int r = 0; r < nr; ++r) {
        h[r] = (set == 0 ? 0 : lv.nL) + r;  // row in Phi
        h[nr + r] = fun[r];                 // basis function index
      }
      int* d = nullptr;
      st = dalloc_t(p, &d, size_t(2) * nr, "gather staging");
      if (st) return st;
      st = cuda_check(p, cudaMemcpyAsync(d, h.data(), sizeof(int) * 2 * nr, cudaMemcpyHostToDevice, s), "copy");
      if (st) return st;
      const int64_t tot = int64_t(nr) * lv.k;
      count_launches(1);
      k_gather_pivots<<<unsigned((tot + 255) / 256), 256, 0, s>>>(nr, d, d + nr, lv.k, lv.d_pg, lv.phi, lv.ng,
                                                                  set == 0 ? p->XL : p->XN, nip, p->poff[l]);
      st = cuda_check(p, cudaGetLastError(), "k_gather_pivots");
      if (st) return st;
      st = cuda_check(p, cudaStreamSynchronize(s), "gather");
      dfree(d);
      if (st) return st;
    }
  }
  return ISDF_OK;
}

}  // namespace isdf
