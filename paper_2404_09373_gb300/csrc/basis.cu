// Basis evaluation on the grid levels (kernel family (a)).
//
// A periodic uncontracted Cartesian Gaussian on an orthorhombic cell is the
// product of three 1-D image sums (the Gaussian and the monomial both
// separate over x, y, z, and the kept lattice translations form a box), so
//   phi_mu(i, j, k) = N_mu T^x_mu(i) T^y_mu(j) T^z_mu(k).
// k_tab1d evaluates the 1-D factors (the only exp work); k_phi expands them
// into the basis matrix Phi[f][g] of a level, an HBM-write-bound outer product.
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace isdf {
namespace {

// One descriptor per (plan, level, axis) of a batch of plans: the 1-D factors
// tab[r * n + i] = scale[r] * sum_{t = tlo[r]}^{thi[r]} u^l exp(-alpha u^2),
// u = x_i - A[r] - t L, for the level's nG functions, at the grid points
// x_i = ((o + i) mod pn) L / pn (o = 0, pn = n for a full-cell grid; a local
// box's points are those of its parent grid); the per-function data sit at
// offset `fo` of the batch's staging arrays.
struct TabDesc {
  int64_t e0;  // first element of this descriptor in the batch's enumeration
  int nG, n;
  int o, pn;
  double L;
  int64_t fo;
  double* tab;
};

// Every element of every descriptor of the batch: one launch for all cells,
// levels and axes (the only exp work of the basis).
__global__ void k_tab1d(const TabDesc* __restrict__ D, int nd, int64_t total, const double* __restrict__ A,
                        const double* __restrict__ alpha, const int* __restrict__ lpow, const int* __restrict__ tlo,
                        const int* __restrict__ thi, const double* __restrict__ scale) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= total) return;
  int lo = 0, hi = nd - 1;  // last descriptor with e0 <= e
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (D[mid].e0 <= e) lo = mid;
    else hi = mid - 1;
  }
  const TabDesc d = D[lo];
  const int64_t le = e - d.e0;
  const int r = int(le / d.n), i = int(le % d.n);
  const int64_t f = d.fo + r;
  const int gi = ((d.o + i) % d.pn + d.pn) % d.pn;
  const double x = double(gi) * (d.L / double(d.pn));
  const double a = alpha[f];
  double s = 0.0;
  for (int t = tlo[f]; t <= thi[f]; ++t) {
    const double u = x - A[f] - double(t) * d.L;
    const double g = exp(-a * u * u);
    s += (lpow[f] ? u * g : g);
  }
  d.tab[le] = scale[f] * s;
}

// One descriptor per (plan, level): Phi[r][g] = tx[r][i] ty[r][j] tz[r][k],
// g = i + nx (j + ny k); on a local box zero outside the sphere
// ((o + i) h - c)^2 summed over the axes (x, y, then z) <= r2 (r2 < 0: no sphere).
struct PhiDesc {
  int64_t l0;  // first grid line of this descriptor in the batch's enumeration
  int nG, nx, ny, nz;
  const double *tx, *ty, *tz;
  double* phi;
  int o[3];
  double h[3], c[3], r2;
};

// One warp per grid line (function r, y index j, z index k) of any
// descriptor: the line's factor ty * tz is formed once, the lanes walk x with
// coalesced stores, so every value costs one FP64 multiply.  One launch
// expands the basis of every level of every plan of a batch.
__global__ void k_phi(const PhiDesc* __restrict__ D, int nd, int64_t nlines) {
  const int lane = threadIdx.x & 31;
  const int64_t wstride = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t line = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); line < nlines; line += wstride) {
    int lo = 0, hi = nd - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (D[mid].l0 <= line) lo = mid;
      else hi = mid - 1;
    }
    const PhiDesc d = D[lo];
    const int64_t nyz = int64_t(d.ny) * d.nz, ll = line - d.l0;
    const int64_t r = ll / nyz;
    const int rem = int(ll - r * nyz);
    const int k = rem / d.ny, j = rem - k * d.ny;
    const double yz = d.ty[r * d.ny + j] * d.tz[r * d.nz + k];
    const double* __restrict__ xr = d.tx + r * d.nx;
    double* __restrict__ out = d.phi + r * (nyz * d.nx) + (int64_t(k) * d.ny + j) * d.nx;
    if (d.r2 < 0.0) {
      for (int i = lane; i < d.nx; i += 32) out[i] = xr[i] * yz;
    } else {
      // the sphere test in the host's order and rounding (no contraction)
      const double dy = __dsub_rn(__dmul_rn(double(d.o[1] + j), d.h[1]), d.c[1]);
      const double dz = __dsub_rn(__dmul_rn(double(d.o[2] + k), d.h[2]), d.c[2]);
      const double dy2 = __dmul_rn(dy, dy), dz2 = __dmul_rn(dz, dz);
      for (int i = lane; i < d.nx; i += 32) {
        const double dx = __dsub_rn(__dmul_rn(double(d.o[0] + i), d.h[0]), d.c[0]);
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), dy2), dz2);
        out[i] = d2 <= d.r2 ? xr[i] * yz : 0.0;
      }
    }
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

// Basis of every level of every plan in one k_tab1d and one k_phi launch on
// `s` (the plans' buffers must be allocated and visible to `s`).  Per-function
// data of all (plan, level, axis) go to the device in one staging copy.
isdf_status basis_eval(Plan* const* plans_in, int nplans_in, cudaStream_t s) {
  Plan* p0 = plans_in[0];
  // a plan with local grids brings its atoms' sub-plans
  std::vector<Plan*> all;
  for (int b = 0; b < nplans_in; ++b) {
    all.insert(all.end(), plans_in[b]->sub.begin(), plans_in[b]->sub.end());
    all.push_back(plans_in[b]);
  }
  Plan* const* plans = all.data();
  const int nplans = int(all.size());
  std::vector<TabDesc> td;
  std::vector<PhiDesc> pd;
  std::vector<double> hA, hal, hsc;
  std::vector<int> hlp, hlo, hhi;
  int64_t e = 0, lines = 0;
  double tab_bytes = 0.0, phi_bytes = 0.0;
  for (int b = 0; b < nplans; ++b) {
    Plan* p = plans[b];
    for (int l = 0; l < p->nlev; ++l) {
      Level& lv = p->lev[l];
      const int nG = lv.nG;
      if (nG == 0) continue;
      std::vector<int> rows(lv.L);  // rows of Phi: L then N
      rows.insert(rows.end(), lv.N.begin(), lv.N.end());
      for (int a = 0; a < 3; ++a) {
        const int pn = lv.pn[0] ? lv.pn[a] : lv.n[a];
        TabDesc d{e, nG, lv.n[a], lv.pn[0] ? lv.o[a] : 0, pn, p->edge[a], int64_t(hA.size()), lv.tab[a]};
        for (int r = 0; r < nG; ++r) {
          const int mu = rows[r];
          int lo = 0, hi = 0;
          hA.push_back(p->xyz[3 * p->f_atom[mu] + a]);
          hal.push_back(p->f_alpha[mu]);
          hlp.push_back(p->f_l[a][mu]);
          hsc.push_back(a == 0 ? p->f_norm[mu] : 1.0);
          image_range(hA.back(), p->edge[a], hal.back(), p->image_tol, &lo, &hi);
          hlo.push_back(lo);
          hhi.push_back(hi);
        }
        td.push_back(d);
        e += int64_t(nG) * lv.n[a];
      }
      PhiDesc q{lines, nG, lv.n[0], lv.n[1], lv.n[2], lv.tab[0], lv.tab[1], lv.tab[2], lv.phi, {0, 0, 0},
                {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, lv.mr2};
      for (int a = 0; a < 3; ++a) {
        q.o[a] = lv.o[a];
        q.h[a] = lv.pn[0] ? p->edge[a] / double(lv.pn[a]) : 0.0;
        q.c[a] = lv.mc[a];
      }
      pd.push_back(q);
      lines += int64_t(nG) * lv.n[1] * lv.n[2];
      phi_bytes += 8.0 * double(nG) * double(lv.ng);
    }
  }
  if (td.empty()) return ISDF_OK;
  tab_bytes = 8.0 * double(e);
  const size_t nf = hA.size();
  // staging: descriptors, then A, alpha, scale (double), then lpow, tlo, thi (int)
  const size_t b_td = td.size() * sizeof(TabDesc), b_pd = pd.size() * sizeof(PhiDesc);
  const size_t off_pd = (b_td + 15) & ~size_t(15), off_f = (off_pd + b_pd + 15) & ~size_t(15);
  const size_t bytes = off_f + nf * (3 * sizeof(double) + 3 * sizeof(int));
  std::vector<unsigned char> h(bytes);
  std::memcpy(h.data(), td.data(), b_td);
  std::memcpy(h.data() + off_pd, pd.data(), b_pd);
  double* hd = reinterpret_cast<double*>(h.data() + off_f);
  int* hi3 = reinterpret_cast<int*>(hd + 3 * nf);
  for (size_t r = 0; r < nf; ++r) {
    hd[r] = hA[r], hd[nf + r] = hal[r], hd[2 * nf + r] = hsc[r];
    hi3[r] = hlp[r], hi3[nf + r] = hlo[r], hi3[2 * nf + r] = hhi[r];
  }
  unsigned char* dd = nullptr;
  isdf_status st = dalloc_t(p0, &dd, bytes, "basis staging");
  if (st) return st;
  st = cuda_check(p0, cudaMemcpyAsync(dd, h.data(), bytes, cudaMemcpyHostToDevice, s), "copy");
  const double* dA = reinterpret_cast<const double*>(dd + off_f);
  const int* di = reinterpret_cast<const int*>(dA + 3 * nf);
  if (!st) {
    Prof pr(nplans_in == 1 ? p0 : nullptr, "basis_tab1d", tab_bytes, "byte", 1);
    k_tab1d<<<unsigned((e + 255) / 256), 256, 0, s>>>(reinterpret_cast<const TabDesc*>(dd), int(td.size()), e, dA,
                                                      dA + nf, di, di + nf, di + 2 * nf, dA + 2 * nf);
    st = cuda_check(p0, cudaGetLastError(), "k_tab1d");
  }
  if (!st) {
    Prof pr(nplans_in == 1 ? p0 : nullptr, "basis_phi", phi_bytes, "byte", 1);
    k_phi<<<152 * 16, 256, 0, s>>>(reinterpret_cast<const PhiDesc*>(dd + off_pd), int(pd.size()), lines);
    st = cuda_check(p0, cudaGetLastError(), "k_phi");
  }
  // the staging buffer must outlive the kernels
  isdf_status st2 = cuda_check(p0, cudaStreamSynchronize(s), "basis");
  dfree(dd);
  return st ? st : st2;
}

// Allocate the 1-D factor tables and the basis matrix of every level.
isdf_status basis_alloc(Plan* p) {
  for (Plan* q : p->sub) {
    isdf_status st = basis_alloc(q);
    if (st) {
      p->err = q->err;
      return st;
    }
  }
  for (int l = 0; l < p->nlev; ++l) {
    Level& lv = p->lev[l];
    if (lv.nG == 0) continue;
    isdf_status st;
    for (int a = 0; a < 3; ++a)
      if ((st = dalloc_t(p, &lv.tab[a], size_t(lv.nG) * lv.n[a], "basis 1-D tables"))) return st;
    if ((st = dalloc_t(p, &lv.phi, size_t(lv.nG) * lv.ng, "basis values Phi"))) return st;
  }
  return ISDF_OK;
}

isdf_status basis_build(Plan* p) {
  isdf_status st = basis_alloc(p);
  if (!st) st = basis_eval(&p, 1, p->stream);
  return st;
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
