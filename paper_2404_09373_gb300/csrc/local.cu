// Atom-centred local dense grids (Section III, Eq. 5 and Fig. Grids): the
// finest level's functions are represented on a sphere of radius
//   r_max = sqrt(-ln eps_r / alpha_min)
// around their atom, and each atom runs its own ISDF there (the local form of
// Eq. 7: products mu^L_A nu^G_A on the grid R_A, fitted by the greedy of
// Eq. 2 and the least squares of Eq. 3).
//
// Layout.  Atom A's grid is a box of the finest full grid around A's nearest
// grid index; the basis values outside the sphere are zero, so the box is the
// sphere exactly (zero residuals are never pivots, the fit is zero there).
// Each atom is a single-level sub-plan with its own basis values, selection
// and fit, so the selection and fit kernels run unchanged on it.  The main
// plan's level 0 has no basis values of its own: after the atoms' fits it
// receives their interpolation vectors placed on the full finest grid (rows
// scattered from the boxes), and the Coulomb matrix (one transform per local
// fitting function, Section III) and the exchange build treat it like any
// other level.  X^N of a local pivot also holds the finest-level functions of
// higher-index atoms.
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace isdf {
namespace {

// dst[r][parent(b)] = src[r][b] for the k rows of one box (dst rows zeroed by
// the caller; rows are ld apart in dst, box-sized in src).
__global__ void k_embed_box(int k, const double* __restrict__ src, int bx, int by, int bz, int ox, int oy, int oz,
                            int nx, int ny, int nz, double* __restrict__ dst, int64_t ld) {
  const int64_t nb = int64_t(bx) * by * bz;
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= nb * k) return;
  const int64_t r = e / nb, b = e % nb;
  const int i = int(b % bx), j = int((b / bx) % by), kk = int(b / (int64_t(bx) * by));
  const int gx = ((ox + i) % nx + nx) % nx, gy = ((oy + j) % ny + ny) % ny, gz = ((oz + kk) % nz + nz) % nz;
  dst[r * ld + gx + int64_t(nx) * (gy + int64_t(ny) * gz)] = src[e];
}

void free_sub_fit(Plan* q) {
  Level& lv = q->lev[0];
  dfree(lv.zct), dfree(lv.rinv), dfree(lv.xiT), dfree(lv.resid);
  lv.zct = lv.rinv = lv.xiT = nullptr;
  lv.resid = nullptr;
  dfree(q->XL), dfree(q->XN);
  q->XL = q->XN = nullptr;
}

}  // namespace

bool local_inside(const Plan* q, int64_t b) {
  const Level& lv = q->lev[0];
  const int i = int(b % lv.n[0]), j = int((b / lv.n[0]) % lv.n[1]), k = int(b / (int64_t(lv.n[0]) * lv.n[1]));
  // each operation rounded on its own (no fused multiply-add), as in k_phi
  volatile double d2[3];
  const int ijk[3] = {i, j, k};
  for (int a = 0; a < 3; ++a) {
    volatile double x = double(lv.o[a] + ijk[a]) * (q->edge[a] / double(lv.pn[a]));
    volatile double d = x - lv.mc[a];
    d2[a] = d * d;
  }
  volatile double t = d2[0] + d2[1];
  return t + d2[2] <= lv.mr2;
}

isdf_status local_setup(Plan* p, double alpha_min) {
  const Level& f = p->lev[0];
  p->r_max = std::sqrt(-std::log(p->opt.local_eps_r) / alpha_min);
  int r[3], B[3];
  double h[3];
  for (int a = 0; a < 3; ++a) {
    h[a] = p->edge[a] / double(f.n[a]);
    r[a] = int(std::floor(p->r_max / h[a])) + 1;
    B[a] = 2 * r[a] + 1;
    if (B[a] > f.n[a])
      return fail(p, ISDF_ERR_ARG, "options.local_grids: the local grid (" + std::to_string(B[a]) +
                                       " points) is wider than the cell (" + std::to_string(f.n[a]) + ")");
    if (B[a] > 255) return fail(p, ISDF_ERR_ARG, "options.local_grids: more than 255 box points per axis");
  }
  if (p->natom > 65535) return fail(p, ISDF_ERR_ARG, "options.local_grids: more than 65535 atoms");
  for (int A = 0; A < p->natom; ++A) {
    Plan* q = new (std::nothrow) Plan();
    if (!q) return fail(p, ISDF_ERR_OOM, "host allocation failed");
    p->sub.push_back(q);
    q->stream = p->stream;
    q->opt = p->opt;
    q->opt.local_grids = 0;
    q->opt.coarse_sinc = 0;
    q->opt.profile = 0;
    // an atom takes some tens of pivots over some ten thousand points: the
    // step-by-step selection (four graph-captured kernels per step, same
    // pivots) costs less there than the speculative blocks' set-up
    q->opt.select_block = 0;
    q->fault = p->fault;
    q->fit_slices = 8;
    for (int a = 0; a < 3; ++a) q->edge[a] = p->edge[a];
    q->omega = p->omega;
    q->image_tol = p->image_tol;
    q->natom = p->natom;
    q->xyz = p->xyz;
    q->nfun = p->nfun;
    q->f_atom = p->f_atom;
    for (int a = 0; a < 3; ++a) q->f_l[a] = p->f_l[a];
    q->f_level = p->f_level;
    q->f_alpha = p->f_alpha;
    q->f_norm = p->f_norm;
    q->nlev = 1;
    Level& lv = q->lev[0];
    for (int a = 0; a < 3; ++a) {
      const double x = p->xyz[3 * A + a];
      const int c = int(std::floor(x / h[a] + 0.5));
      lv.n[a] = B[a];
      lv.o[a] = c - r[a];
      lv.pn[a] = f.n[a];
      lv.mc[a] = x;
    }
    lv.mr2 = p->r_max * p->r_max;
    lv.ng = int64_t(B[0]) * B[1] * B[2];
    lv.w = p->omega / double(f.ng);
    for (int mu = 0; mu < p->nfun; ++mu) {
      const bool sharp = p->f_level[mu] == 0;
      if (sharp && p->f_atom[mu] == A) lv.L.push_back(mu);
      if ((sharp && p->f_atom[mu] > A) || p->f_level[mu] > 0) lv.N.push_back(mu);
    }
    lv.nL = int(lv.L.size());
    lv.nN = int(lv.N.size());
    lv.nG = lv.nL + lv.nN;
    q->off[0] = 0;
    q->off[1] = lv.ng;
    q->ntot = lv.ng;
    isdf_status st = dalloc_t(p, &q->d_err, 1, "error word");
    if (!st) st = dalloc_t(p, &q->d_ozerr, 1, "error word");
    if (!st) st = cuda_check(p, cudaMemsetAsync(q->d_ozerr, 0, sizeof(int), p->stream), "memset");
    if (st) return st;
  }
  // level 0 of this plan: no functions of its own (no basis values); its
  // points are those of the full finest grid, for the Coulomb matrix only
  Level& l0 = p->lev[0];
  l0.L.clear();
  l0.N.clear();
  l0.nL = l0.nN = l0.nG = 0;
  p->sel_lo = 1;
  return ISDF_OK;
}

isdf_status local_select(Plan* p, std::vector<int64_t>& piv, std::vector<double>& dval) {
  cudaStream_t s = p->stream;
  Prof pr(p, "local_select", 0.0, "flop", kLaunchesInside);
  for (int A = 0; A < int(p->sub.size()); ++A) {
    Plan* q = p->sub[A];
    const int cap = int(std::min<int64_t>(p->opt.local_cap, q->ntot));
    int found = 0;
    isdf_status st = select_run(q, cap, p->opt.local_tol, nullptr, &found);
    if (st) {
      p->err = "atom " + std::to_string(A) + ": " + q->err;
      return st;
    }
    std::vector<int64_t> c(found);
    std::vector<double> d(found);
    if (found) {
      cudaMemcpyAsync(c.data(), q->d_piv, sizeof(int64_t) * found, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(d.data(), q->d_dval, sizeof(double) * found, cudaMemcpyDeviceToHost, s);
      if ((st = cuda_check(p, cudaStreamSynchronize(s), "local pivots"))) return st;
    }
    for (int i = 0; i < found; ++i) {
      piv.push_back((int64_t(A) << kLocalAtomShift) | (c[i] & kPivMask));
      dval.push_back(d[i]);
    }
    // the factor columns and candidate arrays go with the call
    dfree(q->d_diag);
    q->d_diag = nullptr;
  }
  return ISDF_OK;
}

isdf_status local_fit(Plan* p, const std::vector<std::vector<int64_t>>& per_atom) {
  cudaStream_t s = p->stream;
  Prof pr(p, "local_fit", 0.0, "flop", kLaunchesInside);
  for (int A = 0; A < int(p->sub.size()); ++A) {
    Plan* q = p->sub[A];
    Level& lv = q->lev[0];
    free_sub_fit(q);
    dfree(lv.d_pg);
    lv.d_pg = nullptr;
    lv.pg = per_atom[A];
    lv.k = int(lv.pg.size());
    q->nip = lv.k;
    q->poff[0] = 0;
    q->poff[1] = lv.k;
    q->piv_lo = lv.pg;
    if (lv.k == 0) continue;
    isdf_status st;
    if ((st = dalloc_t(p, &lv.d_pg, size_t(lv.k), "pivot indices")) ||
        (st = cuda_check(p, cudaMemcpyAsync(lv.d_pg, lv.pg.data(), sizeof(int64_t) * lv.k, cudaMemcpyHostToDevice, s),
                         "copy pivots")) ||
        (st = dalloc_t(p, &q->XL, size_t(p->nfun) * lv.k, "X^L")) ||
        (st = dalloc_t(p, &q->XN, size_t(p->nfun) * lv.k, "X^N")))
      return st;
    if ((st = fit_run(q))) {
      p->err = "atom " + std::to_string(A) + ": " + q->err;
      return st;
    }
  }
  return ISDF_OK;
}

isdf_status local_assemble(Plan* p) {
  cudaStream_t s = p->stream;
  Level& l0 = p->lev[0];
  dfree(l0.zct), dfree(l0.rinv), dfree(l0.xiT), dfree(l0.resid);
  l0.zct = l0.rinv = l0.xiT = nullptr;
  l0.resid = nullptr;
  const int64_t K0 = l0.k, nip = p->nip;
  if (K0 == 0) return ISDF_OK;
  // Level 0 holds the interpolation vectors themselves, not the factored
  // form ZC with W = (CC^T)^-1: an atom's threshold-driven CC^T can be
  // conditioned far beyond the inverse of local_tol, and applying an explicit
  // W on both sides of the Coulomb matrix loses accuracy as cond(CC^T)^2,
  // where forming Xi first (R^-T (R^-1 ZC^T), FP64-grade products on the
  // atom's small box) loses it as cond(CC^T)
  isdf_status st;
  for (Plan* q : p->sub)
    if (q->lev[0].k && (st = fit_xi_run(q, 0))) {
      p->err = q->err;
      return st;
    }
  if ((st = dalloc_t(p, &l0.xiT, size_t(K0) * l0.ng, "Xi (local grids)"))) return st;
  Prof pr(p, "local_assemble", 8.0 * double(K0) * double(l0.ng), "byte", kLaunchesInside);
  cudaMemsetAsync(l0.xiT, 0, sizeof(double) * size_t(K0) * l0.ng, s);
  int64_t c0 = 0;
  for (Plan* q : p->sub) {
    Level& lv = q->lev[0];
    const int64_t k = lv.k;
    if (!k) continue;
    const int64_t tot = k * lv.ng;
    k_embed_box<<<unsigned((tot + 255) / 256), 256, 0, s>>>(int(k), lv.xiT, lv.n[0], lv.n[1], lv.n[2], lv.o[0], lv.o[1],
                                                            lv.o[2], l0.n[0], l0.n[1], l0.n[2], l0.xiT + c0 * l0.ng,
                                                            l0.ng);
    count_launches(1);
    if ((st = cuda_check(p, cudaGetLastError(), "k_embed_box"))) return st;
    // X^L, X^N columns of this atom's pivots (after the plan's own gather,
    // which cleared both matrices)
    const int64_t col = p->poff[0] + c0;
    if ((st = cuda_check(p, cudaMemcpy2DAsync(p->XL + col, sizeof(double) * nip, q->XL, sizeof(double) * k,
                                              sizeof(double) * k, p->nfun, cudaMemcpyDeviceToDevice, s),
                         "X^L columns")) ||
        (st = cuda_check(p, cudaMemcpy2DAsync(p->XN + col, sizeof(double) * nip, q->XN, sizeof(double) * k,
                                              sizeof(double) * k, p->nfun, cudaMemcpyDeviceToDevice, s),
                         "X^N columns")))
      return st;
    c0 += k;
  }
  st = cuda_check(p, cudaStreamSynchronize(s), "local assembly");
  // the atoms' copies are no longer needed
  for (Plan* q : p->sub) free_sub_fit(q);
  return st;
}

}  // namespace isdf
