// C ABI of the multigrid ISDF library: argument checks, plan life cycle,
// host/device marshalling and the call-order state machine.  Every step of
// the computation runs in this library's kernels (basis.cu, select.cu,
// fit.cu, coulomb.cu, exchange.cu, dgemm.cu).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>
#include <set>

#include <mutex>
#include <unordered_map>

#include "internal.cuh"

struct isdf_plan_s {
  isdf::Plan p;
};

namespace isdf {

static thread_local std::string g_plan_error;  // failures before a plan exists
std::atomic<long long> g_launches{0};
thread_local long long t_launches = 0;

Prof::Prof(Plan* p_, const char* name, double work, const char* unit, int64_t launches) : p(p_) {
  if (launches > 0) count_launches(launches);
  t0 = t_launches;
  if (!p || !p->opt.profile) return;
  e.name = name;
  e.work = work;
  e.unit = unit;
  e.launches = launches;
  cudaEventCreate(&e.a);
  cudaEventCreate(&e.b);
  cudaEventRecord(e.a, p->stream);
}

Prof::~Prof() {
  if (!p || !p->opt.profile || !e.a) return;
  if (e.launches == kLaunchesInside) e.launches = t_launches - t0;
  cudaEventRecord(e.b, p->stream);
  p->pend.push_back(e);
}

void prof_flush(Plan* p) {
  for (ProfEvent& e : p->pend) {
    float ms = 0.0f;
    if (cudaEventSynchronize(e.b) == cudaSuccess && cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) {
      KStat& k = p->stats[e.name];
      k.launches += e.launches;
      k.ms += ms;
      k.work += e.work;
      k.flop += e.flop;
      k.unit = e.unit;
    }
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  p->pend.clear();
  cudaGetLastError();
}

isdf_status fail(Plan* p, isdf_status s, const std::string& msg) {
  if (p) p->err = msg;
  return s;
}

isdf_status cuda_check(Plan* p, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return ISDF_OK;
  return fail(p, ISDF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Plan buffers are stream-ordered: allocated with cudaMallocAsync on the
// plan's stream from the device's default pool (whose release threshold is
// raised once, so freed memory stays cached for the next allocation or the
// next plan) and freed with cudaFreeAsync on the same stream.  The stream of
// every live allocation is remembered for dfree.  Buffers without a plan
// (the stand-alone product) use cudaMalloc / cudaFree.
namespace {
std::mutex g_alloc_mu;
std::unordered_map<void*, cudaStream_t> g_async_owner;
bool g_pool_ready[64] = {false};

void pool_setup() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return;
  }
  if (g_pool_ready[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  g_pool_ready[dev] = true;
}
}  // namespace

isdf_status dalloc(Plan* p, void** ptr, size_t bytes, const char* what) {
  *ptr = nullptr;
  if (p && p->fault == "oom") return fail(p, ISDF_ERR_OOM, std::string("device allocation failed (injected): ") + what);
  if (bytes == 0) bytes = 16;
  cudaError_t e;
  if (p) {
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    pool_setup();
    e = cudaMallocAsync(ptr, bytes, p->stream);
    if (e == cudaErrorMemoryAllocation && !p->capturing) {
      // the pool keeps freed memory (raised release threshold); when a large
      // request finds it fragmented, give the unused part back once and retry
      cudaGetLastError();
      int dev = 0;
      cudaMemPool_t pool;
      if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        cudaDeviceSynchronize();  // frees pending on other streams complete first
        cudaMemPoolTrimTo(pool, 0);
        e = cudaMallocAsync(ptr, bytes, p->stream);
      }
    }
    if (e == cudaSuccess) g_async_owner[*ptr] = p->stream;
  } else {
    e = cudaMalloc(ptr, bytes);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return fail(p, e == cudaErrorMemoryAllocation ? ISDF_ERR_OOM : ISDF_ERR_CUDA,
                std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes for " + what + ": " +
                    cudaGetErrorString(e));
  }
  return ISDF_OK;
}

isdf_status oz_check(Plan* p) {
  int h = 0;
  isdf_status st = cuda_check(p, cudaMemcpyAsync(&h, p->d_ozerr, sizeof(int), cudaMemcpyDeviceToHost, p->stream),
                              "error word copy");
  if (!st) st = cuda_check(p, cudaStreamSynchronize(p->stream), "tensor-core products");
  if (!st && h) {
    cudaMemsetAsync(p->d_ozerr, 0, sizeof(int), p->stream);
    return fail(p, ISDF_ERR_TIMEOUT, "a tensor-core pipeline wait expired (code " + std::to_string(h) + ")");
  }
  return st;
}

void dfree(void* ptr) {
  if (!ptr) return;
  {
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    auto it = g_async_owner.find(ptr);
    if (it != g_async_owner.end()) {
      cudaFreeAsync(ptr, it->second);
      g_async_owner.erase(it);
      return;
    }
  }
  cudaFree(ptr);
}

bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

namespace {

void free_plan(Plan* p) {
  for (Plan* q : p->sub) {
    free_plan(q);
    delete q;
  }
  p->sub.clear();
  for (int l = 0; l < ISDF_MAX_LEVELS; ++l) {
    Level& lv = p->lev[l];
    for (int a = 0; a < 3; ++a) dfree(lv.tab[a]);
    dfree(lv.phi);
    dfree(lv.fac);
    dfree(lv.d_pg);
    dfree(lv.xiT);
    dfree(lv.resid);
    dfree(lv.zct);
    dfree(lv.rinv);
    dfree(lv.spec);
    lv = Level();
  }
  dfree(p->d_diag);
  dfree(p->d_selstate);
  dfree(p->d_piv);
  dfree(p->d_dval);
  dfree(p->XL);
  dfree(p->XN);
  dfree(p->V);
  dfree(p->d_err);
  dfree(p->d_ozerr);
  dfree(p->d_perm);
  p->d_perm = nullptr;
  dfree(p->VFU);
  p->VFU = nullptr;
  p->d_ozerr = nullptr;
  p->d_diag = nullptr;
  p->d_selstate = nullptr;
  p->d_piv = nullptr;
  p->d_dval = nullptr;
  p->XL = p->XN = p->V = nullptr;
  p->d_err = nullptr;
}

// Copy n elements from a host or device source into a host vector.
template <class T>
isdf_status to_host(Plan* p, const T* src, size_t n, std::vector<T>& out) {
  out.resize(n);
  if (n == 0) return ISDF_OK;
  if (is_device_ptr(src)) {
    isdf_status st = cuda_check(p, cudaMemcpyAsync(out.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost, p->stream),
                                "device to host copy");
    if (st) return st;
    return cuda_check(p, cudaStreamSynchronize(p->stream), "device to host copy");
  }
  std::memcpy(out.data(), src, n * sizeof(T));
  return ISDF_OK;
}

// Copy n elements from device memory to a host or device destination.
template <class T>
isdf_status from_device(Plan* p, T* dst, const T* dsrc, size_t n, bool sync) {
  if (n == 0) return ISDF_OK;
  const bool dev = is_device_ptr(dst);
  isdf_status st = cuda_check(
      p, cudaMemcpyAsync(dst, dsrc, n * sizeof(T), dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->stream),
      "copy out");
  if (st) return st;
  if (!dev || sync) return cuda_check(p, cudaStreamSynchronize(p->stream), "copy out");
  return ISDF_OK;
}

isdf_status validate_system(const isdf_system* sys, std::string& why) {
  auto bad = [&](const std::string& m) {
    why = m;
    return ISDF_ERR_ARG;
  };
  if (!sys) return bad("system is NULL");
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double v = sys->lattice[3 * i + j];
      if (i != j && v != 0.0) return bad("lattice must be diagonal (orthorhombic cell)");
      if (i == j && !(v > 0.0 && std::isfinite(v))) return bad("lattice edge lengths must be positive");
    }
  if (sys->natom < 1 || !sys->xyz) return bad("need natom >= 1 and xyz");
  for (int i = 0; i < 3 * sys->natom; ++i)
    if (!std::isfinite(sys->xyz[i])) return bad("atom coordinates must be finite");
  if (sys->nshell < 1 || !sys->shell_atom || !sys->shell_l || !sys->shell_exp) return bad("need nshell >= 1 and shells");
  for (int i = 0; i < sys->nshell; ++i) {
    if (sys->shell_atom[i] < 0 || sys->shell_atom[i] >= sys->natom) return bad("shell_atom out of range");
    if (sys->shell_l[i] != 0 && sys->shell_l[i] != 1) return bad("only s and p shells (l = 0, 1) are supported");
    if (!(sys->shell_exp[i] > 0.0 && std::isfinite(sys->shell_exp[i]))) return bad("shell exponents must be > 0");
  }
  if (sys->nlevel < 1 || sys->nlevel > ISDF_MAX_LEVELS || !sys->grid) return bad("need 1 <= nlevel <= 4 and grid");
  for (int l = 0; l < sys->nlevel; ++l)
    for (int a = 0; a < 3; ++a) {
      const int n = sys->grid[3 * l + a];
      if (n < 2 || (n % 2) != 0) return bad("grid counts must be even and >= 2");
      if (n > (1 << 20)) return bad("grid count too large");
      if (l > 0 && !(n < sys->grid[3 * (l - 1) + a])) return bad("grid counts must decrease from level to level");
    }
  if (sys->nlevel > 1) {
    if (!sys->level_min_exp) return bad("level_min_exp is NULL");
    for (int l = 0; l + 1 < sys->nlevel; ++l) {
      const double e = sys->level_min_exp[l];
      if (!(e > 0.0 && std::isfinite(e))) return bad("level edges must be positive");
      if (l > 0 && !(e < sys->level_min_exp[l - 1])) return bad("level edges must decrease");
    }
  }
  if (!(sys->image_tol > 0.0 && sys->image_tol < 1.0)) return bad("image_tol must be in (0, 1)");
  return ISDF_OK;
}

isdf_status validate_options(const isdf_options* o, std::string& why) {
  auto bad = [&](const std::string& m) {
    why = m;
    return ISDF_ERR_ARG;
  };
  if (o->precision != 0 && o->precision != 1) return bad("precision must be 0 or 1");
  if (!(o->tie_rel >= 0.0) || !(o->tie_abs >= 0.0) || !(o->reg_rel >= 0.0)) return bad("tolerances must be >= 0");
  if (o->col_batch < 0 || o->timeout_ms < 0) return bad("col_batch and timeout_ms must be >= 0");
  if (o->prefilter != 0 && o->prefilter != 1) return bad("prefilter must be 0 or 1");
  if (o->profile != 0 && o->profile != 1) return bad("profile must be 0 or 1");
  if (o->coarse_sinc != 0 && o->coarse_sinc != 1) return bad("coarse_sinc must be 0 or 1");
  if (o->select_block < 0 || o->select_block > 256) return bad("select_block must be in [0, 256]");
  if (o->local_grids != 0 && o->local_grids != 1) return bad("local_grids must be 0 or 1");
  if (o->local_grids) {
    if (!(o->local_eps_r > 0.0 && o->local_eps_r < 1.0)) return bad("local_eps_r must be in (0, 1)");
    if (!(o->local_tol >= 0.0)) return bad("local_tol must be >= 0");
    if (o->local_cap < 1) return bad("local_cap must be >= 1");
  }
  return ISDF_OK;
}

}  // namespace
}  // namespace isdf

using namespace isdf;

extern "C" {

void isdf_options_default(isdf_options* o) {
  if (!o) return;
  o->precision = 0;
  o->tie_rel = 1e-9;
  o->tie_abs = 1e-13;
  o->reg_rel = 0.0;
  o->col_batch = 0;
  o->coarse_sinc = 0;
  o->timeout_ms = 0;
  o->prefilter = 0;
  o->profile = 0;
  o->select_block = 0;
  o->local_grids = 0;
  o->local_eps_r = 1e-5;
  o->local_tol = 1e-6;
  o->local_cap = 64;
}

namespace {

// Plan creation; with defer_basis the basis buffers are allocated but not
// evaluated (isdf_plan_batch evaluates every plan's basis in one launch).
isdf_status plan_create(const isdf_system* sys, const isdf_options* opt, void* stream, bool defer_basis,
                        isdf_plan_t* out) {
  if (!out) {
    g_plan_error = "out is NULL";
    return ISDF_ERR_ARG;
  }
  *out = nullptr;
  std::string why;
  if (validate_system(sys, why)) {
    g_plan_error = why;
    return ISDF_ERR_ARG;
  }
  isdf_options o;
  isdf_options_default(&o);
  if (opt) o = *opt;
  if (validate_options(&o, why)) {
    g_plan_error = why;
    return ISDF_ERR_ARG;
  }
  if (o.coarse_sinc && sys->nlevel < 2) {
    g_plan_error = "options.coarse_sinc needs at least two grid levels";
    return ISDF_ERR_ARG;
  }
  if (o.local_grids && sys->nlevel < 2) {
    g_plan_error = "options.local_grids needs at least two grid levels";
    return ISDF_ERR_ARG;
  }
  if (o.local_grids && o.coarse_sinc && sys->nlevel < 3) {
    g_plan_error = "options.local_grids with options.coarse_sinc needs at least three grid levels";
    return ISDF_ERR_ARG;
  }
  isdf_plan_s* h = new (std::nothrow) isdf_plan_s();
  if (!h) {
    g_plan_error = "host allocation failed";
    return ISDF_ERR_OOM;
  }
  Plan* p = &h->p;
  p->stream = static_cast<cudaStream_t>(stream);
  p->opt = o;
  if (const char* f = std::getenv("ISDF_FAULT")) p->fault = f;
  for (int a = 0; a < 3; ++a) p->edge[a] = sys->lattice[4 * a];
  p->omega = p->edge[0] * p->edge[1] * p->edge[2];
  p->image_tol = sys->image_tol;
  p->natom = sys->natom;
  p->xyz.assign(sys->xyz, sys->xyz + 3 * sys->natom);
  // functions and their levels (Section III: split by exponent)
  for (int i = 0; i < sys->nshell; ++i) {
    const double e = sys->shell_exp[i];
    int lev = 0;
    for (int l = 0; l + 1 < sys->nlevel; ++l)
      if (e < sys->level_min_exp[l]) ++lev;
    const int ncomp = sys->shell_l[i] == 0 ? 1 : 3;
    for (int c = 0; c < ncomp; ++c) {
      p->f_atom.push_back(sys->shell_atom[i]);
      p->f_alpha.push_back(e);
      double nrm = std::pow(2.0 * e / M_PI, 0.75);
      if (sys->shell_l[i] == 1) nrm *= 2.0 * std::sqrt(e);
      p->f_norm.push_back(nrm);
      for (int a = 0; a < 3; ++a) p->f_l[a].push_back(sys->shell_l[i] == 1 && a == c ? 1 : 0);
      p->f_level.push_back(lev);
    }
  }
  p->nfun = int(p->f_atom.size());
  p->nlev = sys->nlevel;
  p->off[0] = 0;
  for (int l = 0; l < p->nlev; ++l) {
    Level& lv = p->lev[l];
    for (int a = 0; a < 3; ++a) lv.n[a] = sys->grid[3 * l + a];
    lv.ng = int64_t(lv.n[0]) * lv.n[1] * lv.n[2];
    lv.w = p->omega / double(lv.ng);
    for (int mu = 0; mu < p->nfun; ++mu) {
      if (p->f_level[mu] == l) lv.L.push_back(mu);
      if (p->f_level[mu] > l) lv.N.push_back(mu);
    }
    lv.nL = int(lv.L.size());
    lv.nN = int(lv.N.size());
    lv.nG = lv.nL + lv.nN;
    p->off[l + 1] = p->off[l] + lv.ng;
  }
  p->ntot = p->off[p->nlev];
  // device checks
  int dev = 0;
  cudaDeviceProp prop;
  isdf_status st = cuda_check(p, cudaGetDevice(&dev), "cudaGetDevice");
  if (!st) st = cuda_check(p, cudaGetDeviceProperties(&prop, dev), "cudaGetDeviceProperties");
  if (!st && !(prop.major == 10 && prop.minor == 3))
    st = fail(p, ISDF_ERR_CUDA,
              "this library is built for sm_103a; device compute capability is " + std::to_string(prop.major) + "." +
                  std::to_string(prop.minor));
  if (!st) st = dalloc_t(p, &p->d_err, 1, "error word");
  if (!st) st = dalloc_t(p, &p->d_ozerr, 1, "error word");
  if (!st) st = cuda_check(p, cudaMemsetAsync(p->d_ozerr, 0, sizeof(int), p->stream), "memset");
  if (!st && o.local_grids) st = local_setup(p, sys->level_min_exp[0]);
  if (!st) st = defer_basis ? basis_alloc(p) : basis_build(p);
  if (!st) st = cuda_check(p, cudaStreamSynchronize(p->stream), "plan");
  if (st) {
    g_plan_error = p->err;
    free_plan(p);
    delete h;
    return st;
  }
  *out = h;
  return ISDF_OK;
}

}  // namespace

isdf_status isdf_plan(const isdf_system* sys, const isdf_options* opt, void* stream, isdf_plan_t* out) {
  return plan_create(sys, opt, stream, false, out);
}

isdf_status isdf_plan_batch(const isdf_system* systems, int ncells, const isdf_options* opt, void* const* streams,
                            isdf_plan_t* out) {
  if (!systems || !out || ncells < 1) {
    g_plan_error = "invalid arguments to isdf_plan_batch";
    return ISDF_ERR_ARG;
  }
  for (int i = 0; i < ncells; ++i) out[i] = nullptr;
  // a batch is a new, large working set: give the memory the stream-ordered
  // pool kept from earlier work back first, so the cells' buffers are not
  // fragmented around it
  {
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      cudaDeviceSynchronize();
      cudaMemPoolTrimTo(pool, 0);
    }
    cudaGetLastError();
  }
  std::vector<Plan*> plans;
  auto undo = [&](isdf_status st) {
    const std::string why = g_plan_error;
    for (int i = 0; i < ncells; ++i) {
      isdf_destroy(out[i]);
      out[i] = nullptr;
    }
    g_plan_error = why;
    return st;
  };
  for (int i = 0; i < ncells; ++i) {
    isdf_status st = plan_create(&systems[i], opt, streams ? streams[i] : nullptr, true, &out[i]);
    if (st) {
      g_plan_error = "cell " + std::to_string(i) + ": " + g_plan_error;
      return undo(st);
    }
    plans.push_back(&out[i]->p);
  }
  // every plan's buffers exist (each plan synchronised its stream); one
  // k_tab1d and one k_phi launch evaluate the basis of all cells and levels
  isdf_status st = basis_eval(plans.data(), ncells, plans[0]->stream);
  if (st) {
    g_plan_error = plans[0]->err;
    return undo(st);
  }
  return ISDF_OK;
}

isdf_status isdf_select_points(isdf_plan_t h, int nip, double tol, const int64_t* cand, int64_t ncand,
                               int64_t* piv_out, double* dval_out, int* nip_out) {
  if (!h) return ISDF_ERR_ARG;
  Plan* p = &h->p;
  if (p->released) return fail(p, ISDF_ERR_STATE, "the plan's basis values were released (isdf_release_fit)");
  if (nip < 1 || !piv_out || !nip_out || !(tol >= 0.0) || (cand && ncand < 1) || (!cand && ncand != 0))
    return fail(p, ISDF_ERR_ARG, "invalid arguments to isdf_select_points");
  if (nip > (p->opt.coarse_sinc ? p->off[p->nlev - 1] : p->ntot) - p->off[p->sel_lo])
    return fail(p, ISDF_ERR_ARG, "nip exceeds the number of grid points that take part in the selection");
  std::vector<int64_t> cv;
  if (cand) {
    isdf_status st = to_host(p, cand, size_t(ncand), cv);
    if (st) return st;
    for (int64_t c : cv) {
      const int64_t l = c >> kPivShift, g = c & kPivMask;
      if (c < 0 || l >= p->nlev || g >= p->lev[l].ng) return fail(p, ISDF_ERR_ARG, "candidate code out of range");
      if (p->opt.coarse_sinc && l == p->nlev - 1)
        return fail(p, ISDF_ERR_ARG, "with options.coarse_sinc the coarsest level has no candidates");
      if (l < p->sel_lo) return fail(p, ISDF_ERR_ARG, "with options.local_grids level 0 has no candidates");
    }
  }
  // local grids: every atom's own selection first
  std::vector<int64_t> lpiv;
  std::vector<double> ldv;
  if (p->opt.local_grids) {
    isdf_status st = local_select(p, lpiv, ldv);
    if (st) return st;
  }
  int found = 0;
  isdf_status st = select_run(p, nip, tol, cand ? &cv : nullptr, &found);
  if (st && st != ISDF_ERR_TIMEOUT) return st;
  isdf_status st2 = ISDF_OK;
  if (p->opt.local_grids) {
    std::vector<int64_t> pv(found);
    std::vector<double> dv(found);
    if (found) {
      cudaMemcpyAsync(pv.data(), p->d_piv, sizeof(int64_t) * found, cudaMemcpyDeviceToHost, p->stream);
      cudaMemcpyAsync(dv.data(), p->d_dval, sizeof(double) * found, cudaMemcpyDeviceToHost, p->stream);
      st2 = cuda_check(p, cudaStreamSynchronize(p->stream), "pivots");
    }
    lpiv.insert(lpiv.end(), pv.begin(), pv.end());
    ldv.insert(ldv.end(), dv.begin(), dv.end());
    found = int(lpiv.size());
    auto put = [&](void* dst, const void* src, size_t bytes) -> isdf_status {
      if (!bytes) return ISDF_OK;
      if (!is_device_ptr(dst)) {
        std::memcpy(dst, src, bytes);
        return ISDF_OK;
      }
      return cuda_check(p, cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice), "copy out");
    };
    if (!st2) st2 = put(piv_out, lpiv.data(), sizeof(int64_t) * lpiv.size());
    if (!st2 && dval_out) st2 = put(dval_out, ldv.data(), sizeof(double) * ldv.size());
  } else {
    st2 = from_device(p, piv_out, p->d_piv, size_t(found), true);
    if (!st2 && dval_out) st2 = from_device(p, dval_out, p->d_dval, size_t(found), true);
  }
  if (st2) return st2;
  *nip_out = found;
  p->state = 1;
  return st;
}

isdf_status isdf_fit(isdf_plan_t h, const int64_t* piv, int nip) {
  if (!h) return ISDF_ERR_ARG;
  Plan* p = &h->p;
  if (p->released) return fail(p, ISDF_ERR_STATE, "the plan's basis values were released (isdf_release_fit)");
  if (!piv || nip < 1) return fail(p, ISDF_ERR_ARG, "invalid arguments to isdf_fit");
  std::vector<int64_t> pv;
  isdf_status st = to_host(p, piv, size_t(nip), pv);
  if (st) return st;
  std::vector<std::vector<int64_t>> per(p->nlev);
  std::vector<std::vector<int64_t>> per_atom(p->sub.size());
  std::set<int64_t> seen;
  for (int64_t c : pv) {
    const int64_t l = c >> kPivShift, g = c & kPivMask;
    if (p->opt.local_grids && c >= 0 && l == 0) {
      // local pivot: (atom << 24) | box index, inside the atom's sphere
      const int64_t A = g >> kLocalAtomShift, b = g & ((int64_t(1) << kLocalAtomShift) - 1);
      if (A >= int64_t(p->sub.size()) || b >= p->sub[A]->lev[0].ng || !local_inside(p->sub[A], b))
        return fail(p, ISDF_ERR_ARG, "local pivot code out of range or outside its atom's sphere");
      if (!seen.insert(c).second) return fail(p, ISDF_ERR_ARG, "duplicate pivot");
      per_atom[A].push_back(b);
      per[0].push_back(g);
      continue;
    }
    if (c < 0 || l >= p->nlev || g >= p->lev[l].ng) return fail(p, ISDF_ERR_ARG, "pivot code out of range");
    if (p->opt.coarse_sinc && l == p->nlev - 1)
      return fail(p, ISDF_ERR_ARG, "with options.coarse_sinc every coarsest-level point is implicit: pass none");
    if (!seen.insert(c).second) return fail(p, ISDF_ERR_ARG, "duplicate pivot");
    per[l].push_back(g);
  }
  for (int l = 0; l < p->nlev; ++l)
    if (int64_t(per[l].size()) > p->lev[l].ng && !(p->opt.local_grids && l == 0))
      return fail(p, ISDF_ERR_ARG, "too many pivots on a level");
  if (p->opt.local_grids) {
    // level 0 in atom order, each atom's pivots in the order given
    per[0].clear();
    for (size_t A = 0; A < per_atom.size(); ++A)
      for (int64_t b : per_atom[A]) per[0].push_back((int64_t(A) << kLocalAtomShift) | b);
  }
  // level-ordered layout
  p->nip = nip;
  p->piv_lo.clear();
  p->poff[0] = 0;
  for (int l = 0; l < p->nlev; ++l) {
    Level& lv = p->lev[l];
    lv.pg = per[l];
    lv.k = int(per[l].size());
    p->poff[l + 1] = p->poff[l] + lv.k;
    for (int64_t g : per[l]) p->piv_lo.push_back((int64_t(l) << kPivShift) | g);
    dfree(lv.d_pg);
    lv.d_pg = nullptr;
    if (lv.k && l >= p->sel_lo) {
      if ((st = dalloc_t(p, &lv.d_pg, size_t(lv.k), "pivot indices"))) return st;
      if ((st = cuda_check(p, cudaMemcpyAsync(lv.d_pg, lv.pg.data(), sizeof(int64_t) * lv.k, cudaMemcpyHostToDevice,
                                              p->stream),
                           "copy pivots")))
        return st;
    }
  }
  dfree(p->XL);
  dfree(p->XN);
  p->XL = p->XN = nullptr;
  if ((st = dalloc_t(p, &p->XL, size_t(p->nfun) * nip, "X^L")) ||
      (st = dalloc_t(p, &p->XN, size_t(p->nfun) * nip, "X^N")))
    return st;
  p->state = 0;  // an unfinished fit leaves the plan needing a new fit
  if (p->opt.local_grids && (st = local_fit(p, per_atom))) return st;
  if ((st = fit_run(p))) return st;
  if (p->opt.local_grids && (st = local_assemble(p))) return st;
  p->state = 2;
  return ISDF_OK;
}

isdf_status isdf_coulomb(isdf_plan_t h, double* V_out) {
  if (!h) return ISDF_ERR_ARG;
  Plan* p = &h->p;
  if (p->state < 2 || p->released) return fail(p, ISDF_ERR_STATE, "isdf_coulomb needs isdf_fit first");
  p->state = 2;
  isdf_status st = coulomb_run(p);
  if (st) return st;
  if (V_out && (st = from_device(p, V_out, p->V, size_t(p->nip) * p->nip, false))) return st;
  p->state = 3;
  return ISDF_OK;
}

isdf_status isdf_exchange(isdf_plan_t h, const double* C, int n, double* K_out, double* Ex_out) {
  if (!h) return ISDF_ERR_ARG;
  Plan* p = &h->p;
  if (p->state < 3) return fail(p, ISDF_ERR_STATE, "isdf_exchange needs isdf_coulomb first");
  if (!C || n < 1) return fail(p, ISDF_ERR_ARG, "invalid arguments to isdf_exchange");
  const size_t nc = size_t(p->nfun) * n, nk = size_t(p->nfun) * p->nfun;
  const double* dC = C;
  double* stageC = nullptr;
  double* dK = nullptr;
  bool own_k = false;
  isdf_status st = ISDF_OK;
  if (!is_device_ptr(C)) {
    if ((st = dalloc_t(p, &stageC, nc, "C staging"))) return st;
    st = cuda_check(p, cudaMemcpyAsync(stageC, C, nc * sizeof(double), cudaMemcpyHostToDevice, p->stream), "copy C");
    dC = stageC;
  }
  if (!st) {
    if (K_out && is_device_ptr(K_out)) {
      dK = K_out;
    } else {
      own_k = true;
      st = dalloc_t(p, &dK, nk, "K");
    }
  }
  double ex = 0.0;
  if (!st) st = exchange_run(p, dC, n, dK, nullptr, &ex);
  if (!st && K_out && own_k) st = from_device(p, K_out, dK, nk, true);
  if (!st && Ex_out) *Ex_out = ex;
  dfree(stageC);
  if (own_k) dfree(dK);
  return st;
}

isdf_status isdf_exchange_occ(isdf_plan_t h, const double* C, int n, double* KC_out, double* Ex_out) {
  if (!h) return ISDF_ERR_ARG;
  Plan* p = &h->p;
  if (p->state < 3) return fail(p, ISDF_ERR_STATE, "isdf_exchange_occ needs isdf_coulomb first");
  if (!C || n < 1) return fail(p, ISDF_ERR_ARG, "invalid arguments to isdf_exchange_occ");
  const size_t nc = size_t(p->nfun) * n;
  const double* dC = C;
  double* stageC = nullptr;
  double* dKC = nullptr;
  bool own = false;
  isdf_status st = ISDF_OK;
  if (!is_device_ptr(C)) {
    if ((st = dalloc_t(p, &stageC, nc, "C staging"))) return st;
    st = cuda_check(p, cudaMemcpyAsync(stageC, C, nc * sizeof(double), cudaMemcpyHostToDevice, p->stream), "copy C");
    dC = stageC;
  }
  if (!st) {
    if (KC_out && is_device_ptr(KC_out)) {
      dKC = KC_out;
    } else {
      own = true;
      st = dalloc_t(p, &dKC, nc, "K C");
    }
  }
  double ex = 0.0;
  if (!st) st = exchange_run(p, dC, n, nullptr, dKC, &ex);
  if (!st && KC_out && own) st = from_device(p, KC_out, dKC, nc, true);
  if (!st && Ex_out) *Ex_out = ex;
  dfree(stageC);
  if (own) dfree(dKC);
  return st;
}

// ---------------------------------------------------------------- captured exchange builds

struct isdf_exchange_graph_s {
  std::vector<Plan*> plans;
  std::vector<int> n;
  int occ = 0;
  std::vector<double*> dC, dOut;
  double* dEx = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> ev;
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;  // kernels per replay
};

void isdf_exchange_graph_destroy(isdf_exchange_graph_t g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  if (g->exec) {
    cudaGraphExecDestroy(g->exec);
    // the graph's allocations return to the device's graph memory pool, which
    // keeps their physical memory until trimmed: give it back to the device
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGraphMemTrim(dev);
    cudaGetLastError();
  }
  for (double* q : g->dC) cudaFree(q);
  for (double* q : g->dOut) cudaFree(q);
  cudaFree(g->dEx);
  for (cudaStream_t b : g->branch) cudaStreamDestroy(b);
  for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
  delete g;
}

isdf_status isdf_exchange_graph(isdf_plan_t* plans, int nplans, const int* n_occ, int occ, void* stream,
                                isdf_exchange_graph_t* out) {
  if (!out || !plans || !n_occ || nplans < 1 || (occ != 0 && occ != 1)) {
    g_plan_error = "invalid arguments to isdf_exchange_graph";
    return ISDF_ERR_ARG;
  }
  *out = nullptr;
  for (int i = 0; i < nplans; ++i)
    if (plans[i] && plans[i]->p.opt.coarse_sinc) {
      g_plan_error = "isdf_exchange_graph: plan " + std::to_string(i) + " uses options.coarse_sinc";
      return ISDF_ERR_ARG;
    } else if (!plans[i] || plans[i]->p.state < 3 || n_occ[i] < 1) {
      g_plan_error = "isdf_exchange_graph: plan " + std::to_string(i) + " needs isdf_coulomb first and n >= 1";
      return plans[i] ? ISDF_ERR_STATE : ISDF_ERR_ARG;
    }
  auto* g = new (std::nothrow) isdf_exchange_graph_s();
  if (!g) return ISDF_ERR_OOM;
  g->occ = occ;
  g->stream = static_cast<cudaStream_t>(stream);
  auto undo = [&](isdf_status st, const std::string& why) {
    for (Plan* p : g->plans) p->capturing = false, p->d_ex_slot = nullptr;
    isdf_exchange_graph_destroy(g);
    g_plan_error = why;
    return st;
  };
  cudaError_t e = cudaMalloc(&g->dEx, sizeof(double) * size_t(nplans));
  for (int i = 0; i < nplans && e == cudaSuccess; ++i) {
    Plan* p = &plans[i]->p;
    g->plans.push_back(p);
    g->n.push_back(n_occ[i]);
    double *c = nullptr, *o = nullptr;
    const size_t nc = size_t(p->nfun) * n_occ[i], no = occ ? nc : size_t(p->nfun) * p->nfun;
    e = cudaMalloc(&c, sizeof(double) * nc);
    if (e == cudaSuccess) e = cudaMalloc(&o, sizeof(double) * no);
    if (e == cudaSuccess) e = cudaMemset(c, 0, sizeof(double) * nc);
    g->dC.push_back(c);
    g->dOut.push_back(o);
    cudaStream_t b = nullptr;
    cudaEvent_t ev = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking);
    g->branch.push_back(b);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    g->ev.push_back(ev);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return undo(ISDF_ERR_OOM, std::string("isdf_exchange_graph: buffers: ") + cudaGetErrorString(e));
  }
  cudaEvent_t fork = nullptr;
  cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  g->ev.push_back(fork);
  // one exchange per plan outside the capture, on the plan's own stream:
  // uploads each plan's level order (a plan-owned buffer, freed with the
  // plan on its stream) and fills the autotuner's table for these shapes
  for (size_t i = 0; i < g->plans.size(); ++i) {
    Plan* p = g->plans[i];
    double ex = 0.0;
    const isdf_status st = exchange_run(p, g->dC[i], g->n[i], occ ? nullptr : g->dOut[i], occ ? g->dOut[i] : nullptr, &ex);
    if (st) return undo(st, "isdf_exchange_graph: plan " + std::to_string(i) + ": " + p->err);
  }
  // capture on a stream of the graph's own (the caller's stream may be the
  // legacy default stream, which cannot be captured): it forks into one
  // branch per plan (every plan's exchange build is an independent chain of
  // the graph) and joins again
  cudaStream_t cap = nullptr;
  if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) {
    cudaGetLastError();
    return undo(ISDF_ERR_CUDA, std::string("isdf_exchange_graph: stream: ") + cudaGetErrorString(e));
  }
  g->branch.push_back(cap);  // destroyed with the graph
  cudaGraph_t graph = nullptr;
  const long long l0 = g_launches.load();
  isdf_status st = ISDF_OK;
  std::string why;
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = cudaEventRecord(fork, cap);
  for (size_t i = 0; i < g->plans.size() && e == cudaSuccess && !st; ++i) {
    Plan* p = g->plans[i];
    e = cudaStreamWaitEvent(g->branch[i], fork, 0);
    if (e != cudaSuccess) break;
    const cudaStream_t keep = p->stream;
    const int prof = p->opt.profile;
    p->stream = g->branch[i];
    p->opt.profile = 0;
    p->capturing = true;
    p->d_ex_slot = g->dEx + i;
    double ex = 0.0;
    st = exchange_run(p, g->dC[i], g->n[i], occ ? nullptr : g->dOut[i], occ ? g->dOut[i] : nullptr, &ex);
    if (st) why = "plan " + std::to_string(i) + ": " + p->err;
    p->capturing = false;
    p->d_ex_slot = nullptr;
    p->stream = keep;
    p->opt.profile = prof;
    if (!st) e = cudaEventRecord(g->ev[i], g->branch[i]);
    if (!st && e == cudaSuccess) e = cudaStreamWaitEvent(cap, g->ev[i], 0);
  }
  const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
  if (e == cudaSuccess) e = e2;
  g->launches = g_launches.load() - l0;
  if (!st && e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (st || e != cudaSuccess) {
    cudaGetLastError();
    return undo(st ? st : ISDF_ERR_CUDA,
                st ? "isdf_exchange_graph: " + why : std::string("isdf_exchange_graph: capture: ") + cudaGetErrorString(e));
  }
  *out = g;
  return ISDF_OK;
}

isdf_status isdf_exchange_graph_run(isdf_exchange_graph_t g, const double* const* C, double* const* out,
                                    double* Ex_out) {
  if (!g || !C) {
    g_plan_error = "invalid arguments to isdf_exchange_graph_run";
    return ISDF_ERR_ARG;
  }
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < g->plans.size() && e == cudaSuccess; ++i) {
    if (!C[i]) {
      g_plan_error = "isdf_exchange_graph_run: C[" + std::to_string(i) + "] is NULL";
      return ISDF_ERR_ARG;
    }
    const size_t nc = size_t(g->plans[i]->nfun) * g->n[i];
    e = cudaMemcpyAsync(g->dC[i], C[i], sizeof(double) * nc, cudaMemcpyDefault, g->stream);
  }
  if (e == cudaSuccess) e = cudaGraphLaunch(g->exec, g->stream);
  count_launches(g->launches);
  for (size_t i = 0; i < g->plans.size() && e == cudaSuccess; ++i) {
    if (!out || !out[i]) continue;
    const Plan* p = g->plans[i];
    const size_t no = g->occ ? size_t(p->nfun) * g->n[i] : size_t(p->nfun) * p->nfun;
    e = cudaMemcpyAsync(out[i], g->dOut[i], sizeof(double) * no, cudaMemcpyDefault, g->stream);
  }
  std::vector<double> ex(g->plans.size());
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ex.data(), g->dEx, sizeof(double) * ex.size(), cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    g_plan_error = std::string("isdf_exchange_graph_run: ") + cudaGetErrorString(e);
    return ISDF_ERR_CUDA;
  }
  for (Plan* p : g->plans) {
    int h = 0;
    if (cudaMemcpy(&h, p->d_ozerr, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && h) {
      cudaMemset(p->d_ozerr, 0, sizeof(int));
      g_plan_error = "isdf_exchange_graph_run: a tensor-core pipeline wait expired (code " + std::to_string(h) + ")";
      return ISDF_ERR_TIMEOUT;
    }
  }
  if (Ex_out)
    for (size_t i = 0; i < ex.size(); ++i) Ex_out[i] = ex[i];
  return ISDF_OK;
}

// ---------------------------------------------------------------- checkpoint
//
// File: "ISDFCKP1", int32 nfun, nlev, nip, int32 grid[nlev][3], double
// edges[3], int64 pivot codes (level order) [nip], double X^L [nfun][nip],
// X^N [nfun][nip], V [nip][nip]; native byte order.

namespace {
constexpr char kCkpMagic[8] = {'I', 'S', 'D', 'F', 'C', 'K', 'P', '1'};
}

const char* isdf_autotune_table(void) {
  static thread_local std::string t;
  t = oz_tune_json();
  return t.c_str();
}

isdf_status isdf_release_fit(isdf_plan_t h) {
  if (!h) return ISDF_ERR_ARG;
  Plan* p = &h->p;
  if (p->state < 3) return fail(p, ISDF_ERR_STATE, "isdf_release_fit needs isdf_coulomb first");
  isdf_status st = cuda_check(p, cudaStreamSynchronize(p->stream), "release");
  if (st) return st;
  auto release = [&](Plan* q, bool keep_coarse_phi) {
    for (int l = 0; l < q->nlev; ++l) {
      Level& lv = q->lev[l];
      const bool keep = keep_coarse_phi && l == q->nlev - 1;  // the sinc grid's exchange reads them
      if (!keep) {
        for (int a = 0; a < 3; ++a) dfree(lv.tab[a]), lv.tab[a] = nullptr;
        dfree(lv.phi), lv.phi = nullptr;
      }
      dfree(lv.fac), dfree(lv.xiT), dfree(lv.resid), dfree(lv.zct), dfree(lv.rinv), dfree(lv.spec);
      lv.fac = lv.xiT = lv.zct = lv.rinv = nullptr;
      lv.resid = nullptr;
      lv.spec = nullptr;
    }
    dfree(q->d_diag), q->d_diag = nullptr;
  };
  for (Plan* q : p->sub) release(q, false);
  release(p, p->opt.coarse_sinc != 0);
  p->released = true;
  return ISDF_OK;
}

isdf_status isdf_save(isdf_plan_t h, const char* path) {
  if (!h) return ISDF_ERR_ARG;
  Plan* p = &h->p;
  if (p->state < 3) return fail(p, ISDF_ERR_STATE, "isdf_save needs isdf_coulomb first");
  if (!path) return fail(p, ISDF_ERR_ARG, "isdf_save: path is NULL");
  if (p->opt.coarse_sinc) return fail(p, ISDF_ERR_ARG, "isdf_save: options.coarse_sinc plans are not saved");
  if (p->opt.local_grids) return fail(p, ISDF_ERR_ARG, "isdf_save: options.local_grids plans are not saved");
  const size_t nx = size_t(p->nfun) * p->nip, nv = size_t(p->nip) * p->nip;
  std::vector<double> xl(nx), xn(nx), v(nv);
  isdf_status st;
  if ((st = from_device(p, xl.data(), p->XL, nx, false)) || (st = from_device(p, xn.data(), p->XN, nx, false)) ||
      (st = from_device(p, v.data(), p->V, nv, true)))
    return st;
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(p, ISDF_ERR_ARG, std::string("isdf_save: cannot open ") + path);
  const int32_t hdr[3] = {p->nfun, p->nlev, p->nip};
  int32_t grid[3 * ISDF_MAX_LEVELS];
  for (int l = 0; l < p->nlev; ++l)
    for (int a = 0; a < 3; ++a) grid[3 * l + a] = p->lev[l].n[a];
  bool ok = std::fwrite(kCkpMagic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(int32_t), 3, f) == 3 &&
            std::fwrite(grid, sizeof(int32_t), size_t(3 * p->nlev), f) == size_t(3 * p->nlev) &&
            std::fwrite(p->edge, sizeof(double), 3, f) == 3 &&
            std::fwrite(p->piv_lo.data(), sizeof(int64_t), p->piv_lo.size(), f) == p->piv_lo.size() &&
            std::fwrite(xl.data(), sizeof(double), nx, f) == nx && std::fwrite(xn.data(), sizeof(double), nx, f) == nx &&
            std::fwrite(v.data(), sizeof(double), nv, f) == nv;
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return fail(p, ISDF_ERR_ARG, std::string("isdf_save: write failed: ") + path);
  return ISDF_OK;
}

isdf_status isdf_load(isdf_plan_t h, const char* path) {
  if (!h) return ISDF_ERR_ARG;
  Plan* p = &h->p;
  if (!path) return fail(p, ISDF_ERR_ARG, "isdf_load: path is NULL");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(p, ISDF_ERR_ARG, std::string("isdf_load: cannot open ") + path);
  auto bad = [&](const char* why) {
    std::fclose(f);
    return fail(p, ISDF_ERR_ARG, std::string("isdf_load: ") + why + ": " + path);
  };
  char magic[8];
  int32_t hdr[3];
  if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, kCkpMagic, 8) != 0) return bad("not a checkpoint");
  if (std::fread(hdr, sizeof(int32_t), 3, f) != 3) return bad("truncated header");
  if (hdr[0] != p->nfun || hdr[1] != p->nlev || hdr[2] < 1) return bad("basis or levels differ from the plan's");
  const int nip = hdr[2];
  int32_t grid[3 * ISDF_MAX_LEVELS];
  double edge[3];
  if (std::fread(grid, sizeof(int32_t), size_t(3 * p->nlev), f) != size_t(3 * p->nlev) ||
      std::fread(edge, sizeof(double), 3, f) != 3)
    return bad("truncated header");
  for (int l = 0; l < p->nlev; ++l)
    for (int a = 0; a < 3; ++a)
      if (grid[3 * l + a] != p->lev[l].n[a]) return bad("grids differ from the plan's");
  for (int a = 0; a < 3; ++a)
    if (edge[a] != p->edge[a]) return bad("cell differs from the plan's");
  std::vector<int64_t> piv(nip);
  const size_t nx = size_t(p->nfun) * nip, nv = size_t(nip) * nip;
  std::vector<double> xl(nx), xn(nx), v(nv);
  if (std::fread(piv.data(), sizeof(int64_t), size_t(nip), f) != size_t(nip) ||
      std::fread(xl.data(), sizeof(double), nx, f) != nx || std::fread(xn.data(), sizeof(double), nx, f) != nx ||
      std::fread(v.data(), sizeof(double), nv, f) != nv)
    return bad("truncated data");
  char extra;
  if (std::fread(&extra, 1, 1, f) != 0) return bad("trailing data");
  std::fclose(f);
  // pivots: in range, level-ordered, no duplicates
  std::vector<std::vector<int64_t>> per(p->nlev);
  std::set<int64_t> seen;
  int64_t last_level = 0;
  for (int64_t c : piv) {
    const int64_t l = c >> kPivShift, g = c & kPivMask;
    if (c < 0 || l >= p->nlev || g >= p->lev[l].ng || l < last_level || !seen.insert(c).second)
      return fail(p, ISDF_ERR_ARG, std::string("isdf_load: invalid pivot codes: ") + path);
    last_level = l;
    per[l].push_back(g);
  }
  // the plan now holds the loaded factors; nothing of an earlier fit survives
  isdf_status st;
  p->state = 0;
  for (int l = 0; l < p->nlev; ++l) {
    Level& lv = p->lev[l];
    dfree(lv.xiT), dfree(lv.zct), dfree(lv.rinv), dfree(lv.spec), dfree(lv.resid), dfree(lv.d_pg);
    lv.xiT = nullptr, lv.zct = nullptr, lv.rinv = nullptr, lv.spec = nullptr, lv.resid = nullptr, lv.d_pg = nullptr;
    lv.pg = per[l];
    lv.k = int(per[l].size());
  }
  p->resid_ready = false;
  p->nip = nip;
  p->piv_lo = piv;
  p->poff[0] = 0;
  for (int l = 0; l < p->nlev; ++l) p->poff[l + 1] = p->poff[l] + p->lev[l].k;
  dfree(p->XL), dfree(p->XN), dfree(p->V);
  p->XL = p->XN = p->V = nullptr;
  if ((st = dalloc_t(p, &p->XL, nx, "X^L")) || (st = dalloc_t(p, &p->XN, nx, "X^N")) ||
      (st = dalloc_t(p, &p->V, nv, "V")))
    return st;
  if ((st = cuda_check(p, cudaMemcpyAsync(p->XL, xl.data(), nx * 8, cudaMemcpyHostToDevice, p->stream), "load X^L")) ||
      (st = cuda_check(p, cudaMemcpyAsync(p->XN, xn.data(), nx * 8, cudaMemcpyHostToDevice, p->stream), "load X^N")) ||
      (st = cuda_check(p, cudaMemcpyAsync(p->V, v.data(), nv * 8, cudaMemcpyHostToDevice, p->stream), "load V")) ||
      (st = cuda_check(p, cudaStreamSynchronize(p->stream), "load")))
    return st;
  p->state = 3;
  return ISDF_OK;
}

int64_t isdf_get_size(isdf_plan_t h, int what) {
  if (!h) return 0;
  Plan* p = &h->p;
  switch (what) {
    case ISDF_GET_NBASIS:
      return 1;
    case ISDF_GET_NIP_LEVEL:
      return p->nlev;
    case ISDF_GET_PIVOTS:
      return p->state >= 2 ? p->nip : 0;
    case ISDF_GET_XL:
    case ISDF_GET_XN:
      return p->state >= 2 ? int64_t(p->nfun) * p->nip : 0;
    case ISDF_GET_V:
      return p->state >= 3 ? int64_t(p->nip) * p->nip : 0;
    case ISDF_GET_NPOINTS:
      return 1;
    case ISDF_GET_FIT_RESIDUAL:
      return (p->state >= 2 && (!p->released || p->resid_ready)) ? 2 * p->nlev : 0;
    case ISDF_GET_SELECT_STATS:
      return p->state >= 1 ? 3 : 0;
    case ISDF_GET_V_COARSE:
      return (p->state >= 3 && p->VFU) ? int64_t(p->nip) * p->lev[p->nlev - 1].ng : 0;
    case ISDF_GET_LOCAL_BOX:
      return p->opt.local_grids ? 4 : 0;
    case ISDF_GET_LOCAL_NIP:
      return (p->opt.local_grids && p->state >= 2) ? int64_t(p->sub.size()) : 0;
    default:
      break;
  }
  if (what >= ISDF_GET_XI_LEVEL0 && what < ISDF_GET_XI_LEVEL0 + p->nlev) {
    const Level& lv = p->lev[what - ISDF_GET_XI_LEVEL0];
    return (p->state >= 2 && (lv.xiT || lv.zct)) ? int64_t(lv.k) * lv.ng : 0;
  }
  if (what >= ISDF_GET_PHI_LEVEL0 && what < ISDF_GET_PHI_LEVEL0 + p->nlev) {
    const Level& lv = p->lev[what - ISDF_GET_PHI_LEVEL0];
    return lv.phi ? int64_t(lv.nG) * lv.ng : 0;
  }
  return 0;
}

isdf_status isdf_get(isdf_plan_t h, int what, void* dst) {
  if (!h) return ISDF_ERR_ARG;
  Plan* p = &h->p;
  if (!dst) return fail(p, ISDF_ERR_ARG, "dst is NULL");
  const int64_t n = isdf_get_size(h, what);
  if (n == 0) return fail(p, ISDF_ERR_STATE, "requested data is not available yet");
  const bool dev = is_device_ptr(dst);
  auto put_host = [&](const void* src, size_t bytes) -> isdf_status {
    if (dev)
      return cuda_check(p, cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice), "isdf_get copy");
    std::memcpy(dst, src, bytes);
    return ISDF_OK;
  };
  switch (what) {
    case ISDF_GET_NBASIS: {
      const int32_t v = p->nfun;
      return put_host(&v, sizeof(v));
    }
    case ISDF_GET_NIP_LEVEL: {
      std::vector<int32_t> v(p->nlev);
      for (int l = 0; l < p->nlev; ++l) v[l] = p->lev[l].k;
      return put_host(v.data(), sizeof(int32_t) * v.size());
    }
    case ISDF_GET_PIVOTS:
      return put_host(p->piv_lo.data(), sizeof(int64_t) * p->piv_lo.size());
    case ISDF_GET_XL:
      return from_device(p, static_cast<double*>(dst), p->XL, size_t(n), true);
    case ISDF_GET_V_COARSE:
      return from_device(p, static_cast<double*>(dst), p->VFU, size_t(n), true);
    case ISDF_GET_XN:
      return from_device(p, static_cast<double*>(dst), p->XN, size_t(n), true);
    case ISDF_GET_V:
      return from_device(p, static_cast<double*>(dst), p->V, size_t(n), true);
    case ISDF_GET_NPOINTS: {
      const int64_t v = p->ntot;
      return put_host(&v, sizeof(v));
    }
    case ISDF_GET_FIT_RESIDUAL: {
      isdf_status st = fit_residual_run(p);  // a factored fit computes it on request
      if (st) return st;
      return put_host(p->fit_resid, sizeof(double) * 2 * p->nlev);
    }
    case ISDF_GET_SELECT_STATS: {
      const int64_t v[3] = {p->sel_blocks, p->sel_plain_steps, p->sel_compactions};
      return put_host(v, sizeof(v));
    }
    case ISDF_GET_LOCAL_BOX: {
      const Level& b = p->sub[0]->lev[0];
      const double v[4] = {p->r_max, double(b.n[0]), double(b.n[1]), double(b.n[2])};
      return put_host(v, sizeof(v));
    }
    case ISDF_GET_LOCAL_NIP: {
      std::vector<int32_t> v;
      for (Plan* q : p->sub) v.push_back(q->lev[0].k);
      return put_host(v.data(), sizeof(int32_t) * v.size());
    }
    default:
      break;
  }
  if (what >= ISDF_GET_XI_LEVEL0 && what < ISDF_GET_XI_LEVEL0 + p->nlev) {
    isdf_status st = fit_xi_run(p, what - ISDF_GET_XI_LEVEL0);  // a factored fit makes Xi on request
    if (st) return st;
    return from_device(p, static_cast<double*>(dst), p->lev[what - ISDF_GET_XI_LEVEL0].xiT, size_t(n), true);
  }
  if (what >= ISDF_GET_PHI_LEVEL0 && what < ISDF_GET_PHI_LEVEL0 + p->nlev)
    return from_device(p, static_cast<double*>(dst), p->lev[what - ISDF_GET_PHI_LEVEL0].phi, size_t(n), true);
  return fail(p, ISDF_ERR_ARG, "unknown isdf_get selector");
}

const char* isdf_profile_json(isdf_plan_t h) {
  if (!h) return "{}";
  Plan* p = &h->p;
  cudaStreamSynchronize(p->stream);
  prof_flush(p);
  std::string s = "{\"kernels\": {";
  bool first = true;
  for (const auto& kv : p->stats) {
    char buf[512];
    snprintf(buf, sizeof(buf),
             "%s\"%s\": {\"launches\": %lld, \"ms\": %.6f, \"work\": %.6e, \"unit\": \"%s\", \"flop\": %.6e}",
             first ? "" : ", ", kv.first.c_str(), (long long)kv.second.launches, kv.second.ms, kv.second.work,
             kv.second.unit.c_str(), kv.second.flop);
    s += buf;
    first = false;
  }
  s += "}}";
  p->prof_json = s;
  return p->prof_json.c_str();
}

int64_t isdf_kernel_launches(void) { return g_launches.load(); }

int isdf_mlp_num_params(void) { return mlp_num_params(); }

isdf_status isdf_features(isdf_plan_t h, float* feat_out) {
  if (!h) return ISDF_ERR_ARG;
  Plan* p = &h->p;
  if (!feat_out) return fail(p, ISDF_ERR_ARG, "feat_out is NULL");
  if (p->released) return fail(p, ISDF_ERR_STATE, "the plan's basis values were released (isdf_release_fit)");
  if (p->opt.local_grids) return fail(p, ISDF_ERR_ARG, "the learned proposal does not take options.local_grids");
  const size_t n = size_t(p->ntot) * 8;
  float* d = feat_out;
  float* stage = nullptr;
  const bool dev = is_device_ptr(feat_out);
  isdf_status st = ISDF_OK;
  if (!dev && (st = dalloc_t(p, &stage, n, "features"))) return st;
  if (!dev) d = stage;
  st = learn_features(p, d);
  if (!st && !dev) st = from_device(p, feat_out, stage, n, true);
  dfree(stage);
  return st;
}

isdf_status isdf_mlp_train_step(float* params, float* adam_m, float* adam_v, int step, float lr, const float* X,
                                const float* y, const float* w, int64_t n, float* loss_out, float* grad_out,
                                void* stream) {
  if (!params || !X || !y || !w || n < 1 || step < 1 || !(lr >= 0.0f) || (lr > 0.0f && (!adam_m || !adam_v))) {
    g_plan_error = "invalid arguments to isdf_mlp_train_step";
    return ISDF_ERR_ARG;
  }
  if (!is_device_ptr(params) || !is_device_ptr(X) || !is_device_ptr(y) || !is_device_ptr(w)) {
    g_plan_error = "isdf_mlp_train_step takes device pointers";
    return ISDF_ERR_ARG;
  }
  std::string why;
  const isdf_status st = mlp_grad_step(params, adam_m, adam_v, step, lr, X, y, w, n, loss_out, grad_out,
                                       static_cast<cudaStream_t>(stream), why);
  if (st) g_plan_error = why;
  return st;
}

isdf_status isdf_mlp_score(const float* params, const float* X, int64_t n, float* scores, void* stream) {
  if (!params || !X || !scores || n < 1) {
    g_plan_error = "invalid arguments to isdf_mlp_score";
    return ISDF_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mlp_score(params, X, n, scores, s);
  const cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    g_plan_error = std::string("isdf_mlp_score: ") + cudaGetErrorString(e);
    return ISDF_ERR_CUDA;
  }
  return ISDF_OK;
}

isdf_status isdf_propose(isdf_plan_t h, const float* params, const int64_t* quota, int64_t* cand_out) {
  if (!h) return ISDF_ERR_ARG;
  Plan* p = &h->p;
  if (!params || !quota || !cand_out) return fail(p, ISDF_ERR_ARG, "invalid arguments to isdf_propose");
  if (p->released) return fail(p, ISDF_ERR_STATE, "the plan's basis values were released (isdf_release_fit)");
  if (p->opt.local_grids) return fail(p, ISDF_ERR_ARG, "the learned proposal does not take options.local_grids");
  std::vector<int64_t> q(p->nlev);
  int64_t ncand = 0;
  for (int l = 0; l < p->nlev; ++l) {
    if (quota[l] < 0 || quota[l] > p->lev[l].ng) return fail(p, ISDF_ERR_ARG, "quota out of range");
    q[l] = quota[l];
    ncand += q[l];
  }
  if (ncand < 1) return fail(p, ISDF_ERR_ARG, "empty candidate quota");
  int64_t* d = cand_out;
  int64_t* stage = nullptr;
  const bool dev = is_device_ptr(cand_out);
  isdf_status st = ISDF_OK;
  if (!dev && (st = dalloc_t(p, &stage, size_t(ncand), "candidates"))) return st;
  if (!dev) d = stage;
  st = learn_propose(p, params, q.data(), d);
  if (!st && !dev) st = from_device(p, cand_out, stage, size_t(ncand), true);
  dfree(stage);
  return st;
}

isdf_status isdf_propose_residual(isdf_plan_t h, const int64_t* quota, int64_t* cand_out) {
  if (!h) return ISDF_ERR_ARG;
  Plan* p = &h->p;
  if (!quota || !cand_out) return fail(p, ISDF_ERR_ARG, "invalid arguments to isdf_propose_residual");
  if (p->opt.local_grids) return fail(p, ISDF_ERR_ARG, "the learned proposal does not take options.local_grids");
  if (p->state < 2 || p->released) return fail(p, ISDF_ERR_STATE, "isdf_propose_residual needs isdf_fit first");
  std::vector<int64_t> q(p->nlev);
  int64_t ncand = 0;
  for (int l = 0; l < p->nlev; ++l) {
    if (quota[l] < 0 || quota[l] > p->lev[l].ng) return fail(p, ISDF_ERR_ARG, "quota out of range");
    if (quota[l] > 0 && !p->lev[l].resid) return fail(p, ISDF_ERR_STATE, "no fit residual on this level");
    q[l] = quota[l];
    ncand += q[l];
  }
  if (ncand < 1) return fail(p, ISDF_ERR_ARG, "empty candidate quota");
  int64_t* d = cand_out;
  int64_t* stage = nullptr;
  const bool dev = is_device_ptr(cand_out);
  isdf_status st = ISDF_OK;
  if (!dev && (st = dalloc_t(p, &stage, size_t(ncand), "candidates"))) return st;
  if (!dev) d = stage;
  st = fit_residual_run(p);
  if (!st) st = learn_propose_residual(p, q.data(), d);
  if (!st && !dev) st = from_device(p, cand_out, stage, size_t(ncand), true);
  dfree(stage);
  return st;
}

isdf_status isdf_gemm_f64(const double* A, const double* B, double* C, int64_t M, int64_t N, int64_t K, int64_t lda,
                          int64_t ldb, int64_t ldc, double alpha, int slices, int splits, void* stream) {
  if (!A || !B || !C || M < 1 || N < 1 || K < 1 || lda < K || ldb < K || ldc < N ||
      (slices < 5 || slices > 8) || splits < 1 || splits > 1024) {
    g_plan_error = "invalid arguments to isdf_gemm_f64";
    return ISDF_ERR_ARG;
  }
  if (!is_device_ptr(A) || !is_device_ptr(B) || !is_device_ptr(C)) {
    g_plan_error = "isdf_gemm_f64 takes device pointers";
    return ISDF_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  OzOperand a, b;
  double* work = nullptr;
  int* err = nullptr;
  isdf_status st = oz_alloc(nullptr, a, M, K, 128, slices, "A slices");
  if (!st) st = oz_alloc(nullptr, b, N, K, oz_bn(slices), slices, "B slices");
  if (!st && splits > 1) st = dalloc_t(nullptr, &work, size_t(splits) * M * N, "split-K partials");
  if (!st) st = dalloc_t(nullptr, &err, 1, "error word");
  int herr = 0;
  if (!st) {
    cudaMemsetAsync(err, 0, sizeof(int), s);
    oz_slice(A, lda, 1, nullptr, 1.0, a, s);
    oz_slice(B, ldb, 1, nullptr, 1.0, b, s);
    oz_gemm(a, b, C, ldc, 0, alpha, 0, 0, splits, work, err, s);
    cudaError_t e = cudaGetLastError();  // a launch that could not start
    if (e == cudaSuccess) {
      cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
      e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) {
      g_plan_error = std::string("isdf_gemm_f64: ") + cudaGetErrorString(e);
      st = ISDF_ERR_CUDA;
    } else if (herr) {
      g_plan_error = "isdf_gemm_f64: tensor-core pipeline wait expired (code " + std::to_string(herr) + ")";
      st = ISDF_ERR_TIMEOUT;
    }
  } else {
    g_plan_error = "isdf_gemm_f64: allocation failed";
  }
  oz_free(a);
  oz_free(b);
  dfree(work);
  dfree(err);
  return st;
}

isdf_status isdf_gemm_f64_noalloc(const double* A, const double* B, double* C, int64_t M, int64_t N, int64_t K,
                                  int64_t lda, int64_t ldb, int64_t ldc, double alpha, int slices, void* stream) {
  if (!A || !B || !C || M < 1 || N < 1 || K < 1 || lda < K || ldb < K || ldc < N || (slices < 5 || slices > 8)) {
    g_plan_error = "invalid arguments to isdf_gemm_f64_noalloc";
    return ISDF_ERR_ARG;
  }
  // a host or stale pointer would reach the kernels as an address: refuse it
  // here, before anything is launched
  if (!is_device_ptr(A) || !is_device_ptr(B) || !is_device_ptr(C)) {
    g_plan_error = "isdf_gemm_f64_noalloc takes device pointers";
    return ISDF_ERR_ARG;
  }
  std::string why;
  const isdf_status st = gemm_noalloc(A, B, C, M, N, K, lda, ldb, ldc, alpha, slices,
                                      static_cast<cudaStream_t>(stream), why);
  if (st) g_plan_error = why;
  return st;
}

int64_t isdf_gemm_f64_noalloc_capacity(void) { return int64_t(gemm_noalloc_capacity()); }

isdf_status isdf_grids_for_threshold(const isdf_system* sys, double eps_K, int* grid_out) {
  // Section III, Eq. 6: a Gaussian exp(-a r^2) has the Fourier transform
  // exp(-G^2 / 4a), which falls to eps_K at G_max = sqrt(-4 a ln eps_K); a
  // grid of n points over an edge L carries wave numbers up to pi n / L.
  if (!sys || !grid_out || !(eps_K > 0.0 && eps_K < 1.0) || sys->nlevel < 1 || sys->nlevel > ISDF_MAX_LEVELS ||
      sys->nshell < 1 || !sys->shell_exp || (sys->nlevel > 1 && !sys->level_min_exp)) {
    g_plan_error = "invalid arguments to isdf_grids_for_threshold (0 < eps_K < 1, 1 <= nlevel <= 4, shells)";
    return ISDF_ERR_ARG;
  }
  double L[3];
  for (int a = 0; a < 3; ++a) {
    L[a] = sys->lattice[4 * a];
    if (!(L[a] > 0.0) || !std::isfinite(L[a])) {
      g_plan_error = "isdf_grids_for_threshold: the lattice must be diagonal with positive edges";
      return ISDF_ERR_ARG;
    }
  }
  for (int l = 0; l + 1 < sys->nlevel; ++l)
    if (!(sys->level_min_exp[l] > 0.0) || (l > 0 && !(sys->level_min_exp[l] < sys->level_min_exp[l - 1]))) {
      g_plan_error = "isdf_grids_for_threshold: level edges must be positive and decreasing";
      return ISDF_ERR_ARG;
    }
  // admissible sizes: even 2^a 3^b, ascending
  std::vector<int> sizes;
  for (long long p2 = 2; p2 <= 4096; p2 *= 2)
    for (long long n = p2; n <= 4096; n *= 3) sizes.push_back(int(n));
  std::sort(sizes.begin(), sizes.end());
  // sharpest exponent of each level (its own functions, else the coarser ones)
  double own[ISDF_MAX_LEVELS] = {0, 0, 0, 0};
  for (int i = 0; i < sys->nshell; ++i) {
    const double e = sys->shell_exp[i];
    if (!(e > 0.0) || !std::isfinite(e)) {
      g_plan_error = "isdf_grids_for_threshold: shell exponents must be > 0";
      return ISDF_ERR_ARG;
    }
    int lev = 0;
    for (int l = 0; l + 1 < sys->nlevel; ++l) lev += (e < sys->level_min_exp[l]) ? 1 : 0;
    own[lev] = std::max(own[lev], e);
  }
  int out[ISDF_MAX_LEVELS][3];
  for (int l = 0; l < sys->nlevel; ++l) {
    double alpha = own[l];
    for (int m = l + 1; m < sys->nlevel && alpha == 0.0; ++m) alpha = std::max(alpha, own[m]);
    for (int a = 0; a < 3; ++a) {
      if (alpha == 0.0) {
        out[l][a] = 2;
        continue;
      }
      const double gmax = std::sqrt(-4.0 * alpha * std::log(eps_K));
      int n = 0;
      for (int c : sizes)
        if (M_PI * double(c) / L[a] >= gmax) {
          n = c;
          break;
        }
      if (!n) {
        g_plan_error = "isdf_grids_for_threshold: the threshold needs more than 4096 points per axis";
        return ISDF_ERR_ARG;
      }
      out[l][a] = n;
    }
  }
  // strictly decreasing from level to level: raise a finer level where needed
  for (int l = sys->nlevel - 2; l >= 0; --l)
    for (int a = 0; a < 3; ++a)
      if (out[l][a] <= out[l + 1][a]) out[l][a] = *std::upper_bound(sizes.begin(), sizes.end(), out[l + 1][a]);
  for (int l = 0; l < sys->nlevel; ++l)
    for (int a = 0; a < 3; ++a) grid_out[3 * l + a] = out[l][a];
  return ISDF_OK;
}

isdf_status isdf_rfft3(const double* f, int nx, int ny, int nz, int64_t batch, double* S, void* stream) {
  if (!f || !S || batch < 1 || !rfft3_df_supported(nx, ny, nz)) {
    g_plan_error = "invalid arguments to isdf_rfft3 (every axis must be 2^a 3^b <= 128)";
    return ISDF_ERR_ARG;
  }
  if (!is_device_ptr(f) || !is_device_ptr(S)) {
    g_plan_error = "isdf_rfft3 takes device pointers";
    return ISDF_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  isdf_status st = rfft3_df(nullptr, f, nx, ny, nz, batch, reinterpret_cast<double2*>(S), s);
  const cudaError_t e = cudaStreamSynchronize(s);
  if (!st && e != cudaSuccess) {
    g_plan_error = std::string("isdf_rfft3: ") + cudaGetErrorString(e);
    st = ISDF_ERR_CUDA;
  }
  return st;
}

const char* isdf_last_error(isdf_plan_t h) {
  if (!h) return g_plan_error.c_str();
  return h->p.err.c_str();
}

void isdf_destroy(isdf_plan_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->p.stream);
  prof_flush(&h->p);
  free_plan(&h->p);
  delete h;
}

}  // extern "C"
