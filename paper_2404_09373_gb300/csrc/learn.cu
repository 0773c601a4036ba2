// Learned point proposer: a small MLP scores every grid point from local
// features so that pivoted Cholesky (Section II.A) can run on a short
// candidate list.  Not part of the paper's method; the full greedy selection
// stays the reference and the fallback.
//
//   k_point_stats   per point aL = sum_{L} phi^2, aN = sum_{N} phi^2
//   k_features      8 FP32 features per point (level-major, grid order)
//   k_mlp_grad      fused forward + backward of 8-64-64-1 (ReLU, logistic,
//                   class-weighted BCE) over 64-sample chunks, gradients summed
//                   per block in shared memory, one atomicAdd per parameter
//   k_adam          Adam update with bias correction
//   k_mlp_score     inference with BF16 weights and activations, FP32 sums
//   top-K           exact K largest scores (bisection on an order-preserving
//                   key, ties broken by the smallest (level, g)), ordered output
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace isdf {
namespace {

constexpr int NI = 8, NH = 64;
constexpr int OFF_W1 = 0, OFF_B1 = NI * NH, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH, OFF_W3 = OFF_B2 + NH,
              OFF_B3 = OFF_W3 + NH, NPARAM = OFF_B3 + 1;
constexpr int CHUNK = 64;

__global__ void k_point_stats(const double* __restrict__ phi, int64_t ng, int nL, int nG, double* __restrict__ st) {
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < ng; g += int64_t(gridDim.x) * blockDim.x) {
    double aL = 0.0, aN = 0.0;
    for (int r = 0; r < nL; ++r) aL = fma(phi[int64_t(r) * ng + g], phi[int64_t(r) * ng + g], aL);
    for (int r = nL; r < nG; ++r) aN = fma(phi[int64_t(r) * ng + g], phi[int64_t(r) * ng + g], aN);
    st[2 * g] = aL;
    st[2 * g + 1] = aN;
  }
}

struct FeatLevel {
  const double* st;  // (aL, aN) per point
  int n[3];
  double h[3];
  double w;
  int level, nlev;
};

__global__ void k_features(FeatLevel F, const double* __restrict__ xyz, int natom, double Lx, double Ly, double Lz,
                           double d0max, float* __restrict__ feat) {
  const int64_t ng = int64_t(F.n[0]) * F.n[1] * F.n[2];
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < ng; g += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(g % F.n[0]), j = int((g / F.n[0]) % F.n[1]), k = int(g / (int64_t(F.n[0]) * F.n[1]));
    const double aL = F.st[2 * g], aN = F.st[2 * g + 1];
    const double d0 = F.w * aL * (aL + 2.0 * aN);
    auto rho = [&](int ii, int jj, int kk) {
      ii = (ii + F.n[0]) % F.n[0];
      jj = (jj + F.n[1]) % F.n[1];
      kk = (kk + F.n[2]) % F.n[2];
      const int64_t e = ii + int64_t(F.n[0]) * (jj + int64_t(F.n[1]) * kk);
      return F.st[2 * e] + F.st[2 * e + 1];
    };
    const double gx = (rho(i + 1, j, k) - rho(i - 1, j, k)) / (2.0 * F.h[0]);
    const double gy = (rho(i, j + 1, k) - rho(i, j - 1, k)) / (2.0 * F.h[1]);
    const double gz = (rho(i, j, k + 1) - rho(i, j, k - 1)) / (2.0 * F.h[2]);
    const double x = i * F.h[0], y = j * F.h[1], z = k * F.h[2];
    double m1 = 1e300, m2 = 1e300;
    for (int a = 0; a < natom; ++a) {
      double dx = x - xyz[3 * a], dy = y - xyz[3 * a + 1], dz = z - xyz[3 * a + 2];
      dx -= Lx * rint(dx / Lx);
      dy -= Ly * rint(dy / Ly);
      dz -= Lz * rint(dz / Lz);
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < m1) {
        m2 = m1;
        m1 = r2;
      } else if (r2 < m2) {
        m2 = r2;
      }
    }
    float* f = feat + g * NI;
    f[0] = float(log10(fmax(d0, 1e-300) / d0max) / 10.0);
    f[1] = float(log10(aL + 1e-30) / 10.0);
    f[2] = float(log10(aN + 1e-30) / 10.0);
    f[3] = float(log10(sqrt(gx * gx + gy * gy + gz * gz) + 1e-30) / 10.0);
    f[4] = float(sqrt(m1) / 4.0);
    f[5] = float(sqrt(m2) / 4.0);
    f[6] = float(aL / (aL + aN + 1e-300));
    f[7] = float(F.nlev > 1 ? double(F.level) / double(F.nlev - 1) : 0.0);
  }
}

__global__ void k_diag_max(const double* __restrict__ st, int64_t ng, double w, unsigned long long* out) {
  double m = 0.0;
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < ng; g += int64_t(gridDim.x) * blockDim.x) {
    const double aL = st[2 * g], aN = st[2 * g + 1];
    m = fmax(m, w * aL * (aL + 2.0 * aN));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// ---------------------------------------------------------------- training

__global__ __launch_bounds__(256) void k_mlp_grad(const float* __restrict__ params, const float* __restrict__ X,
                                                  const float* __restrict__ y, const float* __restrict__ wt, int64_t n,
                                                  float inv_wsum, float* __restrict__ grad, float* __restrict__ loss) {
  extern __shared__ float sm[];
  float* P = sm;                 // NPARAM
  float* G = P + NPARAM;         // NPARAM
  float* xc = G + NPARAM;        // CHUNK x NI
  float* h1 = xc + CHUNK * NI;   // CHUNK x NH
  float* h2 = h1 + CHUNK * NH;   // CHUNK x NH
  float* d2 = h2 + CHUNK * NH;   // CHUNK x NH
  float* d1 = d2 + CHUNK * NH;   // CHUNK x NH
  float* dz = d1 + CHUNK * NH;   // CHUNK
  __shared__ float lsum[8];
  const int tid = threadIdx.x;
  for (int e = tid; e < NPARAM; e += blockDim.x) {
    P[e] = params[e];
    G[e] = 0.0f;
  }
  float my_loss = 0.0f;
  __syncthreads();
  for (int64_t c0 = int64_t(blockIdx.x) * CHUNK; c0 < n; c0 += int64_t(gridDim.x) * CHUNK) {
    for (int e = tid; e < CHUNK * NI; e += blockDim.x) {
      const int64_t s = c0 + e / NI;
      xc[e] = s < n ? X[s * NI + e % NI] : 0.0f;
    }
    __syncthreads();
    for (int e = tid; e < CHUNK * NH; e += blockDim.x) {
      const int s = e / NH, jj = e % NH;
      float a = P[OFF_B1 + jj];
      for (int k = 0; k < NI; ++k) a = fmaf(xc[s * NI + k], P[OFF_W1 + k * NH + jj], a);
      h1[e] = fmaxf(a, 0.0f);
    }
    __syncthreads();
    for (int e = tid; e < CHUNK * NH; e += blockDim.x) {
      const int s = e / NH, jj = e % NH;
      float a = P[OFF_B2 + jj];
      for (int i = 0; i < NH; ++i) a = fmaf(h1[s * NH + i], P[OFF_W2 + i * NH + jj], a);
      h2[e] = fmaxf(a, 0.0f);
    }
    __syncthreads();
    if (tid < CHUNK) {
      const int64_t s = c0 + tid;
      float z = P[OFF_B3];
      for (int jj = 0; jj < NH; ++jj) z = fmaf(h2[tid * NH + jj], P[OFF_W3 + jj], z);
      float g = 0.0f;
      if (s < n) {
        const float ys = y[s], ws = wt[s];
        const float sp_pos = fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z)));  // softplus(z)
        const float sp_neg = sp_pos - z;                                  // softplus(-z)
        my_loss += ws * (ys * sp_neg + (1.0f - ys) * sp_pos) * inv_wsum;
        const float p = 1.0f / (1.0f + expf(-z));
        g = ws * (p - ys) * inv_wsum;
      }
      dz[tid] = g;
    }
    __syncthreads();
    for (int e = tid; e < CHUNK * NH; e += blockDim.x) {
      const int s = e / NH, jj = e % NH;
      d2[e] = h2[e] > 0.0f ? dz[s] * P[OFF_W3 + jj] : 0.0f;
    }
    __syncthreads();
    for (int e = tid; e < CHUNK * NH; e += blockDim.x) {
      const int s = e / NH, i = e % NH;
      float a = 0.0f;
      for (int jj = 0; jj < NH; ++jj) a = fmaf(d2[s * NH + jj], P[OFF_W2 + i * NH + jj], a);
      d1[e] = h1[e] > 0.0f ? a : 0.0f;
    }
    __syncthreads();
    // each parameter is owned by one thread: no shared-memory atomics
    for (int e = tid; e < NPARAM; e += blockDim.x) {
      float a = 0.0f;
      if (e < OFF_B1) {
        const int k = e / NH, i = e % NH;
        for (int s = 0; s < CHUNK; ++s) a = fmaf(xc[s * NI + k], d1[s * NH + i], a);
      } else if (e < OFF_W2) {
        const int i = e - OFF_B1;
        for (int s = 0; s < CHUNK; ++s) a += d1[s * NH + i];
      } else if (e < OFF_B2) {
        const int i = (e - OFF_W2) / NH, jj = (e - OFF_W2) % NH;
        for (int s = 0; s < CHUNK; ++s) a = fmaf(h1[s * NH + i], d2[s * NH + jj], a);
      } else if (e < OFF_W3) {
        const int jj = e - OFF_B2;
        for (int s = 0; s < CHUNK; ++s) a += d2[s * NH + jj];
      } else if (e < OFF_B3) {
        const int jj = e - OFF_W3;
        for (int s = 0; s < CHUNK; ++s) a = fmaf(h2[s * NH + jj], dz[s], a);
      } else {
        for (int s = 0; s < CHUNK; ++s) a += dz[s];
      }
      G[e] += a;
    }
    __syncthreads();
  }
  for (int e = tid; e < NPARAM; e += blockDim.x) atomicAdd(&grad[e], G[e]);
  for (int o = 16; o > 0; o >>= 1) my_loss += __shfl_xor_sync(0xffffffffu, my_loss, o);
  if ((tid & 31) == 0) lsum[tid >> 5] = my_loss;
  __syncthreads();
  if (tid == 0) {
    float t = 0.0f;
    for (int i = 0; i < int(blockDim.x / 32); ++i) t += lsum[i];
    atomicAdd(loss, t);
  }
}

__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v, const float* __restrict__ g,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float gi = g[e];
  const float mi = b1 * m[e] + (1.0f - b1) * gi;
  const float vi = b2 * v[e] + (1.0f - b2) * gi * gi;
  m[e] = mi;
  v[e] = vi;
  p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_sum_weights(const float* __restrict__ w, int64_t n, float* out) {
  float t = 0.0f;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    t += w[i];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, t);
}

// ---------------------------------------------------------------- inference

__global__ __launch_bounds__(256) void k_mlp_score(const float* __restrict__ params, const float* __restrict__ X,
                                                   int64_t n, float* __restrict__ out) {
  __shared__ __nv_bfloat16 Pb[NPARAM];
  for (int e = threadIdx.x; e < NPARAM; e += blockDim.x) Pb[e] = __float2bfloat16_rn(params[e]);
  __syncthreads();
  for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x) {
    float x[NI];
#pragma unroll
    for (int k = 0; k < NI; ++k) x[k] = __bfloat162float(__float2bfloat16_rn(X[s * NI + k]));
    float h1[NH];
#pragma unroll
    for (int jj = 0; jj < NH; ++jj) {
      float a = __bfloat162float(Pb[OFF_B1 + jj]);
#pragma unroll
      for (int k = 0; k < NI; ++k) a = fmaf(x[k], __bfloat162float(Pb[OFF_W1 + k * NH + jj]), a);
      h1[jj] = __bfloat162float(__float2bfloat16_rn(fmaxf(a, 0.0f)));
    }
    float z = __bfloat162float(Pb[OFF_B3]);
    for (int jj = 0; jj < NH; ++jj) {
      float a = __bfloat162float(Pb[OFF_B2 + jj]);
#pragma unroll
      for (int i = 0; i < NH; ++i) a = fmaf(h1[i], __bfloat162float(Pb[OFF_W2 + i * NH + jj]), a);
      const float h2 = __bfloat162float(__float2bfloat16_rn(fmaxf(a, 0.0f)));
      z = fmaf(h2, __bfloat162float(Pb[OFF_W3 + jj]), z);
    }
    out[s] = z;
  }
}

// ---------------------------------------------------------------- top-K

__device__ __forceinline__ uint32_t order_key(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__global__ void k_count_ge(const float* __restrict__ s, int64_t n, uint32_t t, unsigned long long* out) {
  unsigned long long c = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    c += order_key(s[i]) >= t;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, c);
}

constexpr int kTopBlock = 1024;
// per block: number above T and number equal to T
__global__ void k_top_counts(const float* __restrict__ s, int64_t n, uint32_t T, int* __restrict__ gt,
                             int* __restrict__ eq) {
  __shared__ int sg[32], se[32];
  const int64_t i = int64_t(blockIdx.x) * kTopBlock + threadIdx.x;
  const uint32_t key = i < n ? order_key(s[i]) : 0u;
  const unsigned bg = __ballot_sync(0xffffffffu, i < n && key > T);
  const unsigned be = __ballot_sync(0xffffffffu, i < n && key == T);
  if ((threadIdx.x & 31) == 0) {
    sg[threadIdx.x >> 5] = __popc(bg);
    se[threadIdx.x >> 5] = __popc(be);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0, b = 0;
    for (int w = 0; w < kTopBlock / 32; ++w) a += sg[w], b += se[w];
    gt[blockIdx.x] = a;
    eq[blockIdx.x] = b;
  }
}

// selected = key > T, or key == T among the first `need_eq` equals (index order)
__global__ void k_top_write(const float* __restrict__ s, int64_t n, uint32_t T, const int* __restrict__ off_sel,
                            const int* __restrict__ off_eq, int64_t need_eq, const int64_t* __restrict__ lev_off,
                            int nlev, int level0, int64_t* __restrict__ out) {
  __shared__ int ws[32], we[32];
  const int64_t i = int64_t(blockIdx.x) * kTopBlock + threadIdx.x;
  const uint32_t key = i < n ? order_key(s[i]) : 0u;
  const bool is_eq = i < n && key == T;
  const unsigned be = __ballot_sync(0xffffffffu, is_eq);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) we[wid] = __popc(be);
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0;
    for (int w = 0; w < kTopBlock / 32; ++w) {
      const int c = we[w];
      we[w] = a;
      a += c;
    }
  }
  __syncthreads();
  const int64_t eq_rank = off_eq[blockIdx.x] + we[wid] + __popc(be & ((1u << lane) - 1u));
  const bool sel = (i < n && key > T) || (is_eq && eq_rank < need_eq);
  const unsigned bs = __ballot_sync(0xffffffffu, sel);
  if (lane == 0) ws[wid] = __popc(bs);
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0;
    for (int w = 0; w < kTopBlock / 32; ++w) {
      const int c = ws[w];
      ws[w] = a;
      a += c;
    }
  }
  __syncthreads();
  if (sel) {
    int l = 0;
    while (l + 1 < nlev && i >= lev_off[l + 1]) ++l;
    out[off_sel[blockIdx.x] + ws[wid] + __popc(bs & ((1u << lane) - 1u))] =
        (int64_t(l + level0) << kPivShift) | (i - lev_off[l]);
  }
}

}  // namespace

int mlp_num_params() { return NPARAM; }

isdf_status learn_features(Plan* p, float* dfeat) {
  cudaStream_t s = p->stream;
  double* st = nullptr;
  double* dxyz = nullptr;
  unsigned long long* dmax = nullptr;
  isdf_status r;
  if ((r = dalloc_t(p, &st, size_t(2) * p->ntot, "point statistics")) ||
      (r = dalloc_t(p, &dxyz, size_t(3) * p->natom, "atoms")) || (r = dalloc_t(p, &dmax, 1, "max slot"))) {
    dfree(st), dfree(dxyz), dfree(dmax);
    return r;
  }
  cudaMemcpyAsync(dxyz, p->xyz.data(), sizeof(double) * 3 * p->natom, cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), s);
  for (int l = 0; l < p->nlev; ++l) {
    const Level& lv = p->lev[l];
    k_point_stats<<<152 * 8, 256, 0, s>>>(lv.phi, lv.ng, lv.nL, lv.nG, st + 2 * p->off[l]);
    k_diag_max<<<152 * 4, 256, 0, s>>>(st + 2 * p->off[l], lv.ng, lv.w, dmax);
  }
  unsigned long long bits = 0;
  cudaMemcpyAsync(&bits, dmax, sizeof(bits), cudaMemcpyDeviceToHost, s);
  if ((r = cuda_check(p, cudaStreamSynchronize(s), "feature statistics"))) {
    dfree(st), dfree(dxyz), dfree(dmax);
    return r;
  }
  double d0max;
  std::memcpy(&d0max, &bits, sizeof(d0max));
  if (!(d0max > 0.0)) d0max = 1.0;
  for (int l = 0; l < p->nlev; ++l) {
    const Level& lv = p->lev[l];
    FeatLevel F;
    F.st = st + 2 * p->off[l];
    for (int a = 0; a < 3; ++a) {
      F.n[a] = lv.n[a];
      F.h[a] = p->edge[a] / lv.n[a];
    }
    F.w = lv.w;
    F.level = l;
    F.nlev = p->nlev;
    k_features<<<152 * 8, 256, 0, s>>>(F, dxyz, p->natom, p->edge[0], p->edge[1], p->edge[2], d0max,
                                       dfeat + int64_t(NI) * p->off[l]);
  }
  count_launches(3 * p->nlev);
  r = cuda_check(p, cudaStreamSynchronize(s), "features");
  dfree(st), dfree(dxyz), dfree(dmax);
  return r;
}

isdf_status mlp_grad_step(float* params, float* m, float* v, int step, float lr, const float* X, const float* y,
                          const float* w, int64_t n, float* loss_host, float* grad_dev, cudaStream_t s,
                          std::string& why) {
  float *grad = nullptr, *scal = nullptr;
  if (cudaMalloc(&grad, sizeof(float) * NPARAM) != cudaSuccess || cudaMalloc(&scal, sizeof(float) * 2) != cudaSuccess) {
    cudaGetLastError();
    if (grad) cudaFree(grad);
    why = "allocation failed";
    return ISDF_ERR_OOM;
  }
  cudaMemsetAsync(grad, 0, sizeof(float) * NPARAM, s);
  cudaMemsetAsync(scal, 0, sizeof(float) * 2, s);
  k_sum_weights<<<152, 256, 0, s>>>(w, n, scal);
  float wsum = 0.0f;
  cudaMemcpyAsync(&wsum, scal, sizeof(float), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  const size_t smem = sizeof(float) * (2 * NPARAM + CHUNK * NI + 4 * CHUNK * NH + CHUNK);
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    configured = true;
  }
  const int64_t chunks = (n + CHUNK - 1) / CHUNK;
  const unsigned blocks = unsigned(std::min<int64_t>(chunks, 152 * 2));
  k_mlp_grad<<<blocks, 256, smem, s>>>(params, X, y, w, n, wsum > 0.0f ? 1.0f / wsum : 0.0f, grad, scal + 1);
  if (grad_dev) cudaMemcpyAsync(grad_dev, grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, s);
  if (m && v && lr > 0.0f) {
    const float b1 = 0.9f, b2 = 0.999f;
    k_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(params, m, v, grad, NPARAM, lr, b1, b2, 1e-8f,
                                                1.0f - std::pow(b1, float(step)), 1.0f - std::pow(b2, float(step)));
  }
  count_launches(3);
  float lh = 0.0f;
  cudaMemcpyAsync(&lh, scal + 1, sizeof(float), cudaMemcpyDeviceToHost, s);
  const cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(grad);
  cudaFree(scal);
  if (e != cudaSuccess) {
    why = cudaGetErrorString(e);
    return ISDF_ERR_CUDA;
  }
  if (loss_host) *loss_host = lh;
  return ISDF_OK;
}

void mlp_score(const float* params, const float* X, int64_t n, float* out, cudaStream_t s) {
  k_mlp_score<<<152 * 8, 256, 0, s>>>(params, X, n, out);
  count_launches(1);
}

namespace {

// The K largest scores of one level (slice [off, off + n) of the score array),
// ties to the smallest g, written as ascending pivot codes of that level.
isdf_status topk_level(Plan* p, const float* score, int64_t n, int level, int64_t K, int64_t* dcand,
                       unsigned long long* cnt) {
  cudaStream_t s = p->stream;
  if (K <= 0) return ISDF_OK;
  const int64_t nb = (n + kTopBlock - 1) / kTopBlock;
  int *gt = nullptr, *eq = nullptr;
  int64_t* loff = nullptr;
  isdf_status r;
  if ((r = dalloc_t(p, &gt, size_t(nb), "top-k counts")) || (r = dalloc_t(p, &eq, size_t(nb), "top-k counts")) ||
      (r = dalloc_t(p, &loff, 2, "offsets"))) {
    dfree(gt), dfree(eq), dfree(loff);
    return r;
  }
  auto cleanup = [&]() { dfree(gt), dfree(eq), dfree(loff); };
  auto count_ge = [&](uint32_t t, unsigned long long* c) -> isdf_status {
    cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s);
    k_count_ge<<<152 * 4, 256, 0, s>>>(score, n, t, cnt);
    count_launches(1);
    cudaMemcpyAsync(c, cnt, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    return cuda_check(p, cudaStreamSynchronize(s), "top-k count");
  };
  // bisection for T = the K-th largest key: count(key >= T) >= K > count(key >= T + 1)
  uint64_t lo = 0, hi = 0xFFFFFFFFull;
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo + 1) / 2;
    unsigned long long c = 0;
    if ((r = count_ge(uint32_t(mid), &c))) return cleanup(), r;
    if (c >= (unsigned long long)K)
      lo = mid;
    else
      hi = mid - 1;
  }
  const uint32_t T = uint32_t(lo);
  k_top_counts<<<unsigned(nb), kTopBlock, 0, s>>>(score, n, T, gt, eq);
  std::vector<int> hg(nb), he(nb);
  cudaMemcpyAsync(hg.data(), gt, sizeof(int) * nb, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(he.data(), eq, sizeof(int) * nb, cudaMemcpyDeviceToHost, s);
  if ((r = cuda_check(p, cudaStreamSynchronize(s), "top-k counts"))) return cleanup(), r;
  int64_t ngt = 0, neq = 0;
  for (int64_t b = 0; b < nb; ++b) ngt += hg[b], neq += he[b];
  const int64_t need_eq = std::min<int64_t>(neq, K - ngt);
  std::vector<int> sel_off(nb), eq_off(nb);
  int64_t acc_s = 0, acc_e = 0;
  for (int64_t b = 0; b < nb; ++b) {
    eq_off[b] = int(acc_e);
    sel_off[b] = int(acc_s);
    const int64_t admit = std::max<int64_t>(0, std::min<int64_t>(he[b], need_eq - acc_e));
    acc_s += hg[b] + admit;
    acc_e += he[b];
  }
  cudaMemcpyAsync(gt, sel_off.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(eq, eq_off.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, s);
  // codes of this level: a one-level offset table (0, n) with the level index folded in below
  const int64_t lo_h[2] = {0, n};
  cudaMemcpyAsync(loff, lo_h, sizeof(lo_h), cudaMemcpyHostToDevice, s);
  k_top_write<<<unsigned(nb), kTopBlock, 0, s>>>(score, n, T, gt, eq, need_eq, loff, 1, level, dcand);
  count_launches(2);
  r = cuda_check(p, cudaStreamSynchronize(s), "top-k write");
  cleanup();
  return r;
}

}  // namespace

isdf_status learn_propose_residual(Plan* p, const int64_t* quota, int64_t* dcand) {
  unsigned long long* cnt = nullptr;
  isdf_status r;
  if ((r = dalloc_t(p, &cnt, 1, "count"))) return r;
  int64_t written = 0;
  for (int l = 0; l < p->nlev; ++l) {
    const int64_t K = std::min<int64_t>(quota[l], p->lev[l].ng);
    if (K <= 0) continue;
    if ((r = topk_level(p, p->lev[l].resid, p->lev[l].ng, l, K, dcand + written, cnt))) break;
    written += K;
  }
  dfree(cnt);
  return r;
}

isdf_status learn_propose(Plan* p, const float* params, const int64_t* quota, int64_t* dcand) {
  cudaStream_t s = p->stream;
  const int64_t n = p->ntot;
  float *feat = nullptr, *score = nullptr;
  unsigned long long* cnt = nullptr;
  auto cleanup = [&]() { dfree(feat), dfree(score), dfree(cnt); };
  isdf_status r;
  if ((r = dalloc_t(p, &feat, size_t(NI) * n, "features")) || (r = dalloc_t(p, &score, size_t(n), "scores")) ||
      (r = dalloc_t(p, &cnt, 1, "count")))
    return cleanup(), r;
  if ((r = learn_features(p, feat))) return cleanup(), r;
  mlp_score(params, feat, n, score, s);
  int64_t written = 0;
  for (int l = 0; l < p->nlev; ++l) {
    const int64_t K = std::min<int64_t>(quota[l], p->lev[l].ng);
    if ((r = topk_level(p, score + p->off[l], p->lev[l].ng, l, K, dcand + written, cnt))) return cleanup(), r;
    written += std::max<int64_t>(K, 0);
  }
  cleanup();
  return ISDF_OK;
}

}  // namespace isdf
