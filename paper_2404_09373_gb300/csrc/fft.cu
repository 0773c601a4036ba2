// Batched 3-D real-to-half-complex DFT in double-float arithmetic: the half
// spectra S(q) = sum_r f(r) exp(-2 pi i q.r / n) (unnormalised, the layout of
// a D2Z transform: [qz][qy][qx], qx in [0, nx/2]) that the Coulomb integrals
// of Section II, Eq. 1 are built from.
//
// Every value is a pair of FP32 numbers (hi, lo) with hi + lo the represented
// number (about 48 significant bits); sums use an error-free two-sum and
// products an FMA-based two-product, so the transform runs on the FP32 pipes
// (tens of times the FP64 rate on this GPU) with an error of a few 2^-48 per
// stage relative to the vector's magnitude.
//
// One pass per axis: a CTA loads a tile of lines into shared memory, runs the
// mixed-radix (4, 2, 3) Stockham stages there and writes the tile back:
//   x: real lines f[v][z][y][0..nx)   -> complex [v][z][y][0..nx/2]  (into the output)
//   y: complex lines along y, in place;  z: along z, in place, converted to FP64.
// A double-float complex value takes 16 bytes like a double2, so the output
// buffer holds the intermediate passes.  Axes other than 2^a 3^b <= 128 are
// not handled here (the caller falls back to cuFFT).
#include <cmath>
#include <vector>

#include "dfloat.cuh"
#include "internal.cuh"

namespace isdf {
namespace {

constexpr int kMaxN = 128;
constexpr int kMaxStages = 8;

struct DC {
  DF re, im;
};
__device__ __forceinline__ DC dc_add(DC a, DC b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ DC dc_sub(DC a, DC b) { return {df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
// x y + sgn u v in double-float as one error-free sum of the two leading
// products, their exact rounding errors and the cross terms (the lo * lo
// terms, below 2^-48 of the result, are dropped as in df_mul)
__device__ __forceinline__ DF df_dot2(DF x, DF y, DF u, DF v, float sgn) {
  const float p = __fmul_rn(x.hi, y.hi), q = __fmul_rn(sgn * u.hi, v.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fadd_rn(e, __fmaf_rn(sgn * u.hi, v.hi, -q));
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  e = __fmaf_rn(sgn * u.hi, v.lo, e);
  e = __fmaf_rn(sgn * u.lo, v.hi, e);
  const DF s = two_sum(p, q);
  return quick_two_sum(s.hi, __fadd_rn(s.lo, e));
}
__device__ __forceinline__ DC dc_mul(DC a, DC b) {
  return {df_dot2(a.re, b.re, a.im, b.im, -1.0f), df_dot2(a.re, b.im, a.im, b.re, 1.0f)};
}
__device__ __forceinline__ DC dc_mul_mi(DC a) { return {a.im, df_neg(a.re)}; }  // a * (-i)
__device__ __forceinline__ DC dc_mul_pi(DC a) { return {df_neg(a.im), a.re}; }  // a * (+i)

__device__ __forceinline__ float4 dc_pack(DC a) { return make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo); }
__device__ __forceinline__ DC dc_unpack(float4 v) { return {{v.x, v.y}, {v.z, v.w}}; }

struct FftPass {
  int n;                    // transform length
  int nstage;
  int radix[kMaxStages];
  int64_t nlines;
  // line l starts at (l / lin) * lso + (l % lin) * lsi; element e at + e * es
  // (all in values of the input / output arrays)
  int64_t lin, lso, lsi, es;
  int nout;                 // elements written per line (x pass: n / 2 + 1)
  const float4* tw;         // exp(-2 pi i k / n), k < n
  const double* in_real;    // x pass input (real), else nullptr
  float4* io;               // complex data (double-float), in/out
  double2* out64;           // last pass: FP64 output (same buffer), else nullptr
};

// floor(x / d) for x < 2^16, 1 <= d <= 128: with M = ceil(2^32 / d) the high
// word of x M is exact (the rounding error x (M - 2^32/d) / 2^32 < 2^-16 stays
// below the gap 1/d between x/d and the next integer).  M = 0 encodes d = 1.
struct FastDiv {
  unsigned int d, M;
};
__host__ __device__ inline FastDiv fast_div(unsigned int d) {
  return {d, d == 1 ? 0u : (unsigned int)((0xFFFFFFFFull + d) / d)};
}
__device__ __forceinline__ int fdiv(int x, FastDiv f) { return f.M ? int(__umulhi(unsigned(x), f.M)) : x; }

// one Stockham stage on LPB lines held in shared memory
template <int R>
__device__ __forceinline__ void stage(const float4* __restrict__ x, float4* __restrict__ y, const float4* tw, int n,
                                      int ld, int s, int lines, int tid, int nthreads) {
  const int m = n / (R * s);  // butterflies per line: m * s
  const int per_line = m * s;
  const FastDiv dl = fast_div(per_line), ds = fast_div(s);
  for (int b = tid; b < lines * per_line; b += nthreads) {
    const int li = fdiv(b, dl), j = b - li * per_line;
    const int p = fdiv(j, ds), q = j - p * s;
    const float4* xl = x + li * ld;
    float4* yl = y + li * ld;
    DC a[R];
#pragma unroll
    for (int t = 0; t < R; ++t) a[t] = dc_unpack(xl[q + s * (p + t * m)]);
    DC o[R];
    if (R == 2) {
      o[0] = dc_add(a[0], a[1]);
      o[1] = dc_sub(a[0], a[1]);
    } else if (R == 4) {
      const DC s02 = dc_add(a[0], a[2]), d02 = dc_sub(a[0], a[2]);
      const DC s13 = dc_add(a[1], a[3]), d13 = dc_sub(a[1], a[3]);
      o[0] = dc_add(s02, s13);
      o[2] = dc_sub(s02, s13);
      o[1] = dc_add(d02, dc_mul_mi(d13));  // a0 - i a1 - a2 + i a3
      o[3] = dc_add(d02, dc_mul_pi(d13));  // a0 + i a1 - a2 - i a3
    } else {  // R == 3: w = exp(-2 pi i / 3) = -1/2 - i sqrt(3)/2
      const DF k = {0.8660253882408142f, 1.5543625053737742e-08f};  // sqrt(3)/2 as hi + lo
      const DC b = dc_add(a[1], a[2]), c = dc_sub(a[1], a[2]);
      o[0] = dc_add(a[0], b);
      const DC t0 = {df_sub(a[0].re, df_half(b.re)), df_sub(a[0].im, df_half(b.im))};
      const DC kc = {df_mul(k, c.re), df_mul(k, c.im)};
      o[1] = dc_add(t0, dc_mul_mi(kc));  // t0 - i (sqrt3/2) c
      o[2] = dc_add(t0, dc_mul_pi(kc));  // t0 + i (sqrt3/2) c
    }
#pragma unroll
    for (int u = 0; u < R; ++u) {
      DC v = o[u];
      const int e = p * u * s;  // < (m - 1)(R - 1) s < n
      if (e) v = dc_mul(v, dc_unpack(tw[e]));
      yl[q + s * (R * p + u)] = dc_pack(v);
    }
  }
}

template <int LPB>
__global__ void __launch_bounds__(256) k_fft_pass(FftPass P) {
  extern __shared__ float4 sm[];
  __shared__ float4 tws[kMaxN];
  const int n = P.n, tid = threadIdx.x, nt = blockDim.x;
  // lines n + 1 values apart: consecutive lines of one element fall in
  // different shared-memory banks
  const int ld = n + 1;
  float4* buf0 = sm;
  float4* buf1 = sm + LPB * ld;
  for (int i = tid; i < n; i += nt) tws[i] = P.tw[i];
  const int64_t l0 = int64_t(blockIdx.x) * LPB;
  const int lines_in = int(P.nlines - l0 < LPB ? P.nlines - l0 : LPB);
  // x pass: two real lines per complex line (z = f_2c + i f_2c+1), split after
  const bool pairs = P.in_real != nullptr;
  const int lines = pairs ? (lines_in + 1) / 2 : lines_in;
  // load: consecutive threads take consecutive elements of a line when the
  // line is contiguous, else consecutive lines of one element
  const bool contiguous = P.es == 1;
  const FastDiv dn = fast_div(n), dlines = fast_div(lines_in), dout = fast_div(P.nout);
  if (pairs && (lines_in & 1)) {  // the last complex line has no partner: imaginary part 0
    float2* h = reinterpret_cast<float2*>(buf0);
    for (int e = tid; e < n; e += nt) h[2 * ((lines - 1) * ld + e) + 1] = make_float2(0.0f, 0.0f);
  }
  for (int idx = tid; idx < lines_in * n; idx += nt) {
    int li, e;
    if (contiguous) {
      li = fdiv(idx, dn), e = idx - li * n;
    } else {
      e = fdiv(idx, dlines), li = idx - e * lines_in;
    }
    const int64_t l = l0 + li;
    const int64_t base = (P.lin ? (l / P.lin) * P.lso + (l % P.lin) * P.lsi : l * P.lsi) + int64_t(e) * P.es;
    if (pairs) {
      const DF v = df_from_double(P.in_real[base]);
      reinterpret_cast<float2*>(buf0)[2 * ((li >> 1) * ld + e) + (li & 1)] = make_float2(v.hi, v.lo);
    } else {
      buf0[li * ld + e] = P.io[base];
    }
  }
  __syncthreads();
  float4* x = buf0;
  float4* y = buf1;
  int s = 1;
  for (int st = 0; st < P.nstage; ++st) {
    const int r = P.radix[st];
    if (r == 4)
      stage<4>(x, y, tws, n, ld, s, lines, tid, nt);
    else if (r == 2)
      stage<2>(x, y, tws, n, ld, s, lines, tid, nt);
    else
      stage<3>(x, y, tws, n, ld, s, lines, tid, nt);
    __syncthreads();
    float4* t = x;
    x = y;
    y = t;
    s *= r;
  }
  // store the first nout elements of every line
  const int nout = P.nout;
  for (int idx = tid; idx < lines_in * nout; idx += nt) {
    int li, e;
    if (contiguous) {
      li = fdiv(idx, dout), e = idx - li * nout;
    } else {
      e = fdiv(idx, dlines), li = idx - e * lines_in;
    }
    const int64_t l = l0 + li;
    DC v;
    int64_t base;
    if (pairs) {
      // Z = F_a + i F_b with F_a, F_b Hermitian:  F_a = (Z_k + conj Z_{n-k}) / 2,
      // F_b = -i (Z_k - conj Z_{n-k}) / 2
      const float4* zl = x + (li >> 1) * ld;
      const DC zk = dc_unpack(zl[e]);
      const DC zc = dc_unpack(zl[e == 0 ? 0 : n - e]);
      const DC w = {zc.re, df_neg(zc.im)};
      if (li & 1) {
        const DC d = dc_sub(zk, w);
        v = {df_half(d.im), df_half(df_neg(d.re))};
      } else {
        const DC sm2 = dc_add(zk, w);
        v = {df_half(sm2.re), df_half(sm2.im)};
      }
      base = l * nout + e;
    } else {
      v = dc_unpack(x[li * ld + e]);
      base = (P.lin ? (l / P.lin) * P.lso + (l % P.lin) * P.lsi : l * P.lsi) + int64_t(e) * P.es;
    }
    if (P.out64)
      P.out64[base] = make_double2(df_to_double(v.re), df_to_double(v.im));
    else
      P.io[base] = dc_pack(v);
  }
}

bool factor(int n, int* radix, int* nstage) {
  int k = 0, m = n;
  while (m % 4 == 0 && m > 4 && k < kMaxStages) radix[k++] = 4, m /= 4;
  while (m % 2 == 0 && k < kMaxStages) radix[k++] = 2, m /= 2;
  while (m % 3 == 0 && k < kMaxStages) radix[k++] = 3, m /= 3;
  *nstage = k;
  return m == 1;
}

constexpr int kLPB = 16;

}  // namespace

bool rfft3_df_supported(int nx, int ny, int nz) {
  int r[kMaxStages], k;
  for (int n : {nx, ny, nz})
    if (n < 1 || n > kMaxN || !factor(n, r, &k)) return false;
  return true;
}

// f: batch x (nz ny nx) FP64, S: batch x (nz ny (nx/2+1)) double2 (device);
// tw: device scratch of 2 (nx + ny + nz) float4 (twiddle tables).
isdf_status rfft3_df(Plan* p, const double* f, int nx, int ny, int nz, int64_t batch, double2* S, cudaStream_t s) {
  if (!rfft3_df_supported(nx, ny, nz)) return fail(p, ISDF_ERR_ARG, "double-float transform: unsupported grid");
  if (batch <= 0) return ISDF_OK;
  const int nxh = nx / 2 + 1;
  // twiddle tables exp(-2 pi i k / n) as double-float, from FP64
  std::vector<float> tw(size_t(4) * (nx + ny + nz));
  size_t o = 0;
  int64_t toff[3];
  const int ns[3] = {nx, ny, nz};
  for (int a = 0; a < 3; ++a) {
    toff[a] = int64_t(o / 4);
    for (int k = 0; k < ns[a]; ++k) {
      const double th = -2.0 * 3.14159265358979323846 * double(k) / double(ns[a]);
      const double c = std::cos(th), sn = std::sin(th);
      const float ch = float(c), sh = float(sn);
      tw[o++] = ch;
      tw[o++] = float(c - double(ch));
      tw[o++] = sh;
      tw[o++] = float(sn - double(sh));
    }
  }
  float4* dtw = nullptr;
  isdf_status st;
  if ((st = dalloc_t(p, &dtw, tw.size() / 4, "transform twiddles"))) return st;
  if ((st = cuda_check(p, cudaMemcpyAsync(dtw, tw.data(), sizeof(float) * tw.size(), cudaMemcpyHostToDevice, s),
                       "twiddle copy"))) {
    dfree(dtw);
    return st;
  }
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_fft_pass<kLPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(size_t(2) * kLPB * (kMaxN + 1) * sizeof(float4)));
    configured = true;
  }
  float4* io = reinterpret_cast<float4*>(S);
  const int64_t nq = int64_t(nz) * ny * nxh;
  auto launch = [&](FftPass P) {
    const int64_t blocks = (P.nlines + kLPB - 1) / kLPB;
    const size_t smem = size_t(2) * kLPB * (P.n + 1) * sizeof(float4);  // two tiles of lines
    k_fft_pass<kLPB><<<unsigned(blocks), 256, smem, s>>>(P);
    count_launches(1);
  };
  // x: lines (v, z, y), contiguous
  FftPass P{};
  P.n = nx;
  factor(nx, P.radix, &P.nstage);
  P.nlines = batch * nz * ny;
  P.lin = 0;
  P.lsi = nx;
  P.es = 1;
  P.nout = nxh;
  P.tw = dtw + toff[0];
  P.in_real = f;
  P.io = io;
  launch(P);
  // y: lines (v, z, qx), element stride nxh, in place
  FftPass Q{};
  Q.n = ny;
  factor(ny, Q.radix, &Q.nstage);
  Q.nlines = batch * nz * nxh;
  Q.lin = nxh;
  Q.lso = int64_t(ny) * nxh;
  Q.lsi = 1;
  Q.es = nxh;
  Q.nout = ny;
  Q.tw = dtw + toff[1];
  Q.io = io;
  launch(Q);
  // z: lines (v, qy, qx), element stride ny nxh, in place, FP64 out
  FftPass R{};
  R.n = nz;
  factor(nz, R.radix, &R.nstage);
  R.nlines = batch * ny * nxh;
  R.lin = int64_t(ny) * nxh;
  R.lso = nq;
  R.lsi = 1;
  R.es = int64_t(ny) * nxh;
  R.nout = nz;
  R.tw = dtw + toff[2];
  R.io = io;
  R.out64 = S;
  launch(R);
  dfree(dtw);
  return ISDF_OK;
}

}  // namespace isdf
