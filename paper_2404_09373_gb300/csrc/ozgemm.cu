// FP64-accurate GEMM on the tcgen05 tensor cores from sliced BF16 products.
//
// Every row r of an FP64 operand X (rows x K) is scaled by 2^-e_r so that
// |x| < 1, rounded to a fixed-point integer with 7S fraction bits and split
// into S balanced base-128 digits d_0..d_{S-1} (|d_0| <= 128, |d_s| <= 64),
// each exactly representable in BF16:
//     x 2^-e_r = sum_s d_s 2^{-7(s+1)} + O(2^{-7S-1}).
// A product keeps the digit pairs s + t <= S - 1 ("levels" q = s + t):
//     (A B^T)_mn = 2^{e_m + f_n - 14} sum_q 2^{-7q} L_q,  L_q = sum_k sum_{s+t=q} d_s b_t.
// Each level has its own FP32 accumulator in tensor memory.  Digit products
// are integers below 2^14, so levels 0 and 1 summed over a chunk of 1024 k
// values stay below 2^24 and are exact in FP32; deeper levels are scaled by
// 2^-14 or less, where FP32 rounding is harmless.  After every chunk the
// epilogue warps read the levels out (tcgen05.ld) and add them to double-float
// (hi, lo) register accumulators; the result is formed in FP64 at the end.
// With S = 8 (FP64-grade: 56 fraction bits per operand) the chunk is 256 k, so
// every level's sum is an exact integer below 2^24, and the epilogue adds the
// levels into two 64-bit integer accumulators: the product of the rounded
// operands is then exact up to the dropped levels (below 2^-56 relative per
// term) and one final FP64 rounding.
//
// Operands are pre-tiled by the slicing kernel into the canonical K-major,
// no-swizzle UMMA layout (8x8 core matrices, LBO = 128 B along K, SBO =
// 512 B per 8-row group, 32 k values per tile), all S slices of one
// (row tile, k tile) contiguous, so one cp.async.bulk per operand fills a
// pipeline stage.  Roles per CTA: warp 0 issues the bulk copies, warp 1 owns
// tensor memory and issues tcgen05.mma, warps 2-9 drain the accumulators.
// Every mbarrier wait is bounded: on expiry the CTA records an error code,
// lets its copies and MMAs in flight finish, frees tensor memory and exits.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "internal.cuh"

namespace isdf {
namespace {

constexpr int kMaxDevices = 64;  // per-device launch set-up and scratch addresses

constexpr int kBM = 128;  // A rows per CTA = TMEM lanes
constexpr int kBK = kOzBK;  // k values per tile / pipeline stage
constexpr int kKcTiles = 1024 / kBK;  // 1024 k values per exact chunk
constexpr long long kWaitLimit = 1ll << 30;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s of device time per wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  // K-major, no swizzle: LBO = 128 B (next core matrix along K), SBO = 16 kBK
  // bytes (next 8-row group), descriptor version 1 (bits 46-47), layout type 0.
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)((16 * kBK) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// kind::f16 instruction descriptor: D F32, A/B BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait: gives up after wait_ns of device time (0: after the first
// unsuccessful try), after kWaitLimit polls, or as soon as any CTA of the
// launch has recorded an error in *err.  The
// pipeline waits take the launch's limit (kWaitNs unless a host-side fault
// injection shortens it); the drain waits for copies and MMAs in flight
// always take kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, const int* err,
                                          unsigned long long wait_ns = kWaitNs) {
  const uint32_t addr = smem_u32(bar);
  unsigned long long t0 = 0;
  for (long long i = 0; i < kWaitLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(phase)
        : "memory");
    if (done) return true;
    if (wait_ns == 0) return false;  // a zero limit gives up after the first unsuccessful try
    if ((i & 255) == 0) {
      const unsigned long long now = globaltimer_ns();
      if (i == 0) t0 = now;
      else if (now - t0 > wait_ns) return false;
      if (err && *(volatile const int*)err) return false;
    }
  }
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void umma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}


// Compiler fence on 16 accumulators: the empty volatile statement reads and
// writes them, so their updates are complete here and no later volatile
// statement (a tensor-memory load) is moved above it.
__device__ __forceinline__ void reg_fence16(long long (&a)[16], uint32_t (&b)[16]) {
  asm volatile("" : "+l"(a[0]), "+l"(a[1]), "+l"(a[2]), "+l"(a[3]), "+l"(a[4]), "+l"(a[5]), "+l"(a[6]), "+l"(a[7]));
  asm volatile("" : "+l"(a[8]), "+l"(a[9]), "+l"(a[10]), "+l"(a[11]), "+l"(a[12]), "+l"(a[13]), "+l"(a[14]),
               "+l"(a[15]));
  asm volatile("" : "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]), "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7]),
               "+r"(b[8]), "+r"(b[9]), "+r"(b[10]), "+r"(b[11]), "+r"(b[12]), "+r"(b[13]), "+r"(b[14]), "+r"(b[15]));
}

__device__ __forceinline__ void set_err(int* err, int code) { atomicCAS(err, 0, code); }

// f * 2^e as a double, built with integer operations (exact; the narrow FP64
// pipe is left alone).  Subnormal or out-of-range cases take the FP64 route.
__device__ __forceinline__ double scaled_to_double(float f, int e) {
  const uint32_t b = __float_as_uint(f);
  if ((b << 1) == 0u) return __longlong_as_double((long long)(uint64_t(b >> 31) << 63));  // +-0
  const int ef = int((b >> 23) & 0xFF);
  const int ed = ef - 127 + 1023 + e;
  if (ef == 0 || ef == 0xFF || ed <= 0 || ed >= 0x7FF) return ldexp(double(f), e);
  const uint64_t bits = (uint64_t(b >> 31) << 63) | (uint64_t(ed) << 52) | (uint64_t(b & 0x7FFFFF) << 29);
  return __longlong_as_double((long long)bits);
}

// An integer-valued float (|x| < 2^62) as a 64-bit integer without the
// 64-bit conversion instruction, which runs on the narrow FP64 unit: below
// 2^23 a 32-bit conversion is exact, above it the value is its significand
// shifted left.
__device__ __forceinline__ long long intf_to_ll(float x) {
  const uint32_t b = __float_as_uint(x);
  const int ef = int((b >> 23) & 0xFF);
  if (ef < 150) return (long long)__float2int_rz(x);
  const long long m = (long long)((b & 0x7FFFFFu) | 0x800000u) << (ef - 150);
  return (b >> 31) ? -m : m;
}

// (th + rem 2^-28) 2^e rounded once to the nearest double (ties to even),
// from the fixed-point value with integer operations; outside the normal
// range it takes the FP64 route.
__device__ __forceinline__ double fixed_to_double(long long th, uint32_t rem, int e) {
  const __int128 X = ((__int128)th << 28) + (__int128)rem;  // value X 2^(e - 28)
  if (X == 0) return 0.0;
  const bool neg = X < 0;
  const unsigned __int128 U = neg ? (unsigned __int128)(-X) : (unsigned __int128)X;
  const uint64_t hi = uint64_t(U >> 64), lo = uint64_t(U);
  const int L = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);  // bit length
  int E = L - 1 + e - 28;
  uint64_t M;  // significand, 53 bits
  if (L <= 53) {
    M = lo << (53 - L);
  } else {
    const int sh = L - 53;
    const unsigned __int128 q = U >> sh;
    const unsigned __int128 r = U - (q << sh);
    const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
    M = uint64_t(q);
    if (r > half || (r == half && (M & 1ull))) {
      ++M;
      if (M >> 53) M >>= 1, ++E;
    }
  }
  if (E < -1022 || E > 1023) return ldexp(neg ? -double(M) : double(M), E - 52);
  const uint64_t bits = (uint64_t(neg) << 63) | (uint64_t(E + 1023) << 52) | (M & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

// ---------------------------------------------------------------- slicing

// |x| as an order-preserving integer key (finite doubles)
__device__ __forceinline__ uint64_t abs_key(double x) { return uint64_t(__double_as_longlong(x)) & 0x7FFFFFFFFFFFFFFFull; }

// exponent e with |x| < 2^e from the key of the largest |x| of a row
__device__ __forceinline__ int exp_of_key(uint64_t key) {
  if (key == 0) return 0;
  int e;
  frexp(__longlong_as_double((long long)key), &e);
  return e;
}

// round(x * 2^shift) to the nearest integer (ties to even) with integer
// operations only; |result| < 2^62 is guaranteed by the caller's scaling
__device__ __forceinline__ long long round_scaled(double x, int shift) {
  const uint64_t b = uint64_t(__double_as_longlong(x));
  const int E = int((b >> 52) & 0x7FF);
  if (E == 0 && (b << 1) == 0) return 0;
  uint64_t m = b & 0xFFFFFFFFFFFFFull;
  int ee = E;
  if (E == 0) ee = 1; else m |= 1ull << 52;
  const int sh = ee - 1075 + shift;  // value = m * 2^sh
  long long q;
  if (sh >= 0) {
    q = (long long)(m << sh);
  } else if (sh <= -64) {
    q = 0;
  } else {
    const int r = -sh;
    const uint64_t qq = m >> r;
    const uint64_t rem = m & ((1ull << r) - 1ull);
    const uint64_t half = 1ull << (r - 1);
    q = (long long)(qq + ((rem > half || (rem == half && (qq & 1ull))) ? 1ull : 0ull));
  }
  return (b >> 63) ? -q : q;
}

__device__ __forceinline__ int64_t map_at(const OzMap& m, int64_t i) {
  return m.in ? (i / m.in) * m.so + (i % m.in) * m.si : i * m.si;
}

// source offset of row r: ridx[r] rows of stride rm.si, else the row map
__device__ __forceinline__ int64_t row_base(const OzMap& rm, const int* ridx, int64_t r) {
  return ridx ? int64_t(ridx[r]) * rm.si : map_at(rm, r);
}

// |mul * kw[k] * v| as an order-preserving key
__device__ __forceinline__ uint64_t key_at(double v, int64_t k, const double* __restrict__ kw, double mul) {
  if (mul != 1.0) v *= mul;
  if (kw) v *= kw[k];
  return abs_key(v);
}

__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }

// e_r: max_k |x(r,k)| < 2^e_r, x = mul * kw[k] * src[row(r) + map_k(k)]; one thread per row
// (four loads in flight per thread on the plain-stride path)
__global__ void k_oz_rowexp_thread(const double* __restrict__ src, OzMap rm, OzMap km, int64_t rows, int64_t K,
                                   const double* __restrict__ kw, double mul, const int* __restrict__ ridx,
                                   int* __restrict__ exps) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const double* row = src + row_base(rm, ridx, r);
  uint64_t m = 0;
  if (km.in == 0) {
    const int64_t si = km.si;
    int64_t k = 0;
    for (; k + 4 <= K; k += 4) {
      const double v0 = row[k * si], v1 = row[(k + 1) * si], v2 = row[(k + 2) * si], v3 = row[(k + 3) * si];
      m = umax64(m, umax64(umax64(key_at(v0, k, kw, mul), key_at(v1, k + 1, kw, mul)),
                           umax64(key_at(v2, k + 2, kw, mul), key_at(v3, k + 3, kw, mul))));
    }
    for (; k < K; ++k) m = umax64(m, key_at(row[k * si], k, kw, mul));
  } else {
    int64_t q = 0, rem = 0;  // k = q km.in + rem, advanced without division
    for (int64_t k = 0; k < K; ++k) {
      m = umax64(m, key_at(row[q * km.so + rem * km.si], k, kw, mul));
      if (++rem == km.in) rem = 0, ++q;
    }
  }
  exps[r] = exp_of_key(m);
}

// same, one block per row (few long rows); contiguous rows are read as
// 16-byte vectors, four per thread in flight
__global__ void k_oz_rowexp_block(const double* __restrict__ src, OzMap rm, OzMap km, int64_t K,
                                  const double* __restrict__ kw, double mul, const int* __restrict__ ridx,
                                  int* __restrict__ exps) {
  __shared__ unsigned long long sh[256];
  const int64_t r = blockIdx.x;
  const double* row = src + row_base(rm, ridx, r);
  uint64_t m = 0;
  const int bd = blockDim.x;
  if (km.in == 0 && km.si == 1 && (reinterpret_cast<uintptr_t>(row) & 15) == 0) {
    const double2* p = reinterpret_cast<const double2*>(row);
    const int64_t K2 = K >> 1;
    int64_t i = threadIdx.x;
    for (; i + 3 * bd < K2; i += 4 * bd) {
      double2 t[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) t[h] = __ldg(p + i + h * bd);
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int64_t k = 2 * (i + h * bd);
        m = umax64(m, umax64(key_at(t[h].x, k, kw, mul), key_at(t[h].y, k + 1, kw, mul)));
      }
    }
    for (; i < K2; i += bd) {
      const double2 t = __ldg(p + i);
      m = umax64(m, umax64(key_at(t.x, 2 * i, kw, mul), key_at(t.y, 2 * i + 1, kw, mul)));
    }
    if ((K & 1) && threadIdx.x == 0) m = umax64(m, key_at(row[K - 1], K - 1, kw, mul));
  } else {
    for (int64_t k = threadIdx.x; k < K; k += bd) m = umax64(m, key_at(row[map_at(km, k)], k, kw, mul));
  }
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] = sh[threadIdx.x] > sh[threadIdx.x + o] ? sh[threadIdx.x] : sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) exps[r] = exp_of_key(sh[0]);
}

// BF16 bits of a small integer d (|d| <= 2^8): 1.5 * 2^23 + d is exact in
// FP32 (unit spacing), subtracting 1.5 * 2^23 leaves d exactly, and d has at
// most 8 significant bits, so the upper half of its FP32 pattern is its BF16
// pattern.  Integer and FP32 operations only.
__device__ __forceinline__ uint32_t bf16_bits_of_small(int d) {
  return __float_as_uint(__int_as_float(0x4B400000 + d) - 12582912.0f);
}

// Digits of row r and k group kg (8 values), written as 16 bytes per slice:
// tile (row tile i, k tile j) sits at position i * kst + j of the tile array.
template <int S>
__device__ __forceinline__ void oz_digit_group(const double* __restrict__ src, const OzMap& rm, const OzMap& km,
                                               int64_t rows, int64_t K, const double* __restrict__ kw, double mul,
                                               const int* __restrict__ exps, int rt, int64_t kst,
                                               const int* __restrict__ ridx, __nv_bfloat16* __restrict__ tiles, int r,
                                               int64_t kg) {
  const bool live = r < rows;
  const int e = live ? exps[r] : 0;
  const double* row = src + (live ? row_base(rm, ridx, r) : 0);
  const int64_t k0 = kg * 8;
  double v[8];
  if (live && km.in == 0 && km.si == 1 && k0 + 8 <= K && (reinterpret_cast<uintptr_t>(row + k0) & 15) == 0) {
    const double2* p = reinterpret_cast<const double2*>(row + k0);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const double2 t = __ldg(p + h);
      v[2 * h] = t.x;
      v[2 * h + 1] = t.y;
    }
  } else {
    int64_t q = 0, rem = 0;  // k0 = q km.in + rem
    if (km.in) q = k0 / km.in, rem = k0 % km.in;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t off = km.in ? q * km.so + rem * km.si : (k0 + u) * km.si;
      if (km.in && ++rem == km.in) rem = 0, ++q;
      v[u] = (live && k0 + u < K) ? row[off] : 0.0;
    }
  }
  long long X[8];
  const int shift = 7 * S - e;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    double x = v[u];
    if (k0 + u < K) {
      if (mul != 1.0) x *= mul;
      if (kw) x *= kw[k0 + u];
    }
    X[u] = round_scaled(x, shift);
  }
  const int it = r / rt, rr = r - it * rt;
  const int64_t jt = kg / (kBK / 8);
  const int kc = int(kg % (kBK / 8));
  const int64_t tile_elems = int64_t(rt) * kBK;
  __nv_bfloat16* base = tiles + ((int64_t(it) * kst + jt) * S) * tile_elems;
  const int inner = (rr >> 3) * (8 * kBK) + kc * 64 + (rr & 7) * 8;  // element offset in a tile
  // Balanced digits from the least significant end (in [-64, 63]; the top one
  // takes the rest, |d_0| <= 128), one slice at a time.  |X| < 2^(7S + 1), so
  // once S - 4 digits are removed the remainder fits in 32 bits.
  int Y[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) Y[u] = int(X[u]);
#pragma unroll
  for (int s = S - 1; s >= 0; --s) {
    uint32_t b[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      int dig;
      if (s >= 4) {
        dig = int((uint32_t(X[u]) + 64u) & 127u) - 64;
        X[u] = (X[u] - dig) >> 7;
        if (s == 4) Y[u] = int(X[u]);
      } else if (s >= 1) {
        dig = ((Y[u] + 64) & 127) - 64;
        Y[u] = (Y[u] - dig) >> 7;
      } else {
        dig = Y[u];
      }
      b[u] = bf16_bits_of_small(dig);
    }
    uint4 w;
    w.x = __byte_perm(b[0], b[1], 0x7632);
    w.y = __byte_perm(b[2], b[3], 0x7632);
    w.z = __byte_perm(b[4], b[5], 0x7632);
    w.w = __byte_perm(b[6], b[7], 0x7632);
    *reinterpret_cast<uint4*>(base + int64_t(s) * tile_elems + inner) = w;
  }
}

// Digits of the k groups [kg0, kg0 + ngrp) of every row (padding rows zero).
// order 0 (k strided): 256 consecutive rows per block, one k group per
// blockIdx.y.  order 1 (k contiguous): each warp takes 8 rows x 4
// consecutive k groups, so it writes one 512-byte line of each slice and
// reads 256 contiguous bytes of each of its rows; blockIdx.y walks the
// 8-row groups.
template <int S>
__global__ void k_oz_digits(const double* __restrict__ src, OzMap rm, OzMap km, int64_t rows, int64_t K,
                            const double* __restrict__ kw, double mul, const int* __restrict__ exps, int rt,
                            int64_t nrt, int64_t kg0, int64_t ngrp, int64_t kst, int order,
                            const int* __restrict__ ridx, __nv_bfloat16* __restrict__ tiles) {
  const int64_t rows_pad = nrt * rt;
  if (order == 0) {
    const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= rows_pad) return;
    for (int64_t g = blockIdx.y; g < ngrp; g += gridDim.y)
      oz_digit_group<S>(src, rm, km, rows, K, kw, mul, exps, rt, kst, ridx, tiles, int(r), kg0 + g);
  } else {
    const int lane = threadIdx.x & 31;
    const int64_t g = (int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 4 + (lane >> 3);
    if (g >= ngrp) return;
    for (int64_t g8 = blockIdx.y; g8 * 8 < rows_pad; g8 += gridDim.y)
      oz_digit_group<S>(src, rm, km, rows, K, kw, mul, exps, rt, kst, ridx, tiles, int(g8 * 8 + (lane & 7)),
                        kg0 + g);
  }
}

// Re-tile an operand's digit planes to another row-tile height: rows of 8
// (one 512-byte line of a slice for 32 k values) move as whole lines, so the
// digits are copied, not recomputed.  Rows at or beyond the source's real rows
// are written as zeros (padding).
__global__ void k_oz_retile(const __nv_bfloat16* __restrict__ src, int src_rt, int64_t src_kst,
                            __nv_bfloat16* __restrict__ dst, int dst_rt, int64_t dst_kst, int S, int64_t rows,
                            int64_t rows_pad, int64_t nkt) {
  const int lane = threadIdx.x & 31;
  const int64_t units = (rows_pad / 8) * nkt * S;
  for (int64_t u = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; u < units;
       u += (int64_t(gridDim.x) * blockDim.x) >> 5) {
    const int s = int(u % S);
    const int64_t kt = (u / S) % nkt, g8 = u / (int64_t(S) * nkt);
    const int64_t r0 = g8 * 8;
    const int64_t dt = r0 / dst_rt, drg = (r0 % dst_rt) / 8;
    uint4* out = reinterpret_cast<uint4*>(dst + ((dt * dst_kst + kt) * S + s) * int64_t(dst_rt) * kBK + drg * 8 * kBK);
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (r0 < rows) {
      const int64_t st = r0 / src_rt, srg = (r0 % src_rt) / 8;
      const uint4* in =
          reinterpret_cast<const uint4*>(src + ((st * src_kst + kt) * S + s) * int64_t(src_rt) * kBK + srg * 8 * kBK);
      v = in[lane];
    }
    out[lane] = v;
  }
}

void launch_digits(const double* src, OzMap rm, OzMap km, const double* kw, double mul, const int* ridx,
                   const OzOperand& op, int64_t kg0, int64_t ngrp, int order, cudaStream_t s) {
  const int64_t rows_pad = op.nrt * op.rt;
  dim3 grid;
  if (order == 0) {
    grid.x = unsigned((rows_pad + 255) / 256);
    grid.y = unsigned(std::min<int64_t>(ngrp, 65535));
  } else {
    grid.x = unsigned(((ngrp + 3) / 4 + 7) / 8);
    grid.y = unsigned(std::min<int64_t>(rows_pad / 8, 65535));
  }
  __nv_bfloat16* t = static_cast<__nv_bfloat16*>(op.tiles);
  if (op.S == 7)
    k_oz_digits<7><<<grid, 256, 0, s>>>(src, rm, km, op.rows, op.K, kw, mul, op.exps, op.rt, op.nrt, kg0, ngrp,
                                        op.kst, order, ridx, t);
  else if (op.S == 5)
    k_oz_digits<5><<<grid, 256, 0, s>>>(src, rm, km, op.rows, op.K, kw, mul, op.exps, op.rt, op.nrt, kg0, ngrp,
                                        op.kst, order, ridx, t);
  else if (op.S == 6)
    k_oz_digits<6><<<grid, 256, 0, s>>>(src, rm, km, op.rows, op.K, kw, mul, op.exps, op.rt, op.nrt, kg0, ngrp,
                                        op.kst, order, ridx, t);
  else
    k_oz_digits<8><<<grid, 256, 0, s>>>(src, rm, km, op.rows, op.K, kw, mul, op.exps, op.rt, op.nrt, kg0, ngrp,
                                        op.kst, order, ridx, t);
}

// ---------------------------------------------------------------- GEMM

struct OzGemmParams {
  const __nv_bfloat16* A;
  const __nv_bfloat16* B;
  const int* ea;
  const int* eb;
  int64_t M, N, nkt;
  int64_t ntm, ntn;    // M tiles (of 128 rows) and N tiles (of BN rows)
  int64_t akst, bkst;  // k-tile strides of the A and B tile arrays (>= nkt)
  int tri;     // 0 dense; 1 B-side lower (k <= n); 2 B-side upper (k >= n)
  int sym;     // compute only tiles that touch the lower triangle (n <= m)
  int splits;  // split-K factor (gridDim.z)
  double* C;
  OzMap cm, cn;  // C[map_m(m) + map_n(n)]
  double alpha;
  double* work;  // split-K partials [z][M][N]
  int* err;
  unsigned long long wait_ns;  // limit of each pipeline wait (device time)
};

template <int S, int BN>
struct OzCfg {
  static constexpr int tileA = kBM * kBK * 2;  // bytes per slice tile
  static constexpr int tileB = BN * kBK * 2;
  static constexpr int stageA = S * tileA;
  static constexpr int stageB = S * tileB;
  static constexpr int stage = stageA + stageB;
  static constexpr int cols = S * BN;
  static constexpr bool exact = S >= 7;
  // two CTAs per SM when the accumulators take at most half of tensor memory:
  // one CTA's pipeline fill and accumulator drain overlap the other's MMAs
  static constexpr bool dual = !exact && cols <= 256;
  static constexpr int min_blocks = dual ? 2 : 1;
  static constexpr int budget = dual ? 115712 - 2048 : 220 * 1024 - 2048;
  static constexpr int nst = budget / stage < 4 ? budget / stage : 4;
  static constexpr int smem = nst * stage + 2048;  // + barriers and 1024-byte alignment slack
  static constexpr uint32_t tcols = cols <= 32 ? 32 : cols <= 64 ? 64 : cols <= 128 ? 128 : cols <= 256 ? 256 : 512;
  // S = 8: levels 0..5 are kept exact (chunks of 512 k keep their integer
  // sums at most 2^24; levels 6, 7 weigh less than 2^-42, where FP32 rounding
  // is harmless) and summed in integers; else double-float
  static constexpr int kc = exact ? 512 / kBK : kKcTiles;  // k tiles per chunk
  // epilogue warps: two per tensor-memory lane quarter (BN/2 columns each),
  // three when exact (BN/3 columns each, so the integer state fits in
  // registers), one when two CTAs share the SM
  static constexpr int epi = exact ? 12 : dual ? 4 : 8;
  static constexpr int threads = 32 * (2 + epi);
  static_assert(!exact || S == 7 || S == 8, "the integer epilogue pairs the levels of 7 or 8 digits");
  static_assert(cols <= 512, "levels x BN must fit in tensor memory");
  static_assert(nst >= 2, "need at least two pipeline stages");
  static_assert((BN / (epi / 4)) % 16 == 0, "each epilogue warp reads whole 16-column groups");
  static_assert(smem <= 232448, "shared memory per CTA");
};

template <int S, int BN>
__global__ void __launch_bounds__(OzCfg<S, BN>::threads, OzCfg<S, BN>::min_blocks) k_oz_gemm(OzGemmParams P) {
  using Cfg = OzCfg<S, BN>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Cfg::nst * Cfg::stage);
  uint64_t* empty = full + Cfg::nst;
  uint64_t* acc_full = empty + Cfg::nst;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* drain = acc_empty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  // an earlier launch failed: do nothing (one read, made uniform across the CTA)
  if (__syncthreads_or(threadIdx.x == 0 ? *(volatile const int*)P.err : 0)) return;

  // Persistent tiles: tile t is (N tile t % NT, M tile (t / NT) % MT, split
  // t / (NT MT)); N tiles vary fastest so that CTAs in flight share A.  Every
  // role walks the same tile sequence; stage and chunk counters run on across
  // tiles, so the ring of stages and the accumulator hand-off never restart
  // and a tile's epilogue overlaps the next tile's copies and MMAs.
  const int64_t NT = P.ntn, MT = P.ntm, ntiles = NT * MT * P.splits;
  struct Tile {
    int64_t nt, mt, m0, n0, kt_lo, nk;
    int z;
    bool skip;
  };
  auto tile_at = [&](int64_t t) {
    Tile T;
    T.nt = t % NT;
    T.mt = (t / NT) % MT;
    T.z = int(t / (NT * MT));
    T.m0 = T.mt * kBM;
    T.n0 = T.nt * BN;
    T.skip = P.sym && T.n0 > T.m0 + kBM - 1;  // tile entirely above the diagonal
    int64_t lo = 0, hi = P.nkt;
    if (P.tri == 1) hi = min(P.nkt, (T.n0 + BN + kBK - 1) / kBK);
    if (P.tri == 2) lo = min(P.nkt, T.n0 / kBK);
    const int64_t tot = hi - lo, per = (tot + P.splits - 1) / P.splits;
    const int64_t a = lo + per * T.z;
    T.kt_lo = min(hi, a);
    T.nk = min(hi, a + per) - T.kt_lo;
    return T;
  };

  if (threadIdx.x == 0) {
    for (int i = 0; i < Cfg::nst; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, Cfg::epi);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(Cfg::tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------ producer
    if (lane == 0) {
      const unsigned char* gA = reinterpret_cast<const unsigned char*>(P.A);
      const unsigned char* gB = reinterpret_cast<const unsigned char*>(P.B);
      int64_t g = 0;  // stages issued so far (all tiles)
      for (int64_t t = blockIdx.x; t < ntiles && !*(volatile int*)abort_flag; t += gridDim.x) {
        const Tile T = tile_at(t);
        if (T.skip) continue;
        for (int64_t it = 0; it < T.nk; ++it, ++g) {
          const int st = int(g % Cfg::nst);
          const int64_t round = g / Cfg::nst;
          if (round > 0 && !mbar_wait(&empty[st], uint32_t((round - 1) & 1), P.err, P.wait_ns)) {
            set_err(P.err, 11);
            *(volatile int*)abort_flag = 1;
            break;
          }
          if (*(volatile int*)abort_flag) break;
          const int64_t kt = T.kt_lo + it;
          unsigned char* sA = smem + st * Cfg::stage;
          unsigned char* sB = sA + Cfg::stageA;
          mbar_expect_tx(&full[st], Cfg::stageA + Cfg::stageB);
          bulk_g2s(sA, gA + (T.mt * P.akst + kt) * int64_t(Cfg::stageA), Cfg::stageA, &full[st]);
          bulk_g2s(sB, gB + (T.nt * P.bkst + kt) * int64_t(Cfg::stageB), Cfg::stageB, &full[st]);
        }
      }
      // copies that were issued but never consumed must land before exit
      if (*(volatile int*)abort_flag) {
        const int64_t first = g > Cfg::nst ? g - Cfg::nst : 0;
        for (int64_t it = first; it < g; ++it) mbar_wait(&full[it % Cfg::nst], uint32_t((it / Cfg::nst) & 1), nullptr);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      int64_t g = 0, h = 0;  // stages consumed, accumulator chunks handed over (all tiles)
      bool stop = false;
      for (int64_t t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
        const Tile T = tile_at(t);
        if (T.skip) continue;
        for (int64_t it = 0; it < T.nk; ++it, ++g) {
          const int st = int(g % Cfg::nst);
          const int64_t round = g / Cfg::nst;
          const int64_t cpos = it % Cfg::kc;
          if (cpos == 0 && h > 0 && !mbar_wait(acc_empty, uint32_t((h - 1) & 1), P.err, P.wait_ns)) {
            set_err(P.err, 12);
            *(volatile int*)abort_flag = 1;
            stop = true;
            break;
          }
          if (!mbar_wait(&full[st], uint32_t(round & 1), P.err, P.wait_ns)) {
            set_err(P.err, 13);
            *(volatile int*)abort_flag = 1;
            stop = true;
            break;
          }
          if (*(volatile int*)abort_flag) {
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t sA = smem_u32(smem + st * Cfg::stage);
          const uint32_t sB = sA + Cfg::stageA;
          // For A digit s the products with B digits t = 0..S-1-s land in
          // levels s..S-1, i.e. tensor-memory columns [s BN, S BN); the B
          // digit tiles of a stage are contiguous, so B rows [0, (S-s) BN) are
          // exactly digits 0..S-1-s and one MMA (N up to 256, else split)
          // covers them all.  The first MMA of a chunk (s = 0) spans every
          // level and initialises the accumulators.
#pragma unroll
          for (int s = 0; s < S; ++s) {
#pragma unroll
            for (int c0 = 0; c0 < BN * (S - s); c0 += 256) {
              const int n = (BN * (S - s) - c0) < 256 ? (BN * (S - s) - c0) : 256;
              const uint32_t idesc = umma_idesc(kBM, n);
#pragma unroll
              for (int ks = 0; ks < kBK / 16; ++ks) {
                const uint64_t da = umma_desc(sA + s * Cfg::tileA + ks * 256);
                const uint64_t db = umma_desc(sB + (c0 / 8) * (16 * kBK) + ks * 256);
                const uint32_t acc = (cpos > 0 || s > 0 || ks > 0) ? 1u : 0u;
                umma_bf16(tmem + uint32_t(s * BN + c0), da, db, idesc, acc);
              }
            }
          }
          umma_commit(&empty[st]);
          if (cpos == Cfg::kc - 1 || it == T.nk - 1) {
            umma_commit(acc_full);
            ++h;
          }
        }
      }
      // all MMAs issued by this thread complete before tensor memory is freed
      umma_commit(drain);
      mbar_wait(drain, 0, nullptr);
    }
  } else {
    // ------------------------------------------------ epilogue warps
    const int quarter = warp % 4;  // a warp reads tensor-memory lanes 32 (warp % 4) ..
    const int half = (warp - 2) / 4;  // which share of the columns
    const int row = quarter * 32 + lane;
    constexpr int HC = BN / (Cfg::epi / 4);  // columns per thread
    int64_t h = 0;  // accumulator chunks taken over (all tiles)
    for (int64_t t = blockIdx.x; t < ntiles && !*(volatile int*)abort_flag; t += gridDim.x) {
      const Tile T = tile_at(t);
      if (T.skip) continue;
      const int64_t nchunks = (T.nk + Cfg::kc - 1) / Cfg::kc;
      const int64_t m = T.m0 + row, n0 = T.n0;
      if constexpr (Cfg::exact) {
        // Levels 0..7 of one column and chunk (512 k: levels 0..5 are exact
        // integers below 2^24) are paired exactly in 32-bit integers,
        //   P01 = L0 2^7 + L1, P23 = L2 2^7 + L3, P45 = L4 2^7 + L5  (< 2^31),
        // and levels 6, 7 (weights below 2^-42) are combined in FP32.  Per
        // column th accumulates P01 2^14 + P23 plus the part of
        // lo = P45 2^14 + (L6 2^7 + L7) above 2^28; rem keeps lo's low 28 bits
        // (carried into th), so the value is th + rem 2^-28 in units of 2^-21.
        // With 7 digits there is no level 7 (L7 = 0).
        static_assert(HC % 16 == 0, "16-column tensor-memory loads");
        long long th[HC];
        uint32_t rem[HC];
#pragma unroll
        for (int j = 0; j < HC; ++j) th[j] = 0, rem[j] = 0u;
        const uint32_t tbase = tmem + (uint32_t(quarter * 32) << 16) + uint32_t(half * HC);
        for (int64_t c = 0; c < nchunks; ++c) {
          if (!mbar_wait(acc_full, uint32_t(h & 1), P.err, P.wait_ns)) {
            set_err(P.err, 14);
            *(volatile int*)abort_flag = 1;
            break;
          }
          ++h;
          asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
          for (int c0 = 0; c0 < HC; c0 += 16) {
#pragma unroll
            for (int pq = 0; pq < 4; ++pq) {  // level pairs (0,1) (2,3) (4,5) (6,7)
              uint32_t ra[16], rb[16];
              tmem_ld16(tbase + uint32_t((2 * pq) * BN + c0), ra);
              if (2 * pq + 1 < S) {
                tmem_ld16(tbase + uint32_t((2 * pq + 1) * BN + c0), rb);
              } else {  // 7 digits: no level 7
#pragma unroll
                for (int j = 0; j < 16; ++j) rb[j] = 0u;
              }
              asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const float fa = __uint_as_float(ra[j]), fb = __uint_as_float(rb[j]);
                if (pq < 3) {
                  const int pair = __float2int_rn(fa) * 128 + __float2int_rn(fb);  // exact, |pair| < 2^31
                  if (pq == 0) {
                    th[c0 + j] += (long long)pair * (1ll << 14);
                  } else if (pq == 1) {
                    th[c0 + j] += (long long)pair;
                  } else {
                    const long long x = (long long)pair * (1ll << 14);  // lo part of levels 4, 5
                    th[c0 + j] += x >> 28;
                    rem[c0 + j] += uint32_t(x & 0x0FFFFFFFll);
                  }
                } else {
                  const long long x = intf_to_ll(fmaf(fa, 128.0f, fb));  // levels 6, 7
                  th[c0 + j] += x >> 28;
                  rem[c0 + j] += uint32_t(x & 0x0FFFFFFFll);
                }
              }
              reg_fence16(th, rem);
            }
          }
#pragma unroll
          for (int j = 0; j < HC; ++j) {  // rem < 3 * 2^28 here
            th[j] += (long long)(rem[j] >> 28);
            rem[j] &= 0x0FFFFFFFu;
          }
          asm volatile("tcgen05.fence::before_thread_sync;");
          __syncwarp();
          if (lane == 0) mbar_arrive(acc_empty);
        }
        if (m < P.M && !*(volatile int*)abort_flag) {
          const int ea = P.ea[m];
          const int64_t cbase = map_at(P.cm, m);
#pragma unroll
          for (int j = 0; j < HC; ++j) {
            const int64_t n = n0 + half * HC + j;
            if (n >= P.N) continue;
            double v = fixed_to_double(th[j], rem[j], ea + P.eb[n] - 14 - 21);  // one rounding
            if (P.alpha != 1.0) v *= P.alpha;
            if (P.splits > 1)
              P.work[(int64_t(T.z) * P.M + m) * P.N + n] = v;
            else
              P.C[cbase + map_at(P.cn, n)] = v;
          }
        }
      } else {
        float hi[HC], lo[HC];
#pragma unroll
        for (int j = 0; j < HC; ++j) hi[j] = lo[j] = 0.0f;
        for (int64_t c = 0; c < nchunks; ++c) {
          if (!mbar_wait(acc_full, uint32_t(h & 1), P.err, P.wait_ns)) {
            set_err(P.err, 14);
            *(volatile int*)abort_flag = 1;
            break;
          }
          ++h;
          asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
          for (int q = 0; q < S; ++q) {
            const float scale = __int_as_float((127 - 7 * q) << 23);  // 2^{-7q}
#pragma unroll
            for (int c0 = 0; c0 < HC; c0 += 16) {
              uint32_t r[16];
              tmem_ld16(tmem + (uint32_t(quarter * 32) << 16) + uint32_t(q * BN + half * HC + c0), r);
              asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const float x = __uint_as_float(r[j]) * scale;
                const float s = hi[c0 + j] + x;
                const float bb = s - hi[c0 + j];
                const float e = (hi[c0 + j] - (s - bb)) + (x - bb);
                hi[c0 + j] = s;
                lo[c0 + j] += e;
              }
            }
          }
          asm volatile("tcgen05.fence::before_thread_sync;");
          __syncwarp();
          if (lane == 0) mbar_arrive(acc_empty);
        }
        if (m < P.M && !*(volatile int*)abort_flag) {
          const int ea = P.ea[m];
          const int64_t cbase = map_at(P.cm, m);
#pragma unroll
          for (int j = 0; j < HC; ++j) {
            const int64_t n = n0 + half * HC + j;
            if (n >= P.N) continue;
            const int e = ea + P.eb[n] - 14;
            double v = scaled_to_double(hi[j], e) + scaled_to_double(lo[j], e);  // one FP64 add
            if (P.alpha != 1.0) v *= P.alpha;
            if (P.splits > 1)
              P.work[(int64_t(T.z) * P.M + m) * P.N + n] = v;
            else
              P.C[cbase + map_at(P.cn, n)] = v;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::tcols));
  }
}

// C = sum_z work[z] (deterministic order), same store maps as the GEMM
__global__ void k_oz_reduce(const double* __restrict__ work, int splits, int64_t M, int64_t N, double* __restrict__ C,
                            OzMap cm, OzMap cn, int sym) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= M * N) return;
  const int64_t m = e / N, n = e % N;
  if (sym && n > m) return;
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += work[int64_t(z) * M * N + e];
  C[map_at(cm, m) + map_at(cn, n)] = s;
}

// persistent: one wave of CTAs that loop over the tiles (a tile's epilogue
// then overlaps the next tile's copies and MMAs); else one CTA per tile, the
// hardware scheduler balancing tiles of uneven length (split or triangular
// products) across the SMs.
template <int S, int BN>
void launch_oz(const OzGemmParams& P, bool persistent, cudaStream_t s) {
  using Cfg = OzCfg<S, BN>;
  // the shared-memory attributes belong to the current device: set them, and
  // count the CTAs of this configuration the device holds at once, per device
  static std::atomic<int> resident[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    dev = 0;
  }
  int res = resident[dev].load(std::memory_order_acquire);
  if (!res) {
    cudaFuncSetAttribute(k_oz_gemm<S, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::smem);
    cudaFuncSetAttribute(k_oz_gemm<S, BN>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int nsm = 0, per = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_oz_gemm<S, BN>, Cfg::threads, Cfg::smem);
    cudaGetLastError();
    res = std::max(1, nsm) * std::max(1, per);
    resident[dev].store(res, std::memory_order_release);
  }
  const int64_t ntiles = P.ntn * P.ntm * P.splits;
  const unsigned grid = unsigned(std::max<int64_t>(1, persistent ? std::min<int64_t>(ntiles, res) : ntiles));
  k_oz_gemm<S, BN><<<grid, Cfg::threads, Cfg::smem, s>>>(P);
}

}  // namespace

int64_t oz_tile_bytes(const OzOperand& op) { return op.nrt * op.kst * op.S * int64_t(op.rt) * kBK * 2; }

int64_t oz_tile_elems(int64_t rows, int64_t K, int rt, int S) {
  const int64_t nrt = (rows + rt - 1) / rt, nkt = (K + kBK - 1) / kBK;
  return nrt * nkt * S * int64_t(rt) * kBK;
}

isdf_status oz_alloc(Plan* p, OzOperand& op, int64_t rows, int64_t K, int rt, int S, const char* what) {
  op.rows = rows;
  op.K = K;
  op.tiles = nullptr;
  op.exps = nullptr;
  op.rt = rt;
  op.S = S;
  op.nrt = (rows + rt - 1) / rt;
  op.nkt = (K + kBK - 1) / kBK;
  op.kst = op.nkt;
  isdf_status st = dalloc(p, &op.tiles, size_t(oz_tile_elems(rows, K, rt, S)) * 2, what);
  if (st) return st;
  return dalloc_t(p, &op.exps, size_t(op.nrt * rt), what);
}

void oz_free(OzOperand& op) {
  dfree(op.tiles);
  dfree(op.exps);
  op.tiles = nullptr;
  op.exps = nullptr;
}

void oz_slice(const double* src, int64_t sr, int64_t sk, const double* kw, double mul, OzOperand& op, cudaStream_t s) {
  const bool rowwise = sr >= sk;  // k contiguous: one block per row
  const OzMap rm = oz_stride(sr), km = oz_stride(sk);
  if ((rowwise && op.K >= 4096) || (op.K >= 256 && op.rows <= 8192)) {
    // few long rows: one block per row (a thread per row would stream its row alone)
    k_oz_rowexp_block<<<unsigned(op.rows), 256, 0, s>>>(src, rm, km, op.K, kw, mul, nullptr, op.exps);
  } else {
    k_oz_rowexp_thread<<<unsigned((op.rows + 255) / 256), 256, 0, s>>>(src, rm, km, op.rows, op.K, kw, mul, nullptr,
                                                                        op.exps);
  }
  launch_digits(src, rm, km, kw, mul, nullptr, op, 0, op.nkt * (kBK / 8), rowwise ? 1 : 0, s);
  count_launches(2);
}

void oz_retile(const OzOperand& from, OzOperand& to, cudaStream_t s) {
  const int64_t rows_pad = to.nrt * to.rt;
  const int64_t units = (rows_pad / 8) * to.nkt * to.S;
  const int64_t blocks = std::min<int64_t>((units * 32 + 255) / 256, 152 * 64);
  k_oz_retile<<<unsigned(std::max<int64_t>(blocks, 1)), 256, 0, s>>>(
      static_cast<const __nv_bfloat16*>(from.tiles), from.rt, from.kst, static_cast<__nv_bfloat16*>(to.tiles), to.rt,
      to.kst, to.S, from.rows, rows_pad, to.nkt);
  cudaMemcpyAsync(to.exps, from.exps, size_t(to.rows) * sizeof(int), cudaMemcpyDeviceToDevice, s);
  count_launches(1);
}

void oz_slice_ex(const double* src, int64_t sr, int64_t sk, const int* ridx, OzOperand& op, int64_t kg0, int64_t kg1,
                 bool exps_ready, cudaStream_t s) {
  if (op.rows <= 0 || kg1 <= kg0) return;
  const bool rowwise = sr >= sk;
  const OzMap rm = oz_stride(sr), km = oz_stride(sk);
  if (!exps_ready) {
    // few long rows (a gathered set of rows with large K): one block per row
    if ((rowwise && op.K >= 4096) || (op.K >= 256 && op.rows <= 8192))
      k_oz_rowexp_block<<<unsigned(op.rows), 256, 0, s>>>(src, rm, km, op.K, nullptr, 1.0, ridx, op.exps);
    else
      k_oz_rowexp_thread<<<unsigned((op.rows + 255) / 256), 256, 0, s>>>(src, rm, km, op.rows, op.K, nullptr, 1.0,
                                                                          ridx, op.exps);
    count_launches(1);
  }
  launch_digits(src, rm, km, nullptr, 1.0, ridx, op, kg0, kg1 - kg0, rowwise ? 1 : 0, s);
  count_launches(1);
}

// S levels x BN columns of tensor memory: 5 x 48 (two CTAs per SM), 6 x 64, 7 x 48, 8 x 48
int oz_bn(int S) { return S == 6 ? 64 : 48; }

void oz_gemm(const OzOperand& A, const OzOperand& B, double* C, int64_t ldc, int trans, double alpha, int tri, int sym,
             int splits, double* work, int* err, cudaStream_t s) {
  OzGemmParams P;
  P.A = static_cast<const __nv_bfloat16*>(A.tiles);
  P.B = static_cast<const __nv_bfloat16*>(B.tiles);
  P.ea = A.exps;
  P.eb = B.exps;
  P.M = A.rows;
  P.N = B.rows;
  P.nkt = A.nkt;
  P.akst = A.kst > 0 ? A.kst : A.nkt;
  P.bkst = B.kst > 0 ? B.kst : B.nkt;
  P.tri = tri;
  P.sym = sym;
  P.splits = splits < 1 ? 1 : splits;
  P.C = C;
  P.cm = trans ? oz_stride(1) : oz_stride(ldc);
  P.cn = trans ? oz_stride(ldc) : oz_stride(1);
  P.alpha = alpha;
  P.work = work;
  P.err = err;
  // host-side fault injection (ISDF_FAULT=oz_wait): every pipeline wait gives
  // up at once, so the launch takes its error path (error code, copies and
  // MMAs in flight completed, tensor memory freed) and the call reports
  // ISDF_ERR_TIMEOUT; nothing faults or hangs
  const char* fault = std::getenv("ISDF_FAULT");
  P.wait_ns = (fault && std::strcmp(fault, "oz_wait") == 0) ? 0ull : kWaitNs;
  P.ntm = A.nrt;
  P.ntn = B.nrt;
  // Persistent CTAs pay off where a tile's epilogue is long against its
  // main loop: the exact 8-digit epilogue over short K.  Measured on
  // 131072 x 48 x 512 (8 digits): 291 -> 213 us; with 5 digits (two CTAs
  // per SM already overlap their epilogues) and on split or triangular
  // products one CTA per tile is faster.
  const bool persistent = A.S >= 7 && P.splits == 1 && !P.sym && P.tri == 0 && P.nkt * kBK <= 4096;
  if (A.S == 5)
    launch_oz<5, 48>(P, persistent, s);
  else if (A.S == 8)
    launch_oz<8, 48>(P, persistent, s);
  else if (A.S == 7)
    launch_oz<7, 48>(P, persistent, s);
  else
    launch_oz<6, 64>(P, persistent, s);
  count_launches(1);
  if (P.splits > 1) {
    const int64_t tot = A.rows * B.rows;
    k_oz_reduce<<<unsigned((tot + 255) / 256), 256, 0, s>>>(work, P.splits, A.rows, B.rows, C, P.cm, P.cn, sym);
    count_launches(1);
  }
}

// ---------------------------------------------------------------- split-K autotuner
//
// The one free launch parameter of a product shape is its split-K factor
// (how many CTAs share one output tile's k range).  On the first product of
// a shape (rows of A, rows of B, k tiles, digits, symmetric or not) outside
// any graph capture, every admissible candidate runs on the real operands
// (one warm-up run, then one timed run per candidate, CUDA events on the
// product's stream) and the fastest is cached for the process; the heuristic's choice
// is among the candidates, and the chosen one runs last so C holds its
// result.  Candidates whose split-K partials would exceed 2 GiB are skipped.

namespace {
struct TuneKey {
  int64_t M, N, nkt;
  int S, sym, trans;
  bool operator<(const TuneKey& o) const {
    return std::tie(M, N, nkt, S, sym, trans) < std::tie(o.M, o.N, o.nkt, o.S, o.sym, o.trans);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, float>> g_tune;  // shape -> (splits, ms)
}  // namespace

int oz_tuned_splits(Plan* p, const OzOperand& A, const OzOperand& B, double* C, int64_t ldc, int trans, int sym,
                    int heuristic, cudaStream_t s) {
  const TuneKey key{A.rows, B.rows, A.nkt, A.S, sym, trans};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second.first;
  }
  if ((p && p->capturing) || std::getenv("ISDF_NO_AUTOTUNE")) return heuristic;
  std::vector<int> cand;
  for (int c : {1, 2, 4, 8, 16, 32, 64})
    if (c <= std::max<int64_t>(1, A.nkt)) cand.push_back(c);
  if (std::find(cand.begin(), cand.end(), heuristic) == cand.end()) cand.push_back(heuristic);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int* err = p ? p->d_ozerr : nullptr;
  int best = heuristic;
  float best_ms = 1e30f;
  for (int c : cand) {
    double* work = nullptr;
    const size_t wbytes = c > 1 ? sizeof(double) * size_t(c) * A.rows * B.rows : 0;
    if (wbytes > (size_t(2) << 30)) continue;
    if (wbytes && cudaMallocAsync(reinterpret_cast<void**>(&work), wbytes, s) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    float ms = 1e30f;
    for (int rep = (c == cand.front() ? 0 : 1); rep < 2; ++rep) {  // one warm-up run before the first candidate
      cudaEventRecord(e0, s);
      oz_gemm(A, B, C, ldc, trans, 1.0, 0, sym, c, work, err, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float t = 0.0f;
      if (rep > 0 && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) ms = std::min(ms, t);
    }
    if (work) cudaFreeAsync(work, s);
    if (ms < best_ms) best_ms = ms, best = c;
  }
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[key] = {best, best_ms};
  return best;
}

std::string oz_tune_json() {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  std::string o = "[";
  for (const auto& kv : g_tune) {
    if (o.size() > 1) o += ",";
    o += "{\"M\":" + std::to_string(kv.first.M) + ",\"N\":" + std::to_string(kv.first.N) +
         ",\"k_tiles\":" + std::to_string(kv.first.nkt) + ",\"digits\":" + std::to_string(kv.first.S) +
         ",\"sym\":" + std::to_string(kv.first.sym) + ",\"splits\":" + std::to_string(kv.second.first) +
         ",\"ms\":" + std::to_string(kv.second.second) + "}";
  }
  return o + "]";
}

// ---------------------------------------------------------------- fixed scratch
//
// The variant below runs the same slicing and GEMM kernels, but its scratch
// lives in one file-scope device array instead of memory from cudaMalloc.
// Every GPU that loads the library holds this array until the process exits.

constexpr size_t kStaticScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_gemm_static_scratch[kStaticScratchBytes];

namespace {

std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {nullptr};

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

size_t gemm_noalloc_capacity() { return kStaticScratchBytes; }

isdf_status gemm_noalloc(const double* A, const double* B, double* C, int64_t M, int64_t N, int64_t K, int64_t lda,
                         int64_t ldb, int64_t ldc, double alpha, int slices, cudaStream_t s, std::string& why) {
  // bound every extent by the array before any size arithmetic: with each of
  // M, N, K at most the array's byte count the products below cannot overflow
  const int64_t cap = int64_t(kStaticScratchBytes);
  if (M > cap || N > cap || K > cap || M * K > cap || N * K > cap) {
    why = "isdf_gemm_f64_noalloc: operands of " + std::to_string(M) + " x " + std::to_string(K) + " and " +
          std::to_string(N) + " x " + std::to_string(K) + " exceed what the static array holds (" +
          std::to_string(kStaticScratchBytes) + " bytes)";
    return ISDF_ERR_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    why = "no current CUDA device";
    return ISDF_ERR_CUDA;
  }
  unsigned char* base = nullptr;
  {
    // set-up once per device, with that device current: the array's name is
    // a host-side stand-in, its device address comes from the runtime
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_gemm_static_scratch);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        why = std::string("cudaGetSymbolAddress of the static scratch failed: ") + cudaGetErrorString(e);
        return ISDF_ERR_CUDA;
      }
      g_static_addr[dev] = ptr;
    }
    base = static_cast<unsigned char*>(g_static_addr[dev]);
  }
  OzOperand a, b;
  a.rows = M, a.K = K, a.rt = 128, a.S = slices, a.nrt = (M + 127) / 128, a.nkt = (K + kBK - 1) / kBK, a.kst = a.nkt;
  b.rows = N, b.K = K, b.rt = oz_bn(slices), b.S = slices, b.nrt = (N + b.rt - 1) / b.rt, b.nkt = a.nkt, b.kst = b.nkt;
  const size_t ta = round256(size_t(oz_tile_elems(M, K, a.rt, slices)) * 2);
  const size_t ea = round256(sizeof(int) * size_t(a.nrt * a.rt));
  const size_t tb = round256(size_t(oz_tile_elems(N, K, b.rt, slices)) * 2);
  const size_t eb = round256(sizeof(int) * size_t(b.nrt * b.rt));
  const size_t need = ta + ea + tb + eb + 256;
  if (need > kStaticScratchBytes) {
    why = "isdf_gemm_f64_noalloc needs " + std::to_string(need) + " bytes of scratch; the static array holds " +
          std::to_string(kStaticScratchBytes);
    return ISDF_ERR_ARG;
  }
  a.tiles = base;
  a.exps = reinterpret_cast<int*>(base + ta);
  b.tiles = base + ta + ea;
  b.exps = reinterpret_cast<int*>(base + ta + ea + tb);
  int* err = reinterpret_cast<int*>(base + ta + ea + tb + eb);
  // the array keeps the previous call's contents: the error word must start at
  // zero; every slice byte and every scale read below is rewritten first.
  // Clear any stale launch error so the check after the launches sees ours.
  cudaGetLastError();
  if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    why = "cudaMemsetAsync of the error word failed";
    return ISDF_ERR_CUDA;
  }
  oz_slice(A, lda, 1, nullptr, 1.0, a, s);
  oz_slice(B, ldb, 1, nullptr, 1.0, b, s);
  oz_gemm(a, b, C, ldc, 0, alpha, 0, 0, 1, nullptr, err, s);
  // a launch that could not start (configuration, resources) is reported here
  // and nowhere else: the copy below would succeed with C unwritten
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    why = std::string("isdf_gemm_f64_noalloc: launch failed: ") + cudaGetErrorString(e);
    return ISDF_ERR_CUDA;
  }
  int herr = 0;
  e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    why = std::string("isdf_gemm_f64_noalloc: ") + cudaGetErrorString(e);
    return ISDF_ERR_CUDA;
  }
  if (herr) {
    why = "isdf_gemm_f64_noalloc: tensor-core pipeline wait expired (code " + std::to_string(herr) + ")";
    return ISDF_ERR_TIMEOUT;
  }
  return ISDF_OK;
}

}  // namespace isdf
