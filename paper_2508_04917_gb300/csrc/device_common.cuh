// Device helpers: shared-memory mbarriers, the fixed reduction order,
// precision conversions. sm_103a only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace ilu0dd {

// Shared-memory mbarriers at CTA scope: arrive has release semantics,
// try_wait acquire semantics.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// True once the phase with the given parity has completed. The thread may be
// suspended for a hardware-chosen interval (woken when the phase completes)
// before a false return.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ float bf16_to_f32(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

// Factor loads from the packed stream (read-only path), converted to the
// apply's compute type.
template <typename TF>
struct FactorLoad;
template <>
struct FactorLoad<double> {
  using compute = double;
  __device__ __forceinline__ static double getg(const unsigned char* p) {
    return __ldg(reinterpret_cast<const double*>(p));
  }
};
template <>
struct FactorLoad<float> {
  using compute = float;
  __device__ __forceinline__ static float getg(const unsigned char* p) {
    return __ldg(reinterpret_cast<const float*>(p));
  }
};
struct bf16s {
  uint16_t v;
};
template <>
struct FactorLoad<bf16s> {
  using compute = float;
  __device__ __forceinline__ static float getg(const unsigned char* p) {
    return bf16_to_f32(__ldg(reinterpret_cast<const unsigned short*>(p)));
  }
};

// ---- double-float arithmetic (the DF64 factor mode) -----------------------
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits, computed on the FP32 pipe (this GPU's FP64 pipe
// runs at 1/55 of its FP32 rate). Built from error-free transformations: the
// exact error of a float product, fma(a, b, -a*b); Knuth's two-sum, exact for
// any a, b; Dekker's fast two-sum, exact when |a| >= |b|. Every step uses the
// explicitly rounded intrinsics, so no contraction can break them.
struct df64s {  // storage of one factor entry: hi then lo (8 bytes)
  float hi, lo;
};
struct df64 {
  float hi, lo;
  __device__ __forceinline__ df64() {}
  __device__ __forceinline__ df64(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ explicit df64(int z) : hi((float)z), lo(0.f) {}
};

// Nearest float pair of a double: hi = fl(v), lo = fl(v - hi) (v - hi is exact).
__device__ __forceinline__ df64 df_from_double(double v) {
  const float h = __double2float_rn(v);
  return df64(h, __double2float_rn(v - (double)h));
}
__device__ __forceinline__ double df_to_double(df64 a) { return (double)a.hi + (double)a.lo; }

// The same two conversions by integer and FP32 operations, from the bit
// layouts of IEEE 754 binary64 and binary32, for the apply's load and store of
// its subdomain vector: on this GPU every FP64 operation, conversions
// included, takes the FP64 pipe, which the DF64 apply otherwise leaves idle
// (measured: the load and store phases cost 13 % of the DF64 apply at 160^3).
// They give the FP64 operations' bits exactly where every intermediate is a
// normal number and return false elsewhere (zero, subnormal, infinite or NaN
// values, exponents at the ends of the ranges), where the caller uses the FP64
// operations.

// A float from its integer bits' sum x < 2^23 (exact: 2^23 + x - 2^23).
__device__ __forceinline__ float small_uint_to_float(uint32_t x) {
  return __fsub_rn(__uint_as_float(0x4B000000u | x), 8388608.0f);
}

// df_from_double(v * 2^-k): hi = v * 2^-k rounded to nearest float (ties to
// even), lo = (v * 2^-k - hi) rounded to nearest float.
__device__ __forceinline__ bool df_from_double_scaled_bits(double v, int k, df64* out) {
  const uint64_t u = (uint64_t)__double_as_longlong(v);
  const uint32_t h32 = (uint32_t)(u >> 32), l32 = (uint32_t)u;
  const int eb = (int)((h32 >> 20) & 0x7FFu);  // biased binary64 exponent of v
  const int e = eb - k;                         // ... of v * 2^-k (exact while it stays normal)
  const int E = e - 896;                        // binary32 biased exponent (bias 127 = 1023 - 896)
  if (eb == 0 || eb == 0x7FF || E < 1 || E > 253) return false;
  const uint32_t sign = h32 & 0x80000000u;
  const uint32_t m23 = ((h32 & 0xFFFFFu) << 3) | (l32 >> 29);  // the 23 stored bits binary32 keeps
  const uint32_t rest = l32 & 0x1FFFFFFFu;                      // the 29 bits it drops
  const bool up = rest > 0x10000000u || (rest == 0x10000000u && (m23 & 1u));
  // rounding up carries into the exponent field when m23 is all ones
  out->hi = __uint_as_float(sign | ((((uint32_t)E << 23) | m23) + (up ? 1u : 0u)));
  // v * 2^-k - hi = +-R units of 2^(e - 1075): the dropped bits, or their
  // complement to 2^29 when hi was rounded up (R <= 2^28 either way)
  const uint32_t R = up ? 0x20000000u - rest : rest;
  if (R == 0) {
    out->lo = 0.0f;
    return true;
  }
  const int se = e - 1075;
  if (se < -126) return false;  // lo would not be a normal float
  // RNE(R) as a float: R = a 2^16 + b, a and b exact, one rounding in the fma
  const float r = __fmaf_rn(small_uint_to_float(R >> 16), 65536.0f, small_uint_to_float(R & 0xFFFFu));
  const float mag = __fmul_rn(r, __uint_as_float((uint32_t)(se + 127) << 23));  // exact: normal result
  out->lo = __uint_as_float(__float_as_uint(mag) ^ (up ? sign ^ 0x80000000u : sign));
  return true;
}

// The binary64 value of a normal binary32 f times 2^k, by its bits (exact),
// when its biased binary64 exponent lies in [min_e, 2046].
__device__ __forceinline__ bool double_from_float_scaled_bits(float f, int k, int min_e, double* out) {
  const uint32_t b = __float_as_uint(f);
  const int E = (int)((b >> 23) & 0xFFu);
  const int e = E + 896 + k;
  if (E == 0 || E == 0xFF || e < min_e || e > 2046) return false;
  const uint64_t bits = ((uint64_t)(b & 0x80000000u) << 32) | ((uint64_t)e << 52) | ((uint64_t)(b & 0x7FFFFFu) << 29);
  *out = __longlong_as_double((long long)bits);
  return true;
}

// df_to_double(a) * 2^k with one FP64 operation (the add) where both floats
// and their scaled values are normal numbers: rounding hi 2^k + lo 2^k once
// gives the bits of rounding hi + lo and scaling by 2^k, since nothing
// leaves the normal range (hi's scaled exponent is kept 64 above the bottom,
// so even a cancelling lo cannot take the sum out of it).
__device__ __forceinline__ double df_to_double_scaled(df64 a, int k) {
  double h, l;
  if (double_from_float_scaled_bits(a.hi, k, 64, &h)) {
    if (a.lo == 0.0f) return h;  // hi + (+-0) = hi for a normal hi
    if (double_from_float_scaled_bits(a.lo, k, 1, &l)) return h + l;
  }
  return df_to_double(a) * ldexp(1.0, k);
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }

// a * b (the lo * lo term, below 2^-48 relative, is dropped)
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float h = __fadd_rn(p, e);
  return df64(h, __fsub_rn(e, __fsub_rn(h, p)));
}

// a * b + c: the product's head and tail as above, two-sum of the head with
// c.hi, then the tails, then a fast two-sum to renormalise.
__device__ __forceinline__ df64 df_fma(df64 a, df64 b, df64 c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float s = __fadd_rn(p, c.hi);
  const float v = __fsub_rn(s, p);
  float t = __fadd_rn(__fsub_rn(p, __fsub_rn(s, v)), __fsub_rn(c.hi, v));
  t = __fadd_rn(t, __fadd_rn(e, c.lo));
  const float h = __fadd_rn(s, t);
  return df64(h, __fsub_rn(t, __fsub_rn(h, s)));
}

// Generic helpers of the apply over its compute types (float, double, df64).
template <typename T>
__device__ __forceinline__ T mac(T a, T b, T c) {  // a * b + c
  return fma(a, b, c);
}
template <>
__device__ __forceinline__ df64 mac<df64>(df64 a, df64 b, df64 c) {
  return df_fma(a, b, c);
}
template <typename T>
__device__ __forceinline__ T shfl(T v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}
template <>
__device__ __forceinline__ df64 shfl<df64>(df64 v, int src) {
  return df64(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
}
template <typename T>
__device__ __forceinline__ T to_compute(double v) {
  return (T)v;
}
template <>
__device__ __forceinline__ df64 to_compute<df64>(double v) {
  return df_from_double(v);
}
__device__ __forceinline__ double to_double(float v) { return (double)v; }
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(df64 v) { return df_to_double(v); }

template <>
struct FactorLoad<df64s> {
  using compute = df64;
  __device__ __forceinline__ static df64 getg(const unsigned char* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return df64(v.x, v.y);
  }
};

// Fixed-order block reduction of kDotTile values, one per thread of a
// kDotTile-thread block: halving sums s[i] += s[i + h], h = 128 .. 1. `buf`
// holds kDotTile doubles of shared memory. Result valid in thread 0.
template <int NV>
__device__ __forceinline__ void tile_halving_sum(double (&q)[NV], double (*buf)[kDotTile]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int v = 0; v < NV; ++v) buf[v][t] = q[v];
  __syncthreads();
#pragma unroll
  for (int h = kDotTile / 2; h >= 32; h >>= 1) {
    if (t < h) {
#pragma unroll
      for (int v = 0; v < NV; ++v) buf[v][t] = buf[v][t] + buf[v][t + h];
    }
    __syncthreads();
  }
  if (t < 32) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      double s = buf[v][t];
#pragma unroll
      for (int h = 16; h >= 1; h >>= 1) {
        double o = __shfl_down_sync(0xffffffffu, s, h);
        s = s + o;  // lanes < h hold s[i] + s[i+h]; others are ignored
      }
      q[v] = s;
    }
  }
}

// Levels h >= kDotTile of the final halving sum for K = m / kDotTile values per
// thread (indices t + k * kDotTile): a halving sum over k, kept in registers.
template <int K, int NV>
__device__ __forceinline__ void fold_strided(const double* const (&part)[NV], double (&q)[NV]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double a[K];
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] = __ldcg(part[v] + t + k * kDotTile);
#pragma unroll
    for (int h = K / 2; h >= 1; h >>= 1) {
#pragma unroll
      for (int k = 0; k < h; ++k) a[k] = a[k] + a[k + h];
    }
    q[v] = a[0];
  }
}

// The same levels for K >= 16 with O(log K) registers, evaluated depth first.
// With R(k, h) the value at index k after the levels of stride >= h,
// R(k, h) = R(k, 2h) + R(k + h, 2h) and R(k, K) = the k-th partial, so the
// result R(0, 1) is built by visiting the partials in bit-reversed order and
// merging each finished pair of equal subtrees, left (smaller index) operand
// first: the same additions on the same operands as the halving loops. Loads
// are issued eight at a time (a compiler barrier between batches) so only a
// few are live at once.
template <int K, int NV>
__device__ __forceinline__ void fold_strided_deep(const double* const (&part)[NV], double (&q)[NV]) {
  constexpr int LOG = K <= 1 ? 0 : K <= 2 ? 1 : K <= 4 ? 2 : K <= 8 ? 3 : K <= 16 ? 4 : K <= 32 ? 5 : 6;
  static_assert((1 << LOG) == K, "K must be a power of two up to 64");
  const int t = threadIdx.x;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double stack[LOG + 1];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      int k = 0;  // bit reversal of j over LOG bits
#pragma unroll
      for (int b = 0; b < LOG; ++b) k |= ((j >> b) & 1) << (LOG - 1 - b);
      double val = __ldcg(part[v] + t + k * kDotTile);
      int l = 0;
#pragma unroll
      for (; l < LOG; ++l) {
        if (!((j >> l) & 1)) break;
        val = stack[l] + val;
      }
      stack[l] = val;
      if ((j & 7) == 7) asm volatile("" ::: "memory");
    }
    q[v] = stack[LOG];
  }
}

// Same for larger K: the partial sums are updated in place in global memory
// (only the block that owns the final reduction runs this).
template <int NV>
__device__ __forceinline__ void fold_strided_global(const double* const (&part)[NV], int64_t K, double (&q)[NV]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double* p = const_cast<double*>(part[v]);
    for (int64_t h = K / 2; h >= 1; h >>= 1)
      for (int64_t k = 0; k < h; ++k)
        p[t + k * kDotTile] = __ldcg(p + t + k * kDotTile) + __ldcg(p + t + (k + h) * kDotTile);
    q[v] = __ldcg(p + t);
  }
}

// Final fixed-order reduction over `m` (power of two) tile partials held in
// global memory, by a kDotTile-thread block: halving sums from h = m/2 down to
// 1. Levels with h >= kDotTile combine indices of equal residue mod kDotTile,
// so each thread finishes them alone; the rest use shared memory. For
// m < kDotTile the partials are padded with zeros to kDotTile: the extra
// levels then add zeros and leave the sums unchanged. Result in thread 0.
template <int NV>
__device__ __forceinline__ void final_halving_sum(const double* const (&part)[NV], int64_t m,
                                                  double (&out)[NV], double (*buf)[kDotTile]) {
  const int t = threadIdx.x;
  double q[NV];
  if (m >= kDotTile) {
    switch (m / kDotTile) {
      case 1: fold_strided<1, NV>(part, q); break;
      case 2: fold_strided<2, NV>(part, q); break;
      case 4: fold_strided<4, NV>(part, q); break;
      case 8: fold_strided<8, NV>(part, q); break;
      case 16: fold_strided_deep<16, NV>(part, q); break;
      case 32: fold_strided_deep<32, NV>(part, q); break;
      case 64: fold_strided_deep<64, NV>(part, q); break;
      default: fold_strided_global<NV>(part, m / kDotTile, q); break;
    }
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = t < m ? __ldcg(part[v] + t) : 0.0;
  }
  tile_halving_sum<NV>(q, buf);
#pragma unroll
  for (int v = 0; v < NV; ++v) out[v] = q[v];
}

}  // namespace ilu0dd
