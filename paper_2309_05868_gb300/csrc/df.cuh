// df.cuh -- pair ("double-float") arithmetic on FP32 pipes and FP64 <-> pair conversion
// by integer bit manipulation (no FP64 instruction).  Dekker's (1971) pair arithmetic with
// Knuth's TwoSum and the FMA-based TwoProd.
#pragma once

#include "common.cuh"

namespace rq {

// ---------------------------------------------------------------------------------------
// FP64 -> (hi, lo) without FP64 instructions.  hi keeps the top 24 significant bits
// (truncated), lo is the remaining 29-bit tail rounded to FP32 by an integer->float
// conversion and scaled by an exactly representable power of two.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float2 d2df(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7ff);  // biased FP64 exponent
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFULL;
  if (e <= 896) return make_float2(__uint_as_float(sign), 0.0f);           // |x| < 2^-126
  if (e >= 1151) return make_float2(__uint_as_float(sign | 0x7f800000u), 0.0f);  // overflow
  const float hi = __uint_as_float(sign | ((unsigned int)(e - 896) << 23) | (unsigned int)(mant >> 29));
  const unsigned int tail = (unsigned int)(mant & 0x1FFFFFFFULL);  // 29 bits, weight 2^(e-1075)
  const int pe = e - 1075 + 127;                                    // biased exponent of 2^(e-1075)
  float lo = 0.0f;
  if (tail != 0 && pe > 0) {
    lo = __uint2float_rn(tail) * __uint_as_float((unsigned int)pe << 23);
    lo = __uint_as_float(__float_as_uint(lo) | sign);
  }
  return make_float2(hi, lo);
}

// (hi, lo) -> FP64 without FP64 instructions: assemble hi's FP64 bit pattern and add lo's
// significand, aligned to hi's FP64 ulp (truncated below it), in 64-bit integer arithmetic.
__device__ __forceinline__ double df2d(float hi, float lo) {
  const unsigned int hb = __float_as_uint(hi), lb = __float_as_uint(lo);
  const int eh = (int)((hb >> 23) & 0xff);
  if (eh == 0) return __longlong_as_double((long long)((unsigned long long)(hb >> 31) << 63));
  if (eh == 255) return __longlong_as_double((long long)(((unsigned long long)(hb >> 31) << 63) | 0x7ff0000000000000ULL));
  long long M = (long long)((1ULL << 52) | ((unsigned long long)(hb & 0x7fffff) << 29));
  int E = eh - 127;  // value = M * 2^(E - 52)
  const int el = (int)((lb >> 23) & 0xff);
  if (el != 0 && el != 255) {
    const long long ml = (long long)((1u << 23) | (lb & 0x7fffff));  // value = ml * 2^(el-127-23)
    const int s = (el - 127 - 23) - (E - 52);                       // shift into hi's units
    long long add = 0;
    if (s >= 0)
      add = (s < 40) ? (ml << s) : 0;
    else
      add = (-s < 63) ? (ml >> (-s)) : 0;
    if ((lb >> 31) != (hb >> 31)) add = -add;
    M += add;
    if (M >= (1LL << 53)) { M >>= 1; ++E; }
    while (M > 0 && M < (1LL << 52)) { M <<= 1; --E; }
  }
  if (M <= 0) return 0.0;
  const unsigned long long out = ((unsigned long long)(hb >> 31) << 63) |
                                 ((unsigned long long)(E + 1023) << 52) |
                                 ((unsigned long long)M & 0xFFFFFFFFFFFFFULL);
  return __longlong_as_double((long long)out);
}

// s -= a * b with s kept as an unnormalised pair (sh, sl).
__device__ __forceinline__ void df_fms(float &sh, float &sl, float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float t = __fsub_rn(sh, p);
  const float z = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(-p, z));
  sl = __fadd_rn(__fsub_rn(sl, e), err);
  sh = t;
}

// s += a * b.
__device__ __forceinline__ void df_fma(float &sh, float &sl, float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float t = __fadd_rn(sh, p);
  const float z = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(p, z));
  sl = __fadd_rn(__fadd_rn(sl, e), err);
  sh = t;
}

// s[c] -= a * b[c] for c < N, written stage by stage across the N independent updates so
// their dependent chains interleave (same arithmetic as N calls of df_fms).
template <int N>
__device__ __forceinline__ void df_fms_n(float (&sh)[N], float (&sl)[N], float2 a, const float2 (&b)[N]) {
  float p[N], e[N], t[N], z[N];
#pragma unroll
  for (int c = 0; c < N; ++c) p[c] = a.x * b[c].x;
#pragma unroll
  for (int c = 0; c < N; ++c) e[c] = __fmaf_rn(a.x, b[c].x, -p[c]);
#pragma unroll
  for (int c = 0; c < N; ++c) t[c] = __fsub_rn(sh[c], p[c]);
#pragma unroll
  for (int c = 0; c < N; ++c) e[c] = __fmaf_rn(a.x, b[c].y, e[c]);
#pragma unroll
  for (int c = 0; c < N; ++c) z[c] = __fsub_rn(t[c], sh[c]);
#pragma unroll
  for (int c = 0; c < N; ++c) e[c] = __fmaf_rn(a.y, b[c].x, e[c]);
#pragma unroll
  for (int c = 0; c < N; ++c) {
    const float err = __fadd_rn(__fsub_rn(sh[c], __fsub_rn(t[c], z[c])), __fsub_rn(-p[c], z[c]));
    sl[c] = __fadd_rn(__fsub_rn(sl[c], e[c]), err);
    sh[c] = t[c];
  }
}

// s[c] -= a[c] * b[c] for c < N, stage by stage across the N independent updates.
template <int N>
__device__ __forceinline__ void df_fms_nn(float (&sh)[N], float (&sl)[N], const float2 (&a)[N],
                                          const float2 (&b)[N]) {
  float p[N], e[N], t[N], z[N];
#pragma unroll
  for (int c = 0; c < N; ++c) p[c] = a[c].x * b[c].x;
#pragma unroll
  for (int c = 0; c < N; ++c) e[c] = __fmaf_rn(a[c].x, b[c].x, -p[c]);
#pragma unroll
  for (int c = 0; c < N; ++c) t[c] = __fsub_rn(sh[c], p[c]);
#pragma unroll
  for (int c = 0; c < N; ++c) e[c] = __fmaf_rn(a[c].x, b[c].y, e[c]);
#pragma unroll
  for (int c = 0; c < N; ++c) z[c] = __fsub_rn(t[c], sh[c]);
#pragma unroll
  for (int c = 0; c < N; ++c) e[c] = __fmaf_rn(a[c].y, b[c].x, e[c]);
#pragma unroll
  for (int c = 0; c < N; ++c) {
    const float err = __fadd_rn(__fsub_rn(sh[c], __fsub_rn(t[c], z[c])), __fsub_rn(-p[c], z[c]));
    sl[c] = __fadd_rn(__fsub_rn(sl[c], e[c]), err);
    sh[c] = t[c];
  }
}

// (ah + al) += (bh + bl), accurate pair addition (two TwoSums, renormalised).
__device__ __forceinline__ void df_add(float &ah, float &al, float bh, float bl) {
  const float s = __fadd_rn(ah, bh);
  const float v = __fsub_rn(s, ah);
  float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, v)), __fsub_rn(bh, v));
  const float t = __fadd_rn(al, bl);
  const float w = __fsub_rn(t, al);
  const float f = __fadd_rn(__fsub_rn(al, __fsub_rn(t, w)), __fsub_rn(bl, w));
  e = __fadd_rn(e, t);
  float h = __fadd_rn(s, e);
  float l = __fsub_rn(e, __fsub_rn(h, s));
  l = __fadd_rn(l, f);
  ah = __fadd_rn(h, l);
  al = __fsub_rn(l, __fsub_rn(ah, h));
}

__device__ __forceinline__ float2 df_norm(float sh, float sl) {
  const float h = __fadd_rn(sh, sl);
  return make_float2(h, __fsub_rn(sl, __fsub_rn(h, sh)));
}

// (sh + sl) * r, normalised.
__device__ __forceinline__ float2 df_mul(float sh, float sl, float2 r) {
  const float p = sh * r.x;
  float e = __fmaf_rn(sh, r.x, -p);
  e = __fmaf_rn(sh, r.y, e);
  e = __fmaf_rn(sl, r.x, e);
  return df_norm(p, e);
}


// 2^e * FP64 value, by adding e to the exponent field (integer ops); the value must be normal
// and stay normal.
__device__ __forceinline__ double scale_pow2(double v, int e) {
  const long long b = __double_as_longlong(v);
  if ((b & 0x7FF0000000000000LL) == 0) return 0.0;
  return __longlong_as_double(b + ((long long)e << 52));
}

}  // namespace rq
