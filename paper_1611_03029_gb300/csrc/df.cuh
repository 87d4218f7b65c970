// Double-float arithmetic on the FP32 pipes: a value is the unevaluated sum
// hi + lo of two floats (about 48 significant bits).  Built from the
// error-free transformations TwoSum (Knuth) and FMA-based TwoProd (Dekker's
// product with a fused multiply-add); every operation uses the _rn
// intrinsics so that the compiler cannot contract or reassociate them.
#pragma once

namespace mfp {
namespace {

struct df {
  float h, l;
};

__device__ __forceinline__ df df_make(float h, float l = 0.f) {
  df r;
  r.h = h;
  r.l = l;
  return r;
}

// s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df_make(s, e);
}

// s + e = a + b exactly when |a| >= |b| (Dekker's Fast2Sum)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return df_make(s, e);
}

__device__ __forceinline__ df operator+(df a, df b) {
  df s = two_sum(a.h, b.h);
  const float e = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  return fast_two_sum(s.h, e);
}

__device__ __forceinline__ df operator-(df a) { return df_make(-a.h, -a.l); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return fast_two_sum(p, e);
}

// multiplication by a power of two is exact
__device__ __forceinline__ df df_scale2(df a, float pow2) {
  return df_make(__fmul_rn(a.h, pow2), __fmul_rn(a.l, pow2));
}

// Accumulator of a dot product: (h, l) unnormalised, h carries the TwoSum
// chain of the leading product parts, l the collected rounding errors.
struct dacc {
  float h, l;
};

__device__ __forceinline__ dacc acc_first(float ah, float al, float bh,
                                          float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  dacc r;
  r.h = p;
  r.l = e;
  return r;
}

__device__ __forceinline__ void acc_mac(dacc& s, float ah, float al, float bh,
                                        float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  const float t = __fadd_rn(s.h, p);
  const float bv = __fsub_rn(t, s.h);
  const float er =
      __fadd_rn(__fsub_rn(s.h, __fsub_rn(t, bv)), __fsub_rn(p, bv));
  s.l = __fadd_rn(s.l, __fadd_rn(e, er));
  s.h = t;
}

__device__ __forceinline__ void acc_add(dacc& s, df b) {
  const float t = __fadd_rn(s.h, b.h);
  const float bv = __fsub_rn(t, s.h);
  const float er =
      __fadd_rn(__fsub_rn(s.h, __fsub_rn(t, bv)), __fsub_rn(b.h, bv));
  s.l = __fadd_rn(s.l, __fadd_rn(b.l, er));
  s.h = t;
}

__device__ __forceinline__ df acc_get(dacc s) { return two_sum(s.h, s.l); }

// float64 -> double-float with integer operations only (the conversion
// instructions run on the 2-per-clock FP64 pipe): hi keeps the sign, the
// exponent and the top 23 mantissa bits (truncation), lo the next 23 bits,
// built exactly as q * 2^(e-1069) via the 2^23 magic constant.  Exact to
// 2^-46 relative for 2^-80 <= |x| < 2^128; smaller values keep only hi
// (values below 2^-126 become 0), larger ones saturate to +-inf.
__device__ __forceinline__ df df_from_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int hi32 = (unsigned int)(b >> 32);
  const unsigned int sign = hi32 & 0x80000000u;
  const int e = (int)((hi32 >> 20) & 0x7FFu);
  const int fe = e - 896;
  const unsigned int mh = (unsigned int)(b >> 29) & 0x7FFFFFu;
  const unsigned int q = (unsigned int)(b >> 6) & 0x7FFFFFu;
  const int se = e - 942;
  float h, l;
  if (fe >= 1 && fe <= 254) {
    h = __uint_as_float(sign | ((unsigned int)fe << 23) | mh);
    const float qf =
        __fsub_rn(__uint_as_float(0x4B000000u | q), 8388608.0f);  // exact
    l = se >= 1 ? __fmul_rn(qf, __uint_as_float((unsigned int)se << 23))
                : 0.f;
    l = sign ? -l : l;
  } else {
    h = fe > 254 ? __uint_as_float(sign | 0x7F800000u) : 0.f;
    l = 0.f;
  }
  return df_make(h, l);
}

// float -> float64 exactly with integer operations (subnormal floats -> 0)
__device__ __forceinline__ double float_to_double_exact(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xFFu;
  const unsigned int de = e == 255u ? 2047u : e + 896u;  // inf / nan kept
  const unsigned long long bits =
      ((unsigned long long)(u & 0x80000000u) << 32) |
      ((unsigned long long)de << 52) |
      ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return e == 0 ? 0.0 : __longlong_as_double(bits);
}

// double-float -> float64: one FP64 addition
__device__ __forceinline__ double df_to_double(df a) {
  return __dadd_rn(float_to_double_exact(a.h), float_to_double_exact(a.l));
}

}  // namespace
}  // namespace mfp
