// gv_ff.cuh -- float-float ("double-float") arithmetic for the grid
// refinement's compression.  A value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.  The
// refinement is a chain of dependent operations; on this chip a dependent
// FP64 operation costs ~120 cycles and an FP32 one a few, so the compression
// ((1 - rho)/(-ln rho))^(3/2) and the slope runs in FP32 pairs, to ~1e-13
// relative, well inside what the grid's edges need.
// The error-free transforms are the published ones: Knuth's TwoSum (The Art
// of Computer Programming, vol. 2, 4.2.2), Dekker's FastTwoSum (Numer. Math.
// 18 (1971) 224), and the product's rounding error from one fused
// multiply-add; the pair operations follow Dekker's and the standard
// double-double algorithms with FP32 in place of FP64.
#pragma once
#include <cstdint>

struct GvFF {
  float hi, lo;
};

// a + b = s + e exactly (any a, b).
__device__ __forceinline__ GvFF gv_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
  return {s, e};
}

// a + b = s + e exactly for |a| >= |b| (or a = 0).
__device__ __forceinline__ GvFF gv_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a b = p + e exactly (no overflow or underflow).
__device__ __forceinline__ GvFF gv_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ GvFF gv_ff_add(GvFF x, GvFF y) {
  GvFF s = gv_two_sum(x.hi, y.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return gv_fast_two_sum(s.hi, e);
}

__device__ __forceinline__ GvFF gv_ff_mul(GvFF x, GvFF y) {
  GvFF p = gv_two_prod(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.lo, p.lo);
  e = __fmaf_rn(x.lo, y.hi, e);
  return gv_fast_two_sum(p.hi, e);
}

__device__ __forceinline__ GvFF gv_ff_mul_f(GvFF x, float f) {
  GvFF p = gv_two_prod(x.hi, f);
  return gv_fast_two_sum(p.hi, __fmaf_rn(x.lo, f, p.lo));
}

// x / y: a quotient q1 of the leading parts, the remainder x - q1 y formed
// exactly enough from a two-product, and one correction term.
__device__ __forceinline__ GvFF gv_ff_div(GvFF x, GvFF y) {
  const float q1 = __fdiv_rn(x.hi, y.hi);
  GvFF p = gv_two_prod(q1, y.hi);
  const float pe = __fmaf_rn(q1, y.lo, p.lo);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p.hi), pe), x.lo);
  return gv_fast_two_sum(q1, __fdiv_rn(r, y.hi));
}

// sqrt x for x > 0: the correctly rounded root of the leading part and one
// Newton correction (x - s^2)/(2 s).
__device__ __forceinline__ GvFF gv_ff_sqrt(GvFF x) {
  const float s = __fsqrt_rn(x.hi);
  GvFF p = gv_two_prod(s, s);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p.hi), p.lo), x.lo);
  return gv_fast_two_sum(s, __fdiv_rn(r, __fmul_rn(2.0f, s)));
}

// A positive double d with 2^-100 < d < 2^20 as a pair, by integer
// operations on its bits: hi = d rounded to 24 bits (nearest, ties to even),
// lo = d - hi (its 29-bit remainder, rounded to 24 bits: the pair keeps 48).
__device__ __forceinline__ GvFF gv_ff_from_double(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int E = (int)((b >> 52) & 0x7FF);
  const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  unsigned long long keep = M >> 29;
  const unsigned rem = (unsigned)(M & 0x1FFFFFFFull);
  if (rem > 0x10000000u || (rem == 0x10000000u && (keep & 1ull))) ++keep;
  const long long R = (long long)M - (long long)(keep << 29);  // in [-2^28, 2^28]
  // d = keep 2^(E - 1046) + R 2^(E - 1075); keep <= 2^24 is exact in FP32
  const float s_hi = __int_as_float((E - 1046 + 127) << 23);
  const float s_lo = __int_as_float((E - 1075 + 64 + 127) << 23);  // times 2^-64 below
  const float hi = __fmul_rn((float)keep, s_hi);
  const float lo = __fmul_rn(__fmul_rn((float)R, s_lo), 0x1p-64f);
  return {hi, lo};
}

__device__ __forceinline__ double gv_ff_to_double(GvFF x) {
  return (double)x.hi + (double)x.lo;  // exact: at most 48 bits
}
