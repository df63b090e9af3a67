// gv_plus_stat.cuh -- VEGAS+ (Lepage, J. Comput. Phys. 439 (2021) 110386)
// statistics of one hypercube from its sums over its events: the sample
// variance v_h of F = J g, v_h / n_h (summed over the hypercubes and divided
// by nh^2: sigma_k^2) and the allocation weight v_h^(beta/2).  The
// stratified fill forms them for every hypercube whose events lie in one
// tile, and the finishing kernel for the hypercubes that cross a tile
// boundary; both call these functions, so every hypercube's values are the
// same wherever they are formed.
#pragma once
#include "gv_common.cuh"

// v^(j/8) (beta = j/4) from correctly rounded operations only: v = t 2^(8q)
// with t in [1/2, 128) rounded to FP32, three FP32 square roots, j - 1 FP32
// products, and 2^(q j) exactly.
// The exponent split, the FP32 rounding of t, the widening of the FP32
// result and the final scaling are exact bit operations here (frexp, a
// conversion to nearest, a widening and ldexp, written with integers: their
// library and hardware forms run on the FP64 pipe, which this chip has little
// of); a subnormal v takes the library path.
__device__ __forceinline__ double gv_plus_weight(double v, int j) {
  const long long bits = __double_as_longlong(v);
  if (j == 0) return 1.0;
  if (bits <= 0) return 0.0;  // +0 (v is finite and not negative)
  const int eb = (int)(bits >> 52);  // biased exponent
  int e, q, r;
  unsigned tb;  // FP32 bits of t = m 2^r in [1/2, 128), m in [1/2, 1)
  if (eb == 0) {
    const double m = frexp(v, &e);
    q = e >= 0 ? e / 8 : -((-e + 7) / 8);
    r = e - 8 * q;
    tb = __float_as_uint(__double2float_rn(ldexp(m, r)));
  } else {
    e = eb - 1022;  // v = m 2^e
    q = e >= 0 ? e / 8 : -((-e + 7) / 8);
    r = e - 8 * q;
    // round the 52-bit mantissa to 23 bits, to nearest, ties to even (a carry
    // runs into the exponent, as it should)
    const unsigned long long M = (unsigned long long)bits & 0x000FFFFFFFFFFFFFull;
    tb = ((unsigned)(126 + r) << 23) | (unsigned)(M >> 29);
    const unsigned half = (unsigned)(M >> 28) & 1u;
    const unsigned sticky = (M & ((1ull << 28) - 1ull)) != 0ull ? 1u : 0u;
    tb += half & (sticky | (tb & 1u));
  }
  const float t = __uint_as_float(tb);
  const float y = __fsqrt_rn(__fsqrt_rn(__fsqrt_rn(t)));
  float p = y;
  for (int k = 1; k < j; ++k) p = __fmul_rn(p, y);
  // (double)p 2^(q j): p is normal and so is the product (|q j| <= 540)
  const unsigned pb = __float_as_uint(p);
  const long long db = ((long long)(((pb >> 23) & 0xFFu) - 127 + 1023) << 52) |
                       ((long long)(pb & 0x7FFFFFu) << 29);
  return __longlong_as_double(db + ((long long)(q * j) << 52));
}

// (1/n, 1/(n - 1)) beyond the tables (kept out of line, so that the common
// path does not carry two FP64 divisions; returned by value, which keeps
// both reciprocals out of local memory on the common path)
static __device__ __noinline__ double2 gv_plus_recips(double n) {
  return make_double2(1.0 / n, 1.0 / (n - 1.0));
}

// Hypercube statistics from s1 = sum F, s2 = sum F^2 over its m >= 2 events:
// v = (s2 - s1^2/m)/(m - 1) (0 where rounding makes it negative), v/m, and
// the weight v^(beta/2) with beta = beta_j/4; 1/m and 1/(m - 1) from the
// table inv (entries below GV_PLUS_NTAB) or divided out.
struct GvPlusStat {
  double v, vn, w;
};
__device__ __forceinline__ GvPlusStat gv_plus_stat(double s1, double s2, int m, const double* inv,
                                                   int beta_j) {
  double inv_n, inv_m1;
  if (m < GV_PLUS_NTAB) {
    inv_n = __ldg(inv + m);
    inv_m1 = __ldg(inv + m - 1);
  } else {
    const double2 rc = gv_plus_recips((double)m);
    inv_n = rc.x;
    inv_m1 = rc.y;
  }
  double v = (s2 - s1 * s1 * inv_n) * inv_m1;
  v = __double_as_longlong(v) > 0ll ? v : 0.0;  // negative (rounding) or -0 -> 0
  return GvPlusStat{v, v * inv_n, gv_plus_weight(v, beta_j)};
}
