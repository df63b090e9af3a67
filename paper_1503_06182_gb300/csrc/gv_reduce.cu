// gv_reduce.cu -- combination of all events of an iteration and the grid
// optimisation (Section 2.1: the grid optimisation is serial so that it can
// use the results of all events).
//
// gv_reduce_kernel sums the tile partials exactly.  Its grid is (slot blocks
// of 32) x (tile ranges): each CTA owns 32 slots and a range of tiles; its 8
// warps stride over the tiles, align every partial to the largest exponent
// the slot has in the range (channel sums: the tiles' scales; bin sums: the
// bins' own exponents, formed by the fill kernel with order-free atomicMax)
// and add in 192-bit integers; the warps' sums are combined in shared memory
// and published with that exponent.  No sum is formed with atomics.  Integer
// addition is associative, and the alignment depends only on the data and on
// the reduce grid, a function of the tile count alone: the totals do not
// depend on the fill's launch shape or on timing.
//
// Tickets instead of waiting: each CTA publishes its sums and counts itself
// on its block of 32 slots; the CTA that completes a block combines the
// block's sums, rounds them once to FP64 and counts the block on each axis
// its bins belong to.  The CTA whose count completes an axis refines that
// axis at once (Lepage's VEGAS, cited in Section 2.1: smoothing,
// normalisation, compression ((1-rho)/(-ln rho))^alpha, redistribution into
// N equal shares), so the axes are refined in parallel by different CTAs
// while others still reduce; the CTA that completes block 0 (the channel
// sums) records I_k and sigma_k and combines the stage.  No CTA ever waits
// for another.
//
// On this chip a dependent FP64 operation waits ~56-64 cycles, a warp-wide
// FP64 instruction occupies the SM's FP64 pipe for ~19 cycles, and the FP64
// library log takes ~2000 cycles: the serial code here keeps its FP64 chains
// short (reciprocals passed in, a table-driven log, one thread per bin).
#include <algorithm>

#include "gv_combine.cuh"
#include "gv_ff.cuh"
#include "gv_integrands.cuh"

struct u192 {
  unsigned long long l0, l1, l2;
};

__device__ __forceinline__ void add192(u192& r, const u192& x) {
  const unsigned long long a0 = r.l0 + x.l0;
  const unsigned long long c0 = a0 < r.l0 ? 1ull : 0ull;
  const unsigned long long t1 = r.l1 + x.l1;
  const unsigned long long c1 = t1 < r.l1 ? 1ull : 0ull;
  const unsigned long long a1 = t1 + c0;
  const unsigned long long c1b = a1 < t1 ? 1ull : 0ull;
  r.l0 = a0;
  r.l1 = a1;
  r.l2 = r.l2 + x.l2 + c1 + c1b;
}

// Arithmetic shift right of a 192-bit two's complement value.
__device__ __forceinline__ u192 sar192(u192 v, int s) {
  const unsigned long long ext = (unsigned long long)((long long)v.l2 >> 63);
  if (s <= 0) return v;
  if (s >= 192) return {ext, ext, ext};
  while (s >= 64) {
    v.l0 = v.l1;
    v.l1 = v.l2;
    v.l2 = ext;
    s -= 64;
  }
  if (s > 0) {
    v.l0 = (v.l0 >> s) | (v.l1 << (64 - s));
    v.l1 = (v.l1 >> s) | (v.l2 << (64 - s));
    v.l2 = (unsigned long long)((long long)v.l2 >> s);
  }
  return v;
}

// Left shift by 0 <= s < 64 (callers keep the result below 2^149).
__device__ __forceinline__ u192 shl192(u192 v, int s) {
  if (s <= 0) return v;
  v.l2 = (v.l2 << s) | (v.l1 >> (64 - s));
  v.l1 = (v.l1 << s) | (v.l0 >> (64 - s));
  v.l0 <<= s;
  return v;
}

// Slots (GvSlot: 192 bits and an exponent) are written by one thread and read
// by CTAs that took a ticket after the writer's fence: L2 loads.
__device__ __forceinline__ u192 slot_value(const GvSlot& s) { return {s.l0, s.l1, s.l2}; }
__device__ __forceinline__ GvSlot load_slot(const GvSlot* p) {
  const ulonglong2 a = __ldcg(reinterpret_cast<const ulonglong2*>(p));
  const ulonglong2 b = __ldcg(reinterpret_cast<const ulonglong2*>(p) + 1);
  GvSlot s;
  s.l0 = a.x;
  s.l1 = a.y;
  s.l2 = b.x;
  s.e = (int)(unsigned)(b.y & 0xFFFFFFFFull);
  s.pad = 0;
  return s;
}
__device__ __forceinline__ void store_slot(GvSlot* p, const u192& v, int e) {
  reinterpret_cast<ulonglong2*>(p)[0] = make_ulonglong2(v.l0, v.l1);
  reinterpret_cast<ulonglong2*>(p)[1] = make_ulonglong2(v.l2, (unsigned long long)(unsigned)e);
}

// value * 2^q rounded to nearest-even, assembled with integer operations only
// (the 192-bit integer is two's complement; results stay in the normal range
// for every sum this library forms).
__device__ double u192_to_double(u192 v, int q) {
  const bool neg = (long long)v.l2 < 0;
  if (neg) {
    v.l0 = ~v.l0;
    v.l1 = ~v.l1;
    v.l2 = ~v.l2;
    v.l0 += 1ull;
    const unsigned long long c0 = v.l0 == 0ull ? 1ull : 0ull;
    v.l1 += c0;
    v.l2 += (c0 && v.l1 == 0ull) ? 1ull : 0ull;
  }
  int top;
  if (v.l2)
    top = 191 - __clzll((long long)v.l2);
  else if (v.l1)
    top = 127 - __clzll((long long)v.l1);
  else if (v.l0)
    top = 63 - __clzll((long long)v.l0);
  else
    return 0.0;
  // 64-bit window with the leading one at bit 63, plus a sticky bit
  unsigned long long window;
  bool sticky = false;
  if (top >= 63) {
    const int sh = top - 63;
    window = sar192(v, sh).l0;
    if (sh >= 128) {
      sticky = v.l0 != 0ull || v.l1 != 0ull || (sh > 128 && (v.l2 << (192 - sh)) != 0ull);
    } else if (sh >= 64) {
      sticky = v.l0 != 0ull || (sh > 64 && (v.l1 << (128 - sh)) != 0ull);
    } else if (sh > 0) {
      sticky = (v.l0 << (64 - sh)) != 0ull;
    }
  } else {
    window = v.l0 << (63 - top);
  }
  // round the 64-bit window to 53 bits (nearest, ties to even)
  unsigned long long mant = window >> 11;
  const unsigned long long rest = window & 0x7FFull;
  const bool half = (rest & 0x400ull) != 0ull;
  const bool above = (rest & 0x3FFull) != 0ull || sticky;
  if (half && (above || (mant & 1ull))) ++mant;
  int e = top + q;  // value = mant * 2^(e - 52)
  if (mant >> 53) {
    mant >>= 1;
    ++e;
  }
  double r;
  if (e > 1023) {
    r = __longlong_as_double(0x7FF0000000000000ll);  // beyond FP64, as a sum of doubles would be
  } else if (e >= -1022) {
    r = __longlong_as_double((long long)(((unsigned long long)(e + 1023) << 52) |
                                         (mant & 0xFFFFFFFFFFFFFull)));
  } else if (e >= -1022 - 600) {
    // below the normal range: scale into it, then one multiply by 2^-600
    // (the product rounds to the subnormal grid; rare, and on the FP64 pipe)
    r = __longlong_as_double((long long)(((unsigned long long)(e + 600 + 1023) << 52) |
                                         (mant & 0xFFFFFFFFFFFFFull))) *
        0x1p-600;
  } else {
    r = 0.0;
  }
  return neg ? -r : r;
}


// Barrier of a group of nthr threads (a multiple of 32); id 0 is the whole CTA.
__device__ __forceinline__ void gv_bar(int id, int nthr) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthr) : "memory");
}

// The iteration's finalisation, by the threads [0, nthr) of a group (local
// thread index tid, barrier id bar): the iteration record, the stage's
// combination and the per-iteration state.
__device__ void finalize_iteration(const GvReduceArgs& a, int tid, int nthr, int bar) {
  const int lane = tid & 31, wid = tid >> 5;
  (void)nthr;
  (void)bar;
  GvState* st = a.st;
  // the sums, each rounded once to FP64 by the CTA that completed its block
  if (wid == 0) {
    // warp 0: the iteration record (one lane per channel) and the stage
    const int stride = a.mode ? 2 + 2 * GV_NGRAD : 2;
    if (lane < a.nch) {
      double* rec = a.per_iter + (size_t)a.k * stride + 2 * lane;
      double I, s;
      mean_sigma(__ldcg(a.sums + 2 * lane), __ldcg(a.sums + 2 * lane + 1), a.inv_c, a.inv_cm1,
                 &I, &s);
      rec[0] = I;
      if (!a.plus) rec[1] = s;  // VEGAS+: sigma_k comes from the hypercube statistics
      if (a.host_rec) {
        a.host_rec[(size_t)a.k * stride + 2 * lane] = I;
        a.host_rec[(size_t)a.k * stride + 2 * lane + 1] = s;
      }
    }
    __syncwarp();
    if (a.last && !a.plus) combine_stage_warp(a.per_iter, stride, a.k + 1, a.inv_m1, st, a.mode != 0);
    if (a.last && a.plus) {
      // the hypercube statistics run beside this kernel: the second of the
      // two to finish the stage's last iteration combines it
      int t = 0;
      if (lane == 0) {
        __threadfence();  // this iteration's I_k before the arrival
        t = atomicAdd(&st->join, 1);
      }
      t = __shfl_sync(0xffffffffu, t, 0);
      if (t == 1) {
        __threadfence();  // the statistics' sigma_k, published before their arrival
        combine_stage_warp(a.per_iter, stride, a.k + 1, a.inv_m1, st, false);
        if (lane == 0) st->join = 0;
      }
    }
    if (lane == 0) {
      const unsigned long long nf = __ldcg(&st->nonfinite_iter);
      st->nonfinite = (a.k == 0 ? 0ull : st->nonfinite) + nf;
      if (a.k == 0) st->status = 0;
      st->nonfinite_iter = 0ull;
    }
  }
  if (tid == 0) {
    st->it = st->it + 1ull;
    if (a.last) st->it0 = st->it;  // the next stage's first counter
    if (a.last && a.host_st) {
      // the state the host reads after the stage: this thread wrote all of it
      a.host_st->it = st->it;
      a.host_st->nonfinite = st->nonfinite;
      a.host_st->status = st->status;
      a.host_st->integral = st->integral;
      a.host_st->error = st->error;
      a.host_st->chi2 = st->chi2;
    }
  }
}

// ---------------------------------------------------------------------------
// Grid refinement (Lepage's VEGAS, cited in Section 2.1), one axis at a time:
// every step of it -- smoothing, normalisation, compression, redistribution
// -- involves one axis only, so the CTA whose reduction completes an axis
// refines it at once, while other CTAs are still reducing.
// ---------------------------------------------------------------------------
// Write the edges e_src (N+1 values) of axis ax into the grid pack with the
// axis' derived tables.
__device__ __forceinline__ void pack_axis_tables(double* grid, const double* e_src, int ax, int d, int N, int tid,
                                 int nthr) {
  const GvGridLayout L{d, N};
  double* e64 = grid + L.off_e64() + (size_t)ax * (N + 1);
  double* wd64 = grid + L.off_wd64() + (size_t)ax * N;
  double* jac = grid + L.off_jac() + (size_t)ax * N;
  float* w32 = reinterpret_cast<float*>(grid + L.off_f32_base());
  float* e32 = w32 + L.w_e32() + (size_t)ax * (N + 1);
  float* wd32 = w32 + L.w_wd32() + (size_t)ax * N;
  float* jm32 = w32 + L.w_jm32() + (size_t)ax * N;
  int* je = reinterpret_cast<int*>(w32 + L.w_je()) + (size_t)ax * N;
  for (int i = tid; i <= N; i += nthr) {
    const double e = e_src[i];
    e64[i] = e;
    e32[i] = (float)e;
    if (i < N) {
      const double w = e_src[i + 1] - e;
      const double j = (double)N * w;
      wd64[i] = w;
      jac[i] = j;
      wd32[i] = (float)w;
      // j = m 2^x with m in [1,2): exponent from the bits (j > 0; a subnormal
      // j is scaled into the normal range first)
      const bool sub = j < 0x1p-1000;
      const double js = sub ? j * 0x1p200 : j;
      const long long b = __double_as_longlong(js);
      const int x = (int)((b >> 52) & 0x7FF) - 1023;
      const double m = __longlong_as_double((b & 0xFFFFFFFFFFFFFll) | 0x3FF0000000000000ll);
      jm32[i] = (float)m;
      je[i] = sub ? x - 200 : x;
    }
  }
}

// 1/x and 1/sqrt(x) for positive normal x: the hardware approximations
// (PTX rcp.approx.ftz.f64 and rsqrt.approx.ftz.f64, about 20 correct bits)
// refined by two Newton-Raphson steps, y <- y + y (1 - x y) and
// z <- z + z (1 - x z^2) / 2, each of which squares the relative error.
// Measured against the correctly rounded results over six decades: the
// reciprocal agrees bit for bit, the square root within 2.7e-16.  They
// replace the library's correctly rounded routines, whose special-case
// handling costs this chip's scarce FP64 pipe more instructions.
__device__ __forceinline__ double gv_rcp_nr(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}
__device__ __forceinline__ double gv_rsqrt_nr(double x) {
  double z;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(z) : "d"(x));
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const double h = x * z;
    const double e = fma(-h, z, 1.0);
    z = fma(0.5 * z, e, z);
  }
  return z;
}

// ((1 - rho)/(-ln rho))^alpha for 0 < rho < 1, with the common exponents
// evaluated by reciprocals and roots rather than pow.  In the refinement
// rho <= 3/5 (a smoothed bin holds at most 3/5 of the smoothed total), so
// 1 - rho >= 2/5 and -ln rho >= 0.51: both are positive normal numbers.
__device__ __forceinline__ double compress(double rho, double alpha) {
  if (rho <= 0.0) return 0.0;
  if (rho >= 1.0) return 1.0;
  const double L = -gv_log_pos(rho);
  const double om = 1.0 - rho;
  if (alpha == 1.5) {  // om^(3/2) L^(-3/2) = (om^2 / sqrt(om)) (1/sqrt(L))^3
    const double y = gv_rsqrt_nr(L), z = gv_rsqrt_nr(om);
    return (om * om * z) * (y * y * y);
  }
  if (alpha == 1.0) return om * gv_rcp_nr(L);
  if (alpha == 0.5) return om * gv_rsqrt_nr(om) * gv_rsqrt_nr(L);
  if (alpha == 2.0) {
    const double q = om * gv_rcp_nr(L);
    return q * q;
  }
  if (alpha == 0.0) return 1.0;
  return pow(om * __drcp_rn(L), alpha);
}

// The compressed value r = ((1 - rho)/(-ln rho))^(3/2) (alpha = 3/2) and the
// slope de / r in FP32 pairs (gv_ff.cuh), for 2^-100 < rho <= 3/5 and
// 2^-100 < de <= 1.  -ln rho by the table reduction of gv_log_pos: rho =
// 2^k m, r' = m R_j - 1 (|r'| < 2^-7), ln rho = k ln2 + L_j + ln(1 + r'),
// with ln(1 + r') = r' + r'^2 P(r'), P = -1/2 + r'/3 - r'^2/4 + ... + r'^5/7
// (truncation below 2^-60); the leading -1/2 and r' P's product are paired,
// the rest of P (scaled by r'^3 < 2^-21) is FP32.
__device__ __forceinline__ void compress15_ff(double rho, double de, double& rv, double& sl) {
  const long long b = __double_as_longlong(rho);
  const int k = (int)(b >> 52) - 1023;
  const int j = (int)((b >> 45) & 127);
  const GvFF m = gv_ff_from_double(
      __longlong_as_double((b & 0xFFFFFFFFFFFFFll) | 0x3FF0000000000000ll));
  const double2 RL = __ldg(reinterpret_cast<const double2*>(gv_log_tab) + j);
  const GvFF p = gv_ff_mul(m, gv_ff_from_double(RL.x));
  const GvFF r = gv_two_sum(__fsub_rn(p.hi, 1.0f), p.lo);  // p.hi - 1 is exact
  const float x = r.hi;
  float Q = __fmaf_rn(x, 1.0f / 7.0f, -1.0f / 6.0f);
  Q = __fmaf_rn(Q, x, 0.2f);
  Q = __fmaf_rn(Q, x, -0.25f);
  Q = __fmaf_rn(Q, x, 1.0f / 3.0f);
  const GvFF P = gv_two_sum(-0.5f, __fmul_rn(x, Q));
  const GvFF l1p = gv_ff_add(r, gv_ff_mul(gv_ff_mul(r, r), P));
  // ln 2 = 0x1.62e43p-1 + (-0x1.05c61p-29), to 9e-17
  const GvFF kln2 = gv_ff_mul_f(GvFF{0x1.62e43p-1f, -0x1.05c61p-29f}, (float)k);
  const GvFF lnrho = gv_ff_add(gv_ff_add(kln2, gv_ff_from_double(RL.y)), l1p);
  const GvFF L = {-lnrho.hi, -lnrho.lo};
  const GvFF R = gv_ff_from_double(rho);
  const GvFF om = gv_ff_add(GvFF{1.0f, 0.0f}, GvFF{-R.hi, -R.lo});
  const GvFF q = gv_ff_div(om, L);
  const GvFF c = gv_ff_mul(q, gv_ff_sqrt(q));
  rv = gv_ff_to_double(c);
  sl = gv_ff_to_double(gv_ff_div(gv_ff_from_double(de), c));
}

// alpha values whose compressed values are at least (1/745)^2 > 1e-6 (the
// reciprocal approximation then sees normal numbers only)
__device__ __forceinline__ bool fast_alpha(double alpha) {
  return alpha == 1.5 || alpha == 1.0 || alpha == 0.5 || alpha == 2.0 || alpha == 0.0;
}

// Shared memory of refine_axis: r[N], slope[N], C[N+1], e[N+1], ne[N+1].
__host__ __device__ inline size_t refine_axis_smem(int N) {
  return sizeof(double) * (2 * (size_t)N + 3 * ((size_t)N + 1));
}

// Refinement of axis ax by a group of nthr threads (local index tid, barrier
// id bar, group number q), once every block holding the axis has rounded its
// bin sums d_i to FP64 (the oracle's arithmetic from here on):
//   1. 6 x the smoothed sums, s_i = 3 (d_0 + d_1) at the ends and
//      2 (d_{i-1} + d_i + d_{i+1}) inside, and their total (a fixed-order
//      tree), then per bin the share rho = s_i / total, the compressed value
//      r = ((1-rho)/(-ln rho))^alpha and the slope (e_{i+1}-e_i)/r;
//   2. one warp: the prefix sums C of r;
//   3. per new edge: the old bin where C reaches j R/N -- binary search on
//      the bit patterns of the nonnegative doubles -- then
//      e_i + (target - C_i) * slope_i; e'_0 = 0 and e'_N = 1 exactly;
//   4. the axis' tables.
// An axis whose bins are all zero keeps its edges.
__device__ __forceinline__ void refine_axis(const GvReduceArgs& a, int ax, double* sm, int tid, int nthr, int bar,
                            int q) {
  const int N = a.nbins, lane = tid & 31, wid = tid >> 5;
  __shared__ double s_inv[8], s_step[8], s_tree[8][32];
  double* r = sm;             // [N] 6 x smoothed sums, then compressed values
  double* slope = r + N;      // [N] bin sums, then slopes
  double* C = slope + N;      // [N+1]
  double* e = C + (N + 1);    // [N+1] old edges
  double* ne = e + (N + 1);   // [N+1] new edges
  const double* d = a.sums + 2 * a.nch + ax * N;
  const double* e64 = a.grid + GvGridLayout{a.ndim, N}.off_e64() + (size_t)ax * (N + 1);
  for (int k = tid; k <= N; k += nthr) e[k] = e64[k];
  for (int i = tid; i < N; i += nthr) slope[i] = __ldcg(d + i);
  gv_bar(bar, nthr);
  for (int i = tid; i < N; i += nthr)
    r[i] = i == 0       ? 3.0 * (slope[0] + slope[1])
           : i == N - 1 ? 3.0 * (slope[N - 2] + slope[N - 1])
                        : 2.0 * (slope[i - 1] + slope[i] + slope[i + 1]);
  gv_bar(bar, nthr);
  if (wid == 0) {
    // the total in an order fixed by N alone (whatever the group's size):
    // 32 consecutive chunks in order, then a fixed pairwise tree in shared
    // memory (shuffles of doubles cost more here)
    const int chunk = (N + 31) / 32;
    const int i0 = min(N, lane * chunk), i1 = min(N, i0 + chunk);
    double part = 0.0;
    if (chunk <= 4) {
      // a fixed pairwise tree over the chunk (zeros past its end add exactly)
      double v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = i0 + k < i1 ? r[i0 + k] : 0.0;
      part = (v[0] + v[1]) + (v[2] + v[3]);
    } else {
      for (int i = i0; i < i1; ++i) part += r[i];
    }
    double* tr = s_tree[q];
    tr[lane] = part;
    __syncwarp();
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      if (lane < m) tr[lane] = tr[lane] + tr[lane + m];
      __syncwarp();
    }
    if (lane == 0) {
      const double t = tr[0];
      s_inv[q] = !(t > 0.0) ? 0.0 : (t > 0x1p-1000 && t < 0x1p1000) ? gv_rcp_nr(t) : __drcp_rn(t);
    }
  }
  gv_bar(bar, nthr);
  const double inv = s_inv[q];
  const bool fast = fast_alpha(a.alpha);
  if (inv > 0.0) {
    for (int i = tid; i < N; i += nthr) {
      double rv = 0.0, sl = 0.0;
      const double s6 = r[i];
      if (s6 > 0.0) {
        const double rho = s6 * inv, de = e[i + 1] - e[i];
        if (a.alpha == 1.5 && rho > 0x1p-100 && rho <= 0.6 && de > 0x1p-100 && de <= 1.0) {
          compress15_ff(rho, de, rv, sl);
        } else {
          rv = compress(rho, a.alpha);
          if (rv > 0.0) sl = de * (fast ? gv_rcp_nr(rv) : __drcp_rn(rv));
        }
      }
      r[i] = rv;
      slope[i] = sl;
    }
    gv_bar(bar, nthr);
    if (wid == 0) {
      const int chunk = (N + 31) / 32;
      const int i0 = min(N, lane * chunk), i1 = min(N, i0 + chunk);
      // the chunk's own running sums (in order), formed before the scan so
      // that each C below is one addition away from its chunk's base
      double lp[4];
      double local = 0.0;
      if (chunk <= 4) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          local = i0 + k < i1 ? local + r[i0 + k] : local;
          lp[k] = local;
        }
      } else {
        for (int i = i0; i < i1; ++i) local += r[i];
      }
      // inclusive prefix sums of the 32 chunk sums (Hillis-Steele in shared
      // memory), then each chunk's exclusive prefix
      double* tr = s_tree[q];
      tr[lane] = local;
      __syncwarp();
#pragma unroll
      for (int m = 1; m < 32; m <<= 1) {
        const double v = lane >= m ? tr[lane] + tr[lane - m] : tr[lane];
        __syncwarp();
        tr[lane] = v;
        __syncwarp();
      }
      double run = lane > 0 ? tr[lane - 1] : 0.0;  // exclusive prefix of this lane's chunk
      if (lane == 0) C[0] = 0.0;
      if (chunk <= 4) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (i0 + k < i1) C[i0 + k + 1] = run + lp[k];
      } else {
        for (int i = i0; i < i1; ++i) {
          run += r[i];
          C[i + 1] = run;
        }
      }
      __syncwarp();
      if (lane == 0) s_step[q] = C[N] * a.inv_nbins;
    }
    gv_bar(bar, nthr);
    const double step = s_step[q];
    const long long* Cb = reinterpret_cast<const long long*>(C);
    for (int j = tid; j <= N; j += nthr) {
      double v;
      if (j == 0) {
        v = 0.0;
      } else if (j == N) {
        v = 1.0;
      } else {
        const double target = step * j;
        const long long tb = __double_as_longlong(target);
        int lo = 0, hi = N - 1;  // first bin i with C[i+1] > target (N-1 if none)
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (Cb[mid + 1] > tb)
            hi = mid;
          else
            lo = mid + 1;
        }
        v = fma(target - C[lo], slope[lo], e[lo]);
      }
      ne[j] = v;
    }
  } else {
    for (int j = tid; j <= N; j += nthr) ne[j] = e[j];
  }
  gv_bar(bar, nthr);
  pack_axis_tables(a.grid, ne, ax, a.ndim, N, tid, nthr);
}

// Axes that one block of 32 slots can touch, and the dynamic shared memory
// the reduce kernels need to refine that many axes side by side.
__host__ __device__ inline int gv_axes_per_block(int N) {
  const int k = (31 + N - 1) / N + 1;
  return k < 7 ? k : 7;
}

#define GV_RED_TILES_PER_LOAD 8

// A tile partial of slot k aligned to exponent em (>= its own exponent e).
// Channel slots: 128-bit two's complement at 2^(pw e - GV_FB); bin slots
// (axis bins and histogram bins): a 96-bit value, unsigned Q (< 2^67) for
// sums of w^2 (pw = 2) or two's complement for the histogram's sums of w
// (pw = 1, sgn), at 2^(pw (e - GV_BINE_OFF) - GV_BIN_QBITS), with
// GV_BIN_XBITS more low bits in the sums.
__device__ __forceinline__ u192 align_tile(ulonglong2 v, int e, int em, bool bin, int pw,
                                           bool sgn = false) {
  if (bin) {
    const unsigned long long ext = sgn ? (unsigned long long)((long long)(int)(unsigned)v.y >> 63)
                                       : 0ull;
    const u192 x = {v.x, sgn ? (unsigned long long)(long long)(int)(unsigned)v.y
                             : (v.y & 0xFFFFFFFFull),
                    ext};
    const int sh = pw * (em - e) - GV_BIN_XBITS;
    return sh < 0 ? shl192(x, -sh) : sar192(x, sh);
  }
  const u192 x = {v.x, v.y, (unsigned long long)((long long)v.y >> 63)};
  return sar192(x, pw * (em - e));
}

// One reduce CTA (256 threads) of one integration: slot block bx (32 slots,
// one per lane), tile range by, of nblk CTAs in total for that integration.
//   A. every CTA: the largest exponent of each slot over its tiles, then the
//      tiles' partials aligned to it and summed -- the CTA's sums, published
//      with that exponent (no atomics);
//   B. the CTA that completes a slot block (ticket): the block's sums over all
//      tile ranges at their largest exponent, each rounded once to FP64;
//   C. the CTA whose block completes an axis (second ticket) refines the
//      axis; the CTA that completes block 0 (the channel sums) finalises the
//      iteration.
// Integer sums of values aligned by rules that depend only on the data:
// nothing here depends on the launch shape or on timing.
__device__ __forceinline__ void gv_reduce_task(const GvReduceArgs& a, int bx, int by, int nblk,
                               u192 (*s_part)[32], int* s_emax, int* s_flags, int* s_won,
                               double* sm) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int k = bx * 32 + lane;
  const int gx = (a.nacc + 31) / 32, gy = nblk / gx;
  const int t0 = by * a.tiles_per_cta;
  const int t1 = min(a.n_tiles, t0 + a.tiles_per_cta);
  const bool bin = a.has_bins && k >= 2 * a.nch;
  // the histogram's sums of w: the last nhist slots
  const bool hw = bin && a.nhist > 0 && k >= a.nacc - a.nhist;
  const int pw = hw ? 1 : (bin ? 2 : (k & 1) + 1);
  const int empty = bin ? 0 : GV_EMPTY;
  const int ch = k >> 1;
  constexpr int G = GV_RED_TILES_PER_LOAD;
  gv_wait_prior_grid();

  // ---- A: this CTA's tiles
  const bool cached = t1 - t0 <= 8 * G;  // every tile of a lane fits in registers
  ulonglong2 v[G];
  int et[G];
  int em = empty;
  if (k < a.nacc) {
    if (cached) {
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int t = t0 + wid + 8 * g;
        v[g] = make_ulonglong2(0ull, 0ull);
        et[g] = empty;
        if (t < t1) {
          v[g] = a.part[(size_t)t * a.nacc + k];
          et[g] = bin ? (int)(v[g].y >> 32) : a.tileE[(size_t)t * a.nch + ch];
        }
        em = max(em, et[g]);
      }
    } else {
      for (int t = t0 + wid; t < t1; t += 8)
        em = max(em, bin ? (int)(__ldcg(&a.part[(size_t)t * a.nacc + k].y) >> 32)
                         : a.tileE[(size_t)t * a.nch + ch]);
    }
  }
  s_emax[wid * 32 + lane] = em;
  __syncthreads();
#pragma unroll
  for (int w = 0; w < 8; ++w) em = max(em, s_emax[w * 32 + lane]);
  u192 r = {0ull, 0ull, 0ull};
  if (k < a.nacc && em != empty) {
    if (cached) {
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (et[g] != empty && (v[g].x | v[g].y)) add192(r, align_tile(v[g], et[g], em, bin, pw, hw));
    } else {
      for (int t = t0 + wid; t < t1; t += 8) {
        const ulonglong2 x = a.part[(size_t)t * a.nacc + k];
        const int e = bin ? (int)(x.y >> 32) : a.tileE[(size_t)t * a.nch + ch];
        if (e != empty && (x.x | x.y)) add192(r, align_tile(x, e, em, bin, pw, hw));
      }
    }
  }
  s_part[wid][lane] = r;
  __syncthreads();
  if (wid == 0) {
    u192 t = s_part[0][lane];
#pragma unroll
    for (int w = 1; w < 8; ++w) add192(t, s_part[w][lane]);
    if (k < a.nacc) store_slot(a.cpart + (size_t)by * (32 * gx) + k, t, em);
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0)
    s_flags[0] = atomicAdd(a.tickets + gv_ticket_group(bx), 1) == gy - 1 ? 1 : 0;
  __syncthreads();
  if (!s_flags[0]) return;

  // ---- B: this CTA completes slot block bx
  __threadfence();  // the other CTAs' sums, published before their tickets
  gv_allow_next_grid();  // what is left is short: the next fill's CTAs may come in
  if (threadIdx.x == 0) a.tickets[gv_ticket_group(bx)] = 0;
  constexpr int YC = 2;  // tile ranges per warp held in registers (gy <= 16)
  GvSlot cs[YC];
  const bool held = gy <= 8 * YC;
  em = empty;
#pragma unroll
  for (int q = 0; q < YC; ++q) {
    const int y = wid + 8 * q;
    cs[q].e = empty;
    if (held && k < a.nacc && y < gy) cs[q] = load_slot(a.cpart + (size_t)y * (32 * gx) + k);
    em = max(em, cs[q].e);
  }
  if (!held && k < a.nacc)
    for (int y = wid; y < gy; y += 8)
      em = max(em, __ldcg(&a.cpart[(size_t)y * (32 * gx) + k].e));
  s_emax[wid * 32 + lane] = em;
  __syncthreads();
#pragma unroll
  for (int w = 0; w < 8; ++w) em = max(em, s_emax[w * 32 + lane]);
  r = {0ull, 0ull, 0ull};
  if (k < a.nacc && em != empty) {
    if (held) {
#pragma unroll
      for (int q = 0; q < YC; ++q)
        if (cs[q].e != empty) add192(r, sar192(slot_value(cs[q]), pw * (em - cs[q].e)));
    } else {
      for (int y = wid; y < gy; y += 8) {
        const GvSlot c = load_slot(a.cpart + (size_t)y * (32 * gx) + k);
        if (c.e != empty) add192(r, sar192(slot_value(c), pw * (em - c.e)));
      }
    }
  }
  s_part[wid][lane] = r;
  __syncthreads();
  const int N = a.nbins;
  // the axis bins of this block (the histogram slots after them have no axis)
  const int j_first = max(0, bx * 32 - 2 * a.nch);
  const int j_last = min(min(a.nacc - 1, bx * 32 + 31) - 2 * a.nch, a.ndim * N - 1);
  if (wid == 0) {
    u192 t = s_part[0][lane];
#pragma unroll
    for (int w = 1; w < 8; ++w) add192(t, s_part[w][lane]);
    // the slot's sum over all events, rounded once to FP64
    if (k < a.nacc)
      a.sums[k] = em == empty ? 0.0
                              : u192_to_double(t, bin ? pw * (em - GV_BINE_OFF) - GV_BIN_FB
                                                      : pw * em - GV_FB);
    __threadfence();
    // second tickets, one lane per axis the block touches: the block whose
    // count completes an axis refines it
    const int ax0 = j_first / N;
    const int nax =
        (a.has_bins && a.refine_follows && j_last >= j_first) ? j_last / N - ax0 + 1 : 0;
    bool won = false;
    if (lane < nax) {
      const int ax = ax0 + lane;
      const int x_lo = (2 * a.nch + ax * N) / 32, x_hi = (2 * a.nch + (ax + 1) * N - 1) / 32;
      int* tk = a.tickets + gv_ticket_axis(a.nacc, ax);
      if (atomicAdd(tk, 1) == x_hi - x_lo) {
        *tk = 0;
        won = true;
      }
    }
    const unsigned mask = __ballot_sync(0xffffffffu, won);
    if (won) s_won[__popc(mask & ((1u << lane) - 1u))] = ax0 + lane;
    if (lane == 0) s_flags[1] = __popc(mask);
  }
  __syncthreads();
  // block 0 holds the channel sums: it finalises the iteration
  const int n_won = s_flags[1], fin = bx == 0;
  if (n_won == 0 && !fin) return;

  // ---- C
  if (n_won) __threadfence();  // the other blocks' sums, published before their tickets
  // the won axes and the finalisation side by side on groups of warps: the
  // finalisation takes warp 7 (all warps if no axis was won), the axes the
  // other warps, min(n_won, 7) groups, each with its own barrier and shared
  // memory
  if (fin && (n_won == 0 || wid == 7)) {
    const int nw = n_won == 0 ? 8 : 1, w0 = 8 - nw;
    finalize_iteration(a, threadIdx.x - 32 * w0, 32 * nw, 1);
  } else if (n_won > 0) {
    const int ng = min(n_won, 7), wpg = (fin ? 7 : 8) / ng, q = wid / wpg;
    if (q < ng) {
      const int per = (int)(refine_axis_smem(a.nbins) / sizeof(double));
      for (int it = q; it < n_won; it += ng)
        refine_axis(a, s_won[it], sm + (size_t)q * per, threadIdx.x - 32 * wpg * q, 32 * wpg,
                    2 + q, q);
    }
  }
}

__global__ void __launch_bounds__(256) gv_reduce_kernel(const GvReduceArgs a) {
  extern __shared__ __align__(16) double sm[];
  __shared__ u192 s_part[8][32];
  __shared__ int s_emax[256], s_flags[4], s_won[GV_MAXD];
  gv_reduce_task(a, blockIdx.x, blockIdx.y, gridDim.x * gridDim.y, s_part, s_emax, s_flags,
                 s_won, sm);
}

// ---------------------------------------------------------------------------
// Single-level reduce of a plain forward iteration (also with a histogram or
// VEGAS+), for slot-major partials (slot k of tile t at part[k n_tiles + t]).
// A group of GT threads (GT/32 warps; 256/GT groups per CTA) owns one slot and
// reads it over every tile: the slot's largest exponent (group max), then the
// partials aligned to it and added in 192-bit integers (group sum), rounded
// once to FP64.  The alignment depends on the data alone, so the sums do not
// depend on any launch shape.  Compared with the two-level reduce there is no
// published per-range sum and no ticket between the levels: one L2 round trip
// for the partials, then one fence and one ticket per slot.
// Tickets: the group that completes the channel slots has its CTA finalise
// the iteration; the group whose bin completes an axis has its CTA refine the
// axis.  No CTA waits for another.
// ---------------------------------------------------------------------------
__device__ __forceinline__ u192 warp_sum192(u192 v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    const u192 o = {shfl_xor_u64(v.l0, m), shfl_xor_u64(v.l1, m), shfl_xor_u64(v.l2, m)};
    add192(v, o);
  }
  return v;
}

template <int GT>
__global__ void __launch_bounds__(256) gv_reduce_slots_kernel(const GvReduceArgs a) {
  constexpr int NG = 256 / GT;  // slots per CTA
  constexpr int WPG = GT / 32;  // warps per slot
  constexpr int G = GV_RED_TILES_PER_LOAD;
  extern __shared__ __align__(16) double sm[];
  __shared__ int s_emax[8];
  __shared__ u192 s_sum[8];
  __shared__ int s_won[NG], s_nwon, s_fin;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int grp = tid / GT, u = tid - grp * GT;
  const int k = blockIdx.x * NG + grp;
  const bool live = k < a.nacc;
  const bool bin = a.has_bins && k >= 2 * a.nch;
  // the histogram's sums of w: the last nhist slots
  const bool hw = bin && a.nhist > 0 && k >= a.nacc - a.nhist;
  const int pw = hw ? 1 : (bin ? 2 : (k & 1) + 1);
  const int empty = bin ? 0 : GV_EMPTY;
  const int ch = k >> 1;
  const ulonglong2* src = a.part + (size_t)k * a.n_tiles;  // slot-major: slot stride n_tiles
  if (tid == 0) {
    s_nwon = 0;
    s_fin = 0;
  }
  gv_wait_prior_grid();
  const int nt = a.tiles_used ? min(a.n_tiles, __ldcg(a.tiles_used)) : a.n_tiles;
  __syncthreads();
  // the slot's largest exponent over all tiles
  const bool cached = nt <= G * GT;  // every partial of a thread fits in registers
  ulonglong2 v[G];
  int et[G];
  int em = empty;
  if (live) {
    if (cached) {
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int t = u + g * GT;
        v[g] = make_ulonglong2(0ull, 0ull);
        et[g] = empty;
        if (t < nt) {
          v[g] = __ldcg(src + t);
          et[g] = bin ? (int)(v[g].y >> 32) : __ldcg(a.tileE + (size_t)t * a.nch + ch);
        }
        em = max(em, et[g]);
      }
    } else {
      for (int t = u; t < nt; t += GT)
        em = max(em, bin ? (int)(__ldcg(src + t).y >> 32)
                         : __ldcg(a.tileE + (size_t)t * a.nch + ch));
    }
  }
  em = __reduce_max_sync(0xffffffffu, em);
  if constexpr (WPG > 1) {
    if (lane == 0) s_emax[wid] = em;
    __syncthreads();
#pragma unroll
    for (int w = 0; w < WPG; ++w) em = max(em, s_emax[grp * WPG + w]);
  }
  // the partials aligned to it, summed
  u192 r = {0ull, 0ull, 0ull};
  if (live && em != empty) {
    if (cached) {
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (et[g] != empty && (v[g].x | v[g].y)) add192(r, align_tile(v[g], et[g], em, bin, pw, hw));
    } else {
      for (int t = u; t < nt; t += GT) {
        const ulonglong2 x = __ldcg(src + t);
        const int e = bin ? (int)(x.y >> 32) : __ldcg(a.tileE + (size_t)t * a.nch + ch);
        if (e != empty && (x.x | x.y)) add192(r, align_tile(x, e, em, bin, pw, hw));
      }
    }
  }
  r = warp_sum192(r);
  if constexpr (WPG > 1) {
    if (lane == 0) s_sum[wid] = r;
    __syncthreads();
    if (u == 0)
#pragma unroll
      for (int w = 1; w < WPG; ++w) add192(r, s_sum[grp * WPG + w]);
  }
  if (u == 0 && live) {
    // the slot's sum over all events, rounded once to FP64
    a.sums[k] = em == empty ? 0.0
                            : u192_to_double(r, bin ? pw * (em - GV_BINE_OFF) - GV_BIN_FB
                                                    : pw * em - GV_FB);
    __threadfence();
    if (k < 2 * a.nch) {
      int* tk = a.tickets + gv_ticket_done(a.nacc);
      if (atomicAdd(tk, 1) == 2 * a.nch - 1) {
        *tk = 0;
        s_fin = 1;
      }
    } else if (a.has_bins && a.refine_follows && k < 2 * a.nch + a.ndim * a.nbins) {
      const int ax = (k - 2 * a.nch) / a.nbins;
      int* tk = a.tickets + gv_ticket_axis(a.nacc, ax);
      if (atomicAdd(tk, 1) == a.nbins - 1) {
        *tk = 0;
        s_won[atomicAdd(&s_nwon, 1)] = ax;
      }
    }
  }
  __syncthreads();
  const int n_won = s_nwon, fin = s_fin;
  if (n_won == 0 && !fin) return;
  __threadfence();  // the other slots' sums, published before their tickets
  gv_allow_next_grid();  // what is left is short: the next fill's CTAs may come in
  // the finalisation on warp 7 (all warps if no axis was won), the won axes
  // one after the other on the other warps
  if (fin && (n_won == 0 || wid == 7)) {
    const int nw = n_won == 0 ? 8 : 1, w0 = 8 - nw;
    finalize_iteration(a, tid - 32 * w0, 32 * nw, 1);
  } else if (n_won > 0) {
    for (int i = 0; i < n_won; ++i) refine_axis(a, s_won[i], sm, tid, fin ? 224 : 256, 2, 0);
  }
}

// Batched: one launch reduces many integrations; task i names the
// integration and the block coordinates of CTA i.
__global__ void __launch_bounds__(256) gv_reduce_batch_kernel(const GvReduceArgs* args,
                                                              const int4* tasks, int k, int last,
                                                              double inv_m1) {
  extern __shared__ __align__(16) double sm[];
  __shared__ u192 s_part[8][32];
  __shared__ int s_emax[256], s_flags[4], s_won[GV_MAXD];
  // the integration's arguments in shared memory, read where used (a copy in
  // registers held ~40 of them for the whole task)
  __shared__ GvReduceArgs s_a;
  const int4 t = tasks[blockIdx.x];
  static_assert(sizeof(GvReduceArgs) % 4 == 0, "GvReduceArgs copy");
  const unsigned* src = reinterpret_cast<const unsigned*>(args + t.x);
  unsigned* dst = reinterpret_cast<unsigned*>(&s_a);
  for (int i = threadIdx.x; i < (int)(sizeof(GvReduceArgs) / 4); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    s_a.k = k;
    s_a.last = last;
    s_a.inv_m1 = inv_m1;
  }
  __syncthreads();
  gv_reduce_task(s_a, t.y, t.z, t.w, s_part, s_emax, s_flags, s_won, sm);
}

// ---------------------------------------------------------------------------
// Histogram of the observable (the paper's differential distributions,
// Section 3.2), after the reduce of iteration k of a call.  Per bin b, from
// the once-rounded sums: H = sum w / C, V = (sum w^2 / C - H^2)/(C-1) (0 if
// rounding makes it negative).  The call's iterations are weighted as the
// integral is: u_k = 1/sigma_k^2, or, if any sigma_k is 0, 1 for those
// iterations and 0 for the others, so that the bins add up to the combined
// integral.  acc holds, in iteration order, sum u H and sum u^2 V over the
// iterations with sigma_k > 0, and sum H and sum V over those with
// sigma_k = 0; the last iteration writes value = sum u H / sum u and
// error = sqrt(sum u^2 V) / sum u.  One thread per bin: nothing depends on
// the launch shape.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) gv_hist_kernel(const GvHistArgs a) {
  const int nh = a.nhist;
  gv_wait_prior_grid();  // the reduce's sums and records
  gv_allow_next_grid();  // the next fill touches nothing this kernel reads or writes
  const double sk = a.per_iter[2 * a.k + 1];
  int nzero = 0;
  double W = 0.0;
  if (a.last) {
    for (int j = 0; j <= a.k; ++j)
      if (!(a.per_iter[2 * j + 1] > 0.0)) ++nzero;
    for (int j = 0; j <= a.k; ++j) {
      const double s = a.per_iter[2 * j + 1];
      W += nzero > 0 ? (s > 0.0 ? 0.0 : 1.0) : 1.0 / (s * s);
    }
  }
  for (int b = threadIdx.x; b < nh; b += blockDim.x) {
    const double h = a.sums[nh + b] * a.inv_c;
    double v = (a.sums[b] * a.inv_c - h * h) * a.inv_cm1;
    v = v > 0.0 ? v : 0.0;
    double A0 = 0.0, A1 = 0.0, A2 = 0.0, A3 = 0.0;
    if (a.k > 0) {
      A0 = a.acc[b];
      A1 = a.acc[nh + b];
      A2 = a.acc[2 * nh + b];
      A3 = a.acc[3 * nh + b];
    }
    if (sk > 0.0) {
      const double u = 1.0 / (sk * sk);
      A0 += u * h;
      A1 += u * u * v;
    } else {
      A2 += h;
      A3 += v;
    }
    a.acc[b] = A0;
    a.acc[nh + b] = A1;
    a.acc[2 * nh + b] = A2;
    a.acc[3 * nh + b] = A3;
    if (a.last) {
      a.out[b] = (nzero > 0 ? A2 : A0) / W;
      a.out[nh + b] = sqrt(nzero > 0 ? A3 : A1) / W;
    }
  }
}

// ---------------------------------------------------------------------------
// Derived constants of an integrand (launched when the parameters change).
// p[GV_MAXPARAMS - 1] carries the number of user parameters.
// ---------------------------------------------------------------------------
__global__ void gv_consts_kernel(int ig, const double* p, double* K) {
  if (threadIdx.x != 0) return;
  const int np = (int)p[GV_MAXPARAMS - 1];
  for (int i = 0; i < GV_NCONST; ++i) K[i] = 0.0;
  if (ig == GV_GAUSS) {
    K[GK_INV2S2] = 1.0 / (2.0 * p[0] * p[0]);
    K[GK_SHIFT] = np > 1 ? p[1] : 0.0;
  } else if (ig == GV_DY || ig == GV_DYNLO) {
    const double sqrt_s = p[0], MZ = p[1], GZ = p[2], sw2 = p[3], alpha = p[4];
    const double mlo = p[5], mhi = p[6];
    const double s = sqrt_s * sqrt_s;
    const double tau_lo = mlo * mlo / s, tau_hi = mhi * mhi / s;
    const double pi = 3.14159265358979323846;
    K[DK_SQRTS] = sqrt_s;
    K[DK_S] = s;
    K[DK_TAULO] = tau_lo;
    K[DK_L] = log(tau_hi / tau_lo);
    K[DK_LOGTAULO] = log(tau_lo);
    K[DK_MZ2] = MZ * MZ;
    K[DK_GM2] = (GZ * MZ) * (GZ * MZ);
    const double kappa = 1.0 / (4.0 * sw2 * (1.0 - sw2));
    K[DK_KAPPA] = kappa;
    // alpha^2/(4 N_c) * (hbar c)^2 [pb GeV^2] * Jacobians of cos(theta) (2) and phi (2 pi)
    K[DK_PREF] = alpha * alpha / (4.0 * 3.0) * 0.3893794e9 * 2.0 * (2.0 * pi);
    // couplings V = T3 - 2 Q sw2, A = T3; muon Q = -1, T3 = -1/2
    const double Vl = -0.5 + 2.0 * sw2, Al = -0.5, dVl = 2.0;
    double cA0 = 0, cA1 = 0, cA2 = 0, cB1 = 0, cB2 = 0, dA1 = 0, dA2 = 0, dB2 = 0;
    for (int t = 0; t < 2; ++t) {
      const double n = t == 0 ? 2.0 : 3.0;  // u, c  |  d, s, b
      const double Q = t == 0 ? 2.0 / 3.0 : -1.0 / 3.0;
      const double T3 = t == 0 ? 0.5 : -0.5;
      const double Vq = T3 - 2.0 * Q * sw2, Aq = T3, dVq = -2.0 * Q;
      cA0 += n * Q * Q;
      cA1 += n * (-2.0 * Q * Vl * Vq);
      cA2 += n * (Al * Al + Vl * Vl) * (Aq * Aq + Vq * Vq);
      cB1 += n * (-4.0 * Q * Al * Aq);
      cB2 += n * (8.0 * Al * Vl * Aq * Vq);
      dA1 += n * (-2.0 * Q * (dVl * Vq + Vl * dVq));
      dA2 += n * (2.0 * Vl * dVl * (Aq * Aq + Vq * Vq) + (Al * Al + Vl * Vl) * 2.0 * Vq * dVq);
      dB2 += n * (8.0 * Al * Aq * (dVl * Vq + Vl * dVq));
    }
    K[DK_CA0] = cA0;
    K[DK_CA1] = cA1;
    K[DK_CA2] = cA2;
    K[DK_CB1] = cB1;
    K[DK_CB2] = cB2;
    K[DK_A] = p[7];
    K[DK_B] = p[8];
    K[DK_NORM] = 0.2 * p[9] * p[9];
    K[DK_MZ] = MZ;
    K[DK_GZ] = GZ;
    K[DK_DKAPPA] = -kappa * (1.0 - 2.0 * sw2) / (sw2 * (1.0 - sw2));
    K[DK_DCA1] = dA1;
    K[DK_DCA2] = dA2;
    K[DK_DCB2] = dB2;
    if (ig == GV_DYNLO) {
      // beta and 1 / I0(beta), I0(beta) = sum_k ((beta/2)^k / k!)^2
      const double beta = p[10];
      double term = 1.0, i0 = 1.0;
      for (int k = 1; k < 200 && term >= 1e-18 * i0; ++k) {
        term *= (0.25 * beta * beta) / ((double)k * (double)k);
        i0 += term;
      }
      K[NK_BETA] = beta;
      K[NK_INVI0] = 1.0 / i0;
    }
  } else if (ig == GV_EE3J) {
    const double Q = np > 1 ? p[1] : 91.1876;
    K[EK_YCUT] = p[0];
    K[EK_Q] = Q;
    K[EK_INVQ2] = 1.0 / (Q * Q);
  }
  float* kf = reinterpret_cast<float*>(K + GV_NCONST_F32);
  for (int i = 0; i < GV_NCONST_F32; ++i) kf[i] = (float)K[i];
}

// Reset the per-iteration state (at creation and after the autotuner's
// trial launches).
__global__ void gv_reset_kernel(GvState* st) {
  if (threadIdx.x == 0) st->nonfinite_iter = 0ull;
}

__global__ void gv_grid_pack_kernel(double* grid, int d, int N) {
  // in place: each axis reads its own edges before writing them back unchanged
  for (int ax = 0; ax < d; ++ax) {
    pack_axis_tables(grid, grid + GvGridLayout{d, N}.off_e64() + (size_t)ax * (N + 1), ax, d, N,
                     threadIdx.x, blockDim.x);
    __syncthreads();
  }
}

__global__ void gv_rng_words_kernel(unsigned long long seed, uint32_t it, uint32_t batch,
                                    unsigned long long ev0, long long n, int d, uint32_t* out) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  uint32_t r[GV_MAXD];
  gv_event_words<GV_MAXD>(seed, it, batch, ev0 + (unsigned long long)j, d, r);
  for (int a = 0; a < d; ++a) out[j * d + a] = r[a];
}

namespace gv {
size_t reduce_smem_bytes(int N) { return gv_axes_per_block(N) * refine_axis_smem(N); }

// Reduce grid: 32 accumulators per CTA; at most 64 tile ranges.
void reduce_grid(int n_tiles, int nacc, int* tiles_per_cta, int* gx, int* gy) {
  const int tpc = n_tiles <= 64 ? std::max(1, n_tiles) : std::max(64, (n_tiles + 63) / 64);
  *tiles_per_cta = tpc;
  *gx = (nacc + 31) / 32;
  *gy = (n_tiles + tpc - 1) / tpc;
}

static cudaError_t allow_smem(const void* k, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_reduce(const GvReduceArgs& a, size_t smem, cudaStream_t s, bool pdl) {
  int tpc, gx, gy;
  reduce_grid(a.n_tiles, a.nacc, &tpc, &gx, &gy);
  if (tpc != a.tiles_per_cta) return cudaErrorInvalidValue;
  cudaError_t e = allow_smem((const void*)gv_reduce_kernel, smem);
  if (e != cudaSuccess) return e;
  return gv_launch(gv_reduce_kernel, dim3(gx, gy), dim3(256), smem, s, pdl, a);
}

// Threads per slot of the single-level reduce: up to 4 tiles per thread
// where that takes at most 256 threads, else 256.
int reduce_slots_threads(int n_tiles) {
  return n_tiles <= 128 ? 32 : (n_tiles <= 256 ? 64 : (n_tiles <= 512 ? 128 : 256));
}

cudaError_t launch_reduce_slots(const GvReduceArgs& a, size_t smem, cudaStream_t s, bool pdl) {
  const int gt = reduce_slots_threads(a.n_tiles);
  const int ng = 256 / gt;
  const dim3 grid((a.nacc + ng - 1) / ng);
  cudaError_t e = cudaSuccess;
  switch (gt) {
    case 32:
      e = allow_smem((const void*)gv_reduce_slots_kernel<32>, smem);
      return e ? e : gv_launch(gv_reduce_slots_kernel<32>, grid, dim3(256), smem, s, pdl, a);
    case 64:
      e = allow_smem((const void*)gv_reduce_slots_kernel<64>, smem);
      return e ? e : gv_launch(gv_reduce_slots_kernel<64>, grid, dim3(256), smem, s, pdl, a);
    case 128:
      e = allow_smem((const void*)gv_reduce_slots_kernel<128>, smem);
      return e ? e : gv_launch(gv_reduce_slots_kernel<128>, grid, dim3(256), smem, s, pdl, a);
    default:
      e = allow_smem((const void*)gv_reduce_slots_kernel<256>, smem);
      return e ? e : gv_launch(gv_reduce_slots_kernel<256>, grid, dim3(256), smem, s, pdl, a);
  }
}

cudaError_t launch_reduce_batch(const GvReduceArgs* args, const int4* tasks, int ntasks, int k,
                                int last, double inv_m1, size_t smem, cudaStream_t s) {
  cudaError_t e = allow_smem((const void*)gv_reduce_batch_kernel, smem);
  if (e != cudaSuccess) return e;
  gv_reduce_batch_kernel<<<ntasks, 256, smem, s>>>(args, tasks, k, last, inv_m1);
  return cudaGetLastError();
}

cudaError_t launch_hist(const GvHistArgs& a, cudaStream_t s, bool pdl) {
  return gv_launch(gv_hist_kernel, dim3(1), dim3(256), 0, s, pdl, a);
}

cudaError_t launch_consts(int integrand, const double* params, double* kconst, cudaStream_t s) {
  gv_consts_kernel<<<1, 32, 0, s>>>(integrand, params, kconst);
  return cudaGetLastError();
}

cudaError_t launch_reset(GvState* st, cudaStream_t s) {
  gv_reset_kernel<<<1, 32, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t launch_grid_pack(int d, int N, double* grid, cudaStream_t s) {
  gv_grid_pack_kernel<<<1, 256, 0, s>>>(grid, d, N);
  return cudaGetLastError();
}

cudaError_t launch_rng_words(unsigned long long seed, uint32_t it, uint32_t batch,
                             unsigned long long ev0, long long n, int d, uint32_t* out,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int thr = 256;
  gv_rng_words_kernel<<<(unsigned)((n + thr - 1) / thr), thr, 0, s>>>(seed, it, batch, ev0, n, d,
                                                                     out);
  return cudaGetLastError();
}
}  // namespace gv
