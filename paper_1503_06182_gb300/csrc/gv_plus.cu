// gv_plus.cu -- VEGAS+ (adaptive stratified sampling on the VEGAS map;
// Lepage, J. Comput. Phys. 439 (2021) 110386, a later form of the VEGAS
// method cited in Section 2.1) after each iteration.  The stratified fill has
// left the sums of J g and its square over each GV_PLUS_SEG-event range's run
// of each hypercube (its segments, in event order): a hypercube's first
// segment at its index, a range's continuation of an earlier one at the
// range's.
//   stats:  one thread per hypercube adds its segments in range order, then
//           forms its sample variance v_h, v_h/n_h and the allocation weight
//           v_h^(beta/2) (divisions by n and n - 1 as products with tabulated
//           reciprocals: FP64 division is a long sequence on the FP64 pipe);
//           the CTA that completes the grid (ticket) forms
//           sigma_k^2 = sum v_h/n_h / nh^2 and D = sum of the weights and
//           writes sigma_k; at the stage's last iteration, of this CTA and the
//           reduce (which runs beside these kernels) the second to arrive
//           combines the stage;
//   alloc:  n_h = max(2, floor(C d_h / D)) (floor(C/nh) if D = 0 or for the
//           uniform start), per-CTA event counts; the completing CTA scans
//           them (exact integers);
//   layout: the offsets of the hypercubes, (C/(nh n_h), sqrt(1/(nh n_h))) (in
//           FP64 and rounded to FP32, for the two forms' fills) and each
//           tile's first hypercube for the next fill.
// Every sum over hypercubes has a shape fixed by nh alone, every count is an
// integer, and no CTA waits for another: the last one to arrive does the rest.
#include "gv_combine.cuh"

namespace {

constexpr int kT = 256;  // threads per CTA, one hypercube each
// 8 CTAs per SM (at most 32 registers): 1216 resident CTAs on 152 SMs hold a
// million-event iteration's 234,256 hypercubes (916 CTAs) in one wave; at 6
// (38 registers) its last four CTAs ran as a second wave, a whole CTA
// lifetime later
constexpr int kMinBlocks = 8;
constexpr int kG = 32;  // CTAs per group of the two-level completion counters

// v^(j/8) (beta = j/4) from correctly rounded operations only: v = t 2^(8q)
// with t in [1/2, 128) rounded to FP32, three FP32 square roots, j - 1 FP32
// products, and 2^(q j) exactly.
// The exponent split, the FP32 rounding of t, the widening of the FP32
// result and the final scaling are exact bit operations here (frexp, a
// conversion to nearest, a widening and ldexp, written with integers: their
// library and hardware forms run on the FP64 pipe, which this chip has little
// of); a subnormal v takes the library path.
__device__ __forceinline__ double plus_weight(double v, int j) {
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

// Two sums over the CTA in a fixed order, with few FP64 instructions (this
// chip's FP64 pipe is narrow) and one latency chain for both: warp 0's lane l
// adds the values of threads 8l..8l+7 in order, then a butterfly over the
// warp.  The result is valid in thread 0.
__device__ __forceinline__ double2 block_sum2(double2 v, double2* s) {
  s[threadIdx.x] = v;
  __syncthreads();
  double2 r = make_double2(0.0, 0.0);
  if (threadIdx.x < 32) {
    const double2* q = s + 8 * threadIdx.x;
    r = q[0];
#pragma unroll
    for (int i = 1; i < 8; ++i) {
      r.x += q[i].x;
      r.y += q[i].y;
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      r.x += __shfl_xor_sync(0xffffffffu, r.x, m);
      r.y += __shfl_xor_sync(0xffffffffu, r.y, m);
    }
  }
  __syncthreads();
  return r;
}

// Exclusive prefix sum over the CTA (integers: any order is exact).
__device__ __forceinline__ long long block_exscan(long long v, long long* s, long long* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) s[wid] = x;
  __syncthreads();
  long long base = 0, all = 0;
#pragma unroll
  for (int w = 0; w < kT / 32; ++w) {
    const long long sw = s[w];
    base += w < wid ? sw : 0ll;
    all += sw;
  }
  __syncthreads();
  *total = all;
  return base + x - v;
}

// 1/n and 1/(n - 1) beyond the tables (kept out of line, so that the common
// path does not carry two FP64 divisions)
__device__ __noinline__ void plus_recips(double n, double* inv_n, double* inv_m1) {
  *inv_n = 1.0 / n;
  *inv_m1 = 1.0 / (n - 1.0);
}

// Per-CTA values a completing CTA's thread holds in registers (up to kT kR
// CTAs: all loads in flight at once; more are read in a loop).
constexpr int kR = 4;

// The completing CTA: the sums of nb per-CTA pairs in CTA order, each thread
// taking a contiguous run, then the fixed tree.
__device__ __forceinline__ double2 sum_parts2(const double2* part, int nb, double2* s) {
  const int chunk = (nb + kT - 1) / kT;
  const int i0 = threadIdx.x * chunk, i1 = min(nb, i0 + chunk);
  double2 v = make_double2(0.0, 0.0);
  if (chunk <= kR) {
    double2 p[kR];
#pragma unroll
    for (int q = 0; q < kR; ++q) p[q] = i0 + q < i1 ? __ldcg(part + i0 + q) : make_double2(0.0, 0.0);
#pragma unroll
    for (int q = 0; q < kR; ++q) {
      if (i0 + q < i1) {
        v.x += p[q].x;
        v.y += p[q].y;
      }
    }
  } else {
    for (int i = i0; i < i1; ++i) {
      const double2 p = __ldcg(part + i);
      v.x += p.x;
      v.y += p.y;
    }
  }
  return block_sum2(v, s);
}

// floor(x / D) with x / D rounded to nearest, as the allocation rule states
// it, for x >= 0 and D > 0 with 1/D rounded to nearest given.  y = x (1/D)
// lies within 3 units in the last place of the rounded quotient q, so when
// no integer lies within 8 units of y, floor(q) = floor(y), read from y's
// bits on the integer pipes; otherwise (equal weights put shares on
// integers) the true division decides.
__device__ __forceinline__ long long floor_quotient(double x, double D, double rD) {
  const double y = x * rD;
  const long long b = __double_as_longlong(y);
  const int E = (int)(b >> 52) - 1023;  // y in [2^E, 2^(E+1)) (y >= 0)
  if (E < 0) {
    // below 1 (and 8 units clear of it): floor 0
    if (b < __double_as_longlong(1.0) - 8) return 0;
  } else if (E < 52) {
    const unsigned long long M = ((unsigned long long)b & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = 52 - E;
    const unsigned long long F = M & ((1ull << sh) - 1ull);  // fraction, in units of y
    if (F > 8ull && (1ull << sh) - F > 8ull) return (long long)(M >> sh);
  }
  return (long long)floor(x / D);
}

}  // namespace

__global__ void __launch_bounds__(kT, kMinBlocks) gv_plus_stats_kernel(const GvPlusArgs a) {
  __shared__ double2 s_red[kT];
  __shared__ int s_last;
  gv_wait_prior_grid();  // the fill's segments and the reduce's I_k
  const long long h = (long long)blockIdx.x * kT + threadIdx.x;
  double vn = 0.0, dd = 0.0;
  if (h < a.nh) {
    const long long o = a.off[h];
    const int m = a.n[h];
    // the hypercube's segments in event order: its first, then the
    // continuations of every later range it reaches
    double2 sg = a.seg_h[h];
    const long long r0 = o / GV_PLUS_SEG, r1 = (o + m - 1) / GV_PLUS_SEG;
    double s1 = sg.x, s2 = sg.y;
    for (long long r = r0 + 1; r <= r1; ++r) {
      sg = a.seg_r[r];
      s1 += sg.x;
      s2 += sg.y;
    }
    const double nd = (double)m;
    double inv_n, inv_m1;
    if (m < GV_PLUS_NTAB) {
      inv_n = __ldg(a.inv + m);
      inv_m1 = __ldg(a.inv + m - 1);
    } else {
      plus_recips(nd, &inv_n, &inv_m1);
    }
    double v = (s2 - s1 * s1 * inv_n) * inv_m1;
    v = __double_as_longlong(v) > 0ll ? v : 0.0;  // negative (rounding) or -0 -> 0
    a.var[h] = v;
    vn = v * inv_n;
    dd = plus_weight(v, a.beta_j);
    a.dw[h] = dd;
  }
  gv_allow_next_grid();
  const double2 sums = block_sum2(make_double2(vn, dd), s_red);
  // two-level completion: the last CTA of each group of kG adds the group's
  // sums (in CTA order, a fixed tree); the last group adds the groups'
  const int b = blockIdx.x, nb = gridDim.x;
  const int g = b / kG, ng = (nb + kG - 1) / kG, gsize = min(kG, nb - g * kG);
  if (threadIdx.x == 0) {
    reinterpret_cast<double2*>(a.part)[b] = sums;
    __threadfence();
    s_last = atomicAdd(a.gctr + g, 1) == gsize - 1;
  }
  __syncthreads();
  if (!s_last) return;
  if (threadIdx.x < 32) {
    __threadfence();  // the group's sums, published before their arrivals
    double2 v = threadIdx.x < gsize ? __ldcg(reinterpret_cast<const double2*>(a.part) + g * kG + threadIdx.x)
                                    : make_double2(0.0, 0.0);
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      v.x += __shfl_xor_sync(0xffffffffu, v.x, m);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, m);
    }
    if (threadIdx.x == 0) {
      a.gpart[g] = v;
      a.gctr[g] = 0;
      __threadfence();
      s_last = atomicAdd(a.gctr + ng, 1) == ng - 1;
    }
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();  // the groups' sums, published before their arrivals
  const double2 VD = sum_parts2(a.gpart, ng, s_red);
  if (threadIdx.x == 0) {
    a.gctr[ng] = 0;
    const double var_k = VD.x * a.inv_nh2;
    const double D = VD.y;
    a.scal[0] = var_k;
    a.scal[1] = D;
    a.scal[2] = D > 0.0 ? 1.0 / D : 0.0;
    a.per_iter[2 * a.k + 1] = var_k > 0.0 ? sqrt(var_k) : 0.0;
    // the stage's last iteration: the reduce runs beside this kernel, and the
    // second of the two to arrive combines the stage
    s_last = 0;
    if (a.last) {
      __threadfence();  // sigma_k before the arrival
      s_last = atomicAdd(&a.st->join, 1) == 1;
    }
  }
  __syncthreads();
  if (s_last && threadIdx.x < 32) {
    __threadfence();  // the reduce's I_k, published before its arrival
    combine_stage_warp(a.per_iter, 2, a.k + 1, a.inv_m1, a.st, false);
    if (threadIdx.x == 0) a.st->join = 0;
  }
}

// The next allocation's count of hypercube h (h < nh): n_h = max(2,
// floor(C d_h / D)), or floor(C / nh) everywhere for the uniform start or
// when every weight is zero.
__device__ __forceinline__ long long plus_count(const GvPlusArgs& a, long long h, double D,
                                                double rD) {
  long long k;
  if (D > 0.0) {
    // floor of the rounded quotient C d_h / D, as the rule states it: shares
    // land on integers exactly (one hypercube, equal weights), where
    // floor(x (1/D)) would fall an ulp short and one event lower
    k = floor_quotient((double)a.ncall * __ldcg(a.dw + h), D, rD);
  } else {
    k = a.ncall / a.nh;
  }
  return k > 2 ? k : 2;
}

// Hypercube h's layout from its count m and first event o: its offset, its
// factors (C/(nh m), sqrt(1/(nh m))) in FP64 and FP32, the tiles whose first
// event lies in it, and after the last hypercube the total and the tiles
// past it.
__device__ __forceinline__ void plus_layout_one(const GvPlusArgs& a, long long h, long long m,
                                                long long o) {
  a.off[h] = o;
  double2 f;
  if (m < GV_PLUS_NTAB) {
    f = __ldg(a.abtab + m);
  } else {
    const double nhd = (double)a.nh * (double)m;
    f = make_double2((double)a.ncall / nhd, sqrt(1.0 / nhd));
  }
  a.ab[h] = f;
  a.ab32[h] = make_float2(__double2float_rn(f.x), __double2float_rn(f.y));
  for (long long t = (o + GV_TILE - 1) / GV_TILE; t * GV_TILE < o + m && t < a.n_tiles; ++t)
    a.tile_h0[t] = (int)h;
  if (h == a.nh - 1) {
    a.off[a.nh] = o + m;
    *a.ncall_dev = o + m;
    // tiles past the last event start in the last hypercube (they hold no event)
    for (long long t = (o + m + GV_TILE - 1) / GV_TILE; t < a.n_tiles; ++t) a.tile_h0[t] = (int)h;
  }
}

// Counts of the next allocation: per CTA their sum (agg); the last CTA of each
// group of kG CTAs (a counter per group, so arrivals spread over many
// addresses) adds its group's (gsum).  Nothing waits; the layout reads them
// after this kernel.
__global__ void __launch_bounds__(kT, kMinBlocks) gv_plus_alloc_kernel(const GvPlusArgs a) {
  __shared__ long long s_scan[kT / 32];
  __shared__ int s_last;
  gv_wait_prior_grid();  // the weights and their sum
  const double D = a.uniform ? 0.0 : __ldcg(a.scal + 1);
  const double rD = a.uniform ? 0.0 : __ldcg(a.scal + 2);
  const int b = blockIdx.x, nb = gridDim.x;
  const long long h = (long long)b * kT + threadIdx.x;
  long long m = 0;
  if (h < a.nh) {
    m = plus_count(a, h, D, rD);
    a.n[h] = (int)m;
  }
  gv_allow_next_grid();
  long long tot;
  block_exscan(m, s_scan, &tot);
  const int g = b / kG, gsize = min(kG, nb - g * kG);
  int* ctr = a.gctr + ((nb + kG - 1) / kG) + 1 + g;
  if (threadIdx.x == 0) {
    a.npart[b] = tot;
    __threadfence();
    s_last = atomicAdd(ctr, 1) == gsize - 1;
  }
  __syncthreads();
  if (!s_last || threadIdx.x >= 32) return;
  __threadfence();  // the group's counts, published before their arrivals
  long long v = threadIdx.x < gsize ? __ldcg(a.npart + g * kG + threadIdx.x) : 0ll;
#pragma unroll
  for (int k = 16; k > 0; k >>= 1) v += __shfl_xor_sync(0xffffffffu, v, k);
  if (threadIdx.x == 0) {
    a.gsum[g] = v;
    *ctr = 0;
  }
}

// The layout: CTA b's first event is the sum of the groups before its group
// (gsum) and of the CTAs before it in its group (agg), then each hypercube's
// by the CTA's scan.
__global__ void __launch_bounds__(kT, kMinBlocks) gv_plus_layout_kernel(const GvPlusArgs a) {
  __shared__ long long s_scan[kT / 32];
  gv_wait_prior_grid();  // the counts and their per-CTA and per-group sums
  // the next fill may come in now: it makes its Philox words, then waits
  // for this kernel to finish
  gv_allow_next_grid();
  const int b = blockIdx.x, g = b / kG;
  const long long h = (long long)b * kT + threadIdx.x;
  const long long m = h < a.nh ? (long long)a.n[h] : 0ll;
  // thread t adds the groups t, t + kT, .. below g and, the CTA t - (kT - kG)
  // of its group below b
  long long pre = 0;
  for (int q = threadIdx.x; q < g; q += kT) pre += __ldcg(a.gsum + q);
  const int c = threadIdx.x - (kT - kG);
  if (c >= 0 && g * kG + c < b) pre += __ldcg(a.npart + g * kG + c);
  long long all, tot;
  block_exscan(pre, s_scan, &all);  // all: the CTA's first event
  const long long o = all + block_exscan(m, s_scan, &tot);
  if (h < a.nh) plus_layout_one(a, h, m, o);
}

namespace gv {

cudaError_t launch_plus_stats(const GvPlusArgs& a, cudaStream_t s, bool pdl) {
  const unsigned nb = (unsigned)((a.nh + kT - 1) / kT);
  return gv_launch_prio(gv_plus_stats_kernel, dim3(nb), dim3(kT), 0, s, pdl, a.prio, a);
}

cudaError_t launch_plus_alloc(const GvPlusArgs& a, cudaStream_t s, bool pdl) {
  const unsigned nb = (unsigned)((a.nh + kT - 1) / kT);
  return gv_launch_prio(gv_plus_alloc_kernel, dim3(nb), dim3(kT), 0, s, pdl, a.prio, a);
}

cudaError_t launch_plus_layout(const GvPlusArgs& a, cudaStream_t s, bool pdl) {
  const unsigned nb = (unsigned)((a.nh + kT - 1) / kT);
  return gv_launch_prio(gv_plus_layout_kernel, dim3(nb), dim3(kT), 0, s, pdl, a.prio, a);
}

}  // namespace gv
