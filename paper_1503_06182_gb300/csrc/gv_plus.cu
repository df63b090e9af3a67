// gv_plus.cu -- VEGAS+ (adaptive stratified sampling on the VEGAS map;
// Lepage, J. Comput. Phys. 439 (2021) 110386, a later form of the VEGAS
// method cited in Section 2.1) after each iteration:
//   seg:    each lane sums J g and its square over GV_PLUS_SEG consecutive
//           events, in event order, split where the hypercube changes (every
//           lane does the same number of steps: the FP64 pipe, which this chip
//           has little of, does no work for idle lanes);
//   stats:  one thread per hypercube adds its segments in range order, then
//           forms its sample variance v_h, v_h/n_h and the allocation weight
//           v_h^(beta/2) (divisions by n and n - 1 as products with tabulated
//           reciprocals: FP64 division is a long sequence on the FP64 pipe);
//           the CTA that completes the grid (ticket) forms
//           sigma_k^2 = sum v_h/n_h / nh^2 and D = sum of the weights, writes
//           sigma_k and, at the last iteration, combines the stage;
//   alloc:  n_h = max(2, floor(C d_h / D)) (floor(C/nh) if D = 0 or for the
//           uniform start), per-CTA event counts; the completing CTA scans
//           them (exact integers);
//   layout: the offsets of the hypercubes, (C/(nh n_h), sqrt(1/(nh n_h))) and
//           each tile's first hypercube for the next fill.
// Every sum over hypercubes has a shape fixed by nh alone, every count is an
// integer, and no CTA waits for another: the last one to arrive does the rest.
#include "gv_combine.cuh"

namespace {

constexpr int kT = 256;  // threads per CTA, one hypercube each

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

// Sum over the CTA in a fixed order, with few FP64 instructions (this chip's
// FP64 pipe is narrow): warp 0's lane l adds the values of threads 8l..8l+7
// in order, then a butterfly over the warp.  The result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* s) {
  s[threadIdx.x] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    const double* q = s + 8 * threadIdx.x;
    r = q[0];
#pragma unroll
    for (int i = 1; i < 8; ++i) r += q[i];
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) r += __shfl_xor_sync(0xffffffffu, r, m);
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

// The completing CTA: the sum of nb per-CTA values in CTA order, each thread
// taking a contiguous run, then the fixed tree.
__device__ __forceinline__ double sum_parts(const double* part, int stride, int nb, double* s) {
  const int chunk = (nb + kT - 1) / kT;
  const int i0 = threadIdx.x * chunk, i1 = min(nb, i0 + chunk);
  double v = 0.0;
  for (int i = i0; i < i1; ++i) v += __ldcg(part + (size_t)i * stride);
  return block_sum(v, s);
}

}  // namespace

// Range r = events [r K, r K + K) (K = GV_PLUS_SEG): its segments, one per
// hypercube it meets, at seg[r K + j] for the j-th hypercube from hc[r K].
__global__ void __launch_bounds__(kT) gv_plus_seg_kernel(const GvPlusArgs a) {
  gv_wait_prior_grid();  // the fill's J g values and hypercubes
  const long long ncall = __ldcg(a.ncall_dev);
  const long long r = (long long)blockIdx.x * kT + threadIdx.x;
  const long long e0 = r * GV_PLUS_SEG;
  gv_allow_next_grid();
  if (e0 >= ncall) return;
  const long long e1 = e0 + GV_PLUS_SEG < ncall ? e0 + GV_PLUS_SEG : ncall;
  int hp = a.hc[e0];
  long long j = e0;
  double s1 = 0.0, s2 = 0.0;
  for (long long e = e0; e < e1; ++e) {
    const int h = a.hc[e];
    if (h != hp) {
      a.seg[j++] = make_double2(s1, s2);
      s1 = 0.0;
      s2 = 0.0;
      hp = h;
    }
    const double f = a.F[e];
    s1 += f;
    s2 += f * f;
  }
  a.seg[j] = make_double2(s1, s2);
}

__global__ void __launch_bounds__(kT) gv_plus_stats_kernel(const GvPlusArgs a) {
  __shared__ double s_red[kT];
  __shared__ int s_last;
  gv_wait_prior_grid();  // the segments and the reduce's I_k
  const long long h = (long long)blockIdx.x * kT + threadIdx.x;
  double vn = 0.0, dd = 0.0;
  if (h < a.nh) {
    const long long o = a.off[h];
    const int m = a.n[h];
    // the hypercube's segments, range by range: in its first range it is the
    // (h - hc[first event])-th segment; every later range starts inside it
    const long long r0 = o / GV_PLUS_SEG, r1 = (o + m - 1) / GV_PLUS_SEG;
    const long long b0 = r0 * GV_PLUS_SEG;
    double2 sg = a.seg[b0 + (h - a.hc[b0])];
    double s1 = sg.x, s2 = sg.y;
    for (long long r = r0 + 1; r <= r1; ++r) {
      sg = a.seg[r * GV_PLUS_SEG];
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
  vn = block_sum(vn, s_red);
  dd = block_sum(dd, s_red);
  if (threadIdx.x == 0) {
    a.part[2 * (size_t)blockIdx.x] = vn;
    a.part[2 * (size_t)blockIdx.x + 1] = dd;
    __threadfence();
    s_last = atomicAdd(a.tickets, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();  // the other CTAs' sums, published before their tickets
  const int nb = gridDim.x;
  const double V = sum_parts(a.part, 2, nb, s_red);
  const double D = sum_parts(a.part + 1, 2, nb, s_red);
  if (threadIdx.x == 0) {
    a.tickets[0] = 0;
    const double var_k = V * a.inv_nh2;
    a.scal[0] = var_k;
    a.scal[1] = D;
    a.per_iter[2 * a.k + 1] = var_k > 0.0 ? sqrt(var_k) : 0.0;
    __threadfence_block();
  }
  __syncthreads();
  if (a.last && threadIdx.x < 32)
    combine_stage_warp(a.per_iter, 2, a.k + 1, a.inv_m1, a.st, false);
}

__global__ void __launch_bounds__(kT) gv_plus_alloc_kernel(const GvPlusArgs a) {
  __shared__ long long s_scan[kT / 32];
  __shared__ int s_last;
  gv_wait_prior_grid();  // the weights and their sum
  const double D = a.uniform ? 0.0 : __ldcg(a.scal + 1);
  const long long h = (long long)blockIdx.x * kT + threadIdx.x;
  long long m = 0;
  if (h < a.nh) {
    long long k;
    if (D > 0.0) {
      // a true division, as the rule states it: shares land on integers
      // exactly (one hypercube, equal weights), where a product with 1/D
      // would fall an ulp short and floor one event lower
      const double x = (double)a.ncall * __ldcg(a.dw + h) / D;
      k = (long long)floor(x);
    } else {
      k = a.ncall / a.nh;
    }
    m = k > 2 ? k : 2;
    a.n[h] = (int)m;
  }
  gv_allow_next_grid();
  long long tot;
  block_exscan(m, s_scan, &tot);
  if (threadIdx.x == 0) {
    a.npart[blockIdx.x] = tot;
    __threadfence();
    s_last = atomicAdd(a.tickets + 1, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // exclusive scan of the per-CTA counts, in place
  const int nb = gridDim.x;
  const int chunk = (nb + kT - 1) / kT;
  const int i0 = threadIdx.x * chunk, i1 = min(nb, i0 + chunk);
  long long run = 0;
  for (int i = i0; i < i1; ++i) run += __ldcg(a.npart + i);
  long long all;
  long long base = block_exscan(run, s_scan, &all);
  for (int i = i0; i < i1; ++i) {
    const long long v = __ldcg(a.npart + i);
    a.npart[i] = base;
    base += v;
  }
  if (threadIdx.x == 0) {
    a.tickets[1] = 0;
    *a.ncall_dev = all;
  }
}

__global__ void __launch_bounds__(kT) gv_plus_layout_kernel(const GvPlusArgs a) {
  __shared__ long long s_scan[kT / 32];
  gv_wait_prior_grid();  // the counts and the per-CTA bases
  const long long h = (long long)blockIdx.x * kT + threadIdx.x;
  const long long m = h < a.nh ? (long long)a.n[h] : 0ll;
  long long tot;
  const long long o = __ldcg(a.npart + blockIdx.x) + block_exscan(m, s_scan, &tot);
  if (h < a.nh) {
    a.off[h] = o;
    if (m < GV_PLUS_NTAB) {
      a.ab[h] = __ldg(a.abtab + m);
    } else {
      const double nhd = (double)a.nh * (double)m;
      a.ab[h] = make_double2((double)a.ncall / nhd, sqrt(1.0 / nhd));
    }
    // the tiles whose first event lies in this hypercube
    for (long long t = (o + GV_TILE - 1) / GV_TILE; t * GV_TILE < o + m; ++t)
      a.tile_h0[t] = (int)h;
    if (h == a.nh - 1) {
      a.off[a.nh] = o + m;
      // tiles past the last event start in the last hypercube (they hold no event)
      for (long long t = (o + m + GV_TILE - 1) / GV_TILE; t < a.n_tiles; ++t)
        a.tile_h0[t] = (int)h;
    }
  }
}

namespace gv {

cudaError_t launch_plus_seg(const GvPlusArgs& a, cudaStream_t s, bool pdl) {
  const long long ranges = (a.cap + GV_PLUS_SEG - 1) / GV_PLUS_SEG;
  const unsigned nb = (unsigned)((ranges + kT - 1) / kT);
  return gv_launch(gv_plus_seg_kernel, dim3(nb), dim3(kT), 0, s, pdl, a);
}

cudaError_t launch_plus_stats(const GvPlusArgs& a, cudaStream_t s, bool pdl) {
  const unsigned nb = (unsigned)((a.nh + kT - 1) / kT);
  return gv_launch(gv_plus_stats_kernel, dim3(nb), dim3(kT), 0, s, pdl, a);
}

cudaError_t launch_plus_alloc(const GvPlusArgs& a, cudaStream_t s, bool pdl) {
  const unsigned nb = (unsigned)((a.nh + kT - 1) / kT);
  return gv_launch(gv_plus_alloc_kernel, dim3(nb), dim3(kT), 0, s, pdl, a);
}

cudaError_t launch_plus_layout(const GvPlusArgs& a, cudaStream_t s, bool pdl) {
  const unsigned nb = (unsigned)((a.nh + kT - 1) / kT);
  return gv_launch(gv_plus_layout_kernel, dim3(nb), dim3(kT), 0, s, pdl, a);
}

}  // namespace gv
