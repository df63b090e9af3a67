// gv_plus.cu -- VEGAS+ (adaptive stratified sampling on the VEGAS map;
// Lepage, J. Comput. Phys. 439 (2021) 110386, a later form of the VEGAS
// method cited in Section 2.1) after each iteration.  The stratified fill has
// formed the statistics of every hypercube whose events lie in one tile, with
// each tile's sums of their v_h/n_h and weights, and left the segments (sums
// of J g and its square over a range's run of a hypercube, in event order) of
// the hypercubes that cross a tile boundary:
//   finish: 16 CTAs add the tiles' sums in tile order and form the
//           statistics of the crossing hypercubes (gv_plus_stat.cuh: the
//           sample variance v_h, v_h/n_h and the allocation weight
//           v_h^(beta/2)), then sigma_k^2 = sum v_h/n_h / nh^2 and D = sum
//           of the weights (the last CTA to arrive adds the CTAs' sums in
//           order), and writes sigma_k; at the stage's last
//           iteration, of this kernel and the reduce (which runs beside it)
//           the second to arrive combines the stage;
//   alloc:  n_h = max(2, floor(C d_h / D)) (floor(C/nh) if D = 0 or for the
//           uniform start), per-CTA event counts; the completing CTA scans
//           them (exact integers);
//   layout: the offsets of the hypercubes, (C/(nh n_h), sqrt(1/(nh n_h))) (in
//           FP64 and rounded to FP32, for the two forms' fills) and each
//           tile's first hypercube for the next fill.
// Every sum over hypercubes has a shape fixed by the allocation alone, every
// count is an integer, and no CTA waits for another: the last one to arrive
// does the rest.
#include "gv_combine.cuh"
#include "gv_plus_stat.cuh"

namespace {

constexpr int kT = 256;  // threads per CTA of the allocation and layout, one hypercube each
// 8 CTAs per SM (at most 32 registers): 1216 resident CTAs on 152 SMs hold a
// million-event iteration's 234,256 hypercubes (916 CTAs) in one wave; at 6
// (38 registers) its last four CTAs ran as a second wave, a whole CTA
// lifetime later
constexpr int kMinBlocks = 8;
constexpr int kG = 32;  // CTAs per group of the two-level completion counters

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

constexpr int kFC = 16;   // CTAs of the finishing kernel
constexpr int kTF = 256;  // their threads

// Two sums over a CTA of kTF threads in a fixed order, with few FP64
// instructions (this chip's FP64 pipe is narrow) and one latency chain for
// both: warp 0's lane l adds the values of threads 8l..8l+7 in order, then a
// butterfly over the warp.  The result is valid in thread 0.
__device__ __forceinline__ double2 block_sum2(double2 v, double2* s) {
  constexpr int L = kTF / 32;
  s[threadIdx.x] = v;
  __syncthreads();
  double2 r = make_double2(0.0, 0.0);
  if (threadIdx.x < 32) {
    const double2* q = s + L * threadIdx.x;
    r = q[0];
#pragma unroll
    for (int i = 1; i < L; ++i) {
      r.x += q[i].x;
      r.y += q[i].y;
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      r.x += __shfl_xor_sync(0xffffffffu, r.x, m);
      r.y += __shfl_xor_sync(0xffffffffu, r.y, m);
    }
  }
  return r;
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

__global__ void __launch_bounds__(kTF) gv_plus_finish_kernel(const GvPlusArgs a) {
  __shared__ double2 s_red[kTF];
  __shared__ int s_last;
  gv_wait_prior_grid();  // the fill's tile sums and crossing segments
  gv_allow_next_grid();
  const long long T = (__ldcg(a.ncall_dev) + GV_TILE - 1) / GV_TILE;  // tiles with events
  // CTA c takes the c-th of kFC equal runs of the tiles and of the
  // boundaries, and each of its threads a contiguous run of those
  const long long c = blockIdx.x, t = threadIdx.x;
  double vn = 0.0, dd = 0.0;
  // the tiles' sums, in tile order
  {
    const long long run = (T + kFC - 1) / kFC, lo = min(T, c * run), hi = min(T, lo + run);
    const long long per = (run + kTF - 1) / kTF;
    const long long b0 = min(hi, lo + t * per), b1 = min(hi, b0 + per);
    for (long long q = b0; q < b1; ++q) {
      const double2 p = __ldcg(a.tpart + q);
      vn += p.x;
      dd += p.y;
    }
  }
  // the hypercubes that cross a tile boundary, each at the first boundary b
  // (between tiles b - 1 and b, 1 <= b < T) it crosses: the one holding tile
  // b's first event when it began in tile b - 1.  Its segments in event
  // order: its first, then the continuations of every later range it reaches.
  {
    const long long run = (T - 1 + kFC - 1) / kFC;
    const long long lo = min(T, 1 + c * run), hi = min(T, lo + run);
    const long long per = (run + kTF - 1) / kTF;
    const long long b0 = min(hi, lo + t * per), b1 = min(hi, b0 + per);
    for (long long b = b0; b < b1; ++b) {
      const long long h = __ldcg(a.tile_h0 + b);
      const long long o = __ldcg(a.off + h);
      if (o >= b * GV_TILE || o < (b - 1) * GV_TILE) continue;
      const long long e = __ldcg(a.off + h + 1);
      double2 sg = __ldcg(a.seg_h + h);
      double s1 = sg.x, s2 = sg.y;
      for (long long r = o / GV_PLUS_SEG + 1; r <= (e - 1) / GV_PLUS_SEG; ++r) {
        sg = __ldcg(a.seg_r + r);
        s1 += sg.x;
        s2 += sg.y;
      }
      const GvPlusStat st = gv_plus_stat(s1, s2, (int)(e - o), a.inv, a.beta_j);
      a.var[h] = st.v;
      a.dw[h] = st.w;
      vn += st.vn;
      dd += st.w;
    }
  }
  const double2 sums = block_sum2(make_double2(vn, dd), s_red);
  // the last CTA to arrive adds the CTAs' sums in CTA order
  if (threadIdx.x == 0) {
    a.fpart[c] = sums;
    __threadfence();
    s_last = atomicAdd(a.fctr, 1) == kFC - 1;
  }
  __syncthreads();
  if (!s_last) return;
  if (threadIdx.x == 0) {
    __threadfence();  // the CTAs' sums, published before their arrivals
    *a.fctr = 0;
    double2 VD = __ldcg(a.fpart);
    for (int q = 1; q < kFC; ++q) {
      const double2 p = __ldcg(a.fpart + q);
      VD.x += p.x;
      VD.y += p.y;
    }
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
  int* ctr = a.gctr + g;
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

cudaError_t launch_plus_finish(const GvPlusArgs& a, cudaStream_t s, bool pdl) {
  return gv_launch_prio(gv_plus_finish_kernel, dim3(kFC), dim3(kTF), 0, s, pdl, a.prio, a);
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
