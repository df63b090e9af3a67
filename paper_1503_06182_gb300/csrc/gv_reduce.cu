// gv_reduce.cu -- combination of all events of an iteration and the serial
// grid optimisation (Section 2.1: "the grid optimization is not parallelized,
// so that all the results can be combined").
//
// gv_reduce_kernel sums the 128-bit tile partials exactly.  Its grid is
// (accumulator blocks of 32) x (tile ranges): each CTA owns 32 accumulators
// and a range of tiles, its 8 warps stride over the tiles, the warps' sums
// are combined in shared memory, and the CTA adds the result to the
// iteration's accumulators with one fire-and-forget integer atomic per limb
// (a handful of CTAs per cache line, so no line becomes a hot spot).  Every
// tile partial is first aligned to the iteration's scale (the max over tiles,
// formed by the fill kernel with an order-free atomicMax).  Integer addition
// is associative: the totals do not depend on the grid or on timing.  The
// last CTA to finish (a ticket, no waiting) rounds the totals to FP64 once,
// records I_k and sigma_k, combines the stage and forms the per-axis totals
// of the smoothed bin sums (accumulated exactly by the reduce CTAs).
//
// gv_refine_kernel then refines the grid (Lepage's VEGAS, cited in Section
// 2.1): smoothing, normalisation, compression ((1-rho)/(-ln rho))^alpha and
// redistribution into N equal shares.  Smoothing is done exactly on the bin
// integers; the compression (an FP64 log per bin) is spread over CTAs; the
// last one places the new edges from shared memory.
//
// On this chip an FP64 instruction occupies a warp's FP64 pipe for ~64 cycles
// and the FP64 library log takes ~2000 cycles: the serial code here keeps its
// FP64 chains short (reciprocals passed in, a table-driven log, one warp per
// independent task).
#include <algorithm>

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

// Accumulators: three 64-bit limbs holding bits [0,43), [43,86) and [86,...)
// (the last one signed), 32 bytes apart.  The two low limbs have 21 bits of
// headroom (up to 2^21 adds), so no carry travels between limbs until the
// final conversion and no atomic waits for a returned value.
#define GV_LIMB 43
#define GV_LIMB_MASK ((1ull << GV_LIMB) - 1ull)
#define GV_ACC_STRIDE 4

__device__ __forceinline__ void red_add_limbs(unsigned long long* p, const u192& v) {
  const unsigned long long l0 = v.l0 & GV_LIMB_MASK;
  const unsigned long long l1 = ((v.l0 >> GV_LIMB) | (v.l1 << (64 - GV_LIMB))) & GV_LIMB_MASK;
  // bits 86.. as a signed 64-bit number (|v| < 2^149 always)
  const unsigned long long l2 = (v.l1 >> (2 * GV_LIMB - 64)) | (v.l2 << (128 - 2 * GV_LIMB));
  if (l0) atomicAdd(p, l0);
  if (l1) atomicAdd(p + 1, l1);
  if (l2) atomicAdd(p + 2, l2);
}

// l0 + l1 2^43 + l2 2^86 (l2 signed) as a 192-bit two's complement integer.
__device__ __forceinline__ u192 limbs_to_u192(unsigned long long l0, unsigned long long l1,
                                              unsigned long long l2) {
  u192 r = {l0, 0ull, 0ull};
  u192 a = {l1 << GV_LIMB, l1 >> (64 - GV_LIMB), 0ull};
  add192(r, a);
  const unsigned long long ext = (unsigned long long)((long long)l2 >> 63);
  u192 b = {0ull, l2 << (2 * GV_LIMB - 64),
            (l2 >> (128 - 2 * GV_LIMB)) | (ext << (2 * GV_LIMB - 64))};
  add192(r, b);
  return r;
}

__device__ __forceinline__ u192 load_acc(const unsigned long long* acc, int k) {
  const unsigned long long* p = acc + GV_ACC_STRIDE * k;
  return limbs_to_u192(__ldcg(p), __ldcg(p + 1), __ldcg(p + 2));
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

// Stored bin exponent (GV_BINE_OFF-offset, 0 = empty) -> q of u192_to_double.
__device__ __forceinline__ int bin_q(int g) { return 2 * (g - GV_BINE_OFF) - GV_BIN_FB; }

// Max of the stored bin exponents of one axis, by one warp (all lanes get it).
__device__ __forceinline__ int axis_bin_exp(const int* binE, int N) {
  int g = 0;
  for (int i = threadIdx.x & 31; i < N; i += 32) g = max(g, __ldcg(binE + i));
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) g = max(g, __shfl_xor_sync(0xffffffffu, g, m));
  return g;
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

// ---------------------------------------------------------------------------
// Natural log of a positive double, table-driven (P. T. P. Tang,
// "Table-driven implementation of the logarithm function in IEEE
// floating-point arithmetic", ACM TOMS 16 (1990)): x = 2^k m, m in [1,2);
// with R_j ~ 1/c_j for the 1/128-wide interval of m, r = m R_j - 1 (one fma,
// one rounding, |r| < 2^-7) and ln x = k ln2 + L_j + log1p(r), L_j = -ln R_j,
// log1p(r) by its Taylor series to r^7 (truncation below 2^-59 relative).
// The table (R_j, L_j for j < 128, then ln2 split into a 42-bit head and a
// tail) is built by the host from its libm when a context is created.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double gv_log1p_series(double r) {
  double p = 1.0 / 7.0;
  p = fma(p, r, -1.0 / 6.0);
  p = fma(p, r, 1.0 / 5.0);
  p = fma(p, r, -1.0 / 4.0);
  p = fma(p, r, 1.0 / 3.0);
  p = fma(p, r, -0.5);
  p = fma(p, r, 1.0);
  return p * r;
}

__device__ double gv_log_pos(double x, const double* __restrict__ tab) {
  // near 1 the reduction would cancel: r = x - 1 is exact there (Sterbenz)
  if (fabs(x - 1.0) <= 0x1p-7) return gv_log1p_series(x - 1.0);
  long long b = __double_as_longlong(x);
  int k = 0;
  if (b < (1ll << 52)) {  // subnormal: scale by 2^54
    x *= 0x1p54;
    b = __double_as_longlong(x);
    k = -54;
  }
  k += (int)(b >> 52) - 1023;
  const int j = (int)((b >> 45) & 127);
  const double m = __longlong_as_double((b & 0xFFFFFFFFFFFFFll) | 0x3FF0000000000000ll);
  const double R = __ldg(tab + 2 * j), L = __ldg(tab + 2 * j + 1);
  const double p = gv_log1p_series(fma(m, R, -1.0));
  const double kd = (double)k;
  return fma(kd, __ldg(tab + 256), L) + fma(kd, __ldg(tab + 257), p);
}

// ---------------------------------------------------------------------------
// Iteration record and stage combination.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mean_sigma(double s1, double s2, double inv_c, double inv_cm1,
                                           double* mean, double* sigma) {
  const double I = s1 * inv_c;
  const double var = (s2 * inv_c - I * I) * inv_cm1;
  *mean = I;
  *sigma = var > 0.0 ? sqrt(var) : 0.0;
}

// Inverse-variance combination of the iterations 0..m-1 of a stage by one
// warp (lanes stride over the iterations, fixed butterfly sums); if any
// iteration has zero variance, those alone are averaged with error 0.
__device__ void combine_stage_warp(const double* per_iter, int stride, int m, double inv_m1,
                                   GvState* st, bool adjoint) {
  const int lane = threadIdx.x & 31;
  if (m == 1 && !adjoint) {
    if (lane == 0) {
      st->integral = per_iter[0];
      st->error = per_iter[1];
      st->chi2 = 0.0;
    }
    return;
  }
  double nz = 0.0;
  for (int k = lane; k < m; k += 32) nz += (per_iter[k * stride + 1] > 0.0) ? 0.0 : 1.0;
  nz = warp_sum_f64(nz);
  double swt = 0.0, swi = 0.0;
  for (int k = lane; k < m; k += 32) {
    const double s = per_iter[k * stride + 1];
    const double wt = nz > 0.0 ? (s > 0.0 ? 0.0 : 1.0) : __drcp_rn(s * s);
    swt += wt;
    swi = fma(wt, per_iter[k * stride], swi);
  }
  swt = warp_sum_f64(swt);
  swi = warp_sum_f64(swi);
  const double inv_swt = __drcp_rn(swt);
  const double mean = swi * inv_swt;
  double chi2 = 0.0;
  if (nz == 0.0)
    for (int k = lane; k < m; k += 32) {
      const double s = per_iter[k * stride + 1];
      const double dev = per_iter[k * stride] - mean;
      chi2 = fma(dev * dev, __drcp_rn(s * s), chi2);
    }
  chi2 = warp_sum_f64(chi2);
  if (lane == 0) {
    st->integral = mean;
    st->error = nz > 0.0 ? 0.0 : rsqrt(swt);
    st->chi2 = (nz > 0.0 || m < 2) ? 0.0 : chi2 * inv_m1;
  }
  if (adjoint) {
    for (int p = 0; p < GV_NGRAD; ++p) {
      double num = 0.0, var = 0.0;
      for (int k = lane; k < m; k += 32) {
        const double s = per_iter[k * stride + 1];
        const double wt = nz > 0.0 ? (s > 0.0 ? 0.0 : 1.0) : __drcp_rn(s * s);
        const double sG = per_iter[k * stride + 3 + 2 * p];
        num = fma(wt, per_iter[k * stride + 2 + 2 * p], num);
        var = fma(wt * wt, sG * sG, var);
      }
      num = warp_sum_f64(num);
      var = warp_sum_f64(var);
      if (lane == 0) {
        st->grad[p] = num * inv_swt;
        st->grad_err[p] = sqrt(var) * inv_swt;
      }
    }
  }
}

// Integer weight c_j of bin j in 6 x (sum of the smoothed bin sums of an axis):
// the end entries (d_0+d_1)/2, (d_{N-2}+d_{N-1})/2 weigh 3, the inner entries
// (d_{i-1}+d_i+d_{i+1})/3 weigh 2.
__device__ __forceinline__ int smooth_weight(int j, int N) {
  int c = 0;
  for (int i = max(0, j - 1); i <= min(N - 1, j + 1); ++i) {
    const bool inside = (i == 0) ? (j <= 1) : (i == N - 1) ? (j >= N - 2) : true;
    if (inside) c += (i == 0 || i == N - 1) ? 3 : 2;
  }
  return c;
}

__device__ __forceinline__ u192 mul192_small(u192 v, int c) {
  u192 r = {0ull, 0ull, 0ull};
  for (int q = 0; q < c; ++q) add192(r, v);
  return r;
}

// The last reduce CTA (256 threads).
__device__ void finalize_iteration(const GvReduceArgs& a) {
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, wid = tid >> 5;
  GvState* st = a.st;
  const int d = a.ndim;
  // channel sums (and the bin sums unless the refine kernel converts them):
  // each rounded once to FP64
  const int nconv = a.refine_follows ? 2 * a.nch : a.nacc;
  for (int k = tid; k < nconv; k += nthr) {
    if (k < 2 * a.nch) {
      const int Eg = st->E[k >> 1];
      a.sums[k] =
          Eg != GV_EMPTY ? u192_to_double(load_acc(a.acc, k), ((k & 1) + 1) * Eg - GV_FB) : 0.0;
    } else {  // a bin, at its own scale
      const int g = __ldcg(a.binE + (k - 2 * a.nch));
      a.sums[k] = g ? u192_to_double(load_acc(a.acc, k), bin_q(g)) : 0.0;
    }
  }
  __syncthreads();
  if (wid == 0) {
    // warp 0: the iteration record (one lane per channel) and the stage
    const int stride = a.mode ? 2 + 2 * GV_NGRAD : 2;
    if (lane < a.nch) {
      double* rec = a.per_iter + (size_t)a.k * stride + 2 * lane;
      mean_sigma(a.sums[2 * lane], a.sums[2 * lane + 1], a.inv_c, a.inv_cm1, &rec[0], &rec[1]);
    }
    __syncwarp();
    if (a.last) combine_stage_warp(a.per_iter, stride, a.k + 1, a.inv_m1, st, a.mode != 0);
    if (lane == 0) {
      const unsigned long long nf = __ldcg(&st->nonfinite_iter);
      st->nonfinite = (a.k == 0 ? 0ull : st->nonfinite) + nf;
      if (a.k == 0) st->status = 0;
      st->nonfinite_iter = 0ull;
    }
  } else if (a.has_bins) {
    // per-axis totals (slots after the bins, at the axis' largest bin scale,
    // summed by the reduce CTAs): one rounding, stored as 1/(6 x total), 0
    // when the axis is empty.  One warp per axis.
    for (int ax = wid - 1; ax < d; ax += (nthr >> 5) - 1) {
      const int g = axis_bin_exp(a.binE + ax * a.nbins, a.nbins);
      if (lane == 0) {
        double inv = 0.0;
        if (g) {
          const double t6 = u192_to_double(load_acc(a.acc, a.nacc + ax), bin_q(g));
          inv = t6 > 0.0 ? __drcp_rn(t6) : 0.0;
        }
        a.inv_total[ax] = inv;
      }
    }
  }
  __syncthreads();  // every read of the accumulators here is done
  const int nslots = a.has_bins ? a.nacc + d : a.nacc;
  for (int k = tid; k < GV_ACC_STRIDE * nslots; k += nthr) {
    const int slot = k / GV_ACC_STRIDE;
    const bool bin_slot = a.has_bins && slot >= 2 * a.nch && slot < a.nacc;
    if (!(bin_slot && a.refine_follows)) a.acc[k] = 0ull;
  }
  if (a.has_bins && !a.refine_follows)
    for (int k = tid; k < d * a.nbins; k += nthr) a.binE[k] = 0;
  if (tid == 0) {
    st->E0_prev = st->E[0];
    for (int c = 0; c < GV_MAXCH; ++c) st->E[c] = GV_EMPTY;
    st->done = 0;
    st->it = st->it + 1ull;
  }
}

#define GV_RED_TILES_PER_LOAD 8

// One reduce CTA (256 threads) of one integration: accumulator block bx, tile
// range by, of nblk CTAs in total for that integration.
__device__ void gv_reduce_task(const GvReduceArgs& a, int bx, int by, int nblk,
                               u192 (*s_part)[32], int* is_last_s) {
  int& is_last = *is_last_s;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int k = bx * 32 + lane;
  const int t0 = by * a.tiles_per_cta;
  const int t1 = min(a.n_tiles, t0 + a.tiles_per_cta);
  u192 r = {0ull, 0ull, 0ull};
  gv_wait_prior_grid();
  const bool bin_slot = a.has_bins && k >= 2 * a.nch && k < a.nacc;
  const int gb = bin_slot ? __ldcg(a.binE + (k - 2 * a.nch)) : 0;
  if (bin_slot) {
    // Q 2^(2 F_tb - GV_BIN_QBITS) aligned to 2^(2 G_b - GV_BIN_FB)
    if (gb) {
      constexpr int G = GV_RED_TILES_PER_LOAD;
      for (int tb = t0 + wid; tb < t1; tb += 8 * G) {
        ulonglong2 v[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const int t = tb + 8 * g;
          v[g] = t < t1 ? a.part[(size_t)t * a.nacc + k] : make_ulonglong2(0ull, 0ull);
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const int f = (int)(v[g].y >> 32);
          if (f) {
            const u192 x = {v[g].x, v[g].y & 0xFFFFFFFFull, 0ull};
            const int sh = 2 * (gb - f) - GV_BIN_XBITS;
            add192(r, sh < 0 ? shl192(x, -sh) : sar192(x, sh));
          }
        }
      }
    }
  } else if (k < a.nacc) {
    const int ch = k >> 1;
    const int pw = (k & 1) + 1;
    const int Eg = a.st->E[ch];
    if (Eg != GV_EMPTY) {
      constexpr int G = GV_RED_TILES_PER_LOAD;
      for (int tb = t0 + wid; tb < t1; tb += 8 * G) {
        ulonglong2 v[G];
        int Et[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const int t = tb + 8 * g;
          if (t < t1) {
            Et[g] = a.tileE[(size_t)t * a.nch + ch];
            v[g] = a.part[(size_t)t * a.nacc + k];
          } else {
            Et[g] = GV_EMPTY;
            v[g] = make_ulonglong2(0ull, 0ull);
          }
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const u192 x = {v[g].x, v[g].y, (unsigned long long)((long long)v[g].y >> 63)};
          const int sh = Et[g] == GV_EMPTY ? 192 : pw * (Eg - Et[g]);
          if (x.l0 | x.l1) add192(r, sar192(x, sh));
        }
      }
    }
  }
  s_part[wid][lane] = r;
  __syncthreads();
  if (wid == 0) {
    u192 t = s_part[0][lane];
#pragma unroll
    for (int w = 1; w < 8; ++w) add192(t, s_part[w][lane]);
    if (k < a.nacc && (t.l0 | t.l1 | t.l2)) red_add_limbs(a.acc + GV_ACC_STRIDE * k, t);
    if (a.has_bins) {
      // this CTA's share of 6 x (sum of the smoothed bin sums) of each axis
      const int N = a.nbins;
      const int j = k - 2 * a.nch;  // bin index within [0, d*N)
      const bool is_bin = k < a.nacc && j >= 0;
      const u192 ct = (is_bin && gb) ? mul192_small(t, smooth_weight(j % N, N))
                                      : u192{0ull, 0ull, 0ull};
      const int k0 = bx * 32;
      const int j_first = max(0, k0 - 2 * a.nch);
      const int j_last = min(a.nacc - 1, k0 + 31) - 2 * a.nch;
      for (int ax = j_first / N; j_last >= 0 && ax <= j_last / N; ++ax) {
        // at the axis' largest bin scale (a fixed truncation of the small bins)
        const int gax = axis_bin_exp(a.binE + ax * N, N);
        u192 v = (is_bin && gb && j / N == ax) ? sar192(ct, 2 * (gax - gb))
                                                : u192{0ull, 0ull, 0ull};
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) {
          u192 o = {__shfl_xor_sync(0xffffffffu, v.l0, m), __shfl_xor_sync(0xffffffffu, v.l1, m),
                    __shfl_xor_sync(0xffffffffu, v.l2, m)};
          add192(v, o);
        }
        if (lane == 0 && (v.l0 | v.l1 | v.l2))
          red_add_limbs(a.acc + GV_ACC_STRIDE * (a.nacc + ax), v);
      }
    }
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(&a.st->done, 1) == nblk - 1) ? 1 : 0;
  __syncthreads();
  if (!is_last) return;
  gv_allow_next_grid();
  __threadfence();
  finalize_iteration(a);
}

__global__ void __launch_bounds__(256) gv_reduce_kernel(const GvReduceArgs a) {
  __shared__ u192 s_part[8][32];
  __shared__ int is_last;
  gv_reduce_task(a, blockIdx.x, blockIdx.y, gridDim.x * gridDim.y, s_part, &is_last);
}

// Batched: one launch reduces many integrations; task i names the
// integration and the block coordinates of CTA i.
__global__ void __launch_bounds__(256) gv_reduce_batch_kernel(const GvReduceArgs* args,
                                                              const int4* tasks, int k, int last,
                                                              double inv_m1) {
  __shared__ u192 s_part[8][32];
  __shared__ int is_last;
  const int4 t = tasks[blockIdx.x];
  GvReduceArgs a = args[t.x];
  a.k = k;
  a.last = last;
  a.inv_m1 = inv_m1;
  gv_reduce_task(a, t.y, t.z, t.w, s_part, &is_last);
}

// ---------------------------------------------------------------------------
// Grid refinement.
// ---------------------------------------------------------------------------
// Write the edges e_src (d x (N+1)) into the grid pack with its derived tables.
__device__ void pack_axis_tables(double* grid, const double* e_src, int d, int N, int tid,
                                 int nthr) {
  const GvGridLayout L{d, N};
  double* e64 = grid + L.off_e64();
  double* wd64 = grid + L.off_wd64();
  double* jac = grid + L.off_jac();
  float* w32 = reinterpret_cast<float*>(grid + L.off_f32_base());
  float* e32 = w32 + L.w_e32();
  float* wd32 = w32 + L.w_wd32();
  float* jm32 = w32 + L.w_jm32();
  int* je = reinterpret_cast<int*>(w32 + L.w_je());
  for (int k = tid; k < d * (N + 1); k += nthr) {
    const int a = k / (N + 1), i = k % (N + 1);
    const size_t ie = (size_t)a * (N + 1) + i;
    const double e = e_src[ie];
    e64[ie] = e;
    e32[ie] = (float)e;
    if (i < N) {
      const double w = e_src[ie + 1] - e;
      const double j = (double)N * w;
      const size_t ib = (size_t)a * N + i;
      wd64[ib] = w;
      jac[ib] = j;
      wd32[ib] = (float)w;
      // j = m 2^x with m in [1,2): exponent from the bits (j > 0; a subnormal
      // j is scaled into the normal range first)
      const bool sub = j < 0x1p-1000;
      const double js = sub ? j * 0x1p200 : j;
      const long long b = __double_as_longlong(js);
      const int x = (int)((b >> 52) & 0x7FF) - 1023;
      const double m = __longlong_as_double((b & 0xFFFFFFFFFFFFFll) | 0x3FF0000000000000ll);
      jm32[ib] = (float)m;
      je[ib] = sub ? x - 200 : x;
    }
  }
}

// ((1 - rho)/(-ln rho))^alpha for 0 < rho < 1, with the common exponents
// evaluated by roots rather than pow.
__device__ __forceinline__ double compress(double rho, double alpha, const double* tab) {
  if (rho <= 0.0) return 0.0;
  if (rho >= 1.0) return 1.0;
  const double L = -gv_log_pos(rho, tab);
  const double om = 1.0 - rho;
  if (alpha == 1.5) {
    const double y = rsqrt(L);
    return om * sqrt(om) * (y * y * y);
  }
  if (alpha == 1.0) return om * __drcp_rn(L);
  if (alpha == 0.5) return sqrt(om) * rsqrt(L);
  if (alpha == 2.0) {
    const double q = om * __drcp_rn(L);
    return q * q;
  }
  if (alpha == 0.0) return 1.0;
  return pow(om * __drcp_rn(L), alpha);
}

#define GV_REFINE_THREADS 512
#define GV_REFINE_BINS 32

// Phase 1, every CTA: warp 0 computes the compressed value r_i of 32 bins and
// the slope (e_{i+1}-e_i)/r_i used to place edges.  Phase 2, the last CTA
// (ticket): per-axis prefix sums C of r (warp scan), new edges where C
// reaches j R/N -- binary search on the bit patterns of the nonnegative
// doubles, then e_i + (target - C_i) * slope_i -- and the tables, with r,
// slope, C and the old edges in shared memory.
__device__ void gv_refine_task(const GvRefineArgs& a, int bx, int nblk, double* sm,
                               int* is_last_s, double* s_step) {
  int& is_last = *is_last_s;
  const int d = a.ndim, N = a.nbins, dN = d * N;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int NWARP = GV_REFINE_THREADS / 32;
  double* gr = a.scratch;                   // [dN] r
  double* gsl = a.scratch + dN;             // [dN] slope
  double* ne = a.scratch + 2 * (size_t)dN;  // [d(N+1)] new edges
  const double* e64 = a.grid;               // the pack starts with e64
  gv_wait_prior_grid();
  if (wid == 0) {
    const int k = bx * GV_REFINE_BINS + lane;
    if (k < dN) {
      const int ax = k / N, i = k - ax * N;
      const int base = 2 * a.nch + ax * N;  // slot of bin 0 of this axis
      const int* G = a.binE + ax * N;
      const u192 z = {0ull, 0ull, 0ull};
      const int gm = i > 0 ? __ldcg(G + i - 1) : 0, gc = __ldcg(G + i),
                gp = i < N - 1 ? __ldcg(G + i + 1) : 0;
      const int gx = max(gm, max(gc, gp));
      // the three bins at the largest of their scales (empty bins hold 0)
      const u192 dc0 = load_acc(a.acc, base + i);
      const u192 dm = gm ? sar192(load_acc(a.acc, base + i - 1), 2 * (gx - gm)) : z;
      const u192 dc = gc ? sar192(dc0, 2 * (gx - gc)) : z;
      const u192 dp = gp ? sar192(load_acc(a.acc, base + i + 1), 2 * (gx - gp)) : z;
      // 6 x the smoothed sum: 3 (d_0 + d_1) at the ends,
      // 2 (d_{i-1} + d_i + d_{i+1}) inside
      u192 s6 = dc;
      if (i == 0) {
        add192(s6, dp);
        s6 = mul192_small(s6, 3);
      } else if (i == N - 1) {
        add192(s6, dm);
        s6 = mul192_small(s6, 3);
      } else {
        add192(s6, dm);
        add192(s6, dp);
        s6 = mul192_small(s6, 2);
      }
      a.dsum[k] = gc ? u192_to_double(dc0, bin_q(gc)) : 0.0;
      const double it = a.inv_total[ax];
      double rv = 0.0, sl = 0.0;
      if (it > 0.0 && gx) {
        rv = compress(u192_to_double(s6, bin_q(gx)) * it, a.alpha, a.logtab);
        if (rv > 0.0)
          sl = (e64[ax * (N + 1) + i + 1] - e64[ax * (N + 1) + i]) * __drcp_rn(rv);
      }
      gr[k] = rv;
      gsl[k] = sl;
    }
    __threadfence();
  }
  __syncthreads();
  if (tid == 0) is_last = (atomicAdd(&a.st->done_refine, 1) == nblk - 1) ? 1 : 0;
  __syncthreads();
  if (!is_last) return;
  gv_allow_next_grid();
  __threadfence();
  // every phase-1 CTA has read the bin slots: reset them for the next iteration
  for (int k = tid; k < GV_ACC_STRIDE * dN; k += GV_REFINE_THREADS)
    a.acc[GV_ACC_STRIDE * 2 * a.nch + k] = 0ull;
  for (int k = tid; k < dN; k += GV_REFINE_THREADS) a.binE[k] = 0;
  double* r = sm;                 // [dN]
  double* slope = r + dN;         // [dN]
  double* cum = slope + dN;       // [d(N+1)]
  double* e = cum + d * (N + 1);  // [d(N+1)] old edges
  for (int k = tid; k < dN; k += GV_REFINE_THREADS) {
    r[k] = __ldcg(gr + k);
    slope[k] = __ldcg(gsl + k);
  }
  for (int k = tid; k < d * (N + 1); k += GV_REFINE_THREADS) e[k] = e64[k];
  __syncthreads();
  for (int ax = wid; ax < d; ax += NWARP) {
    const double* ra = r + ax * N;
    double* ca = cum + ax * (N + 1);
    const int chunk = (N + 31) / 32;
    const int i0 = min(N, lane * chunk), i1 = min(N, i0 + chunk);
    double local = 0.0;
    for (int i = i0; i < i1; ++i) local += ra[i];
    double incl = local;
#pragma unroll
    for (int m = 1; m < 32; m <<= 1) {
      const double o = __shfl_up_sync(0xffffffffu, incl, m);
      if (lane >= m) incl += o;
    }
    double run = incl - local;  // exclusive prefix of this lane's chunk
    if (lane == 0) ca[0] = 0.0;
    for (int i = i0; i < i1; ++i) {
      run += ra[i];
      ca[i + 1] = run;
    }
    __syncwarp();
    if (lane == 0) s_step[ax] = ca[N] * a.inv_nbins;
  }
  __syncthreads();
  for (int kk = tid; kk < d * (N + 1); kk += GV_REFINE_THREADS) {
    const int ax = kk / (N + 1), j = kk % (N + 1);
    double v = e[kk];
    if (a.inv_total[ax] > 0.0) {
      if (j == 0) {
        v = 0.0;
      } else if (j == N) {
        v = 1.0;
      } else {
        const double* C = cum + ax * (N + 1);
        const double target = s_step[ax] * j;
        const long long tb = __double_as_longlong(target);
        const long long* Cb = reinterpret_cast<const long long*>(C);
        int lo = 0, hi = N - 1;  // first bin i with C[i+1] > target (N-1 if none)
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (Cb[mid + 1] > tb)
            hi = mid;
          else
            lo = mid + 1;
        }
        v = fma(target - C[lo], slope[ax * N + lo], e[ax * (N + 1) + lo]);
      }
    }
    ne[kk] = v;
  }
  __syncthreads();
  pack_axis_tables(a.grid, ne, d, N, tid, GV_REFINE_THREADS);
  if (tid == 0) a.st->done_refine = 0;
}

__global__ void __launch_bounds__(GV_REFINE_THREADS) gv_refine_kernel(const GvRefineArgs a) {
  extern __shared__ __align__(16) double sm[];
  __shared__ int is_last;
  __shared__ double s_step[GV_MAXD];
  gv_refine_task(a, blockIdx.x, gridDim.x, sm, &is_last, s_step);
}

__global__ void __launch_bounds__(GV_REFINE_THREADS) gv_refine_batch_kernel(
    const GvRefineArgs* args, const int4* tasks) {
  extern __shared__ __align__(16) double sm[];
  __shared__ int is_last;
  __shared__ double s_step[GV_MAXD];
  const int4 t = tasks[blockIdx.x];
  const GvRefineArgs a = args[t.x];
  gv_refine_task(a, t.y, t.w, sm, &is_last, s_step);
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
  } else if (ig == GV_DY) {
    const double sqrt_s = p[0], MZ = p[1], GZ = p[2], sw2 = p[3], alpha = p[4];
    const double mlo = p[5], mhi = p[6];
    const double s = sqrt_s * sqrt_s;
    const double tau_lo = mlo * mlo / s, tau_hi = mhi * mhi / s;
    const double pi = 3.14159265358979323846;
    K[DK_SQRTS] = sqrt_s;
    K[DK_S] = s;
    K[DK_TAULO] = tau_lo;
    K[DK_L] = log(tau_hi / tau_lo);
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
  } else if (ig == GV_EE3J) {
    const double Q = np > 1 ? p[1] : 91.1876;
    K[EK_YCUT] = p[0];
    K[EK_Q] = Q;
    K[EK_INVQ2] = 1.0 / (Q * Q);
  }
  float* kf = reinterpret_cast<float*>(K + GV_NCONST_F32);
  for (int i = 0; i < GV_NCONST_F32; ++i) kf[i] = (float)K[i];
}

// Reset the per-iteration invariants (at creation and after the autotuner's
// trial launches).
__global__ void gv_reset_kernel(GvState* st, int nacc, unsigned long long* acc, int* binE,
                                int dN) {
  for (int k = threadIdx.x; k < dN; k += blockDim.x) binE[k] = 0;
  if (threadIdx.x == 0) {
    st->nonfinite_iter = 0ull;
    st->done = 0;
    st->done_refine = 0;
    for (int c = 0; c < GV_MAXCH; ++c) st->E[c] = GV_EMPTY;
  }
  for (int k = threadIdx.x; k < GV_ACC_STRIDE * nacc; k += blockDim.x) acc[k] = 0ull;
}

__global__ void gv_grid_pack_kernel(double* grid, int d, int N) {
  pack_axis_tables(grid, grid, d, N, threadIdx.x, blockDim.x);
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
size_t refine_smem_bytes(int d, int N) {
  return sizeof(double) * (2 * (size_t)d * N + 2 * (size_t)d * (N + 1));
}

// Reduce grid: 32 accumulators per CTA; at most 64 tile ranges.
void reduce_grid(int n_tiles, int nacc, int* tiles_per_cta, int* gx, int* gy) {
  const int tpc = n_tiles <= 64 ? std::max(1, n_tiles) : std::max(64, (n_tiles + 63) / 64);
  *tiles_per_cta = tpc;
  *gx = (nacc + 31) / 32;
  *gy = (n_tiles + tpc - 1) / tpc;
}

cudaError_t launch_reduce(const GvReduceArgs& a, cudaStream_t s, bool pdl) {
  int tpc, gx, gy;
  reduce_grid(a.n_tiles, a.nacc, &tpc, &gx, &gy);
  if (tpc != a.tiles_per_cta) return cudaErrorInvalidValue;
  return gv_launch(gv_reduce_kernel, dim3(gx, gy), dim3(256), 0, s, pdl, a);
}

cudaError_t prepare_refine(int d, int N) {
  const size_t smem = refine_smem_bytes(d, N);
  if (smem > 48 * 1024)
    return cudaFuncSetAttribute(gv_refine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  return cudaSuccess;
}

cudaError_t launch_refine(const GvRefineArgs& a, cudaStream_t s, bool pdl) {
  const int ctas = (a.ndim * a.nbins + GV_REFINE_BINS - 1) / GV_REFINE_BINS;
  return gv_launch(gv_refine_kernel, dim3(ctas), dim3(GV_REFINE_THREADS),
                   refine_smem_bytes(a.ndim, a.nbins), s, pdl, a);
}

cudaError_t launch_reduce_batch(const GvReduceArgs* args, const int4* tasks, int ntasks, int k,
                                int last, double inv_m1, cudaStream_t s) {
  gv_reduce_batch_kernel<<<ntasks, 256, 0, s>>>(args, tasks, k, last, inv_m1);
  return cudaGetLastError();
}

cudaError_t launch_refine_batch(const GvRefineArgs* args, const int4* tasks, int ntasks,
                                size_t smem, cudaStream_t s) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(gv_refine_batch_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  gv_refine_batch_kernel<<<ntasks, GV_REFINE_THREADS, smem, s>>>(args, tasks);
  return cudaGetLastError();
}

int refine_ctas(int d, int N) { return (d * N + GV_REFINE_BINS - 1) / GV_REFINE_BINS; }

cudaError_t launch_consts(int integrand, const double* params, double* kconst, cudaStream_t s) {
  gv_consts_kernel<<<1, 32, 0, s>>>(integrand, params, kconst);
  return cudaGetLastError();
}

cudaError_t launch_reset(GvState* st, int nacc, unsigned long long* acc, int* binE, int dN,
                         cudaStream_t s) {
  gv_reset_kernel<<<1, 256, 0, s>>>(st, nacc, acc, binE, dN);
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
