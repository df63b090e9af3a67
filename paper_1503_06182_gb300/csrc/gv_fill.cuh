// gv_fill.cuh -- the fused per-event kernel of one VEGAS iteration.
//
// One CTA evaluates one tile of GV_TILE consecutive events (Section 2.1: each
// event generated and evaluated independently), with EPT events per thread:
//   pass 1: Philox words -> bins and in-bin positions -> x on the adaptive grid
//           ((edge, width) pairs and Jacobian factors staged in shared memory)
//           -> g(x) -> w = J g (J in FP64 in the FP64 form; FP32 mantissas
//           with an integer exponent in the FP32 form); the bins stay in registers
//           (d <= 4) or go to shared memory;
//   tile scale: block max of |w| (order-free) -> E_t (in the FP32 form a
//           32-bit max of exponents: each weight is kept as its FP32 product
//           and Jacobian exponent, a 24-bit significand times a power of two);
//   pass 2: w and the exact square w^2 rounded once to fixed point at the tile
//           scale (FP32 form: from the 24-bit significand, gv_direct*);
//           sums in 128-bit integer registers (warp shuffle + block
//           reduction); per-bin sums of w^2, each bin with its own exponent F
//           (an order-free shared atomicMax in pass 1), w^2 rounded once to
//           2^(2F - 56) and added as three 22-bit limbs with 32-bit shared
//           atomics (32-bit shared atomics run several times faster than
//           64-bit ones here, and 10 bits of headroom cover the 1024 events of
//           a tile).
// With VEGAS+ (PLUS), each thread takes GV_PLUS_SEG consecutive events (one
// range): a binary search finds its first event's hypercube, the next events
// step across hypercube boundaries (every hypercube holds at least 2 events),
// and each event takes stratified words from its hypercube's digits.  The
// estimate's weight is F C/(nh n_h) and the bins' quantity F sqrt(1/(nh n_h)),
// F = J g.  The thread also sums F and F^2 over the run of each hypercube in
// its range, in event order (the range's segments), which the hypercube
// statistics add up after the iteration.
// With a histogram of the observable (HIST), every event with w != 0 also
// adds w and w^2 to its observable's bin, in the same limb scheme: a per-bin
// exponent from pass 1, then w^2 as three unsigned 22-bit limbs and w as two
// unsigned limbs and a signed top limb (two's complement, so negative weights
// add like positive ones).
// Integer sums are order-free, so the tile's result is the same for every
// block size / events-per-thread choice.  Apart from the Jacobian product and
// w = J g, the bookkeeping runs on the integer pipes: the FP64 pipe of this
// chip is a small fraction of its FP32 throughput.
#pragma once
#include "gv_integrands.cuh"
#include "gv_plus_stat.cuh"

template <int IG>
struct GvTraits;
template <>
struct GvTraits<GV_GAUSS> {
  static constexpr int NK = 2;
};
template <>
struct GvTraits<GV_DY> {
  static constexpr int NK = DK_NK;
};
template <>
struct GvTraits<GV_EE3J> {
  static constexpr int NK = 3;
};
template <>
struct GvTraits<GV_DYNLO> {
  static constexpr int NK = NK_NK;
};

template <int IG, typename Real, int MAXD>
__device__ __forceinline__ Real gv_eval(const Real (&x)[MAXD], int d,
                                        const GvConst<Real, GvTraits<IG>::NK>& K) {
  if constexpr (IG == GV_GAUSS) {
    return gv_gauss<Real, MAXD>(x, d, K[GK_INV2S2], K[GK_SHIFT]);
  } else if constexpr (IG == GV_DY) {
    return gv_drell_yan<Real, false>(x, K, nullptr);
  } else if constexpr (IG == GV_DYNLO) {
    return gv_dy_nlo<Real, MAXD>(x, d, K);
  } else {
    return gv_ee3j<Real>(x, K);
  }
}

// The histogram observable of an event (the differential distributions of
// Section 3.2): Gauss x_0; Drell-Yan (both forms) the dilepton mass
// m_ll = sqrt(tau s) in GeV, with tau as the integrand forms it; 3-jet the
// thrust max(x1, x2, x3), x3 = 2 - x1 - x2.
template <int IG, typename Real, int MAXD>
__device__ __forceinline__ Real gv_observable(const Real (&x)[MAXD],
                                              const GvConst<Real, GvTraits<IG>::NK>& K) {
  using Mt = GvMath<Real>;
  if constexpr (IG == GV_GAUSS) {
    return x[0];
  } else if constexpr (IG == GV_DY || IG == GV_DYNLO) {
    const Real tau = Mt::exp(Mt::fma(x[0], K[DK_L], K[DK_LOGTAULO]));
    return Mt::sqrt(tau * K[DK_S]);
  } else {
    const Real x1 = x[0], x2 = x[1], x3 = (Real)2 - x1 - x2;
    const Real t = x1 > x2 ? x1 : x2;
    return t > x3 ? t : x3;
  }
}

// Histogram bin of v among nh bins over [lo, lo + nh / invw): 0 below (and
// for a value that is not a number), nh + 1 above.
template <typename Real>
__device__ __forceinline__ int gv_hist_bin(Real v, Real lo, Real invw, int nh) {
  if (!(v >= lo)) return 0;
  const Real t = (v - lo) * invw;
  if (!(t < (Real)nh)) return nh + 1;
  return 1 + (int)t;
}

// |w| rounded to a multiple of 2^(Fs - GV_BIN_QBITS), Fs the bin's scale
// (|w| < 2^Fs), with w's sign: |result| < 2^56.
__device__ __forceinline__ long long gv_hist_fixed(const GvDecoded& dw, int Fs) {
  const int r = Fs - GV_BIN_QBITS - dw.e2;  // right shift of the mantissa (>= -55)
  unsigned long long q;
  if (r <= 0)
    q = dw.m << (-r);
  else if (r < 64)
    q = ((dw.m >> (r - 1)) + 1ull) >> 1;
  else
    q = 0ull;
  return dw.neg ? -(long long)q : (long long)q;
}

// One bin of one axis as staged in shared memory.
struct __align__(16) GvBin32 {
  float e, w;     // edge and width in FP32
  float jm;       // N * (e_{i+1} - e_i) = jm 2^je, jm in [1,2]
  int je;
};
struct __align__(16) GvBin64 {
  double e, w;
};
// A float widened to double by integer operations (exact; the FP64 pipe of
// this chip is scarce).  Zero, subnormal and non-finite inputs are handled.
__device__ __forceinline__ double gv_widen(float g) {
  const unsigned u = __float_as_uint(g);
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  const unsigned ef = (u >> 23) & 0xFFu;
  unsigned long long m = u & 0x7FFFFFu;
  unsigned long long bits;
  if (ef == 0xFFu) {
    bits = sign | 0x7FF0000000000000ull | (m << 29);
  } else if (ef != 0u) {
    bits = sign | ((unsigned long long)(ef + 896u) << 52) | (m << 29);
  } else if (m == 0ull) {
    bits = sign;
  } else {  // subnormal float m 2^-149, leading one at bit p = 23 - lz
    const int lz = __clzll((long long)m) - 40;
    m = (m << lz) & 0x7FFFFFull;
    bits = sign | ((unsigned long long)(897 - lz) << 52) | (m << 29);
  }
  return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ double gv_widen(double g) { return g; }

// The Jacobian of one event: FP64 in the FP64 form; in the FP32 form the
// product of the FP32 mantissas and the sum of the exponents (no range limit,
// and nothing on the FP64 pipe, of which this chip has little).
template <typename Real>
struct GvJac;
template <>
struct GvJac<double> {
  double v;
};
template <>
struct GvJac<float> {
  float m;
  int e;
};

// x 2^E for a double x, on the integer pipes: zero, infinity and NaN pass
// through, a result beyond FP64 becomes infinity (counted as non-finite by
// the caller), one below the normal range becomes zero.
__device__ __forceinline__ double gv_ldexp_bits(double x, int E) {
  const long long b = __double_as_longlong(x);
  const int ef = (int)((b >> 52) & 0x7FF);
  if (ef == 0 || ef == 0x7FF || E == 0) return x;
  const int nf = ef + E;
  const long long sign = b & (long long)0x8000000000000000ull;
  if (nf >= 0x7FF) return __longlong_as_double(sign | 0x7FF0000000000000ll);
  if (nf <= 0) return __longlong_as_double(sign);
  return __longlong_as_double((b & ~0x7FF0000000000000ll) | ((long long)nf << 52));
}

// w = J g as a double.
__device__ __forceinline__ double gv_weight(const GvJac<double>& J, double g) {
  return __dmul_rn(J.v, g);
}
__device__ __forceinline__ double gv_weight(const GvJac<float>& J, float g) {
  const float p = __fmul_rn(J.m, g);
  const unsigned u = __float_as_uint(p);
  const int ef = (int)((u >> 23) & 0xFFu);
  const int nf = ef + 896 + J.e;  // the double's exponent field
  if (ef != 0 && ef != 0xFF && nf > 0 && nf < 0x7FF)  // normal in and out: one assembly
    return __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) |
                                            ((unsigned long long)nf << 52) |
                                            ((unsigned long long)(u & 0x7FFFFFu) << 29)));
  return gv_ldexp_bits(gv_widen(p), J.e);
}

// FP32 form, for the exact sums: the weight p 2^e of an FP32 product
// p = J.m g.  Where p is normal and p 2^e a normal double ("direct"), the
// weight is m 2^e2 with m the 24-bit significand of p and e2 = nf - 1046, nf
// its FP64 exponent field (the double gv_weight assembles holds m << 29).
// Its tile fixed-point terms are formed from m (a 32 x 32 -> 64 bit square):
// the same exactly rounded integers as through the double, with less integer
// work.  Every other case takes the double, formed as gv_weight forms it.
struct GvDirect {
  bool direct;
  unsigned m;
  int e2;
  bool neg;
};
__device__ __forceinline__ GvDirect gv_direct(unsigned u, int e) {
  const int ef = (int)((u >> 23) & 0xFFu);
  const int nf = ef + 896 + e;
  GvDirect w;
  w.direct = ef != 0 && ef != 0xFF && nf > 0 && nf < 0x7FF;
  w.m = (u & 0x7FFFFFu) | 0x800000u;
  w.e2 = nf - 1046;
  w.neg = (u >> 31) != 0u;
  return w;
}
__device__ __forceinline__ double gv_weight_bits(unsigned u, int e) {
  return gv_ldexp_bits(gv_widen(__uint_as_float(u)), e);
}

// round(m 2^s), half up, for m < 2^24 and s <= 72, with the sign: the tile's
// fixed-point value of a direct weight (|w| < 2^E, s = e2 - E + GV_FB), as
// gv_fixed_tile rounds the equal double.
__device__ __forceinline__ u128 gv_direct_fixed(unsigned long long m, int s, bool neg) {
  u128 v;
  if (s >= 0) {
    v.lo = s < 64 ? m << s : 0ull;
    v.hi = s > 40 ? (s < 64 ? m >> (64 - s) : m << (s - 64)) : 0ull;
  } else {
    const int r = -s;
    v.lo = r < 64 ? ((m >> (r - 1)) + 1ull) >> 1 : 0ull;
    v.hi = 0ull;
  }
  return gv_negate_if(v, neg);
}

// round(M 2^t), half up, for the square M = m^2 < 2^48 of a direct weight's
// significand and t = 2 (e2 - E) + GV_FB <= 48: the tile's fixed-point square,
// as gv_square_tile rounds it.
__device__ __forceinline__ u128 gv_direct_square(unsigned long long M, int t) {
  u128 v;
  if (t >= 0) {
    v.lo = M << t;
    v.hi = t > 16 ? M >> (64 - t) : 0ull;
  } else {
    const int r = -t;
    v.lo = r < 64 ? ((M >> (r - 1)) + 1ull) >> 1 : 0ull;
    v.hi = 0ull;
  }
  return v;
}

template <typename Real>
struct GvPair;
template <>
struct GvPair<float> {
  using T = GvBin32;
};
template <>
struct GvPair<double> {
  using T = GvBin64;
};

// Shared-memory layout of the fill kernel (bytes), 16-byte aligned pieces:
//   hist [4][d*N] u32     per-bin sums of w^2 in three 22-bit limbs, then the
//                         tile's bin exponents F_tb + GV_BINE_OFF (forward only)
//   jac  [d*N]    f64     Jacobian factor N*(e_{i+1}-e_i) (FP64 form only)
//   ew   [d*N]    GvBin32 (e, w, jm, je) in the FP32 form, GvBin64 (e, w) in FP64
//   bins [d][GV_TILE] u16 (forward kernels of the d > 4 classes only)
//   hh   [7][nhist] u32   histogram: w^2 limbs [3], w limbs [3] (the third
//                         signed), the tile's bin exponents (with a histogram)
//   po   [GV_PLUS_WIN] i32 hypercube offsets relative to the tile (VEGAS+)
//   ps   [GV_PLUS_WIN + GV_TILE/GV_PLUS_SEG] double2  the tile's segments
//                         (VEGAS+): each window hypercube's first, then each
//                         range's continuation of an earlier hypercube
//   wd   [ceil(d/4)][GV_TILE] uint4  the tile's Philox words, generated before
//                         the kernel waits for its predecessor (see below)
__host__ __device__ inline size_t gv_align16(size_t b) { return (b + 15) & ~(size_t)15; }

// The forward fill generates its tile's Philox words before it waits for the
// previous kernel (the words depend only on the seed, the counter and the
// event), where the launch overlaps the previous iteration's reduce and
// refinement (VEGAS+: its layout; the stratified fill stratifies the words
// after the wait); not beyond 8 axes, nor where the words' shared memory
// would take the layout past GV_WORDS_SMEM_MAX (the host sets
// GvFillArgs::hoist accordingly).
#define GV_WORDS_SMEM_MAX (200 * 1024)
__host__ __device__ inline bool gv_fill_hoistable(bool forward, bool plus, int d) {
  (void)plus;  // the stratified fill stratifies the hoisted words after its wait
  return forward && d <= 8;
}

// A tile of GV_TILE events meets at most GV_TILE/2 + 1 hypercubes (each has
// at least 2 events): the window holds their offsets and the next one.
#define GV_PLUS_WIN (GV_TILE / 2 + 4)

#define GV_PLUS_SEGS (GV_PLUS_WIN + GV_TILE / GV_PLUS_SEG)

struct GvFillSmem {
  size_t hist, jac, ew, bins, hh, po, ps, wd, total;
  __host__ __device__ GvFillSmem(int d, int N, int real_bytes, bool forward, bool bins_smem,
                                 int nhist = 0, bool plus = false, bool words = false) {
    const size_t dN = (size_t)d * N;
    hist = 0;
    jac = gv_align16(hist + (forward ? dN * 16 : 0));
    ew = gv_align16(jac + (real_bytes == 8 ? dN * 8 : 0));
    bins = gv_align16(ew + dN * 16);
    hh = gv_align16(bins + ((forward && bins_smem) ? (size_t)d * GV_TILE * 2 : 0));
    po = gv_align16(hh + (forward ? (size_t)nhist * 7 * 4 : 0));
    ps = gv_align16(po + (plus ? (size_t)GV_PLUS_WIN * 4 : 0));
    wd = gv_align16(ps + (plus ? (size_t)GV_PLUS_SEGS * 16 : 0));
    total = gv_align16(wd + (words ? (size_t)((d + 3) / 4) * GV_TILE * 16 : 0));
  }
};

// VEGAS+: the hypercube of the tile's local event `local` (the last window
// entry at or below it), and the stratified words of hypercube h:
// r' = floor((c_a 2^32 + r_a) / s) with c_a the base-s digits of h (the
// next two functions).
__device__ __forceinline__ int gv_plus_cube(const int* s_off, int local) {
  int lo = 0, hi = GV_PLUS_WIN;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (s_off[mid] <= local)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// A range's segment of window hypercube j (sums s1, s2): the hypercube's
// first segment if it begins in the range (at or after local event r0),
// else the range's continuation of it.  Staged in shared memory (s_seg:
// first segments by window index, then continuations by the tile's range);
// the segments of a hypercube that crosses a tile boundary (offsets outside
// [0, GV_TILE]: the finishing kernel forms its statistics) go to memory too.
__device__ __forceinline__ void gv_plus_put_segment(const GvPlusFill* pf, const int* s_off,
                                                    double2* s_seg, long long h0, int j,
                                                    long long tile0, int r0, double s1,
                                                    double s2) {
  const double2 v = make_double2(s1, s2);
  const bool crossing = s_off[j] < 0 || s_off[j + 1] > GV_TILE;
  if (s_off[j] >= r0) {
    s_seg[j] = v;
    if (crossing) pf->seg_h[h0 + j] = v;
  } else {
    s_seg[GV_PLUS_WIN + r0 / GV_PLUS_SEG] = v;
    if (crossing) pf->seg_r[(tile0 + r0) / GV_PLUS_SEG] = v;
  }
}

// The statistics of every hypercube whose events all lie in the tile, from
// its staged segments in range order (as the finishing kernel adds a crossing
// hypercube's), and the tile's sums of their v/n and weights: thread t takes
// window hypercubes t, t + B, .. in order; then warp 0's lane l adds threads
// (B/32) l .. (B/32)(l + 1) - 1 in order, and a butterfly adds the lanes.
// Few FP64 instructions, one chain.  Written by thread 0 to tpart[tile].
template <int B>
__device__ __forceinline__ void gv_plus_tile_stats(const GvPlusFill* pf, const int* s_off,
                                                   const double2* s_seg, long long h0,
                                                   long long tile, double2* s_red) {
  const int tid = threadIdx.x;
  double vn = 0.0, dd = 0.0;
  for (int j = tid; j < GV_PLUS_WIN - 1; j += B) {
    const int o = s_off[j], e = s_off[j + 1];
    if (o < 0 || e > GV_TILE || h0 + j >= pf->nh) continue;  // crossing, or past the last
    double s1 = s_seg[j].x, s2 = s_seg[j].y;
    for (int r = o / GV_PLUS_SEG + 1; r <= (e - 1) / GV_PLUS_SEG; ++r) {
      s1 += s_seg[GV_PLUS_WIN + r].x;
      s2 += s_seg[GV_PLUS_WIN + r].y;
    }
    const GvPlusStat st = gv_plus_stat(s1, s2, e - o, pf->inv, pf->beta_j);
    pf->var[h0 + j] = st.v;
    pf->dw[h0 + j] = st.w;
    vn += st.vn;
    dd += st.w;
  }
  constexpr int L = B / 32;
  s_red[tid] = make_double2(vn, dd);
  __syncthreads();
  if (tid < 32) {
    double2 r = s_red[L * tid];
#pragma unroll
    for (int i = 1; i < L; ++i) {
      r.x += s_red[L * tid + i].x;
      r.y += s_red[L * tid + i].y;
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      r.x += __shfl_xor_sync(0xffffffffu, r.x, m);
      r.y += __shfl_xor_sync(0xffffffffu, r.y, m);
    }
    if (tid == 0) pf->tpart[tile] = r;
  }
}

// The base-s digits c_a of hypercube h (h < 2^22 is exact in FP32: h / s
// from a float estimate, corrected to the floor).
template <int MAXD>
__device__ __forceinline__ void gv_plus_digits(unsigned h, int d, unsigned s, float inv_s,
                                               unsigned (&c)[MAXD]) {
#pragma unroll
  for (int ax = 0; ax < MAXD; ++ax) {
    if (ax < d) {
      unsigned q = (unsigned)((float)h * inv_s);
      if (q * s > h)
        --q;
      else if ((q + 1u) * s <= h)
        ++q;
      c[ax] = h - q * s;
      h = q;
    }
  }
}

// The stratified words floor(X / s), X = c_a 2^32 + r_a < 2^54: the product
// with floor((2^64-1)/s) is the quotient or one less.
template <int MAXD>
__device__ __forceinline__ void gv_plus_strat(const unsigned (&c)[MAXD], int d, unsigned s,
                                              unsigned long long magic, uint32_t (&r)[MAXD]) {
#pragma unroll
  for (int ax = 0; ax < MAXD; ++ax) {
    if (ax < d) {
      const unsigned long long X = ((unsigned long long)c[ax] << 32) | r[ax];
      unsigned long long t = __umul64hi(X, magic);
      if ((t + 1ull) * s <= X) ++t;
      r[ax] = (uint32_t)t;
    }
  }
}

// Stage the grid of one integration into shared memory.
template <typename Real>
__device__ __forceinline__ void gv_stage_grid(const double* grid, int d, int N, double* s_jac,
                                              typename GvPair<Real>::T* s_ew, int tid,
                                              int nthr) {
  const GvGridLayout L{d, N};
  const int dN = d * N;
  const float* g32 = reinterpret_cast<const float*>(grid + L.off_f32_base());
  for (int k = tid; k < dN; k += nthr) {
    const int a = k / N, i = k - a * N;
    if constexpr (sizeof(Real) == 4) {
      GvBin32 b;
      b.e = g32[L.w_e32() + a * (N + 1) + i];
      b.w = g32[L.w_wd32() + k];
      b.jm = g32[L.w_jm32() + k];
      b.je = reinterpret_cast<const int*>(g32)[L.w_je() + k];
      s_ew[k] = b;
    } else {
      s_jac[k] = grid[L.off_jac() + k];
      GvBin64 b;
      b.e = grid[L.off_e64() + a * (N + 1) + i];
      b.w = grid[L.off_wd64() + k];
      s_ew[k] = b;
    }
  }
}

// Map one event's words through the grid: x, bins and the Jacobian.
// FP64: x = e_i + f*(e_{i+1}-e_i) with f = (lo + 1/2) 2^-32, rounded as
// written, J the FP64 product of the factors N (e_{i+1}-e_i); FP32: x with
// FP32 edges and one fma, J as FP32 mantissa product and exponent sum.  The
// product starts from the first factor (J = 1 * f0 * f1 ... exactly).
template <typename Real, int MAXD>
__device__ __forceinline__ GvJac<Real> gv_map_event(const uint32_t (&r)[MAXD], int d, int N,
                                                    const double* s_jac,
                                                    const typename GvPair<Real>::T* s_ew,
                                                    Real (&x)[MAXD], int (&bin)[MAXD]) {
  GvJac<Real> J;
#pragma unroll
  for (int a = 0; a < MAXD; ++a) {
    if (a < d) {
      const unsigned long long v = (unsigned long long)r[a] * (unsigned)N;
      const int i = (int)(v >> 32);
      const uint32_t lo = (uint32_t)v;
      const auto ew = s_ew[a * N + i];
      if constexpr (sizeof(Real) == 4) {
        const float f = fmaf(__uint2float_rn(lo), 0x1p-32f, 0x1p-33f);
        x[a] = fmaf(f, ew.w, ew.e);
        J.m = (a == 0) ? ew.jm : __fmul_rn(J.m, ew.jm);
        J.e = (a == 0) ? ew.je : J.e + ew.je;
      } else {
        const double f = ((double)lo + 0.5) * 0x1p-32;
        x[a] = __dadd_rn(ew.e, __dmul_rn(f, ew.w));
        const double jf = s_jac[a * N + i];
        J.v = (a == 0) ? jf : __dmul_rn(J.v, jf);
      }
      bin[a] = i;
    }
  }
  return J;
}

// Block-wide reductions over the NW warps of a CTA (results to every thread).
template <int NW>
__device__ __forceinline__ unsigned long long gv_block_max(unsigned long long v,
                                                           unsigned long long* scratch) {
  v = warp_max_u64(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  unsigned long long m = scratch[0];
#pragma unroll
  for (int w = 1; w < NW; ++w) m = scratch[w] > m ? scratch[w] : m;
  __syncthreads();
  return m;
}

template <int NW>
__device__ __forceinline__ int gv_block_max_int(int v, int* scratch) {
  v = __reduce_max_sync(0xffffffffu, v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  int m = scratch[0];
#pragma unroll
  for (int w = 1; w < NW; ++w) m = max(m, scratch[w]);
  __syncthreads();
  return m;
}

template <int NW>
__device__ __forceinline__ u128 gv_block_sum128(u128 v, u128* scratch) {
  v = warp_sum128(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  u128 s = scratch[0];
#pragma unroll
  for (int w = 1; w < NW; ++w) s = add128(s, scratch[w]);
  __syncthreads();
  return s;
}

// Bins of one event between the two passes: packed u16 pairs in registers for
// d <= 4, shared memory otherwise.
template <int MAXD>
struct GvBinStore {
  static constexpr bool REG = MAXD <= 4;
  uint32_t q[REG ? 2 : 1];
  __device__ __forceinline__ void put(const int (&bin)[MAXD], int d, unsigned short* s_bin,
                                      int local) {
    if constexpr (REG) {
      q[0] = (uint32_t)bin[0] | ((MAXD > 1 && d > 1 ? (uint32_t)bin[1] : 0u) << 16);
      q[1] = (MAXD > 2 && d > 2 ? (uint32_t)bin[2] : 0u) |
             ((MAXD > 3 && d > 3 ? (uint32_t)bin[3] : 0u) << 16);
    } else {
#pragma unroll
      for (int a = 0; a < MAXD; ++a)
        if (a < d) s_bin[a * GV_TILE + local] = (unsigned short)bin[a];
    }
  }
  __device__ __forceinline__ int get(int a, const unsigned short* s_bin, int local) const {
    if constexpr (REG)
      return (int)((q[a >> 1] >> ((a & 1) * 16)) & 0xFFFFu);
    else
      return s_bin[a * GV_TILE + local];
  }
};


// |x| bits of a double, and its finiteness, on the integer pipes.
__device__ __forceinline__ unsigned long long gv_abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ bool gv_finite_bits(unsigned long long absbits) {
  return absbits < 0x7FF0000000000000ull;
}

// The scale exponent of the weight u 2^e (gv_scale_exp of the double) and
// whether that double is finite.
__device__ __forceinline__ int gv_direct_scale(unsigned u, int e, bool& fin) {
  const GvDirect dd = gv_direct(u, e);
  if (dd.direct) {
    fin = true;
    return dd.e2 + 24;
  }
  const unsigned long long ab = gv_abs_bits(gv_weight_bits(u, e));
  fin = gv_finite_bits(ab);
  return gv_scale_exp(ab);
}

// ---------------------------------------------------------------------------
// Forward fill of one tile: channel 0 = w, with per-bin sums of w^2.  The grid
// of the integration must be staged and the histogram zeroed (both followed
// by a barrier) before the call.  Used by the per-integration kernel and by
// the persistent batched kernel, so that a tile's partial is the same
// whichever kernel computes it.
// ---------------------------------------------------------------------------
template <int IG, typename Real, int EPT, int MAXD, bool HIST = false, bool PLUS = false>
__device__ __forceinline__ void gv_fill_tile(const GvFillArgs& a, long long tile,
                                             unsigned char* smem, unsigned long long* red_u64,
                                             u128* red_128, uint32_t it,
                                             const uint4* s_words = nullptr) {
  constexpr int B = GV_TILE / EPT;
  constexpr int NW = B / 32;
  using Pair = typename GvPair<Real>::T;
  const int d = a.ndim, N = a.nbins, dN = d * N;
  const int hb = HIST ? a.nhist : 0;
  const GvFillSmem lay(d, N, (int)sizeof(Real), true, MAXD > 4, hb, PLUS);
  unsigned* hh = reinterpret_cast<unsigned*>(smem + lay.hh);  // [6][hb] limbs
  const int* s_off = reinterpret_cast<const int*>(smem + lay.po);
  double2* s_seg = reinterpret_cast<double2*>(smem + lay.ps);
  const GvPlusFill* pf = a.plus;
  const long long ncall = PLUS ? *pf->ncall : a.ncall;
  const long long h0 = PLUS ? pf->tile_h0[tile] : 0;
  double qv[EPT];  // VEGAS+: the bins' quantity F b_h (w itself otherwise)
  int* hebin = reinterpret_cast<int*>(hh + 6 * hb);             // [hb] exponents
  Real h_lo, h_invw;
  if constexpr (sizeof(Real) == 4) {
    h_lo = a.h_lo_f;
    h_invw = a.h_invw_f;
  } else {
    h_lo = a.h_lo;
    h_invw = a.h_invw;
  }
  int hbin[EPT];
  unsigned* hist = reinterpret_cast<unsigned*>(smem + lay.hist);  // [3][dN] limbs
  int* ebin = reinterpret_cast<int*>(hist + 3 * dN);               // [dN] exponents
  const double* s_jac = reinterpret_cast<const double*>(smem + lay.jac);
  const Pair* s_ew = reinterpret_cast<const Pair*>(smem + lay.ew);
  unsigned short* s_bin = reinterpret_cast<unsigned short*>(smem + lay.bins);
  const int tid = threadIdx.x;
  GvConst<Real, GvTraits<IG>::NK> K;
  K.load(a.kconst);

  // FP32 form: each weight is kept as its FP32 product and Jacobian exponent
  // and summed through gv_direct (VEGAS+: the estimate's weight in wp, the
  // bins' quantity in wq)
  constexpr bool DIRECT = sizeof(Real) == 4;
  const long long tile0 = tile * GV_TILE;
  [[maybe_unused]] double w[EPT];
  [[maybe_unused]] unsigned wp[EPT], wq[EPT];
  [[maybe_unused]] int wj[EPT];
  GvBinStore<MAXD> bs[EPT];
  unsigned long long mx = 0ull;
  int mE = GV_EMPTY;  // the direct form's largest weight scale
  unsigned long long nbad = 0ull;
  // VEGAS+: this thread's range (events tile0 + tid EPT ..), the window index
  // of its current hypercube, that hypercube's digits and factors, and the
  // running segment sums
  static_assert(!PLUS || EPT == GV_PLUS_SEG, "a stratified fill thread holds one range");
  [[maybe_unused]] int jc = PLUS ? gv_plus_cube(s_off, tid * EPT) : 0;
  [[maybe_unused]] int jcur = -1;  // the open segment's window index
  [[maybe_unused]] double sg1 = 0.0, sg2 = 0.0;
  constexpr bool KEEP_DIGITS = MAXD <= 4;  // registers to spare only for few axes
  [[maybe_unused]] unsigned cdig[MAXD];
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int local = PLUS ? tid * EPT + k : k * B + tid;
    const long long ev = tile0 + local;
    if constexpr (DIRECT) {
      wp[k] = 0u;
      wq[k] = 0u;
      wj[k] = 0;
    } else {
      w[k] = 0.0;
    }
    if constexpr (PLUS) qv[k] = 0.0;
    hbin[k] = 0;
    if (ev < ncall) {
      uint32_t r[MAXD];
      if (s_words) {  // generated before the wait (the kernel's barrier precedes this)
#pragma unroll
        for (int j = 0; j < (MAXD + 3) / 4; ++j) {
          if (4 * j < d) {
            const uint4 o = s_words[j * GV_TILE + local];
            if (4 * j + 0 < MAXD) r[4 * j + 0] = o.x;
            if (4 * j + 1 < MAXD) r[4 * j + 1] = o.y;
            if (4 * j + 2 < MAXD) r[4 * j + 2] = o.z;
            if (4 * j + 3 < MAXD) r[4 * j + 3] = o.w;
          }
        }
      } else {
        gv_event_words<MAXD>(a.seed, it, a.batch, (unsigned long long)ev, d, r);
      }
      if constexpr (PLUS) {
        while (jc + 1 < GV_PLUS_WIN && s_off[jc + 1] <= local) ++jc;
        if (jc != jcur) {  // a new hypercube: close the previous segment
          if (jcur >= 0)
            gv_plus_put_segment(pf, s_off, s_seg, h0, jcur, tile0, tid * EPT, sg1, sg2);
          jcur = jc;
          sg1 = 0.0;
          sg2 = 0.0;
          if (KEEP_DIGITS)
            gv_plus_digits<MAXD>((unsigned)(h0 + jc), d, (unsigned)pf->s, pf->inv_s, cdig);
        }
        if (!KEEP_DIGITS)
          gv_plus_digits<MAXD>((unsigned)(h0 + jc), d, (unsigned)pf->s, pf->inv_s, cdig);
        gv_plus_strat<MAXD>(cdig, d, (unsigned)pf->s, pf->magic, r);
      }
      Real x[MAXD];
      int bin[MAXD];
      const GvJac<Real> J = gv_map_event<Real, MAXD>(r, d, N, s_jac, s_ew, x, bin);
      bs[k].put(bin, d, s_bin, local);
      const Real g = gv_eval<IG, Real, MAXD>(x, d, K);
      if constexpr (HIST) hbin[k] = gv_hist_bin<Real>(gv_observable<IG, Real, MAXD>(x, K), h_lo,
                                                      h_invw, hb - 2);
      if constexpr (DIRECT) {
        const unsigned u = __float_as_uint(__fmul_rn(J.m, g));
        if ((u & 0x7FFFFFFFu) != 0u) {
          // VEGAS+: the estimate's weight u a_h and the bins' quantity u b_h,
          // FP32 products with the hypercube's factors rounded to FP32
          unsigned uw = u, uq = u;
          if constexpr (PLUS) {
            const float2 f = pf->ab32[h0 + jc];
            uw = __float_as_uint(__fmul_rn(__uint_as_float(u), f.x));
            uq = __float_as_uint(__fmul_rn(__uint_as_float(u), f.y));
          }
          bool fin, finq = true;
          const int Ev = gv_direct_scale(uw, J.e, fin);
          int Eq = Ev;
          if constexpr (PLUS) Eq = gv_direct_scale(uq, J.e, finq);
          if (fin && finq) {
            if constexpr (PLUS) {
              // F = u 2^e, widened exactly, into the segment (a rounded
              // product, then the sum, as the statistics define them: the
              // variance cancels where a hypercube's values are nearly equal)
              double Fv = gv_weight_bits(u, J.e);
              Fv = gv_finite_bits(gv_abs_bits(Fv)) ? Fv : 0.0;
              sg1 += Fv;
              sg2 += Fv * Fv;
              wq[k] = uq;
            }
            wp[k] = uw;
            wj[k] = J.e;
            if (Ev != GV_EMPTY) mE = max(mE, Ev);
            if (Eq != GV_EMPTY) {
              const int F = Eq + GV_BINE_OFF;
#pragma unroll
              for (int ax = 0; ax < MAXD; ++ax)
                if (ax < d) atomicMax(ebin + ax * N + bin[ax], F);
              if constexpr (HIST) atomicMax(hebin + hbin[k], F);
            }
          } else {
            ++nbad;  // counted, contributes nothing
          }
        }
        continue;
      }
      double wv = gv_weight(J, g);
      [[maybe_unused]] double qk = 0.0;
      if constexpr (PLUS) {
        // F = J g into the segment (0 if not finite); the estimate's weight
        // F C/(nh n_h), the bins' F sqrt(1/(nh n_h))
        // (a rounded product, then the sum, as the statistics define them: the
        // variance cancels where a hypercube's values are nearly equal)
        const double Fv = gv_finite_bits(gv_abs_bits(wv)) ? wv : 0.0;
        sg1 += Fv;
        sg2 += Fv * Fv;
        const double2 f = pf->ab[h0 + jc];
        qk = wv * f.y;
        wv = wv * f.x;
      }
      const unsigned long long ab = gv_abs_bits(wv);
      unsigned long long bb = ab;  // |the bins' quantity|
      bool fin = gv_finite_bits(ab);
      if constexpr (PLUS) {
        bb = gv_abs_bits(qk);
        fin = fin && gv_finite_bits(bb);
      }
      if (fin) {
        w[k] = wv;
        if constexpr (PLUS) qv[k] = qk;
        mx = ab > mx ? ab : mx;
        if (bb != 0ull) {
          const int F = gv_scale_exp(bb) + GV_BINE_OFF;
#pragma unroll
          for (int ax = 0; ax < MAXD; ++ax)
            if (ax < d) atomicMax(ebin + ax * N + bin[ax], F);
          if constexpr (HIST) atomicMax(hebin + hbin[k], F);
        }
      } else {
        ++nbad;  // counted, contributes nothing
      }
    }
  }
  if constexpr (PLUS) {
    // the range's last segment and its first hypercube
    if (jcur >= 0) gv_plus_put_segment(pf, s_off, s_seg, h0, jcur, tile0, tid * EPT, sg1, sg2);
  }
  // the tile's scale (the barrier also orders ebin)
  int E;
  if constexpr (DIRECT)
    E = gv_block_max_int<NW>(mE, reinterpret_cast<int*>(red_u64));
  else
    E = gv_scale_exp(gv_block_max<NW>(mx, red_u64));

  u128 s1 = {0ull, 0ull}, s2 = {0ull, 0ull};
  if (E != GV_EMPTY) {
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      bool any;
      if constexpr (DIRECT)
        any = (wp[k] & 0x7FFFFFFFu) != 0u || (PLUS && (wq[k] & 0x7FFFFFFFu) != 0u);
      else
        any = gv_abs_bits(w[k]) != 0ull || (PLUS && gv_abs_bits(qv[k]) != 0ull);
      if (any) {
        const int local = PLUS ? tid * EPT + k : k * B + tid;
        // bins: w^2 (VEGAS+: q^2) at its bin's scale, a 56-bit value, as three
        // 22-bit limbs, from P = floor(m^2 2^-42) of its 53-bit significand m
        // and c = 2 e2 + 98 + 2 GV_BINE_OFF
        unsigned long long P;
        int c;
        [[maybe_unused]] GvDecoded dw;
        if constexpr (DIRECT) {
          const GvDirect dd = gv_direct(wp[k], wj[k]);
          if (dd.direct) {
            const unsigned long long M = (unsigned long long)dd.m * dd.m;
            s1 = add128(s1, gv_direct_fixed(dd.m, dd.e2 - E + GV_FB, dd.neg));
            s2 = add128(s2, gv_direct_square(M, 2 * (dd.e2 - E) + GV_FB));
            P = M << 16;  // m = dd.m 2^29
            c = 2 * (dd.e2 - 29) + 98 + 2 * GV_BINE_OFF;
            if constexpr (HIST) dw = GvDecoded{(unsigned long long)dd.m << 29, dd.e2 - 29, dd.neg};
          } else {
            dw = gv_decode(gv_weight_bits(wp[k], wj[k]));
            P = gv_square_hi(dw.m);
            c = 2 * dw.e2 + 98 + 2 * GV_BINE_OFF;
            if (dw.m != 0ull) {
              s1 = add128(s1, gv_fixed_tile(dw, E));
              s2 = add128(s2, gv_square_tile(dw, P, E));
            } else if (!PLUS) {
              continue;  // below the FP64 range: zero
            }
          }
          if constexpr (PLUS) {
            // the bins' terms from the bins' quantity
            const GvDirect dq = gv_direct(wq[k], wj[k]);
            if (dq.direct) {
              P = ((unsigned long long)dq.m * dq.m) << 16;
              c = 2 * (dq.e2 - 29) + 98 + 2 * GV_BINE_OFF;
            } else {
              const GvDecoded q = gv_decode(gv_weight_bits(wq[k], wj[k]));
              if (q.m == 0ull) continue;  // below the FP64 range: zero
              P = gv_square_hi(q.m);
              c = 2 * q.e2 + 98 + 2 * GV_BINE_OFF;
            }
          }
        } else {
          dw = gv_decode(w[k]);
          const unsigned long long Pw = gv_square_hi(dw.m);
          s1 = add128(s1, gv_fixed_tile(dw, E));
          s2 = add128(s2, gv_square_tile(dw, Pw, E));
          const GvDecoded dq = PLUS ? gv_decode(qv[k]) : dw;
          P = PLUS ? gv_square_hi(dq.m) : Pw;
          c = 2 * dq.e2 + 98 + 2 * GV_BINE_OFF;
        }
#pragma unroll
        for (int ax = 0; ax < MAXD; ++ax) {
          if (ax < d) {
            const int bi = ax * N + bs[k].get(ax, s_bin, local);
            const unsigned long long q = gv_square_bin(P, 2 * ebin[bi] - c);
            const unsigned l0 = (unsigned)(q & 0x3FFFFFull);
            const unsigned l1 = (unsigned)((q >> 22) & 0x3FFFFFull);
            const unsigned l2 = (unsigned)(q >> 44);
            if (l0) atomicAdd(hist + bi, l0);
            if (l1) atomicAdd(hist + dN + bi, l1);
            if (l2) atomicAdd(hist + 2 * dN + bi, l2);
          }
        }
        if constexpr (HIST) {
          // the observable's bin: w^2 as the axis bins, then w (signed)
          const int hk = hbin[k];
          const int Fh = hebin[hk];
          const unsigned long long q = gv_square_bin(P, 2 * Fh - c);
          const unsigned l0 = (unsigned)(q & 0x3FFFFFull);
          const unsigned l1 = (unsigned)((q >> 22) & 0x3FFFFFull);
          const unsigned l2 = (unsigned)(q >> 44);
          if (l0) atomicAdd(hh + hk, l0);
          if (l1) atomicAdd(hh + hb + hk, l1);
          if (l2) atomicAdd(hh + 2 * hb + hk, l2);
          const long long v = gv_hist_fixed(dw, Fh - GV_BINE_OFF);
          const unsigned m0 = (unsigned)((unsigned long long)v & 0x3FFFFFull);
          const unsigned m1 = (unsigned)(((unsigned long long)v >> 22) & 0x3FFFFFull);
          const unsigned m2 = (unsigned)(int)(v >> 44);  // signed, |v >> 44| <= 2^12
          if (m0) atomicAdd(hh + 3 * hb + hk, m0);
          if (m1) atomicAdd(hh + 4 * hb + hk, m1);
          if (m2) atomicAdd(hh + 5 * hb + hk, m2);
        }
      }
    }
  }
  if constexpr (PLUS) {
    // the hypercubes this tile holds whole (the barrier of the tile's scale
    // ordered the staged segments)
    __shared__ double2 s_pr[PLUS ? B : 1];
    gv_plus_tile_stats<B>(pf, s_off, s_seg, h0, tile, s_pr);
  }
  const u128 t1 = gv_block_sum128<NW>(s1, red_128);
  const u128 t2 = gv_block_sum128<NW>(s2, red_128);
  gv_allow_next_grid();
  // the tile's slots: slot k at out[k ks] (tile-major or slot-major partials)
  const size_t ks = a.slot_major ? (size_t)a.n_tiles : (size_t)1;
  ulonglong2* out = a.part + (a.slot_major ? (size_t)tile : (size_t)tile * a.nacc);
  if (tid == 0) {
    out[0] = make_ulonglong2(t1.lo, t1.hi);
    out[ks] = make_ulonglong2(t2.lo, t2.hi);
    a.tileE[tile] = E;
  }
  if (nbad) atomicAdd(&a.st->nonfinite_iter, nbad);
  for (int k = tid; k < dN; k += B) {
    // Q = l0 + l1 2^22 + l2 2^44 (< 2^67) in units of 2^(2 F_tb - GV_BIN_QBITS),
    // with F_tb + GV_BINE_OFF in bits 96.. of the partial
    const unsigned long long l0 = hist[k], l1 = hist[dN + k], l2 = hist[2 * dN + k];
    u128 v = {l0, 0ull};
    v = add128(v, u128{l1 << 22, l1 >> 42});
    v = add128(v, u128{l2 << 44, l2 >> 20});
    out[(2 + k) * ks] = make_ulonglong2(v.lo, v.hi | ((unsigned long long)(unsigned)ebin[k] << 32));
  }
  if constexpr (HIST) {
    for (int k = tid; k < hb; k += B) {
      const unsigned long long eh = (unsigned long long)(unsigned)hebin[k] << 32;
      // w^2: as the axis bins
      const unsigned long long l0 = hh[k], l1 = hh[hb + k], l2 = hh[2 * hb + k];
      u128 v = {l0, 0ull};
      v = add128(v, u128{l1 << 22, l1 >> 42});
      v = add128(v, u128{l2 << 44, l2 >> 20});
      out[(2 + dN + k) * ks] = make_ulonglong2(v.lo, v.hi | eh);
      // w: M = m0 + m1 2^22 + m2 2^44 with m2 signed (|M| < 2^67) as a 96-bit
      // two's complement value in units of 2^(F_tb - GV_BIN_QBITS)
      const unsigned long long m0 = hh[3 * hb + k], m1 = hh[4 * hb + k];
      const long long m2 = (long long)(int)hh[5 * hb + k];
      u128 t = {m0, 0ull};
      t = add128(t, u128{m1 << 22, m1 >> 42});
      t = add128(t, u128{(unsigned long long)m2 << 44, (unsigned long long)(m2 >> 20)});
      out[(2 + dN + hb + k) * ks] = make_ulonglong2(t.lo, (t.hi & 0xFFFFFFFFull) | eh);
    }
  }
}

// The Philox words of a tile's events at counter `it` into shared memory
// (layout [ceil(d/4)][GV_TILE]); each thread makes the words of the events it
// will evaluate (local index tid + k B), so no barrier is needed before use.
template <int MAXD>
__device__ __forceinline__ void gv_tile_words(const GvFillArgs& a, uint32_t it, long long tile,
                                              uint4* s_words, int B) {
  const int d = a.ndim;
  const long long t0 = tile * GV_TILE;
  for (int local = threadIdx.x; local < GV_TILE; local += B) {
    uint32_t r[MAXD];
    gv_event_words<MAXD>(a.seed, it, a.batch, (unsigned long long)(t0 + local), d, r);
#pragma unroll
    for (int j = 0; j < (MAXD + 3) / 4; ++j)
      if (4 * j < d)
        s_words[j * GV_TILE + local] =
            make_uint4(r[4 * j], 4 * j + 1 < MAXD ? r[4 * j + 1] : 0u,
                       4 * j + 2 < MAXD ? r[4 * j + 2] : 0u, 4 * j + 3 < MAXD ? r[4 * j + 3] : 0u);
  }
}

// Minimum resident CTAs per SM in the fill's launch bound (0: none), i.e. its
// register budget.  FP32 fills of at most 8 axes: 64 registers at any width
// (the stratified fill of at most 4 axes included; the stratified fill of up
// to 8 axes, which keeps its range's segment sums, takes 80 with three
// 256-thread CTAs: at 64 it spilled ~250 bytes).  FP32 fills of up to 16 axes without
// VEGAS+, 4 events per thread: three 256-thread CTAs, 80 registers (111 for
// the 13-axis NLO-shaped weight unbounded).  FP64 fills: none (they would
// spill).
template <typename Real, int EPT, int MAXD, bool PLUS>
struct GvFillBlocks {
  static constexpr int B = GV_TILE / EPT;
  static constexpr int value = sizeof(Real) != 4       ? 0
                               : (PLUS && MAXD == 8)   ? 3
                               : MAXD <= 8             ? 65536 / (64 * B)
                               : (!PLUS && EPT == 4)   ? 3
                                                       : 0;
};

template <int IG, typename Real, int EPT, int MAXD, bool HIST = false, bool PLUS = false>
__global__ void __launch_bounds__(GV_TILE / EPT, (GvFillBlocks<Real, EPT, MAXD, PLUS>::value))
    gv_fill_kernel(const GvFillArgs a) {
  constexpr int B = GV_TILE / EPT;
  constexpr int NW = B / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long red_u64[NW];
  __shared__ u128 red_128[NW];
  const int d = a.ndim, N = a.nbins;
  const bool hoist = MAXD <= 8 && a.hoist;  // set by the host (gv_fill_hoistable)
  const GvFillSmem lay(d, N, (int)sizeof(Real), true, MAXD > 4, HIST ? a.nhist : 0, PLUS, hoist);
  unsigned* hist = reinterpret_cast<unsigned*>(smem + lay.hist);
  for (int k = threadIdx.x; k < 4 * d * N; k += B) hist[k] = 0u;
  if constexpr (HIST) {
    unsigned* hh = reinterpret_cast<unsigned*>(smem + lay.hh);
    for (int k = threadIdx.x; k < 7 * a.nhist; k += B) hh[k] = 0u;
  }
  // the tile's words at the counter this iteration should have (the stage's
  // first counter, which no running kernel writes, plus the iteration index),
  // made while the previous iteration's reduce and refinement finish
  uint4* s_words = reinterpret_cast<uint4*>(smem + lay.wd);
  uint32_t itg = 0u;
  if (hoist) {
    itg = (uint32_t)(a.st->it0 + (unsigned long long)a.kst);
    gv_tile_words<MAXD>(a, itg, blockIdx.x, s_words, B);
  }
  gv_wait_prior_grid();  // grid, constants and iteration counter come from earlier kernels
  if constexpr (PLUS) {
    // VEGAS+ sizes the grid for the most events an allocation can have; the
    // iteration's events fill the first tiles_used tiles, which alone the
    // reduce reads, and a tile past them does nothing
    const long long ncall = *a.plus->ncall;
    if (blockIdx.x == 0 && threadIdx.x == 0)
      *a.plus->tiles_used = (int)((ncall + GV_TILE - 1) / GV_TILE);
    if ((long long)blockIdx.x * GV_TILE >= ncall) return;
  }
  gv_stage_grid<Real>(a.grid, d, N, reinterpret_cast<double*>(smem + lay.jac),
                      reinterpret_cast<typename GvPair<Real>::T*>(smem + lay.ew), threadIdx.x, B);
  if constexpr (PLUS) {
    // the offsets of the hypercubes this tile can meet, relative to its first
    // event and clamped to [-1, GV_TILE + 1]
    int* s_off = reinterpret_cast<int*>(smem + lay.po);
    const GvPlusFill* pf = a.plus;
    const long long h0 = pf->tile_h0[blockIdx.x];
    const long long t0 = (long long)blockIdx.x * GV_TILE;
    for (int j = threadIdx.x; j < GV_PLUS_WIN; j += B) {
      int v = GV_TILE + 1;
      if (h0 + j <= pf->nh) {
        const long long o = pf->off[h0 + j] - t0;
        v = o < -1 ? -1 : (o > GV_TILE ? GV_TILE + 1 : (int)o);
      }
      s_off[j] = v;
    }
  }
  const uint32_t it = (uint32_t)a.st->it;
  if (hoist && it != itg) gv_tile_words<MAXD>(a, it, blockIdx.x, s_words, B);  // (not expected)
  __syncthreads();
  gv_fill_tile<IG, Real, EPT, MAXD, HIST, PLUS>(a, blockIdx.x, smem, red_u64, red_128, it,
                                                hoist ? s_words : nullptr);
}

// Single-event diagnostics (no shared memory): weight and bins of the given
// events at iteration `it`, with the same map and integrand code as the fill.
template <int IG, typename Real>
__global__ void gv_eval_events_kernel(const GvFillArgs a, uint32_t it, const long long* events,
                                      long long n, double* w, int* bins) {
  constexpr int MAXD = GV_MAXD;
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int d = a.ndim, N = a.nbins;
  const GvGridLayout L{d, N};
  const double* e64 = a.grid + L.off_e64();
  const double* wd64 = a.grid + L.off_wd64();
  const double* jac = a.grid + L.off_jac();
  const float* g32 = reinterpret_cast<const float*>(a.grid + L.off_f32_base());
  const float* e32 = g32 + L.w_e32();
  const float* wd32 = g32 + L.w_wd32();
  const float* jm32 = g32 + L.w_jm32();
  const int* je = reinterpret_cast<const int*>(g32 + L.w_je());
  GvConst<Real, GvTraits<IG>::NK> K;
  K.load(a.kconst);
  uint32_t r[MAXD];
  gv_event_words<MAXD>(a.seed, it, a.batch, (unsigned long long)events[j], d, r);
  Real x[MAXD];
  GvJac<Real> J;
#pragma unroll
  for (int ax = 0; ax < MAXD; ++ax) {
    if (ax < d) {
      const unsigned long long v = (unsigned long long)r[ax] * (unsigned)N;
      const int i = (int)(v >> 32);
      const uint32_t lo = (uint32_t)v;
      const int k = ax * N + i;
      if constexpr (sizeof(Real) == 4) {
        const float f = fmaf(__uint2float_rn(lo), 0x1p-32f, 0x1p-33f);
        x[ax] = fmaf(f, wd32[k], e32[ax * (N + 1) + i]);
        J.m = (ax == 0) ? jm32[k] : __fmul_rn(J.m, jm32[k]);
        J.e = (ax == 0) ? je[k] : J.e + je[k];
      } else {
        const double f = ((double)lo + 0.5) * 0x1p-32;
        x[ax] = __dadd_rn(e64[ax * (N + 1) + i], __dmul_rn(f, wd64[k]));
        J.v = (ax == 0) ? jac[k] : __dmul_rn(J.v, jac[k]);
      }
      bins[j * d + ax] = i;
    }
  }
  const Real g = gv_eval<IG, Real, MAXD>(x, d, K);
  w[j] = gv_weight(J, g);
}
