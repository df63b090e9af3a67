// gv_fill.cuh -- the fused per-event kernel of one VEGAS iteration.
//
// One CTA evaluates one tile of GV_TILE consecutive events (Section 2.1: each
// event generated and evaluated independently), with EPT events per thread:
//   pass 1: Philox words -> bins and in-bin positions -> x on the adaptive grid
//           (edges and Jacobian factors staged in shared memory) -> g(x)
//           -> w = J g (J in FP64 always); the bins go to shared memory;
//   tile scale: block max of |w| (order-free) -> E_t;
//   pass 2: w and w^2 rounded once to fixed point at the tile scale; sums in
//           128-bit integer registers (warp-shuffle + block reduction) and
//           per-bin sums of w^2 as 64-bit integer shared-memory atomics.
// Integer sums are order-free, so the tile's result is the same for every
// block size / events-per-thread choice.
#pragma once
#include "gv_integrands.cuh"

template <int IG>
struct GvTraits;
template <>
struct GvTraits<GV_GAUSS> {
  static constexpr int NK = 1;
};
template <>
struct GvTraits<GV_DY> {
  static constexpr int NK = 22;
};
template <>
struct GvTraits<GV_EE3J> {
  static constexpr int NK = 3;
};

template <int IG, typename Real, int MAXD>
__device__ __forceinline__ Real gv_eval(const Real (&x)[MAXD], int d,
                                        const GvConst<Real, GvTraits<IG>::NK>& K) {
  if constexpr (IG == GV_GAUSS) {
    return gv_gauss<Real, MAXD>(x, d, K[GK_INV2S2]);
  } else if constexpr (IG == GV_DY) {
    return gv_drell_yan<Real, false>(x, K, nullptr);
  } else {
    return gv_ee3j<Real>(x, K);
  }
}

// Shared-memory layout of the fill kernel (bytes), 16-byte aligned pieces:
//   hist   [d*N][2] u64     per-bin (low 53 bits, high bits) sums
//   jac    [d*N]    f64     Jacobian factor N*(e_{i+1}-e_i)
//   edges  [d*(N+1)] Real
//   width  [d*N]    Real
//   bins   [d][GV_TILE] u16
__host__ __device__ inline size_t gv_align16(size_t b) { return (b + 15) & ~(size_t)15; }

struct GvFillSmem {
  size_t hist, jac, edges, width, bins, total;
  __host__ __device__ GvFillSmem(int d, int N, int real_bytes, bool with_bins) {
    const size_t dN = (size_t)d * N;
    hist = 0;
    jac = gv_align16(hist + (with_bins ? dN * 16 : 0));
    edges = gv_align16(jac + dN * 8);
    width = gv_align16(edges + (size_t)d * (N + 1) * real_bytes);
    bins = gv_align16(width + dN * real_bytes);
    total = gv_align16(bins + (with_bins ? (size_t)d * GV_TILE * 2 : 0));
  }
};

// Stage the grid of one integration into shared memory.
template <typename Real>
__device__ __forceinline__ void gv_stage_grid(const double* grid, int d, int N, double* s_jac,
                                              Real* s_e, Real* s_w, int tid, int nthr) {
  const GvGridLayout L{d, N};
  const int dN = d * N;
  const float* g32 = reinterpret_cast<const float*>(grid + L.off_f32_base());
  for (int k = tid; k < dN; k += nthr) {
    s_jac[k] = grid[L.off_jac() + k];
    if constexpr (sizeof(Real) == 4)
      s_w[k] = g32[(size_t)d * (N + 1) + k];
    else
      s_w[k] = grid[L.off_wd64() + k];
  }
  for (int k = tid; k < d * (N + 1); k += nthr) {
    if constexpr (sizeof(Real) == 4)
      s_e[k] = g32[k];
    else
      s_e[k] = grid[L.off_e64() + k];
  }
}

// Map one event's words through the grid: x, bins (to shared memory) and the
// FP64 Jacobian.  FP64: x = e_i + f*(e_{i+1}-e_i) with f = (lo + 1/2) 2^-32,
// rounded as written; FP32: the same with FP32 edges and one fma.
template <typename Real, int MAXD>
__device__ __forceinline__ double gv_map_event(const uint32_t (&r)[MAXD], int d, int N,
                                               const double* s_jac, const Real* s_e,
                                               const Real* s_w, Real (&x)[MAXD],
                                               unsigned short* s_bin, int local) {
  double J = 1.0;
#pragma unroll
  for (int a = 0; a < MAXD; ++a) {
    if (a < d) {
      const unsigned long long v = (unsigned long long)r[a] * (unsigned)N;
      const int i = (int)(v >> 32);
      const uint32_t lo = (uint32_t)v;
      if constexpr (sizeof(Real) == 4) {
        const float f = fmaf(__uint2float_rn(lo), 0x1p-32f, 0x1p-33f);
        x[a] = fmaf(f, s_w[a * N + i], s_e[a * (N + 1) + i]);
      } else {
        const double f = ((double)lo + 0.5) * 0x1p-32;
        x[a] = __dadd_rn(s_e[a * (N + 1) + i], __dmul_rn(f, s_w[a * N + i]));
      }
      J = __dmul_rn(J, s_jac[a * N + i]);
      if (s_bin) s_bin[a * GV_TILE + local] = (unsigned short)i;
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

// ---------------------------------------------------------------------------
// Forward fill: channel 0 = w, with per-bin sums of w^2.
// ---------------------------------------------------------------------------
template <int IG, typename Real, int EPT, int MAXD>
__global__ void __launch_bounds__(GV_TILE / EPT)
    gv_fill_kernel(const GvFillArgs a) {
  constexpr int B = GV_TILE / EPT;
  constexpr int NW = B / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long red_u64[NW];
  __shared__ u128 red_128[NW];
  const int d = a.ndim, N = a.nbins, dN = d * N;
  const GvFillSmem lay(d, N, (int)sizeof(Real), true);
  unsigned long long* hist = reinterpret_cast<unsigned long long*>(smem + lay.hist);
  double* s_jac = reinterpret_cast<double*>(smem + lay.jac);
  Real* s_e = reinterpret_cast<Real*>(smem + lay.edges);
  Real* s_w = reinterpret_cast<Real*>(smem + lay.width);
  unsigned short* s_bin = reinterpret_cast<unsigned short*>(smem + lay.bins);
  const int tid = threadIdx.x;

  for (int k = tid; k < 2 * dN; k += B) hist[k] = 0ull;
  gv_stage_grid<Real>(a.grid, d, N, s_jac, s_e, s_w, tid, B);
  GvConst<Real, GvTraits<IG>::NK> K;
  K.load(a.kconst);
  const uint32_t it = (uint32_t)a.st->it;
  __syncthreads();

  const long long tile = blockIdx.x;
  const long long tile0 = tile * GV_TILE;
  double w[EPT];
  unsigned long long mx = 0ull;
  unsigned long long nbad = 0ull;
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int local = k * B + tid;
    const long long ev = tile0 + local;
    w[k] = 0.0;
    if (ev < a.ncall) {
      uint32_t r[MAXD];
      gv_event_words<MAXD>(a.seed, it, a.batch, (unsigned long long)ev, d, r);
      Real x[MAXD];
      const double J = gv_map_event<Real, MAXD>(r, d, N, s_jac, s_e, s_w, x, s_bin, local);
      const Real g = gv_eval<IG, Real, MAXD>(x, d, K);
      double wv = __dmul_rn(J, (double)g);
      if (!isfinite(wv)) {
        ++nbad;
        wv = 0.0;
      }
      w[k] = wv;
      const unsigned long long bits = (unsigned long long)__double_as_longlong(fabs(wv));
      mx = bits > mx ? bits : mx;
    }
  }
  const unsigned long long M = gv_block_max<NW>(mx, red_u64);
  const int E = gv_scale_exp(M);

  u128 s1 = {0ull, 0ull}, s2 = {0ull, 0ull};
  if (E != GV_EMPTY) {
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      if (w[k] != 0.0) {
        const int local = k * B + tid;
        const u128 v1 = gv_to_fixed(w[k], E);
        const u128 v2 = gv_to_fixed(__dmul_rn(w[k], w[k]), 2 * E);
        s1 = add128(s1, v1);
        s2 = add128(s2, v2);
        const unsigned long long lo53 = v2.lo & 0x1FFFFFFFFFFFFFull;
        const unsigned long long hi = (v2.lo >> 53) | (v2.hi << 11);
#pragma unroll
        for (int ax = 0; ax < MAXD; ++ax) {
          if (ax < d) {
            const int i = s_bin[ax * GV_TILE + local];
            unsigned long long* h = hist + 2 * (ax * N + i);
            atomicAdd(h, lo53);
            if (hi) atomicAdd(h + 1, hi);
          }
        }
      }
    }
  }
  const u128 t1 = gv_block_sum128<NW>(s1, red_128);
  const u128 t2 = gv_block_sum128<NW>(s2, red_128);
  ulonglong2* out = a.part + (size_t)tile * a.nacc;
  if (tid == 0) {
    out[0] = make_ulonglong2(t1.lo, t1.hi);
    out[1] = make_ulonglong2(t2.lo, t2.hi);
    a.tileE[tile] = E;
    if (E != GV_EMPTY) atomicMax(&a.st->E[0], E);
  }
  if (nbad) atomicAdd(&a.st->nonfinite, nbad);
  for (int k = tid; k < dN; k += B) {
    const unsigned long long lo = hist[2 * k], hi = hist[2 * k + 1];
    u128 v;
    v.lo = lo + (hi << 53);
    v.hi = (hi >> 11) + (v.lo < lo ? 1ull : 0ull);
    out[2 + k] = make_ulonglong2(v.lo, v.hi);
  }
}

// ---------------------------------------------------------------------------
// Adjoint fill (Drell-Yan): channels w, dw/dM_Z, dw/dGamma_Z, dw/dsw2, dw/da,
// dw/db; no bin sums.  Each channel has its own tile scale.
// ---------------------------------------------------------------------------
template <typename Real, int EPT, int MAXD>
__global__ void __launch_bounds__(GV_TILE / EPT)
    gv_fill_adjoint_kernel(const GvFillArgs a) {
  constexpr int B = GV_TILE / EPT;
  constexpr int NW = B / 32;
  constexpr int NCH = GV_MAXCH;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long red_u64[NW];
  __shared__ u128 red_128[NW];
  const int d = a.ndim, N = a.nbins;
  const GvFillSmem lay(d, N, (int)sizeof(Real), false);
  double* s_jac = reinterpret_cast<double*>(smem + lay.jac);
  Real* s_e = reinterpret_cast<Real*>(smem + lay.edges);
  Real* s_w = reinterpret_cast<Real*>(smem + lay.width);
  const int tid = threadIdx.x;
  gv_stage_grid<Real>(a.grid, d, N, s_jac, s_e, s_w, tid, B);
  GvConst<Real, 22> K;
  K.load(a.kconst);
  const uint32_t it = (uint32_t)a.st->it;
  __syncthreads();

  const long long tile = blockIdx.x;
  const long long tile0 = tile * GV_TILE;
  double v[EPT][NCH];
  unsigned long long mx[NCH];
#pragma unroll
  for (int c = 0; c < NCH; ++c) mx[c] = 0ull;
  unsigned long long nbad = 0ull;
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int local = k * B + tid;
    const long long ev = tile0 + local;
#pragma unroll
    for (int c = 0; c < NCH; ++c) v[k][c] = 0.0;
    if (ev < a.ncall) {
      uint32_t r[MAXD];
      gv_event_words<MAXD>(a.seed, it, a.batch, (unsigned long long)ev, d, r);
      Real x[MAXD];
      const double J = gv_map_event<Real, MAXD>(r, d, N, s_jac, s_e, s_w, x, nullptr, local);
      Real gr[GV_NGRAD];
      const Real g = gv_drell_yan<Real, true>(x, K, gr);
      double vals[NCH];
      vals[0] = __dmul_rn(J, (double)g);
#pragma unroll
      for (int p = 0; p < GV_NGRAD; ++p) vals[1 + p] = __dmul_rn(J, (double)gr[p]);
      bool finite = true;
#pragma unroll
      for (int c = 0; c < NCH; ++c) finite &= (bool)isfinite(vals[c]);
      if (!finite) ++nbad;
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        v[k][c] = finite ? vals[c] : 0.0;
        const unsigned long long bits =
            (unsigned long long)__double_as_longlong(fabs(v[k][c]));
        mx[c] = bits > mx[c] ? bits : mx[c];
      }
    }
  }
  ulonglong2* out = a.part + (size_t)tile * a.nacc;
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    const unsigned long long M = gv_block_max<NW>(mx[c], red_u64);
    const int E = gv_scale_exp(M);
    u128 s1 = {0ull, 0ull}, s2 = {0ull, 0ull};
    if (E != GV_EMPTY) {
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        if (v[k][c] != 0.0) {
          s1 = add128(s1, gv_to_fixed(v[k][c], E));
          s2 = add128(s2, gv_to_fixed(__dmul_rn(v[k][c], v[k][c]), 2 * E));
        }
      }
    }
    const u128 t1 = gv_block_sum128<NW>(s1, red_128);
    const u128 t2 = gv_block_sum128<NW>(s2, red_128);
    if (tid == 0) {
      out[2 * c] = make_ulonglong2(t1.lo, t1.hi);
      out[2 * c + 1] = make_ulonglong2(t2.lo, t2.hi);
      a.tileE[tile * NCH + c] = E;
      if (E != GV_EMPTY) atomicMax(&a.st->E[c], E);
    }
  }
  if (nbad) atomicAdd(&a.st->nonfinite, nbad);
}

// Single-event diagnostics (no shared memory): weight and bins of the given
// events at iteration `it`.
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
  const float* e32 = g32;
  const float* wd32 = g32 + (size_t)d * (N + 1);
  GvConst<Real, GvTraits<IG>::NK> K;
  K.load(a.kconst);
  uint32_t r[MAXD];
  gv_event_words<MAXD>(a.seed, it, a.batch, (unsigned long long)events[j], d, r);
  Real x[MAXD];
  double J = 1.0;
#pragma unroll
  for (int ax = 0; ax < MAXD; ++ax) {
    if (ax < d) {
      const unsigned long long v = (unsigned long long)r[ax] * (unsigned)N;
      const int i = (int)(v >> 32);
      const uint32_t lo = (uint32_t)v;
      if constexpr (sizeof(Real) == 4) {
        const float f = fmaf(__uint2float_rn(lo), 0x1p-32f, 0x1p-33f);
        x[ax] = fmaf(f, wd32[ax * N + i], e32[ax * (N + 1) + i]);
      } else {
        const double f = ((double)lo + 0.5) * 0x1p-32;
        x[ax] = __dadd_rn(e64[ax * (N + 1) + i], __dmul_rn(f, wd64[ax * N + i]));
      }
      J = __dmul_rn(J, jac[ax * N + i]);
      bins[j * d + ax] = i;
    }
  }
  const Real g = gv_eval<IG, Real, MAXD>(x, d, K);
  double wv = __dmul_rn(J, (double)g);
  w[j] = wv;
}
