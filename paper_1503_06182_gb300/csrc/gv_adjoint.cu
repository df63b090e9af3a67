// Adjoint fill kernels (Drell-Yan gradient).
//
// Six channels per event: the weight w and dw/d(M_Z, Gamma_Z, sw2, a, b) from
// the reverse sweep of the integrand.  No bin sums: the grid is frozen during
// a gradient stage.  Each channel gets its own tile scale E_c (the exponent of
// the tile's largest |value| in that channel) and contributes two exact 128-bit
// fixed-point sums (values and squares) to the tile's partial, as the forward
// fill does for its one channel.
//
// The six values of each event are staged in shared memory (FP32 form: the
// FP32 products J.m g and the exponent J.e, 28 KB a tile; FP64 form: the
// weights, 48 KB), not held in registers across the tile's maximum, so that
// two 512-thread or three 256-thread CTAs share an SM.  In the FP32 form a
// weight is a 24-bit significand times a power of two, and its fixed-point
// terms are formed from that significand (gv_direct*: one 32 x 32 -> 64 bit
// square), the same exactly rounded integers as through the double, with
// less integer work.  All six channels share the block-wide
// steps: one barrier after the per-warp maxima, one after the tile scales,
// one after the per-warp sums.  Each warp's twelve 128-bit sums leave the warp
// by a reduce-scatter (every shuffle step halves the values a lane carries),
// so a warp shuffles 13 128-bit values instead of 12 x 5.
#include "gv_fill_inst.cuh"

namespace {

constexpr int kNch = GV_MAXCH;     // channels
constexpr int kNsum = 2 * kNch;    // per channel: sum v, sum v^2
static_assert(kNsum == 12, "the reduce-scatter below is laid out for 12 sums");

// One reduce-scatter step over lane distance `mask`: the lane with that bit
// set keeps the upper half of x, its partner the lower half, and each adds
// the partner's copy of the half it keeps.
template <int N>
__device__ __forceinline__ void rs_step(const u128 (&x)[2 * N], u128 (&y)[N], int mask,
                                        bool up) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const u128 send = up ? x[i] : x[i + N];
    const u128 keep = up ? x[i + N] : x[i];
    const u128 recv = {shfl_xor_u64(send.lo, mask), shfl_xor_u64(send.hi, mask)};
    y[i] = add128(keep, recv);
  }
}

// Bytes of the per-event values staged in shared memory after the grid, for
// the tile's GV_TILE events: FP64 form, the six weights; FP32 form, the six
// FP32 products J.m g and the event's Jacobian exponent J.e.
template <typename Real>
constexpr size_t stage_bytes() {
  return sizeof(Real) == 8 ? (size_t)GV_TILE * kNch * 8 : (size_t)GV_TILE * (kNch + 1) * 4;
}

// A weight's two fixed-point terms through the general FP64 route.
__device__ __forceinline__ void adj_add_double(double x, int E, u128& s1, u128& s2) {
  if (gv_abs_bits(x) == 0ull) return;
  const GvDecoded dv = gv_decode(x);
  s1 = add128(s1, gv_fixed_tile(dv, E));
  s2 = add128(s2, gv_square_tile(dv, gv_square_hi(dv.m), E));
}

// Register budget of the FP32 kernels: 64 registers at 1024 or 512 threads
// (one or two CTAs per SM), 80 at 256 (three CTAs; the staging buffer allows
// no fourth).  The FP64 kernels would spill under it and keep their own.
template <typename Real, int EPT>
struct AdjBlocks {
  static constexpr int value = sizeof(Real) == 4 ? (EPT == 4 ? 3 : (EPT == 2 ? 2 : 1)) : 1;
};

}  // namespace

template <typename Real, int EPT, int MAXD>
__global__ void __launch_bounds__(GV_TILE / EPT, AdjBlocks<Real, EPT>::value)
    gv_fill_adjoint_kernel(const GvFillArgs a) {
  constexpr int B = GV_TILE / EPT;
  constexpr int NW = B / 32;
  constexpr bool F32 = sizeof(Real) == 4;
  using Pair = typename GvPair<Real>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int red_max[NW][kNch];
  __shared__ u128 red_sum[NW][kNsum];
  __shared__ int s_E[kNch];
  const int d = a.ndim, N = a.nbins;
  const GvFillSmem lay(d, N, (int)sizeof(Real), false, false);
  double* s_jac = reinterpret_cast<double*>(smem + lay.jac);
  Pair* s_ew = reinterpret_cast<Pair*>(smem + lay.ew);
  // channel c of the thread's k-th event at [(k kNch + c) B + tid]: FP64
  // form, the weight; FP32 form, the bits of J.m g, and J.e at s_je[k B + tid]
  double* s_v = reinterpret_cast<double*>(smem + lay.total);
  unsigned* s_p = reinterpret_cast<unsigned*>(smem + lay.total);
  int* s_je = reinterpret_cast<int*>(smem + lay.total + (size_t)GV_TILE * kNch * 4);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  gv_wait_prior_grid();
  gv_stage_grid<Real>(a.grid, d, N, s_jac, s_ew, tid, B);
  GvConst<Real, DK_NK> K;
  K.load(a.kconst);
  const uint32_t it = (uint32_t)a.st->it;
  __syncthreads();

  const long long tile = blockIdx.x;
  const long long tile0 = tile * GV_TILE;
  // per channel the largest scale gv_scale_exp(|w|) of the thread's weights
  // (the scale of the largest |w|: the scale is monotonic in |w|)
  int mE[kNch];
#pragma unroll
  for (int c = 0; c < kNch; ++c) mE[c] = GV_EMPTY;
  unsigned long long nbad = 0ull;
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const long long ev = tile0 + k * B + tid;
    int Ev[kNch];
#pragma unroll
    for (int c = 0; c < kNch; ++c) Ev[c] = GV_EMPTY;
    [[maybe_unused]] unsigned pu[kNch];
    [[maybe_unused]] double vals[kNch];
    [[maybe_unused]] int je = 0;
#pragma unroll
    for (int c = 0; c < kNch; ++c) {
      pu[c] = 0u;
      vals[c] = 0.0;
    }
    if (ev < a.ncall) {
      uint32_t r[MAXD];
      gv_event_words<MAXD>(a.seed, it, a.batch, (unsigned long long)ev, d, r);
      Real x[MAXD];
      int bin[MAXD];
      const GvJac<Real> J = gv_map_event<Real, MAXD>(r, d, N, s_jac, s_ew, x, bin);
      Real gr[GV_NGRAD];
      const Real g = gv_drell_yan<Real, true>(x, K, gr);
      bool finite = true;
      if constexpr (F32) {
        je = J.e;
        pu[0] = __float_as_uint(__fmul_rn(J.m, g));
#pragma unroll
        for (int p = 0; p < GV_NGRAD; ++p) pu[1 + p] = __float_as_uint(__fmul_rn(J.m, gr[p]));
#pragma unroll
        for (int c = 0; c < kNch; ++c) {
          if ((pu[c] & 0x7FFFFFFFu) == 0u) continue;
          const GvDirect w = gv_direct(pu[c], je);
          if (w.direct) {
            Ev[c] = w.e2 + 24;  // the double's exponent field - 1022
          } else {
            const unsigned long long bits = gv_abs_bits(gv_weight_bits(pu[c], je));
            finite &= gv_finite_bits(bits);
            Ev[c] = gv_scale_exp(bits);
          }
        }
      } else {
        vals[0] = gv_weight(J, g);
#pragma unroll
        for (int p = 0; p < GV_NGRAD; ++p) vals[1 + p] = gv_weight(J, gr[p]);
#pragma unroll
        for (int c = 0; c < kNch; ++c) {
          const unsigned long long bits = gv_abs_bits(vals[c]);
          finite &= gv_finite_bits(bits);
          Ev[c] = gv_scale_exp(bits);
        }
      }
      if (!finite) {
        ++nbad;
#pragma unroll
        for (int c = 0; c < kNch; ++c) {
          pu[c] = 0u;
          vals[c] = 0.0;
          Ev[c] = GV_EMPTY;
        }
      }
    }
#pragma unroll
    for (int c = 0; c < kNch; ++c) {
      mE[c] = max(mE[c], Ev[c]);
      if constexpr (F32)
        s_p[(k * kNch + c) * B + tid] = pu[c];
      else
        s_v[(k * kNch + c) * B + tid] = vals[c];
    }
    if constexpr (F32) s_je[k * B + tid] = je;
  }
  gv_allow_next_grid();

  // tile scales: warp maxima, then one thread per channel over the warps
#pragma unroll
  for (int c = 0; c < kNch; ++c) {
    const int m = __reduce_max_sync(0xffffffffu, mE[c]);
    if (lane == 0) red_max[wid][c] = m;
  }
  __syncthreads();
  if (tid < kNch) {
    int E = red_max[0][tid];
#pragma unroll
    for (int w = 1; w < NW; ++w) E = max(E, red_max[w][tid]);
    s_E[tid] = E;
  }
  __syncthreads();

  // This thread's exact sums, two channels at a time: channels c and c + 3
  // hold sums 2c, 2c+1 and 2c+6, 2c+7, which meet in the first step of the
  // warp's reduce-scatter (lane distance 16), so that step runs as soon as
  // the pair is formed.
  [[maybe_unused]] int jek[EPT];
  if constexpr (F32) {
#pragma unroll
    for (int k = 0; k < EPT; ++k) jek[k] = s_je[k * B + tid];
  }
  const bool up16 = (lane & 16) != 0;
  u128 a6[6];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    u128 s[4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int ch = c + 3 * h;
      const int E = s_E[ch];
      u128 s1 = {0ull, 0ull}, s2 = {0ull, 0ull};
      if (E != GV_EMPTY) {
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
          if constexpr (F32) {
            const unsigned u = s_p[(k * kNch + ch) * B + tid];
            if ((u & 0x7FFFFFFFu) != 0u) {
              const GvDirect w = gv_direct(u, jek[k]);
              if (w.direct) {
                s1 = add128(s1, gv_direct_fixed(w.m, w.e2 - E + GV_FB, w.neg));
                s2 = add128(s2, gv_direct_square((unsigned long long)w.m * w.m,
                                                   2 * (w.e2 - E) + GV_FB));
              } else {
                adj_add_double(gv_weight_bits(u, jek[k]), E, s1, s2);
              }
            }
          } else {
            adj_add_double(s_v[(k * kNch + ch) * B + tid], E, s1, s2);
          }
        }
      }
      s[2 * h] = s1;
      s[2 * h + 1] = s2;
    }
    const u128 x2[4] = {s[0], s[1], s[2], s[3]};
    u128 y[2];
    rs_step<2>(x2, y, 16, up16);
    a6[2 * c] = y[0];
    a6[2 * c + 1] = y[1];
  }
  // the remaining steps: lane distances 8, 4, 2, then both lanes of a pair
  u128 a3[3], a2[2], a1[1];
  rs_step<3>(a6, a3, 8, (lane & 8) != 0);
  const u128 a4[4] = {a3[0], a3[1], a3[2], u128{0ull, 0ull}};
  rs_step<2>(a4, a2, 4, (lane & 4) != 0);
  rs_step<1>(a2, a1, 2, (lane & 2) != 0);
  const u128 o = {shfl_xor_u64(a1[0].lo, 1), shfl_xor_u64(a1[0].hi, 1)};
  const u128 t = add128(a1[0], o);
  // sum index of this lane: 6 b4 + 3 b3 + (2 b2 + b1), b_i bit i of the
  // lane; 2 b2 + b1 = 3 is padding; of the two lanes holding an index, the
  // even one publishes it
  const int local = ((lane >> 1) & 2) | ((lane >> 1) & 1);
  const int j = 6 * ((lane >> 4) & 1) + 3 * ((lane >> 3) & 1) + local;
  if (local < 3 && (lane & 1) == 0) red_sum[wid][j] = t;
  __syncthreads();
  if (tid < kNsum) {
    u128 tot = red_sum[0][tid];
#pragma unroll
    for (int w = 1; w < NW; ++w) tot = add128(tot, red_sum[w][tid]);
    ulonglong2* out = a.part + (size_t)tile * a.nacc;
    out[tid] = make_ulonglong2(tot.lo, tot.hi);
    if ((tid & 1) == 0) a.tileE[tile * kNch + tid / 2] = s_E[tid / 2];
  }
  if (nbad) atomicAdd(&a.st->nonfinite_iter, nbad);
}

template <typename Real, int EPT, int MAXD>
static cudaError_t gv_launch_adj_t(const GvFillArgs& a, int n_tiles, size_t smem, cudaStream_t s,
                                   bool pdl) {
  auto k = gv_fill_adjoint_kernel<Real, EPT, MAXD>;
  const size_t total = smem + stage_bytes<Real>();  // the grid, then the staged values
  cudaError_t e = gv_prepare(k, total);
  if (e != cudaSuccess) return e;
  return gv_launch(k, dim3(n_tiles), dim3(GV_TILE / EPT), total, s, pdl, a);
}

template <typename Real, int MAXD>
static cudaError_t gv_launch_adj_ept(int ept, const GvFillArgs& a, int n_tiles, size_t smem,
                                     cudaStream_t s, bool pdl) {
  switch (ept) {
    case 1: return gv_launch_adj_t<Real, 1, MAXD>(a, n_tiles, smem, s, pdl);
    case 2: return gv_launch_adj_t<Real, 2, MAXD>(a, n_tiles, smem, s, pdl);
    case 4: return gv_launch_adj_t<Real, 4, MAXD>(a, n_tiles, smem, s, pdl);
  }
  return cudaErrorInvalidValue;
}

namespace gv {
cudaError_t launch_fill_adjoint(int fp32, int ept, const GvFillArgs& a, int n_tiles, size_t smem,
                                cudaStream_t s, bool pdl) {
  if (a.ndim <= 4)
    return fp32 ? gv_launch_adj_ept<float, 4>(ept, a, n_tiles, smem, s, pdl)
                : gv_launch_adj_ept<double, 4>(ept, a, n_tiles, smem, s, pdl);
  if (a.ndim <= 16)
    return fp32 ? gv_launch_adj_ept<float, 16>(ept, a, n_tiles, smem, s, pdl)
                : gv_launch_adj_ept<double, 16>(ept, a, n_tiles, smem, s, pdl);
  return cudaErrorInvalidValue;
}
}  // namespace gv
