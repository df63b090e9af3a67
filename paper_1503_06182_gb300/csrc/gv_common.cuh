// gv_common.cuh -- internal definitions shared by the GB300 VEGAS kernels.
//
// One VEGAS iteration (Section 2.1: events evaluated independently, all events
// combined, serial grid optimisation) runs as two kernels:
//   fill   : one CTA per tile of GV_TILE consecutive events; uniforms from
//            Philox4x32-10, grid map, integrand, then exact integer
//            accumulation of sum w, sum w^2 and the per-bin sums of w^2
//            into a per-tile partial;
//   reduce : exact integer reduction of the tile partials; the CTA that
//            completes an axis refines that axis' grid, and the last CTA to
//            finish converts the sums to FP64 and records the iteration.
//
// Exact accumulation.  Every tile takes its scale from its largest |v| (an
// order-free max): E_t with max|v| < 2^E_t.  Each v is rounded once to an
// integer multiple of 2^(E_t - GV_FB) (v^2 to 2^(2 E_t - GV_FB)); from then on
// only integer additions happen, which are associative.  The result is
// therefore bit-identical for any block size, events per thread, tile-to-CTA
// schedule and batching -- the paper's "independent of the number of
// threads" (Section 2.2) made exact -- and it is more accurate than the
// Kahan sums the paper uses for the same purpose.
//
// Bin sums carry their own scale.  The grid refinement compresses every
// bin's share rho through ((1-rho)/(-ln rho))^alpha, which stays far from 0
// even for rho = 1e-100, so a bin's sum needs relative, not absolute,
// precision.  Each bin therefore has its own exponent: F_b with w^2 < 2^(2 F_b)
// for every event of the bin (an order-free max, per tile and then over the
// iteration).  A tile rounds each w^2 once to a multiple of 2^(2 F_tb - 56);
// the iteration's sum aligns the tile sums to 2^(2 F_b - 88).  Alignment
// truncates only bits ~2^-86 below the bin's largest w^2, in a fixed way, so
// the bin sums stay launch-shape independent; one w^2 is rounded to 2^-56 of
// its bin's scale, so a bin sum is relatively exact to 2^-45 at worst.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define GV_TILE 1024          // canonical events per tile
#define GV_FB 96              // fixed-point bits below a tile's scale
#define GV_MAXD 16            // maximum number of axes
#define GV_NGRAD 5            // Drell-Yan gradient components
#define GV_MAXCH (1 + GV_NGRAD)
#define GV_EMPTY (-0x40000000)  // scale of a tile / iteration with no nonzero value
#define GV_NCONST 48          // derived integrand constants per integration (doubles)
#define GV_NCONST_F32 32      // constants 0..31 in FP64, then their FP32 copies
#define GV_MAXPARAMS 16
#define GV_BINE_OFF 1100      // stored bin exponent F + GV_BINE_OFF (0: no nonzero weight)
#define GV_BIN_QBITS 56       // bits of one w^2 below its bin's scale in a tile
#define GV_BIN_XBITS 32       // extra low bits of the iteration's bin sums
#define GV_BIN_FB (GV_BIN_QBITS + GV_BIN_XBITS)  // bin sums in units of 2^(2F - GV_BIN_FB)
#define GV_HIST_MAX 1000      // histogram bins of the observable (plus underflow and overflow)

enum { GV_GAUSS = 0, GV_DY = 1, GV_EE3J = 2, GV_DYNLO = 3 };

// Device-side state of one integration (one context or one batch member).
// nonfinite_iter and the tickets return to zero at the end of every iteration.
struct GvState {
  unsigned long long it;              // global iteration counter (Philox counter word)
  unsigned long long nonfinite_iter;  // non-finite weights of the running iteration
  unsigned long long nonfinite;       // non-finite weights of the stage
  int status;                         // device error word (0 = ok)
  // VEGAS+: arrivals at the end of a stage's last iteration of the reduce
  // (I_k) and of the hypercube statistics (sigma_k), which run side by side;
  // the second to arrive combines the stage and resets it
  int join;
  double integral, error, chi2;
  double grad[GV_NGRAD], grad_err[GV_NGRAD];
  // the counter at the start of the running stage: the counter of its
  // iteration k is it0 + k.  Written only by the last iteration of a stage
  // (and with `it` by the host), so the fill of iteration k > 0 may read it
  // while the previous iteration's kernels still run.
  unsigned long long it0;
};

// Grid pack of one integration (device memory, rewritten by every refine):
//   e64[d][N+1] | wd64[d][N] | jac[d][N] | e32[d][N+1] | wd32[d][N] | jm32[d][N] | je[d][N]
// wd = e[i+1]-e[i]; jac = N*wd (the axis' Jacobian factor) = jm32 2^je with
// jm32 in [1,2] (FP32, for the FP32 form: mantissas multiplied in FP32,
// exponents summed as integers, so the product has no FP32 range limit).
struct GvGridLayout {
  int d, N;
  __host__ __device__ size_t off_e64() const { return 0; }
  __host__ __device__ size_t off_wd64() const { return (size_t)d * (N + 1); }
  __host__ __device__ size_t off_jac() const { return off_wd64() + (size_t)d * N; }
  // 32-bit parts, counted in doubles from the start of the pack
  __host__ __device__ size_t off_f32_base() const { return off_jac() + (size_t)d * N; }
  // offsets of the 32-bit tables in 32-bit words from off_f32_base()
  __host__ __device__ size_t w_e32() const { return 0; }
  __host__ __device__ size_t w_wd32() const { return (size_t)d * (N + 1); }
  __host__ __device__ size_t w_jm32() const { return w_wd32() + (size_t)d * N; }
  __host__ __device__ size_t w_je() const { return w_jm32() + (size_t)d * N; }
  __host__ __device__ size_t doubles() const {
    const size_t nw = w_je() + (size_t)d * N;  // 32-bit words
    return off_f32_base() + (nw + 1) / 2;
  }
};

// VEGAS+ data of the stratified fill: s strata per axis, nh = s^d
// hypercubes; event e lies in the h with off[h] <= e < off[h+1]; tile t's
// first hypercube is tile_h0[t]; ab[h] = (C/(nh n_h), sqrt(1/(nh n_h)));
// *ncall events in all.  Each GV_PLUS_SEG-event range r of the fill sums
// J g and (J g)^2 over its run of each hypercube, in event order (its
// segments).  A tile forms the statistics (var, dw) of every hypercube whose
// events it holds all of, and the sums of their v/n and weights (tpart[t]);
// the segments of a hypercube that crosses a tile boundary go to memory for
// the finishing kernel: its first to seg_h[h], and a range's continuation of
// it (only a range's first segment can be one) to seg_r[r].
struct GvPlusFill {
  int s;
  float inv_s;
  long long nh;
  unsigned long long magic;  // floor((2^64 - 1) / s)
  const long long* off;
  const double2* ab;
  const float2* ab32;  // ab rounded to FP32 (the FP32 form)
  const int* tile_h0;
  const long long* ncall;
  double2* seg_h;
  double2* seg_r;
  int* tiles_used;  // written by the fill: the tiles that hold events this iteration
  double* var;      // [nh] sample variance of J g in each hypercube
  double* dw;       // [nh] allocation weights v^(beta/2)
  double2* tpart;   // [tiles] per tile: sums of v/n and of the weights of its hypercubes
  const double* inv;  // [GV_PLUS_NTAB] 1/n (entry 0 unused)
  int beta_j;       // damping beta = beta_j / 4
};

// Arguments of the fill kernels (forward and adjoint).
struct GvFillArgs {
  int ndim, nbins, nch, nacc;
  long long ncall;
  unsigned long long seed;
  unsigned batch;
  const double* kconst;          // derived integrand constants
  const double* grid;            // grid pack
  GvState* st;
  ulonglong2* part;              // 128-bit two's complement sums: slot k of tile t at
                                 // part[t nacc + k] (tile-major) or part[k n_tiles + t]
                                 // (slot_major, read by the single-level reduce)
  int* tileE;                    // [tile][nch] scales
  int slot_major = 0, n_tiles = 0;
  int kst = 0;                   // the iteration's index in its stage (counter it0 + kst)
  int hoist = 0;                 // 1: the forward fill makes its words before it waits
  // histogram of the integrand's observable (forward fill only): nhist bins,
  // 0 = underflow, nhist - 1 = overflow (nhist = 0: no histogram); the bin of
  // a value v >= lo is 1 + trunc((v - lo) invw), in the integrand's precision
  int nhist = 0;
  double h_lo = 0.0, h_invw = 0.0;
  float h_lo_f = 0.0f, h_invw_f = 0.0f;
  // VEGAS+: the stratified fill's data (device memory; nullptr otherwise).
  // Kept behind one pointer: the fields inline cost the plain fill kernels
  // registers.
  const struct GvPlusFill* plus = nullptr;
};

// One slot's sum as a 192-bit two's complement integer with its exponent:
// channel slot 2c (sum v) / 2c+1 (sum v^2): value = v 2^(pw e - GV_FB),
// pw = 1 / 2, e a tile scale (GV_EMPTY: nothing nonzero); bin slot: value =
// v 2^(2 (e - GV_BINE_OFF) - GV_BIN_FB), e a stored bin exponent (0: empty).
struct __align__(16) GvSlot {
  unsigned long long l0, l1, l2;
  int e, pad;
};

// Tickets of the reduce kernel, each on its own 128-byte line: one per slot
// block of 32 slots, one per axis (and one spare line).
#define GV_TICKET_STRIDE 32
__host__ __device__ inline int gv_ticket_group(int x) { return x * GV_TICKET_STRIDE; }
__host__ __device__ inline int gv_ticket_axis(int nacc, int ax) {
  return ((nacc + 31) / 32 + ax) * GV_TICKET_STRIDE;
}
__host__ __device__ inline int gv_ticket_done(int nacc) {
  return ((nacc + 31) / 32 + GV_MAXD) * GV_TICKET_STRIDE;
}
__host__ __device__ inline size_t gv_tickets_ints(int nacc) {
  return (size_t)gv_ticket_done(nacc) + GV_TICKET_STRIDE;
}

// Arguments of the reduce/finalize kernel.
// Slots: [0, 2*nch) channel sums, then (forward) ndim*nbins bin sums.
// Slots: [2 nch channel sums | ndim * nbins bin sums of w^2 | nhist
// histogram sums of w^2 | nhist histogram sums of w (signed)].
struct GvReduceArgs {
  int ndim, nbins, nch, nacc, has_bins, k, last, mode;  // k: iteration in the stage, last: k == itmx-1
  int nhist = 0;                 // histogram bins (0: none)
  int plus = 0;                  // VEGAS+: sigma_k and the stage combination come later
  // results written straight to mapped host memory as well (plain forward
  // stages): the iteration records, and the state after the last iteration
  GvState* host_st = nullptr;
  double* host_rec = nullptr;
  int refine_follows;            // 1: each axis is refined by the CTA that completes it
  long long ncall;
  double inv_c, inv_cm1, inv_m1; // 1/C, 1/(C-1), 1/(k) for chi2/dof at the last iteration
  int n_tiles, tiles_per_cta;
  const ulonglong2* part;
  const int* tileE;
  GvState* st;
  GvSlot* cpart;                 // [tile ranges][32 * slot blocks] one CTA's sums
  double* sums;                  // [nacc] FP64 sums of the last iteration
  double* per_iter;              // forward: [itmx][2]; adjoint: [itmx][2 + 2*NGRAD]
  int* tickets;                  // gv_tickets_ints(nacc) counters, one per 128-byte line
  // grid refinement
  double alpha, inv_nbins;
  double* grid;                  // grid pack (refined in place, one axis per CTA)
  // VEGAS+: the tiles the fill gave events (its grid holds the largest
  // allocation; the rest left nothing); nullptr: all n_tiles
  const int* tiles_used = nullptr;
};

// ----------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplications with a Weyl-bumped key.
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint4 gv_philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t a = c.x, b = c.z;
    const uint32_t h0 = __umulhi(0xD2511F53u, a), l0 = 0xD2511F53u * a;
    const uint32_t h1 = __umulhi(0xCD9E8D57u, b), l1 = 0xCD9E8D57u * b;
    c = make_uint4(h1 ^ c.y ^ k0, l1, h0 ^ c.w ^ k1, l0);
  }
  return c;
}

// Words of one event: Philox block j has counter (ev lo, ev hi, it, batch<<8|j)
// and key (seed lo, seed hi); its word k drives axis 4j+k.
template <int MAXD>
__device__ __forceinline__ void gv_event_words(unsigned long long seed, uint32_t it,
                                               uint32_t batch, unsigned long long ev,
                                               int d, uint32_t (&r)[MAXD]) {
#pragma unroll
  for (int j = 0; j < (MAXD + 3) / 4; ++j) {
    if (4 * j < d) {
      uint4 o = gv_philox(make_uint4((uint32_t)ev, (uint32_t)(ev >> 32), it, (batch << 8) | j),
                          (uint32_t)seed, (uint32_t)(seed >> 32));
      if (4 * j + 0 < MAXD) r[4 * j + 0] = o.x;
      if (4 * j + 1 < MAXD) r[4 * j + 1] = o.y;
      if (4 * j + 2 < MAXD) r[4 * j + 2] = o.z;
      if (4 * j + 3 < MAXD) r[4 * j + 3] = o.w;
    }
  }
}

// ----------------------------------------------------------------------------
// Programmatic dependent launch: the kernels of an iteration (fill -> reduce
// -> refine -> next fill) are launched with programmatic stream serialisation,
// so each one is scheduled while its predecessor finishes.  A kernel must wait
// before it reads anything its predecessor (or earlier work) wrote; it lets its
// successor launch once the rest of its own work is short.  Both are no-ops
// for a plain launch.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void gv_wait_prior_grid() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void gv_allow_next_grid() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t gv_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                             cudaStream_t s, bool pdl, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? attr : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// The same with a scheduling priority (cudaDeviceGetStreamPriorityRange's
// scale: lower is more urgent): among launches whose CTAs wait for room on
// the SMs, the more urgent are placed first (a graph keeps it per node when
// instantiated with cudaGraphInstantiateFlagUseNodePriority).
template <typename... KArgs, typename... Args>
inline cudaError_t gv_launch_prio(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                  cudaStream_t s, bool pdl, int prio, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = prio;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ----------------------------------------------------------------------------
// Exact fixed-point helpers.
// ----------------------------------------------------------------------------
struct u128 {
  unsigned long long lo, hi;
};

__device__ __forceinline__ u128 add128(u128 a, u128 b) {
  u128 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
  return r;
}

// Scale exponent of a nonnegative finite double bit pattern: the E with
// value < 2^E <= 2*value (GV_EMPTY for zero).
__device__ __forceinline__ int gv_scale_exp(unsigned long long bits) {
  if (bits == 0) return GV_EMPTY;
  const int ef = (int)(bits >> 52);
  if (ef != 0) return ef - 1022;
  return (64 - __clzll(bits)) - 1074;
}

// A finite double as sign, integer mantissa m and exponent e2 (|x| = m 2^e2).
struct GvDecoded {
  unsigned long long m;
  int e2;
  bool neg;
};

__device__ __forceinline__ GvDecoded gv_decode(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  GvDecoded r;
  r.neg = (b >> 63) != 0;
  const int ef = (int)((b >> 52) & 0x7ff);
  r.m = b & 0xFFFFFFFFFFFFFull;
  if (ef == 0) {
    r.e2 = -1074;
  } else {
    r.m |= 1ull << 52;
    r.e2 = ef - 1075;
  }
  return r;
}

// round(m * 2^s) for a 128-bit m = (hi, lo), s of either sign (round half up).
__device__ __forceinline__ u128 gv_shift_round(u128 v, int s) {
  if (s > 0) {
    if (s >= 64) {
      v.hi = v.lo << (s - 64);
      v.lo = 0ull;
    } else {
      v.hi = (v.hi << s) | (v.lo >> (64 - s));
      v.lo <<= s;
    }
    return v;
  }
  if (s == 0) return v;
  const int rs = -s;
  if (rs > 127) return {0ull, 0ull};
  // add half a unit of the last kept bit, then shift right
  u128 h;
  if (rs - 1 >= 64) {
    h.lo = 0ull;
    h.hi = 1ull << (rs - 1 - 64);
  } else {
    h.lo = 1ull << (rs - 1);
    h.hi = 0ull;
  }
  v = add128(v, h);
  if (rs >= 64) {
    v.lo = v.hi >> (rs - 64);
    v.hi = 0ull;
  } else {
    v.lo = (v.lo >> rs) | (v.hi << (64 - rs));
    v.hi >>= rs;
  }
  return v;
}

__device__ __forceinline__ u128 gv_negate_if(u128 v, bool neg) {
  if (neg) {
    v.lo = ~v.lo + 1ull;
    v.hi = ~v.hi + (v.lo == 0 ? 1ull : 0ull);
  }
  return v;
}

// round(x 2^(GV_FB - E)) from a decoded x with |x| < 2^E, two's complement.
__device__ __forceinline__ u128 gv_fixed_dec(const GvDecoded& d, int E) {
  u128 v = {d.m, 0ull};
  v = gv_shift_round(v, d.e2 - E + GV_FB);
  return gv_negate_if(v, d.neg);
}

// round(x^2 2^(GV_FB - 2E)), with the square formed exactly in integers
// (m^2 has at most 106 bits): the sum of squares is then exact too.
__device__ __forceinline__ u128 gv_square_fixed_dec(const GvDecoded& d, int E) {
  u128 v = {d.m * d.m, __umul64hi(d.m, d.m)};
  return gv_shift_round(v, 2 * d.e2 - 2 * E + GV_FB);
}

// x^2 2^(GV_BIN_QBITS - 2F) for |x| = m 2^e2 < 2^F, from the high word
// P = floor(m^2 2^-42) of the square of m 2^11 (the 64 bits below the leading
// ones of m^2, so the truncation is below 2^-62 relative): rounded half up,
// with rs = 2F - 2 e2 - 98 >= 8, below 2^GV_BIN_QBITS.  Each value is formed
// on its own, so the tile's sum does not depend on the event order.
__device__ __forceinline__ unsigned long long gv_square_hi(unsigned long long m) {
  return __umul64hi(m << 11, m << 11);
}
__device__ __forceinline__ unsigned long long gv_square_bin(unsigned long long P, int rs) {
  return rs <= 64 ? ((P >> (rs - 1)) + 1ull) >> 1 : 0ull;
}

// The same roundings as gv_fixed_dec / gv_square_fixed_dec (half up, bit for
// bit), specialised to the shifts that occur in a tile for normal x (|x| <
// 2^E, so the mantissa shift of x is at most GV_FB - 53 and that of x^2 at
// least 106 - GV_FB; subnormal x take the general routine), on 64-bit
// pieces.  round(v 2^-r) = ((v >> (r-1)) + 1) >> 1.
__device__ __forceinline__ u128 gv_fixed_tile(const GvDecoded& d, int E) {
  const int s = d.e2 - E + GV_FB;  // <= GV_FB - 53 unless x is subnormal
  if (s > GV_FB - 53) return gv_fixed_dec(d, E);
  u128 v;
  if (s > 0) {
    v.lo = d.m << s;
    v.hi = d.m >> (64 - s);
  } else if (s == 0) {
    v.lo = d.m;
    v.hi = 0ull;
  } else {
    const int r = -s;
    v.lo = r <= 54 ? ((d.m >> (r - 1)) + 1ull) >> 1 : 0ull;
    v.hi = 0ull;
  }
  return gv_negate_if(v, d.neg);
}
// x^2 from its exact 128-bit mantissa square (hi = floor(m^2 2^-64) taken
// from P = floor(m^2 2^-42), see gv_square_hi; lo = m^2 mod 2^64).
__device__ __forceinline__ u128 gv_square_tile(const GvDecoded& d, unsigned long long P, int E) {
  const int k = 2 * E - 2 * d.e2 - GV_FB - 1;  // r - 1 >= 105 - GV_FB unless x is subnormal
  if (k < 105 - GV_FB) return gv_square_fixed_dec(d, E);
  const unsigned long long hi = P >> 22, lo = d.m * d.m;
  u128 t;
  if (k < 64) {
    t.lo = (lo >> k) | (hi << (64 - k));
    t.hi = hi >> k;
  } else {
    t.lo = k < 128 ? hi >> (k - 64) : 0ull;
    t.hi = 0ull;
  }
  // (t + 1) >> 1
  t.lo += 1ull;
  t.hi += t.lo == 0ull ? 1ull : 0ull;
  t.lo = (t.lo >> 1) | (t.hi << 63);
  t.hi >>= 1;
  return t;
}

__device__ __forceinline__ unsigned long long shfl_xor_u64(unsigned long long v, int m) {
  return __shfl_xor_sync(0xffffffffu, v, m);
}

__device__ __forceinline__ u128 warp_sum128(u128 v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    u128 o = {shfl_xor_u64(v.lo, m), shfl_xor_u64(v.hi, m)};
    v = add128(v, o);
  }
  return v;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    unsigned long long o = shfl_xor_u64(v, m);
    v = o > v ? o : v;
  }
  return v;
}

// ----------------------------------------------------------------------------
// Host-side launchers (defined in the kernel translation units).
// ----------------------------------------------------------------------------
// Histogram of the observable after an iteration's reduce: the iteration's
// bin estimates from the once-rounded sums, accumulated over the call's
// iterations; the combined histogram at the last one.
struct GvHistArgs {
  const double* sums;      // [2][nhist]: sum w^2, then sum w, per bin
  const double* per_iter;  // [itmx][2] (I_k, sigma_k)
  int nhist, k, last;
  double inv_c, inv_cm1;
  double* acc;             // [4][nhist] running sums of the call (see gv_hist_kernel)
  double* out;             // [2][nhist] value, error (written at the last iteration)
};

#define GV_PLUS_NTAB 4096  // per-count tables of the VEGAS+ kernels (larger counts: computed)
#define GV_PLUS_SEG 4      // consecutive events per thread of the stratified fill (one range)

// VEGAS+ after an iteration (see gv_plus.cu): per-hypercube statistics, the
// next allocation, its layout.
struct GvPlusArgs {
  long long nh = 0;          // hypercubes
  long long ncall = 0;       // the target C of the allocation
  int beta_j = 3;            // damping beta = beta_j / 4
  int uniform = 0;           // allocation: floor(C / nh) everywhere
  int n_tiles = 0;           // tiles of the fill grid
  int k = 0, last = 0;       // iteration in the stage
  double inv_m1 = 0.0;       // 1 / (k) for chi2/dof at the last iteration
  double inv_nh2 = 0.0;      // 1 / nh^2
  // the fill's segment sums (sum F, sum F^2): each hypercube's first, and
  // per GV_PLUS_SEG-event range the one that continues an earlier hypercube
  const double2* seg_h = nullptr;  // [nh]
  const double2* seg_r = nullptr;  // [ranges]
  long long cap = 0;         // events the buffers hold
  long long* off = nullptr;  // [nh + 1] first event of each hypercube, then the count
  int* n = nullptr;          // [nh] events per hypercube
  double2* ab = nullptr;     // [nh] (C/(nh n_h), sqrt(1/(nh n_h)))
  float2* ab32 = nullptr;    // [nh] the same rounded to FP32
  int* tile_h0 = nullptr;    // [n_tiles] hypercube of each tile's first event
  double* var = nullptr;     // [nh] sample variance of J g in each hypercube
  double* dw = nullptr;      // [nh] allocation weights v^(beta/2)
  double2* tpart = nullptr;  // [n_tiles] the fill's per-tile sums of v/n and of the weights
  double2* fpart = nullptr;  // [16] the finishing kernel's per-CTA sums
  int* fctr = nullptr;       // its arrival counter (zero between uses)
  // per CTA of kT = 256 hypercubes, per group of 32 CTAs
  long long* npart = nullptr;  // [CTAs] the CTA's events of the next allocation
  long long* gsum = nullptr;   // [groups] the group's events
  int* gctr = nullptr;         // [groups] arrival counters (zero between uses)
  long long* ncall_dev = nullptr;  // events of the allocation
  double* scal = nullptr;    // [3] sigma_k^2, the weights' sum D, 1/D
  int* tiles_used = nullptr; // the fill's tiles with events (the reduce reads no others)
  const double* inv = nullptr;    // [GV_PLUS_NTAB] 1/n (entry 0 unused)
  const double2* abtab = nullptr; // [GV_PLUS_NTAB] ab for n_h = n (C and nh of the allocation)
  int prio = 0;              // launch priority (the most urgent of the device)
  double* per_iter = nullptr;  // [itmx][2]
  GvState* st = nullptr;
};

namespace gv {
cudaError_t launch_plus_finish(const GvPlusArgs& a, cudaStream_t s, bool pdl);
cudaError_t launch_plus_alloc(const GvPlusArgs& a, cudaStream_t s, bool pdl);
cudaError_t launch_plus_layout(const GvPlusArgs& a, cudaStream_t s, bool pdl);
cudaError_t launch_fill_plus(int ig, int fp32, const GvFillArgs& a, int n_tiles, size_t smem,
                             cudaStream_t s, bool pdl);
cudaError_t launch_fill_adjoint(int fp32, int ept, const GvFillArgs& a, int n_tiles,
                                size_t smem, cudaStream_t s, bool pdl);
void reduce_grid(int n_tiles, int nacc, int* tiles_per_cta, int* gx, int* gy);
size_t reduce_smem_bytes(int N);  // dynamic shared memory of the reduce kernels
cudaError_t launch_reduce(const GvReduceArgs& a, size_t smem, cudaStream_t s, bool pdl);
// the single-level reduce of slot-major partials (plain forward stages)
cudaError_t launch_reduce_slots(const GvReduceArgs& a, size_t smem, cudaStream_t s, bool pdl);
cudaError_t launch_hist(const GvHistArgs& a, cudaStream_t s, bool pdl);
cudaError_t launch_fill_hist(int ig, int fp32, const GvFillArgs& a, int n_tiles, size_t smem,
                             cudaStream_t s, bool pdl);
cudaError_t launch_reduce_batch(const GvReduceArgs* args, const int4* tasks, int ntasks, int k,
                                int last, double inv_m1, size_t smem, cudaStream_t s);
cudaError_t launch_consts(int integrand, const double* params, double* kconst, cudaStream_t s);
cudaError_t launch_reset(GvState* st, cudaStream_t s);
cudaError_t launch_grid_pack(int d, int N, double* grid, cudaStream_t s);
cudaError_t launch_rng_words(unsigned long long seed, uint32_t it, uint32_t batch,
                             unsigned long long ev0, long long n, int d, uint32_t* out,
                             cudaStream_t s);
// The CUDA error behind the last VEGAS_ECUDA status of this host thread.
cudaError_t& last_cuda_error();
}  // namespace gv
