// gv_fill_batch.cuh -- the persistent fill kernel of the batched form and its
// launch helpers, instantiated per precision and dimension class in
// gv_batch_{f,d}{4,8,16}.cu (so that they compile in parallel).  Each class
// (at most 4, 8 or 16 axes) and integrand runs its own work list with code
// unrolled for it: one kernel holding the three integrands needed the
// registers of two (219 instead of 96-126 at 16 axes, one CTA per SM
// instead of two).
#pragma once
#include "gv_fill.cuh"

// ---------------------------------------------------------------------------
// Persistent fill over the work list.
// ---------------------------------------------------------------------------
// At 4 events per thread the single-integration fill's register budget (64 or
// 80 registers); at 8 the kernels would spill under it and keep their own.
template <int IG, typename Real, int EPT, int MAXD>
__global__ void __launch_bounds__(GV_TILE / EPT,
                                  (EPT == 4 ? GvFillBlocks<Real, EPT, MAXD, false>::value : 0))
    gv_fill_batch_kernel(const GvFillArgs* __restrict__ args, const int* __restrict__ order,
                         const long long* __restrict__ item_start, int n, long long total,
                         unsigned long long* counter) {
  constexpr int B = GV_TILE / EPT;
  constexpr int NW = B / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long red_u64[NW];
  __shared__ u128 red_128[NW];
  __shared__ long long s_item;
  __shared__ int s_pos;
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long item = (long long)atomicAdd(counter, 1ull);
      int pos = 0;
      if (item < total) {  // last position whose first item is <= item
        int lo = 0, hi = n - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (item_start[mid] <= item)
            lo = mid;
          else
            hi = mid - 1;
        }
        pos = lo;
      }
      s_item = item;
      s_pos = pos;
    }
    __syncthreads();
    const long long item = s_item;
    if (item >= total) break;
    const int pos = s_pos;
    const int b = order[pos];
    const long long tile = item - item_start[pos];
    const GvFillArgs a = args[b];
    const GvFillSmem lay(a.ndim, a.nbins, (int)sizeof(Real), true, MAXD > 4);
    unsigned* hist = reinterpret_cast<unsigned*>(smem + lay.hist);
    for (int k = threadIdx.x; k < 4 * a.ndim * a.nbins; k += B) hist[k] = 0u;
    if (b != cur) {
      gv_stage_grid<Real>(a.grid, a.ndim, a.nbins, reinterpret_cast<double*>(smem + lay.jac),
                          reinterpret_cast<typename GvPair<Real>::T*>(smem + lay.ew),
                          threadIdx.x, B);
      cur = b;
    }
    const uint32_t it = (uint32_t)a.st->it;
    __syncthreads();
    gv_fill_tile<IG, Real, EPT, MAXD>(a, tile, smem, red_u64, red_128, it);
    __syncthreads();
  }
}

template <int IG, typename Real, int EPT, int MAXD>
inline cudaError_t gv_fill_batch_launch(int ctas, size_t smem, cudaStream_t s,
                                        const GvFillArgs* args, const int* order,
                                        const long long* item_start, int n, long long total,
                                        unsigned long long* counter) {
  auto k = gv_fill_batch_kernel<IG, Real, EPT, MAXD>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k<<<ctas, GV_TILE / EPT, smem, s>>>(args, order, item_start, n, total, counter);
  return cudaGetLastError();
}

template <int IG, typename Real, int EPT, int MAXD>
inline int gv_fill_batch_occupancy(size_t smem) {
  auto k = gv_fill_batch_kernel<IG, Real, EPT, MAXD>;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, GV_TILE / EPT, smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return blocks;
}

// Entry points of one integrand, events per thread 4 or 8 (the 3-jet form
// has at least 5 axes: not in the 4-axis class).
template <int IG, typename Real, int MAXD>
inline cudaError_t gv_fill_batch_ig(int ept, int ctas, size_t smem, cudaStream_t s,
                                    const GvFillArgs* args, const int* order,
                                    const long long* item_start, int n, long long total,
                                    unsigned long long* counter) {
  if constexpr (IG == GV_EE3J && MAXD <= 4) {
    return cudaErrorInvalidValue;
  } else {
    return ept == 8 ? gv_fill_batch_launch<IG, Real, 8, MAXD>(ctas, smem, s, args, order,
                                                              item_start, n, total, counter)
                    : gv_fill_batch_launch<IG, Real, 4, MAXD>(ctas, smem, s, args, order,
                                                              item_start, n, total, counter);
  }
}
template <int IG, typename Real, int MAXD>
inline int gv_fill_batch_occ_ig(int ept, size_t smem) {
  if constexpr (IG == GV_EE3J && MAXD <= 4) {
    return 0;
  } else {
    return ept == 8 ? gv_fill_batch_occupancy<IG, Real, 8, MAXD>(smem)
                    : gv_fill_batch_occupancy<IG, Real, 4, MAXD>(smem);
  }
}

// One precision and dimension class' entry points (GV_DEFINE_FILL_BATCH): the
// integrand ig (Gauss, Drell-Yan, 3-jet), events per thread 4 or 8.
#define GV_FILL_BATCH_SIG(NAME)                                                               \
  cudaError_t NAME(int ig, int ept, int ctas, size_t smem, cudaStream_t s,                    \
                   const GvFillArgs* args, const int* order, const long long* item_start,     \
                   int n, long long total, unsigned long long* counter)
#define GV_DECLARE_FILL_BATCH(SUF)                                                            \
  namespace gv {                                                                              \
  GV_FILL_BATCH_SIG(fill_batch_##SUF);                                                        \
  int fill_batch_occ_##SUF(int ig, int ept, size_t smem);                                     \
  }
#define GV_DEFINE_FILL_BATCH(SUF, REAL, MAXD)                                                 \
  namespace gv {                                                                              \
  GV_FILL_BATCH_SIG(fill_batch_##SUF) {                                                       \
    switch (ig) {                                                                             \
      case GV_GAUSS:                                                                          \
        return gv_fill_batch_ig<GV_GAUSS, REAL, MAXD>(ept, ctas, smem, s, args, order,        \
                                                      item_start, n, total, counter);         \
      case GV_DY:                                                                             \
        return gv_fill_batch_ig<GV_DY, REAL, MAXD>(ept, ctas, smem, s, args, order,           \
                                                   item_start, n, total, counter);            \
      case GV_EE3J:                                                                           \
        return gv_fill_batch_ig<GV_EE3J, REAL, MAXD>(ept, ctas, smem, s, args, order,         \
                                                     item_start, n, total, counter);          \
    }                                                                                         \
    return cudaErrorInvalidValue;                                                             \
  }                                                                                           \
  int fill_batch_occ_##SUF(int ig, int ept, size_t smem) {                                    \
    switch (ig) {                                                                             \
      case GV_GAUSS: return gv_fill_batch_occ_ig<GV_GAUSS, REAL, MAXD>(ept, smem);            \
      case GV_DY: return gv_fill_batch_occ_ig<GV_DY, REAL, MAXD>(ept, smem);                  \
      case GV_EE3J: return gv_fill_batch_occ_ig<GV_EE3J, REAL, MAXD>(ept, smem);              \
    }                                                                                         \
    return 0;                                                                                 \
  }                                                                                           \
  }
GV_DECLARE_FILL_BATCH(f4)
GV_DECLARE_FILL_BATCH(f8)
GV_DECLARE_FILL_BATCH(f16)
GV_DECLARE_FILL_BATCH(d4)
GV_DECLARE_FILL_BATCH(d8)
GV_DECLARE_FILL_BATCH(d16)
