// gv_fill_inst.cuh -- instantiation and launch helpers of the fill kernels.
#pragma once
#include "gv_fill.cuh"

// Above 48 KB of shared memory a kernel must opt in; the fills' static
// shared memory (at most ~4.2 KB: the stratified fill's per-thread sums and
// the reduction scratch) counts toward it, so any launch within 8 KB of the
// default opts in.
template <typename KernelT>
static cudaError_t gv_prepare(KernelT k, size_t smem) {
  if (smem + 8 * 1024 > 48 * 1024)
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

template <int IG, typename Real, int EPT, int MAXD, bool HIST = false, bool PLUS = false>
static cudaError_t gv_launch_fill_t(const GvFillArgs& a, int n_tiles, size_t smem,
                                    cudaStream_t s, bool pdl) {
  auto k = gv_fill_kernel<IG, Real, EPT, MAXD, HIST, PLUS>;
  cudaError_t e = gv_prepare(k, smem);
  if (e != cudaSuccess) return e;
  return gv_launch(k, dim3(n_tiles), dim3(GV_TILE / EPT), smem, s, pdl, a);
}

template <int IG, typename Real, int MAXD>
static cudaError_t gv_launch_fill_ept(int ept, const GvFillArgs& a, int n_tiles, size_t smem,
                                      cudaStream_t s, bool pdl) {
  switch (ept) {
    case 1: return gv_launch_fill_t<IG, Real, 1, MAXD>(a, n_tiles, smem, s, pdl);
    case 2: return gv_launch_fill_t<IG, Real, 2, MAXD>(a, n_tiles, smem, s, pdl);
    case 4: return gv_launch_fill_t<IG, Real, 4, MAXD>(a, n_tiles, smem, s, pdl);
    case 8: return gv_launch_fill_t<IG, Real, 8, MAXD>(a, n_tiles, smem, s, pdl);
  }
  return cudaErrorInvalidValue;
}

template <int IG, typename Real>
static cudaError_t gv_launch_fill_maxd(int ept, const GvFillArgs& a, int n_tiles, size_t smem,
                                       cudaStream_t s, bool pdl) {
  if (a.ndim <= 4 && IG != GV_EE3J)
    return gv_launch_fill_ept<IG, Real, 4>(ept, a, n_tiles, smem, s, pdl);
  if (a.ndim <= 8) return gv_launch_fill_ept<IG, Real, 8>(ept, a, n_tiles, smem, s, pdl);
  if (a.ndim <= 16) return gv_launch_fill_ept<IG, Real, 16>(ept, a, n_tiles, smem, s, pdl);
  return cudaErrorInvalidValue;
}

// The fill with a histogram of the observable: 4 events per thread (the
// sums, and so the results, are the same for every choice).
template <int IG, typename Real>
static cudaError_t gv_launch_fill_hist_t(const GvFillArgs& a, int n_tiles, size_t smem,
                                         cudaStream_t s, bool pdl) {
  if (a.ndim <= 4 && IG != GV_EE3J)
    return gv_launch_fill_t<IG, Real, 4, 4, true>(a, n_tiles, smem, s, pdl);
  if (a.ndim <= 8) return gv_launch_fill_t<IG, Real, 4, 8, true>(a, n_tiles, smem, s, pdl);
  if (a.ndim <= 16) return gv_launch_fill_t<IG, Real, 4, 16, true>(a, n_tiles, smem, s, pdl);
  return cudaErrorInvalidValue;
}

// The stratified (VEGAS+) fill: 4 events per thread.
template <int IG, typename Real>
static cudaError_t gv_launch_fill_plus_t(const GvFillArgs& a, int n_tiles, size_t smem,
                                         cudaStream_t s, bool pdl) {
  if (a.ndim <= 4 && IG != GV_EE3J)
    return gv_launch_fill_t<IG, Real, 4, 4, false, true>(a, n_tiles, smem, s, pdl);
  if (a.ndim <= 8) return gv_launch_fill_t<IG, Real, 4, 8, false, true>(a, n_tiles, smem, s, pdl);
  if (a.ndim <= 16)
    return gv_launch_fill_t<IG, Real, 4, 16, false, true>(a, n_tiles, smem, s, pdl);
  return cudaErrorInvalidValue;
}

#define GV_DEFINE_FILL_PLUS_LAUNCHER(REAL, SUF)                                               \
  namespace gv {                                                                              \
  cudaError_t launch_fill_plus_##SUF(int ig, const GvFillArgs& a, int n_tiles, size_t smem,   \
                                     cudaStream_t s, bool pdl) {                              \
    switch (ig) {                                                                             \
      case GV_GAUSS: return gv_launch_fill_plus_t<GV_GAUSS, REAL>(a, n_tiles, smem, s, pdl);  \
      case GV_DY: return gv_launch_fill_plus_t<GV_DY, REAL>(a, n_tiles, smem, s, pdl);        \
      case GV_EE3J: return gv_launch_fill_plus_t<GV_EE3J, REAL>(a, n_tiles, smem, s, pdl);    \
      case GV_DYNLO: return gv_launch_fill_plus_t<GV_DYNLO, REAL>(a, n_tiles, smem, s, pdl);  \
    }                                                                                         \
    return cudaErrorInvalidValue;                                                             \
  }                                                                                           \
  }

#define GV_DEFINE_FILL_HIST_LAUNCHER(REAL, SUF)                                               \
  namespace gv {                                                                              \
  cudaError_t launch_fill_hist_##SUF(int ig, const GvFillArgs& a, int n_tiles, size_t smem,   \
                                     cudaStream_t s, bool pdl) {                              \
    switch (ig) {                                                                             \
      case GV_GAUSS: return gv_launch_fill_hist_t<GV_GAUSS, REAL>(a, n_tiles, smem, s, pdl);  \
      case GV_DY: return gv_launch_fill_hist_t<GV_DY, REAL>(a, n_tiles, smem, s, pdl);        \
      case GV_EE3J: return gv_launch_fill_hist_t<GV_EE3J, REAL>(a, n_tiles, smem, s, pdl);    \
      case GV_DYNLO: return gv_launch_fill_hist_t<GV_DYNLO, REAL>(a, n_tiles, smem, s, pdl);  \
    }                                                                                         \
    return cudaErrorInvalidValue;                                                             \
  }                                                                                           \
  }

template <int IG, typename Real>
static cudaError_t gv_launch_eval_t(const GvFillArgs& a, uint32_t it, const long long* events,
                                    long long n, double* w, int* bins, cudaStream_t s) {
  const int thr = 128;
  const long long blocks = (n + thr - 1) / thr;
  if (blocks == 0) return cudaSuccess;
  gv_eval_events_kernel<IG, Real><<<(unsigned)blocks, thr, 0, s>>>(a, it, events, n, w, bins);
  return cudaGetLastError();
}

// The launchers of one integrand and one precision (one translation unit
// each, so that they compile in parallel), and the precision dispatch.
#define GV_DEFINE_FILL_LAUNCHER(NAME, IG, REAL, SUF)                                          \
  namespace gv {                                                                              \
  cudaError_t NAME##_##SUF(int ept, const GvFillArgs& a, int n_tiles, size_t smem,            \
                           cudaStream_t s, bool pdl) {                                        \
    return gv_launch_fill_maxd<IG, REAL>(ept, a, n_tiles, smem, s, pdl);                      \
  }                                                                                           \
  cudaError_t NAME##_eval_##SUF(const GvFillArgs& a, uint32_t it, const long long* ev,        \
                                long long n, double* w, int* bins, cudaStream_t s) {          \
    return gv_launch_eval_t<IG, REAL>(a, it, ev, n, w, bins, s);                              \
  }                                                                                           \
  }

#define GV_DEFINE_FILL_DISPATCH(NAME)                                                         \
  namespace gv {                                                                              \
  cudaError_t NAME##_f32(int ept, const GvFillArgs& a, int n_tiles, size_t smem,              \
                         cudaStream_t s, bool pdl);                                           \
  cudaError_t NAME##_f64(int ept, const GvFillArgs& a, int n_tiles, size_t smem,              \
                         cudaStream_t s, bool pdl);                                           \
  cudaError_t NAME##_eval_f32(const GvFillArgs& a, uint32_t it, const long long* ev,          \
                              long long n, double* w, int* bins, cudaStream_t s);             \
  cudaError_t NAME##_eval_f64(const GvFillArgs& a, uint32_t it, const long long* ev,          \
                              long long n, double* w, int* bins, cudaStream_t s);             \
  cudaError_t NAME(int fp32, int ept, const GvFillArgs& a, int n_tiles, size_t smem,          \
                   cudaStream_t s, bool pdl) {                                                \
    return fp32 ? NAME##_f32(ept, a, n_tiles, smem, s, pdl)                                   \
                : NAME##_f64(ept, a, n_tiles, smem, s, pdl);                                  \
  }                                                                                           \
  cudaError_t NAME##_eval(int fp32, const GvFillArgs& a, uint32_t it, const long long* ev,    \
                          long long n, double* w, int* bins, cudaStream_t s) {                \
    return fp32 ? NAME##_eval_f32(a, it, ev, n, w, bins, s)                                   \
                : NAME##_eval_f64(a, it, ev, n, w, bins, s);                                  \
  }                                                                                           \
  }
