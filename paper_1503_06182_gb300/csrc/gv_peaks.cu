// gv_peaks.cu -- measured throughput of the arithmetic pipes the VEGAS
// kernels run on (the denominators of their rooflines).
//
// The per-event kernels are bound by plain arithmetic (Philox and the exact
// integer sums on the integer pipes, the FP32 integrand, FP64 in the plain
// form and in the refinement), not by a dense contraction or by HBM, so their
// peaks are the issue rates of those pipes on this GPU at its current clock.
// Each probe kernel runs NCH independent chains of one instruction per
// thread (enough to cover the pipe's latency; each step depends on the
// previous one non-linearly or inexactly, so no two steps can be merged),
// 8 resident 256-thread CTAs per SM, for a calibrated number of rounds; the
// rate is the operation count over the CUDA-event time of the timed launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/vegas.h"
#include "gv_common.cuh"

namespace {

constexpr int NCH = 8;  // independent chains per thread

template <int PIPE>
__global__ void __launch_bounds__(256) gv_peak_kernel(int rounds, float* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (PIPE == VEGAS_PIPE_FFMA) {
    float x[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = 1.0f + 1e-3f * (float)(t + c);
    for (int r = 0; r < rounds; ++r)
#pragma unroll
      for (int c = 0; c < NCH; ++c) x[c] = fmaf(x[c], 0.9999999f, 1e-7f);
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < NCH; ++c) s += x[c];
    out[t] = s;
  } else if constexpr (PIPE == VEGAS_PIPE_DFMA) {
    double x[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = 1.0 + 1e-3 * (double)(t + c);
    for (int r = 0; r < rounds; ++r)
#pragma unroll
      for (int c = 0; c < NCH; ++c) x[c] = fma(x[c], 0.9999999, 1e-7);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < NCH; ++c) s += x[c];
    out[t] = (float)s;
  } else if constexpr (PIPE == VEGAS_PIPE_IMAD) {
    uint32_t x[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = (uint32_t)(t * NCH + c);
    for (int r = 0; r < rounds; ++r)
#pragma unroll
      for (int c = 0; c < NCH; ++c) x[c] = x[c] * x[c] + (uint32_t)(2 * c + 1);
    uint32_t s = 0u;
#pragma unroll
    for (int c = 0; c < NCH; ++c) s ^= x[c];
    out[t] = (float)s;
  } else {  // VEGAS_PIPE_MUFU: 2^x approximations; x stays in [-1, -1/2]
    float x[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = -0.5f - 1e-4f * (float)c;
    for (int r = 0; r < rounds; ++r)
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        float y;
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[c]));
        x[c] = -y;
      }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < NCH; ++c) s += x[c];
    out[t] = s;
  }
}

template <int PIPE>
cudaError_t time_pipe(int blocks, int rounds, float* out, cudaEvent_t e0, cudaEvent_t e1,
                      float* ms) {
  cudaEventRecord(e0, 0);
  gv_peak_kernel<PIPE><<<blocks, 256>>>(rounds, out);
  cudaEventRecord(e1, 0);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  return e;
}

template <int PIPE>
cudaError_t measure(double target_ms, double* ops_per_s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = 8 * sms;
  float* out = nullptr;
  e = cudaMalloc(&out, (size_t)blocks * 256 * sizeof(float));
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // calibrate the number of rounds to the target duration, then time
  int rounds = 256;
  float ms = 0.0f;
  for (int i = 0; i < 8 && e == cudaSuccess; ++i) {
    e = time_pipe<PIPE>(blocks, rounds, out, e0, e1, &ms);
    if (e != cudaSuccess || ms >= 0.5 * target_ms || rounds >= (1 << 24)) break;
    const double f = ms > 0.0f ? target_ms / ms : 64.0;
    rounds = (int)std::min<double>((double)(1 << 24), rounds * std::min(64.0, std::max(2.0, f)));
  }
  if (e == cudaSuccess) e = time_pipe<PIPE>(blocks, rounds, out, e0, e1, &ms);
  if (e == cudaSuccess) {
    const double per_op = (PIPE == VEGAS_PIPE_FFMA || PIPE == VEGAS_PIPE_DFMA) ? 2.0 : 1.0;
    *ops_per_s = per_op * (double)blocks * 256.0 * NCH * (double)rounds / (ms * 1e-3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return e;
}

}  // namespace

extern "C" int vegas_pipe_peak(int pipe, double ms, double* ops_per_s) {
  if (!ops_per_s || !(ms > 0.0) || ms > 10000.0) return VEGAS_EINVAL;
  cudaError_t e;
  switch (pipe) {
    case VEGAS_PIPE_FFMA: e = measure<VEGAS_PIPE_FFMA>(ms, ops_per_s); break;
    case VEGAS_PIPE_DFMA: e = measure<VEGAS_PIPE_DFMA>(ms, ops_per_s); break;
    case VEGAS_PIPE_IMAD: e = measure<VEGAS_PIPE_IMAD>(ms, ops_per_s); break;
    case VEGAS_PIPE_MUFU: e = measure<VEGAS_PIPE_MUFU>(ms, ops_per_s); break;
    default: return VEGAS_EINVAL;
  }
  if (e != cudaSuccess) {
    gv::last_cuda_error() = e;
    cudaGetLastError();
    return VEGAS_ECUDA;
  }
  return VEGAS_OK;
}
