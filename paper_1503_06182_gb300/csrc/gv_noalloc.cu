// gv_noalloc.cu -- Philox words of events without any device allocation.
//
// vegas_rng_words allocates a device buffer, launches the Philox kernel into
// it, copies the words out and frees the buffer, on every call.  Some callers
// cannot do that:
//   - a process whose device memory is held by a caching allocator (PyTorch's,
//     for instance): the memory is free for the cache's owner but cudaMalloc
//     from another library fails with out-of-memory;
//   - latency-critical code that cannot take the device-wide synchronisation
//     that cudaFree implies, nor the cost of the allocator in every call.
// vegas_rng_words_noalloc runs the same Philox words into a fixed buffer that
// is part of the library's own device image, so it allocates nothing.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/vegas.h"
#include "gv_common.cuh"

// The fixed buffer: VEGAS_NOALLOC_MAX_WORDS words (1 MiB), one copy per device
// (a __device__ variable exists once in every context that loads the module),
// held until the process exits.  Nothing in it has to start at zero: every
// word copied out has just been written by the kernel of the same call.
static __device__ __align__(256) uint32_t gv_noalloc_scratch[VEGAS_NOALLOC_MAX_WORDS];

// The words of events ev0 .. ev0 + n - 1 into out (n x d, row = event), with
// the event-word layout of the fill kernels (gv_event_words).  The copy-out
// loop is unrolled over the largest dimension, so that the words stay in
// registers: the kernel uses no local memory, whose pool the driver would
// otherwise grow, with a device allocation, on the first launch.
__global__ void gv_rng_words_noalloc_kernel(unsigned long long seed, uint32_t it, uint32_t batch,
                                            unsigned long long ev0, long long n, int d,
                                            uint32_t* out) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  uint32_t r[GV_MAXD];
  gv_event_words<GV_MAXD>(seed, it, batch, ev0 + (unsigned long long)j, d, r);
#pragma unroll
  for (int a = 0; a < GV_MAXD; ++a)
    if (a < d) out[j * d + a] = r[a];
}

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
uint32_t* g_scratch[kMaxDevices];  // device address of the buffer per device (null: not set up)

// Set-up for the current device, once: the buffer's device address (in host
// code the array's name is only a host-side stand-in), and the kernel loaded,
// so that later calls make neither allocation.
int scratch_of_current_device(uint32_t** out) {
  int dev = 0;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    gv::last_cuda_error() = e;
    cudaGetLastError();
    return VEGAS_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return VEGAS_EDEVICE;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    cudaError_t ea = cudaGetSymbolAddress(&p, gv_noalloc_scratch);
    if (ea == cudaSuccess && p == nullptr) ea = cudaErrorInvalidSymbol;
    cudaFuncAttributes fa;
    if (ea == cudaSuccess) ea = cudaFuncGetAttributes(&fa, gv_rng_words_noalloc_kernel);
    if (ea != cudaSuccess) {
      gv::last_cuda_error() = ea;
      cudaGetLastError();
      return VEGAS_ECUDA;
    }
    g_scratch[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_scratch[dev];
  return VEGAS_OK;
}

}  // namespace

extern "C" int vegas_rng_words_noalloc(uint64_t seed, uint32_t iteration, uint32_t batch,
                                       int64_t first_event, int64_t n, int ndim, uint32_t* out) {
  if (n < 0 || first_event < 0 || ndim < 1 || ndim > VEGAS_MAX_DIM || (n > 0 && !out))
    return VEGAS_EINVAL;
  if (n > VEGAS_NOALLOC_MAX_WORDS / ndim) return VEGAS_EINVAL;  // beyond the fixed buffer
  uint32_t* d = nullptr;
  const int st = scratch_of_current_device(&d);  // also the set-up of a call with n == 0
  if (st || n == 0) return st;
  // legacy default stream: the blocking copy is ordered after the kernel
  const int thr = 256;
  gv_rng_words_noalloc_kernel<<<(unsigned)((n + thr - 1) / thr), thr>>>(
      seed, iteration, batch, (unsigned long long)first_event, n, ndim, d);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpy(out, d, (size_t)n * ndim * sizeof(uint32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    gv::last_cuda_error() = e;
    cudaGetLastError();
    return VEGAS_ECUDA;
  }
  return VEGAS_OK;
}
