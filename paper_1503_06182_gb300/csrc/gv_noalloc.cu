// gv_noalloc.cu -- Philox words of events without any device allocation.
//
// vegas_rng_words allocates a device buffer, launches the Philox kernel into
// it, copies the words out and frees the buffer, on every call.  Some callers
// cannot do that:
//   - a thread that runs while another thread of the process captures a CUDA
//     graph in global capture mode: cudaMalloc and cudaFree are refused then;
//   - a process whose device memory is held by a caching allocator (PyTorch's,
//     for instance), which can leave nothing for a second allocator;
//   - latency-critical code that cannot take the device-wide synchronisation
//     that cudaFree implies.
// vegas_rng_words_noalloc runs the same kernel into a fixed buffer that is
// part of the library's own device image, so it allocates nothing.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/vegas.h"
#include "gv_common.cuh"

// The fixed buffer: VEGAS_NOALLOC_MAX_WORDS words (1 MiB), one copy per device
// (a __device__ variable exists once in every context that loads the module).
// Nothing in it has to start at zero: every word copied out has just been
// written by the kernel of the same call.
static __device__ __align__(256) uint32_t gv_noalloc_scratch[VEGAS_NOALLOC_MAX_WORDS];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_lookup_mutex;
uint32_t* g_scratch[kMaxDevices];  // device address of the buffer per device (null: not looked up)

// The buffer's device address for the current device, looked up on the first
// call for that device and cached.
int scratch_of_current_device(uint32_t** out) {
  int dev = 0;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return VEGAS_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return VEGAS_EDEVICE;
  std::lock_guard<std::mutex> lock(g_lookup_mutex);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    const cudaError_t ea = cudaGetSymbolAddress(&p, gv_noalloc_scratch);
    if (ea != cudaSuccess || p == nullptr) {
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
  // legacy default stream, as vegas_rng_words: the copy is ordered after the kernel
  cudaError_t e = gv::launch_rng_words(seed, iteration, batch, (unsigned long long)first_event,
                                       n, ndim, d, nullptr);
  if (e == cudaSuccess)
    e = cudaMemcpy(out, d, (size_t)n * ndim * sizeof(uint32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return VEGAS_ECUDA;
  }
  return VEGAS_OK;
}
