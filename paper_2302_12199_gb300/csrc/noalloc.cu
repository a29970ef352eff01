// mst_pivot_noalloc: pivot selection (the same sampling and selection kernels
// as mst_step_pivot) for callers that must not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc / cudaMallocAsync are not
// allowed or not wanted -- a host callback or a real-time thread that must not
// block on the allocator, a caller whose memory is fully reserved up front by
// its own allocator (a serving process that pins its whole budget at start-up),
// or one that may not create a library handle (mst_create allocates).  Such a
// caller can still pass its own input and output buffers.
//
// The step's scratch (the sampled keys) lives in the file-scope device array
// below instead of being allocated per call.  Every GPU that loads this library
// holds that array (512 KiB) until the process exits.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "internal.h"
#include "mst.h"

using namespace mstgpu;

namespace {

constexpr uint32_t kMaxSample = MST_PIVOT_NOALLOC_MAX_SAMPLE;

// Shared scratch: the sample keys of the most recent call (not cleared: the
// sampling kernel writes every entry the selection kernel then reads).
static __device__ __align__(256) u64 g_pivot_scratch[kMaxSample];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
u64 *g_scratch_addr[kMaxDevices] = {};

// Looks up the device address of the scratch array on the current device, once
// per device.  In host code `g_pivot_scratch` only names a host-side shadow, so
// the address must come from cudaGetSymbolAddress with that device current.
mst_status scratch_for_current_device(u64 **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return MST_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_pivot_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return MST_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<u64 *>(p);
  }
  *out = g_scratch_addr[dev];
  return MST_OK;
}

}  // namespace

extern "C" mst_status mst_pivot_noalloc(uint64_t m, const uint32_t *d_w, const uint32_t *d_id, uint64_t state,
                                        uint32_t sample, uint64_t *d_pivot, void *stream) {
  if (!d_pivot || sample == 0 || (m > 0 && !d_w)) return MST_ERR_INVALID_ARG;
  if (sample > kMaxSample || m >= (1ULL << 32)) return MST_ERR_TOO_LARGE;
  // An error that earlier work on this host thread left pending is the
  // caller's: report it without launching and without clearing it, so that
  // the launch check below only ever sees this call's own launch.
  if (cudaPeekAtLastError() != cudaSuccess) return MST_ERR_CUDA;
  u64 *scratch = nullptr;
  const mst_status st = scratch_for_current_device(&scratch);
  if (st != MST_OK) return st;
  launch_pivot(EdgeList{nullptr, nullptr, d_w, d_id}, m, nullptr, state, sample, scratch, (u64 *)d_pivot,
               (cudaStream_t)stream);
  if (cudaGetLastError() != cudaSuccess) return MST_ERR_CUDA;
  return MST_OK;
}
