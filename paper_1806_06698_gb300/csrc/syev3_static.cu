// syev3_static.cu -- syev3_batched_static_ws: the compensated FP32 solve
// with its FP64 refinement deferred to a second kernel (as syev3_batched_ws),
// its scratch list kept in a file-scope __device__ array instead of a
// caller-provided workspace.
//
// For callers that cannot hand the library a workspace: a plain C caller
// with no device allocator of its own, or code that must not call
// cudaMalloc / cudaFree on this path (they synchronise the device and can
// fail under memory pressure) and must not keep a per-caller buffer.  The
// array is part of the module's static device memory, so the call itself
// allocates nothing; its size bounds the batch (kStaticMaxN).
//
// The array is shared by every call on a device: calls that overlap in time
// (other streams, other host threads) race on it and must be ordered by the
// caller.  The first call on a device resolves the array's address with
// cudaGetSymbolAddress (which may load the module); it must happen before
// any stream capture begins on that device.  The address is cached per
// device index for the life of the process, so the entry point must not be
// used on a device after cudaDeviceReset (a new context may load the module
// at another address).

#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/syev3.h"
#include "internal.h"

namespace {

constexpr int64_t kStaticMaxN = SYEV3_STATIC_MAX_N;
constexpr size_t kStaticBytes = syev3::kFlagListOffset + (size_t)kStaticMaxN * sizeof(syev3::FlagRec);

// Two counters at offset 0, the list of flagged lanes from kFlagListOffset.
static __device__ __align__(256) unsigned char g_static_ws[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

}  // namespace

extern "C" {

int syev3_batched_static_ws(const void* A_packed6, int64_t n, void* lambda, void* U, uint64_t* d_counters,
                            syev3_stream_t stream) {
  if (n < 0 || n > kStaticMaxN) return SYEV3_EINVAL;
  if (n == 0) return SYEV3_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return syev3::record_cuda_error(e);
  if (dev < 0 || dev >= kMaxDevices) return SYEV3_EINVAL;
  void* ws = nullptr;
  {
    // Once per device, with that device current.
    std::lock_guard<std::mutex> hold(g_mu);
    if (g_addr[dev] == nullptr) {
      e = cudaGetSymbolAddress(&g_addr[dev], g_static_ws);
      if (e != cudaSuccess) {
        g_addr[dev] = nullptr;
        return syev3::record_cuda_error(e);
      }
    }
    ws = g_addr[dev];
  }
  // The argument checks and the launches of the workspace path (the
  // library clears the list's counter on `stream` before the first kernel).
  return syev3_batched_ws(A_packed6, n, lambda, U, SYEV3_F32_COMPENSATED, d_counters, ws, kStaticBytes, stream);
}

}  // extern "C"
