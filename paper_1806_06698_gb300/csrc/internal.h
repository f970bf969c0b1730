// internal.h -- launchers shared between the translation units of libsyev3.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace syev3 {

// Counters layout (see syev3_batched_ex): [0] capped, [1] non-finite,
// [2] refined in FP64, [3] reserved.
constexpr int kNumCounters = 4;

cudaError_t launch_f64(const double* A, int64_t n, double* lam, double* U, unsigned long long* counters,
                       cudaStream_t stream);

// Reads and clears the __device__ status word of each translation unit
// (synchronises the device).
cudaError_t take_flags_f64(unsigned* flags);

}  // namespace syev3
