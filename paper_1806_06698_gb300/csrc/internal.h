// internal.h -- launchers shared between the translation units of libsyev3.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace syev3 {

// Counters layout (see syev3_batched_ex): [0] capped, [1] non-finite,
// [2] refined in FP64, [3] refined lanes failing the FP64 residual check.
constexpr int kNumCounters = 4;

cudaError_t launch_f64(const double* A, int64_t n, double* lam, double* U, unsigned long long* counters,
                       cudaStream_t stream);

// Method study (syev3_batched_method): values match syev3_zero_finder and
// syev3_deflation_test of syev3.h.
constexpr int kZfProduction = 0, kZfBorgesGragg = 1, kZfNewton = 2;
constexpr int kDeflSimplified = 0, kDeflEispack = 1;
struct Method {
  int zero_finder;
  int deflation_test;
};
// Statistics layout of syev3_batched_method (8 words).
constexpr int kStatCapped = 0, kStatNonFinite = 1, kStatDiagonal = 2, kStatDeflated = 3, kStatReduced = 4,
              kStatSteps = 5, kStatRoots = 6, kStatWarpSlots = 7, kNumStats = 8;

cudaError_t launch_f64_method(const double* A, int64_t n, double* lam, double* U, unsigned long long* stats,
                              Method method, cudaStream_t stream);

cudaError_t launch_f32(const float* A, int64_t n, float* lam, float* U, bool compensated,
                       unsigned long long* counters, cudaStream_t stream);

// Compensated FP32 with the refinement deferred to a second kernel
// (syev3_batched_ws): the workspace holds two counters at offset 0 and, from
// kFlagListOffset, room for n records of flagged lanes: reduced arrows from
// the front (counter 0), the other classes from the back (counter 1).
struct alignas(16) FlagRec {
  float v[9];       // a1 a2 b1 b2 g c s (pre-scaled arrow and rotation), mu, nu
  int code;         // e << 2 | class
  long long gidx;   // index of the matrix in the batch
};
static_assert(sizeof(FlagRec) == 48, "FlagRec layout");
constexpr size_t kFlagListOffset = 256;
size_t f32c_workspace_bytes(int64_t n);
cudaError_t launch_f32c_deferred(const float* A, int64_t n, float* lam, float* U, unsigned long long* counters,
                                 void* work, cudaStream_t stream);

// Serving: the work of one round, built on the device by the admission
// kernel (serve.cu) and read by the solve kernels' serving instantiations.
// Each item is a contiguous run of one request's matrices; the items' tiles
// of 128 matrices are numbered consecutively over the list (tile_begin is
// the prefix sum), so a solve kernel's grid walks all requests of the round
// as one ragged batch.
struct ServeItem {
  const void* A;       // first packed record of the run
  void* lam;           // its eigenvalues
  void* U;             // its eigenvectors, or null (eigenvalues only)
  int64_t count;       // matrices in the run, >= 1
  int64_t tile_begin;  // index of the run's first tile in the list
  int64_t tag;         // the owner's reference (the serving runtime's request slot)
};
constexpr int kServeTile = 128;       // matrices per tile of both solve kernels
constexpr int kServeMaxItems = 16384;  // one item per admitted request per round
struct ServeList {
  int64_t n_items;
  int64_t n_tiles;
  ServeItem items[kServeMaxItems];
};

// Solve every item of a device-resident list (grid sized from the host; the
// kernels read the list's length on the device).
cudaError_t launch_f64_serve(const ServeList* list, unsigned long long* counters, cudaStream_t stream);
cudaError_t launch_f32_serve(const ServeList* list, bool compensated, unsigned long long* counters,
                             cudaStream_t stream);

template <class T>
cudaError_t launch_bwd(const T* lam, const T* U, const T* gl, const T* gU, int64_t n, T* gA, T tau,
                       cudaStream_t stream);

// One CTA whose bounded wait runs out (syev3_selftest_wait_limit).
cudaError_t launch_wait_selftest(cudaStream_t stream);

// The arithmetic helpers of arith.cuh elementwise (syev3_selftest_arith) and
// the FP64 fused multiply-add rate probe (syev3_probe_dfma); selftest.cu.
cudaError_t launch_arith_probe(int op, const void* x, void* y, int64_t n, cudaStream_t stream);
cudaError_t launch_dfma_probe(int64_t iters, double* sink, int64_t* dfma_count, cudaStream_t stream);

// Record e as this host thread's last CUDA error (syev3_last_cuda_error),
// clear the runtime's last-error state, and return SYEV3_ECUDA.
int record_cuda_error(cudaError_t e);

// Read and clear the __device__ status word of each translation unit
// (synchronise the device).
cudaError_t take_flags_f64(unsigned* flags);
cudaError_t take_flags_f32(unsigned* flags);
cudaError_t take_flags_bwd(unsigned* flags);

}  // namespace syev3
