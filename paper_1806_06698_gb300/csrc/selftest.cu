// selftest.cu -- measurement and self-test kernels of libsyev3 (sm_103a).
//
// Neither is part of the method of the paper.  k_arith_probe evaluates the
// kernels' own arithmetic helpers (arith.cuh) elementwise, so that tests can
// check them against IEEE results (the approximations' error bounds, the
// integer-pipe conversions' exactness);
// k_dfma_probe runs long chains of independent FP64 fused multiply-adds, the
// operation rate that bounds the FP64 solver, so the benchmark can report
// its roofline against a measured FP64 peak.

#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/syev3.h"
#include "arith.cuh"
#include "internal.h"

namespace syev3 {
namespace {

__global__ void k_arith_probe(int op, const void* __restrict__ x, void* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (op == SYEV3_ARITH_RCP64) {
      static_cast<double*>(y)[i] = rcp64(static_cast<const double*>(x)[i]);
    } else if (op == SYEV3_ARITH_F2D) {
      static_cast<double*>(y)[i] = f2d_exact(static_cast<const float*>(x)[i]);
    } else if (op == SYEV3_ARITH_D2F) {
      static_cast<float*>(y)[i] = d2f_rn(static_cast<const double*>(x)[i]);
    } else {
      const float v = static_cast<const float*>(x)[i];
      float r;
      if (op == SYEV3_ARITH_RCP32)
        r = rcp32(v);
      else if (op == SYEV3_ARITH_SQRT32)
        r = sqrt32(v);
      else
        r = rsqrt32(v);
      static_cast<float*>(y)[i] = r;
    }
  }
}

// kChains independent chains a <- a * m + c per thread; m and c keep the
// values bounded (|m| < 1) and come from the arguments, so nothing folds.
constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_dfma_probe(int64_t iters, double m, double c,
                                                              double* __restrict__ sink) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (double)(threadIdx.x + k);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == 12345.678) sink[0] = s;  // never true for these m, c: keeps the chains live
}

}  // namespace

cudaError_t launch_arith_probe(int op, const void* x, void* y, int64_t n, cudaStream_t stream) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (n + 255) / 256;
  k_arith_probe<<<(int)(blocks < 8LL * sms ? blocks : 8LL * sms), 256, 0, stream>>>(op, x, y, n);
  return cudaGetLastError();
}

cudaError_t launch_dfma_probe(int64_t iters, double* sink, int64_t* dfma_count, cudaStream_t stream) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfma_probe, kProbeThreads, 0);
  if (e != cudaSuccess) return e;
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  *dfma_count = (int64_t)grid * kProbeThreads * kChains * iters;
  k_dfma_probe<<<grid, kProbeThreads, 0, stream>>>(iters, 0.999999, 1e-3, sink);
  return cudaGetLastError();
}

}  // namespace syev3
