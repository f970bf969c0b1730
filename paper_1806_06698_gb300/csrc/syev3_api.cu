// syev3_api.cu -- the extern "C" boundary of libsyev3 (declared in
// include/syev3.h): argument checks on the host, then one launch on the
// caller's stream.  Nothing here computes; every step runs in the kernels.

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/syev3.h"
#include "internal.h"

namespace {

thread_local int t_last_cuda_error = 0;

int cuda_fail(cudaError_t e) {
  t_last_cuda_error = (int)e;
  return SYEV3_ECUDA;
}

size_t elem_size(int dtype) { return dtype == SYEV3_F64 ? 8 : 4; }

bool valid_dtype(int dtype) {
  return dtype == SYEV3_F64 || dtype == SYEV3_F32 || dtype == SYEV3_F32_COMPENSATED;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  if (a == nullptr || b == nullptr) return false;
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}

// Device-accessible memory only: device, managed, or host memory registered
// with (or allocated by) CUDA.  Plain pageable host memory is refused.
bool device_accessible(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged ||
         (at.type == cudaMemoryTypeHost && at.devicePointer != nullptr);
}

int check_forward(const void* A, int64_t n, const void* lam, const void* U, int dtype) {
  if (!valid_dtype(dtype) || n < 0) return SYEV3_EINVAL;
  if (n == 0) return SYEV3_OK;
  if (A == nullptr || lam == nullptr) return SYEV3_EINVAL;
  const size_t es = elem_size(dtype);
  if (!aligned(A, es) || !aligned(lam, es) || (U && !aligned(U, es))) return SYEV3_EINVAL;
  const size_t nb_A = (size_t)n * 6 * es, nb_l = (size_t)n * 3 * es, nb_U = (size_t)n * 9 * es;
  if (overlap(A, nb_A, lam, nb_l) || overlap(A, nb_A, U, nb_U) || overlap(lam, nb_l, U, nb_U))
    return SYEV3_EINVAL;
  if (!device_accessible(A) || !device_accessible(lam) || (U && !device_accessible(U))) return SYEV3_EINVAL;
  return SYEV3_OK;
}

}  // namespace

int syev3::record_cuda_error(cudaError_t e) {
  cudaGetLastError();
  return cuda_fail(e);
}

extern "C" {

int syev3_abi_version(void) { return 2; }

const char* syev3_status_string(int status) {
  switch (status) {
    case SYEV3_OK: return "SYEV3_OK";
    case SYEV3_EINVAL: return "SYEV3_EINVAL: invalid argument";
    case SYEV3_ECUDA: return "SYEV3_ECUDA: CUDA call failed";
    case SYEV3_ENOCONV: return "SYEV3_ENOCONV: zero finder hit its step cap";
    case SYEV3_ETIMEOUT: return "SYEV3_ETIMEOUT: a device-side wait ran out";
    case SYEV3_EAGAIN: return "SYEV3_EAGAIN: the server's request ring is full";
    default: return "SYEV3: unknown status";
  }
}

int syev3_last_cuda_error(void) { return t_last_cuda_error; }

int syev3_batched_ex(const void* A_packed6, int64_t n, void* lambda, void* U, int dtype, uint64_t* d_counters,
                     syev3_stream_t stream) {
  const int st = check_forward(A_packed6, n, lambda, U, dtype);
  if (st != SYEV3_OK || n == 0) return st;
  if (d_counters && (!aligned(d_counters, 8) || !device_accessible(d_counters))) return SYEV3_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  auto* ctr = reinterpret_cast<unsigned long long*>(d_counters);
  cudaError_t e;
  switch (dtype) {
    case SYEV3_F64:
      e = syev3::launch_f64(static_cast<const double*>(A_packed6), n, static_cast<double*>(lambda),
                            static_cast<double*>(U), ctr, s);
      break;
    case SYEV3_F32:
    case SYEV3_F32_COMPENSATED:
      e = syev3::launch_f32(static_cast<const float*>(A_packed6), n, static_cast<float*>(lambda),
                            static_cast<float*>(U), dtype == SYEV3_F32_COMPENSATED, ctr, s);
      break;
    default:
      return SYEV3_EINVAL;
  }
  return e == cudaSuccess ? SYEV3_OK : cuda_fail(e);
}

int syev3_batched(const void* A_packed6, int64_t n, void* lambda, void* U, int dtype, syev3_stream_t stream) {
  return syev3_batched_ex(A_packed6, n, lambda, U, dtype, nullptr, stream);
}

size_t syev3_workspace_bytes(int64_t n, int dtype) {
  if (n <= 0 || dtype != SYEV3_F32_COMPENSATED) return 0;
  return syev3::f32c_workspace_bytes(n);
}

int syev3_batched_ws(const void* A_packed6, int64_t n, void* lambda, void* U, int dtype, uint64_t* d_counters,
                     void* d_workspace, size_t workspace_bytes, syev3_stream_t stream) {
  if (dtype != SYEV3_F32_COMPENSATED)
    return syev3_batched_ex(A_packed6, n, lambda, U, dtype, d_counters, stream);
  const int st = check_forward(A_packed6, n, lambda, U, dtype);
  if (st != SYEV3_OK || n == 0) return st;
  if (d_counters && (!aligned(d_counters, 8) || !device_accessible(d_counters))) return SYEV3_EINVAL;
  const size_t need = syev3::f32c_workspace_bytes(n);
  if (d_workspace == nullptr || workspace_bytes < need || !aligned(d_workspace, 256) ||
      !device_accessible(d_workspace))
    return SYEV3_EINVAL;
  if (overlap(d_workspace, need, A_packed6, (size_t)n * 24) || overlap(d_workspace, need, lambda, (size_t)n * 12) ||
      overlap(d_workspace, need, U, (size_t)n * 36))
    return SYEV3_EINVAL;
  const cudaError_t e = syev3::launch_f32c_deferred(
      static_cast<const float*>(A_packed6), n, static_cast<float*>(lambda), static_cast<float*>(U),
      reinterpret_cast<unsigned long long*>(d_counters), d_workspace, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SYEV3_OK : cuda_fail(e);
}

int syev3_batched_method(const void* A_packed6, int64_t n, void* lambda, void* U, int dtype,
                         const syev3_method* method, uint64_t* d_stats, syev3_stream_t stream) {
  if (dtype != SYEV3_F64 || method == nullptr) return SYEV3_EINVAL;
  if (method->zero_finder < SYEV3_ZF_PRODUCTION || method->zero_finder > SYEV3_ZF_NEWTON) return SYEV3_EINVAL;
  if (method->deflation_test != SYEV3_DEFLATION_SIMPLIFIED && method->deflation_test != SYEV3_DEFLATION_EISPACK)
    return SYEV3_EINVAL;
  const int st = check_forward(A_packed6, n, lambda, U, dtype);
  if (st != SYEV3_OK || n == 0) return st;
  if (d_stats && (!aligned(d_stats, 8) || !device_accessible(d_stats))) return SYEV3_EINVAL;
  static_assert(SYEV3_ZF_NEWTON == syev3::kZfNewton && SYEV3_ZF_BORGES_GRAGG == syev3::kZfBorgesGragg &&
                    SYEV3_DEFLATION_EISPACK == syev3::kDeflEispack && SYEV3_METHOD_STATS == syev3::kNumStats,
                "syev3.h and internal.h disagree");
  const syev3::Method m{method->zero_finder, method->deflation_test};
  const cudaError_t e = syev3::launch_f64_method(static_cast<const double*>(A_packed6), n,
                                                 static_cast<double*>(lambda), static_cast<double*>(U),
                                                 reinterpret_cast<unsigned long long*>(d_stats), m,
                                                 reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SYEV3_OK : cuda_fail(e);
}

int syev3_batched_bwd(const void* lambda, const void* U, const void* g_lambda, const void* g_U, int64_t n,
                      void* g_A_packed6, double gap_tau, int dtype, syev3_stream_t stream) {
  if (!valid_dtype(dtype) || n < 0 || !(gap_tau >= 0.0) || gap_tau > 1e300) return SYEV3_EINVAL;
  if (n == 0) return SYEV3_OK;
  if (lambda == nullptr || U == nullptr || g_lambda == nullptr || g_A_packed6 == nullptr) return SYEV3_EINVAL;
  const size_t es = elem_size(dtype);
  const void* ins[4] = {lambda, U, g_lambda, g_U};
  const size_t nbs[4] = {(size_t)n * 3 * es, (size_t)n * 9 * es, (size_t)n * 3 * es, (size_t)n * 9 * es};
  const size_t nb_out = (size_t)n * 6 * es;
  for (int i = 0; i < 4; ++i) {
    if (ins[i] == nullptr) continue;
    if (!aligned(ins[i], es) || overlap(ins[i], nbs[i], g_A_packed6, nb_out) || !device_accessible(ins[i]))
      return SYEV3_EINVAL;
  }
  if (!aligned(g_A_packed6, es) || !device_accessible(g_A_packed6)) return SYEV3_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (dtype == SYEV3_F64)
    e = syev3::launch_bwd<double>(static_cast<const double*>(lambda), static_cast<const double*>(U),
                                  static_cast<const double*>(g_lambda), static_cast<const double*>(g_U), n,
                                  static_cast<double*>(g_A_packed6), gap_tau, s);
  else
    e = syev3::launch_bwd<float>(static_cast<const float*>(lambda), static_cast<const float*>(U),
                                 static_cast<const float*>(g_lambda), static_cast<const float*>(g_U), n,
                                 static_cast<float*>(g_A_packed6), (float)gap_tau, s);
  return e == cudaSuccess ? SYEV3_OK : cuda_fail(e);
}

int syev3_selftest_wait_limit(syev3_stream_t stream) {
  const cudaError_t e = syev3::launch_wait_selftest(reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SYEV3_OK : cuda_fail(e);
}

int syev3_selftest_arith(int op, const void* x, void* y, int64_t n, syev3_stream_t stream) {
  if (op < SYEV3_ARITH_RCP64 || op > SYEV3_ARITH_D2F || n < 0) return SYEV3_EINVAL;
  if (n == 0) return SYEV3_OK;
  const size_t xs = (op == SYEV3_ARITH_RCP64 || op == SYEV3_ARITH_D2F) ? 8 : 4;
  const size_t ys = (op == SYEV3_ARITH_RCP64 || op == SYEV3_ARITH_F2D) ? 8 : 4;
  if (x == nullptr || y == nullptr || !aligned(x, xs) || !aligned(y, ys) || overlap(x, n * xs, y, n * ys) ||
      !device_accessible(x) || !device_accessible(y))
    return SYEV3_EINVAL;
  const cudaError_t e = syev3::launch_arith_probe(op, x, y, n, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SYEV3_OK : cuda_fail(e);
}

int syev3_probe_dfma(int64_t iters, double* d_sink, int64_t* dfma_count, syev3_stream_t stream) {
  if (iters < 1 || d_sink == nullptr || dfma_count == nullptr || !aligned(d_sink, 8) || !device_accessible(d_sink))
    return SYEV3_EINVAL;
  const cudaError_t e = syev3::launch_dfma_probe(iters, d_sink, dfma_count, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SYEV3_OK : cuda_fail(e);
}

int syev3_device_flags(uint32_t* flags) {
  if (flags == nullptr) return SYEV3_EINVAL;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e);
  unsigned v = 0;
  e = syev3::take_flags_f64(&v);
  if (e == cudaSuccess) e = syev3::take_flags_f32(&v);
  if (e == cudaSuccess) e = syev3::take_flags_bwd(&v);
  if (e != cudaSuccess) return cuda_fail(e);
  *flags = v;
  return SYEV3_OK;
}

}  // extern "C"
