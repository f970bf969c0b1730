// syev3_bwd.cu -- backward pass of the batched 3x3 symmetric eigensolver
// (sm_103a), FP64 and FP32.
//
// Not part of the paper: the standard first-order perturbation result for
// simple eigenvalues, dlambda_i = u_i^T dA u_i and
// du_i = sum_{j != i} u_j (u_j^T dA u_i) / (lambda_i - lambda_j), gives for a
// loss with gradients (gl, gU) with respect to (lambda, U)
//   Abar = U (diag(gl) + F o (U^T gU)) U^T,   F_ij = 1/(lambda_j - lambda_i),
// with F_ij := 0 where |lambda_i - lambda_j| < tau ||A||_F (||A||_F from the
// eigenvalues).  A symmetric A is parametrised by its packed upper triangle,
// so the packed gradient is Abar_ii on the diagonal and Abar_ij + Abar_ji off
// it, which only depends on the symmetric part of the core matrix C:
//   sym(C)_ii = gl_i,   sym(C)_ij = F_ij (M_ij - M_ji) / 2,   M = U^T gU,
// and packed(Abar) = (S_11, S_22, S_33, 2 S_12, 2 S_13, 2 S_23) with
// S = U sym(C) U^T.  One matrix per thread; the four input arrays arrive by
// 1-D bulk copies into shared memory, double-buffered on mbarriers.

#include <cmath>
#include <cstdint>
#include <type_traits>

#include "arith.cuh"
#include "common.cuh"
#include "internal.h"

namespace syev3 {
namespace {

// Matrices per tile (= threads per CTA): 64 in FP64, 128 in FP32, so the
// double-buffered tiles of the four inputs fit in 48 KB of shared memory.
template <class T>
__host__ __device__ constexpr int tile_of() {
  return sizeof(T) == 8 ? 64 : 128;
}

__device__ unsigned g_flags_bwd;

// Helpers with an FP64 form that keeps compares and exact scalings by 2 off
// the FP64 pipe (the one that bounds the FP64 backward): compares of
// non-negative values as bit patterns, halving and doubling by exponent
// arithmetic.  Both forms return bit-identical values to the plain
// expressions 0.5 / x (from a <= 1 ulp reciprocal in FP64), a < b and 2 x.

// 1 / (2 x), x != 0.
template <class T>
__device__ __forceinline__ T half_recip(T x);
template <>
__device__ __forceinline__ double half_recip<double>(double x) {
  if (hi_mag(x) >= hi_pow2(-1000) && hi_mag(x) <= hi_pow2(1000)) {  // |x| in [2^-1000, 2^1000]
    const double r = rcp64(x);  // normal, far from both ends of the range
    return __hiloint2double(__double2hiint(r) - (1 << 20), __double2loint(r));
  }
  return 0.5 / x;
}
template <>
__device__ __forceinline__ float half_recip<float>(float x) {
  return 0.5f / x;
}

// a < b for a, b >= +0 (not NaN).
template <class T>
__device__ __forceinline__ bool lt_nonneg(T a, T b) {
  return a < b;
}
template <>
__device__ __forceinline__ bool lt_nonneg<double>(double a, double b) {
  return dbits(a) < dbits(b);
}

// 2 x, exactly.
template <class T>
__device__ __forceinline__ T twice(T x) {
  return T(2) * x;
}
template <>
__device__ __forceinline__ double twice<double>(double x) {
  return mul_pow2(x, 1);
}

// Packed gradient of one matrix.  l[3] ascending eigenvalues, U[9] row-major
// with eigenvector columns, gl[3], gU[9] (or has_gU false), tau.
template <class T>
__device__ __forceinline__ void grad_one(const T l[3], const T U[9], const T gl[3], const T gU[9], bool has_gU,
                                         T tau, T out[6]) {
  // sym(C): diagonal gl, off-diagonal F_ij (M_ij - M_ji)/2 (masked).
  T c01 = T(0), c02 = T(0), c12 = T(0);
  if (has_gU) {
    // M_ij - M_ji = sum_k U_ki gU_kj - U_kj gU_ki
    T d01 = T(0), d02 = T(0), d12 = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const T u0 = U[k * 3 + 0], u1 = U[k * 3 + 1], u2 = U[k * 3 + 2];
      const T g0 = gU[k * 3 + 0], g1 = gU[k * 3 + 1], g2 = gU[k * 3 + 2];
      d01 = fma(u0, g1, fma(-u1, g0, d01));
      d02 = fma(u0, g2, fma(-u2, g0, d02));
      d12 = fma(u1, g2, fma(-u2, g1, d12));
    }
    // |gap| < tau ||lambda||_2, compared squared (no square root).
    const T thr2 = (tau * tau) * fma(l[0], l[0], fma(l[1], l[1], l[2] * l[2]));
    const T gap01 = l[1] - l[0], gap02 = l[2] - l[0], gap12 = l[2] - l[1];
    c01 = lt_nonneg(gap01 * gap01, thr2) ? T(0) : d01 * half_recip(gap01);
    c02 = lt_nonneg(gap02 * gap02, thr2) ? T(0) : d02 * half_recip(gap02);
    c12 = lt_nonneg(gap12 * gap12, thr2) ? T(0) : d12 * half_recip(gap12);
  }
  const T C[3][3] = {{gl[0], c01, c02}, {c01, gl[1], c12}, {c02, c12, gl[2]}};
  // P = U sym(C); S = P U^T (upper triangle).
  T P[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      P[r][j] = fma(U[r * 3 + 0], C[0][j], fma(U[r * 3 + 1], C[1][j], U[r * 3 + 2] * C[2][j]));
  auto S = [&](int r, int q) {
    return fma(P[r][0], U[q * 3 + 0], fma(P[r][1], U[q * 3 + 1], P[r][2] * U[q * 3 + 2]));
  };
  out[0] = S(0, 0);
  out[1] = S(1, 1);
  out[2] = S(2, 2);
  out[3] = twice(S(0, 1));
  out[4] = twice(S(0, 2));
  out[5] = twice(S(1, 2));
}

// Stage `count` elements of T from global memory into shared memory: a bulk
// copy of the 16-byte-multiple prefix (bytes counted into *tx) and plain
// loads for the rest (done by the caller after the wait).
template <class T>
__device__ __forceinline__ uint32_t bulk_prefix_bytes(int count) {
  return ((uint32_t)count * (uint32_t)sizeof(T)) & ~15u;
}

template <class T, bool kBulk>
__global__ void __launch_bounds__(tile_of<T>()) k_syev3_bwd(const T* __restrict__ lam, const T* __restrict__ U,
                                                    const T* __restrict__ gl, const T* __restrict__ gU, int64_t n,
                                                    T* __restrict__ gA, T tau) {
  constexpr int kTPB = tile_of<T>();
  __shared__ alignas(16) T s_l[2][kTPB * 3];
  __shared__ alignas(16) T s_U[2][kTPB * 9];
  __shared__ alignas(16) T s_gl[2][kTPB * 3];
  __shared__ alignas(16) T s_gU[2][kTPB * 9];
  __shared__ alignas(16) T s_out[kTPB * 6];
  __shared__ alignas(8) uint64_t s_bar[2];

  const int tid = threadIdx.x;
  const bool has_gU = (gU != nullptr);
  const int64_t n_tiles = (n + kTPB - 1) / kTPB;
  const bool vec_out = ((reinterpret_cast<uintptr_t>(gA) & 15) == 0);

  if (kBulk && tid == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();

  auto issue = [&](int64_t tile, int buf) {
    const int64_t base = tile * kTPB;
    const int cnt = (int)((n - base) < kTPB ? (n - base) : kTPB);
    const uint32_t b3 = bulk_prefix_bytes<T>(cnt * 3), b9 = bulk_prefix_bytes<T>(cnt * 9);
    mbar_arrive_expect_tx(&s_bar[buf], 2 * b3 + (has_gU ? 2 * b9 : b9));
    if (b3) {
      bulk_g2s(s_l[buf], lam + base * 3, b3, &s_bar[buf]);
      bulk_g2s(s_gl[buf], gl + base * 3, b3, &s_bar[buf]);
    }
    if (b9) {
      bulk_g2s(s_U[buf], U + base * 9, b9, &s_bar[buf]);
      if (has_gU) bulk_g2s(s_gU[buf], gU + base * 9, b9, &s_bar[buf]);
    }
  };

  uint32_t phases = 0u;
  int buf = 0;
  int64_t tile = blockIdx.x;
  if (kBulk && tid == 0 && tile < n_tiles) issue(tile, 0);

  for (; tile < n_tiles; tile += gridDim.x, buf ^= 1) {
    const int64_t base = tile * kTPB;
    const int cnt = (int)((n - base) < kTPB ? (n - base) : kTPB);
    const int64_t next = tile + gridDim.x;
    int from3 = 0, from9 = 0;  // first element not covered by a bulk copy
    if (kBulk) {
      if (tid == 0 && next < n_tiles) issue(next, buf ^ 1);
      const bool ok = mbar_wait(&s_bar[buf], (phases >> buf) & 1u);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(&g_flags_bwd, kFlagWaitTimeout);
        mbar_wait(&s_bar[buf], (phases >> buf) & 1u);
        if (next < n_tiles) mbar_wait(&s_bar[buf ^ 1], (phases >> (buf ^ 1)) & 1u);
        return;
      }
      phases ^= 1u << buf;
      from3 = (int)(bulk_prefix_bytes<T>(cnt * 3) / sizeof(T));
      from9 = (int)(bulk_prefix_bytes<T>(cnt * 9) / sizeof(T));
    }
    for (int i = from3 + tid; i < cnt * 3; i += kTPB) {
      s_l[buf][i] = lam[base * 3 + i];
      s_gl[buf][i] = gl[base * 3 + i];
    }
    for (int i = from9 + tid; i < cnt * 9; i += kTPB) {
      s_U[buf][i] = U[base * 9 + i];
      if (has_gU) s_gU[buf][i] = gU[base * 9 + i];
    }
    __syncthreads();

    if (tid < cnt) {
      T l[3], u[9], g[3], gu[9], out[6];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        l[k] = s_l[buf][tid * 3 + k];
        g[k] = s_gl[buf][tid * 3 + k];
      }
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        u[k] = s_U[buf][tid * 9 + k];
        gu[k] = has_gU ? s_gU[buf][tid * 9 + k] : T(0);
      }
      grad_one<T>(l, u, g, gu, has_gU, tau, out);
#pragma unroll
      for (int k = 0; k < 6; ++k) s_out[tid * 6 + k] = out[k];
    }
    __syncthreads();
    T* dst = gA + base * 6;
    const int m = cnt * 6;
    constexpr int kVec = 16 / sizeof(T);
    if (vec_out) {
      using V = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
      V* d = reinterpret_cast<V*>(dst);
      const V* s = reinterpret_cast<const V*>(s_out);
      for (int i = tid; i < m / kVec; i += kTPB) d[i] = s[i];
      for (int i = (m / kVec) * kVec + tid; i < m; i += kTPB) dst[i] = s_out[i];
    } else {
      for (int i = tid; i < m; i += kTPB) dst[i] = s_out[i];
    }
    __syncthreads();
  }
}

template <class T, bool kBulk>
cudaError_t launch_one(const T* lam, const T* U, const T* gl, const T* gU, int64_t n, T* gA, T tau,
                       cudaStream_t stream) {
  static int bps = -1;
  if (bps < 0) {
    int v = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_syev3_bwd<T, kBulk>, tile_of<T>(), 0);
    bps = (e == cudaSuccess && v > 0) ? v : 1;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  constexpr int kTPB = tile_of<T>();
  const int64_t n_tiles = (n + kTPB - 1) / kTPB;
  const int64_t resident = (int64_t)sms * bps;
  const int grid = (int)(n_tiles < resident ? n_tiles : resident);
  k_syev3_bwd<T, kBulk><<<grid, kTPB, 0, stream>>>(lam, U, gl, gU, n, gA, tau);
  return cudaGetLastError();
}

bool a16(const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

template <class T>
cudaError_t launch_bwd(const T* lam, const T* U, const T* gl, const T* gU, int64_t n, T* gA, T tau,
                       cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  if (a16(lam) && a16(U) && a16(gl) && a16(gU))
    return launch_one<T, true>(lam, U, gl, gU, n, gA, tau, stream);
  return launch_one<T, false>(lam, U, gl, gU, n, gA, tau, stream);
}

template cudaError_t launch_bwd<double>(const double*, const double*, const double*, const double*, int64_t,
                                        double*, double, cudaStream_t);
template cudaError_t launch_bwd<float>(const float*, const float*, const float*, const float*, int64_t, float*,
                                       float, cudaStream_t);

cudaError_t take_flags_bwd(unsigned* flags) {
  unsigned v = 0, zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_flags_bwd, sizeof(v));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(g_flags_bwd, &zero, sizeof(zero));
  *flags |= v;
  return e;
}

}  // namespace syev3
