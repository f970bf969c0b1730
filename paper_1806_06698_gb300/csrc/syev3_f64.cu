// syev3_f64.cu -- FP64 batched 3x3 symmetric eigensolver for sm_103a.
//
// One matrix per thread.  Each CTA walks tiles of kTPB packed records in a
// grid-stride loop: a 1-D bulk copy (TMA) brings the next tile's records
// into shared memory while the current tile is solved (double buffering on
// two mbarriers); results are staged in shared memory and written back with
// coalesced 16-byte stores.
//
// The per-matrix arithmetic is the method of C. F. Borges, "Solving the 3x3
// Real Symmetric Eigenproblem" (arXiv 1806.06698):
//   Sec. 1     ordered Jacobi rotation in the (1,2)-plane -> ordered arrow,
//   Sec. 1.1   h, the deflation test, the deflated 2x2 solve,
//   Sec. 1.2   mu, nu, the trace identity, the closed-form eigenvectors,
//   Sec. 1.4.1 the Borges-Gragg zero finder started from +infinity.
// Choices the paper leaves open (pre-scaling, the constants C, ordering and
// sign of the output, acceptance at the rounding level of f) are the same
// readings the CPU oracle makes; the two implementations share no code.

#include <cmath>
#include <cstdint>

#include "common.cuh"
#include "internal.h"

namespace syev3 {
namespace {

constexpr int kTPB = 128;        // matrices (threads) per tile
constexpr int kMaxIt = 64;       // zero-finder step cap
constexpr double kEps = 0x1p-52;
constexpr double kCDefl = 1.0;   // C of the deflation test (Sec. 1.1)
constexpr double kCTerm = 2.0;   // C of the stopping rule (Sec. 1.4.1)

__device__ unsigned g_flags;     // kFlagWaitTimeout when a bulk-copy wait ran out

struct Rot {
  double c, s, l1, l2;
};

// Sec. 1: ordered Jacobi rotation of [[p,q],[q,r]]; l1 >= l2, (c,s) the unit
// eigenvector of l1 and (-s,c) that of l2.  The larger eigenvalue's vector
// is built as (1,t) or (t,1) with t = q/(|d| + hypot(d,q)), |t| <= 1.
__device__ __forceinline__ Rot ordered_rotation(double p, double q, double r) {
  Rot J;
  if (q == 0.0) {
    const bool keep = p >= r;
    J.c = keep ? 1.0 : 0.0;
    J.s = keep ? 0.0 : 1.0;
    J.l1 = keep ? p : r;
    J.l2 = keep ? r : p;
    return J;
  }
  const double d = 0.5 * (p - r);
  const double rad = hypot(d, q);
  const bool right = d >= 0.0;
  const double t = q / (right ? d + rad : rad - d);
  const double hi = right ? p : r, lo = right ? r : p;
  J.l1 = fma(t, q, hi);   // rounding is monotone: l1 >= hi >= lo >= l2
  J.l2 = fma(-t, q, lo);
  const double k = rsqrt(fma(t, t, 1.0));
  J.c = right ? k : t * k;
  J.s = right ? t * k : k;
  return J;
}

// Sec. 1.4.1: zero in (0, inf) of f(x) = x - g - b1/x - b2/(x + abar) by the
// Borges-Gragg iteration started from the zero of the limit model Eq. (7).
// Accepts x_j once f/f' < C eps x_j, or when f(x_j) <= 0 or a step no longer
// decreases x (both only happen at the rounding level of f).
__device__ __forceinline__ double zero_bg(double abar, double b1, double b2, double g, bool& capped) {
  const double hg = 0.5 * g;
  const double bs = b1 + b2;
  const double rt = sqrt(fma(hg, hg, bs));
  double x = (g >= 0.0) ? hg + rt : bs / (rt - hg);
  capped = false;
  for (int it = 0;; ++it) {
    const double r1 = 1.0 / x;
    const double r2 = 1.0 / (x + abar);
    const double f = ((x - g) - b1 * r1) - b2 * r2;
    const double fp = fma(b2 * r2, r2, fma(b1 * r1, r1, 1.0));  // Eq. (3)
    if (!(f > 0.0)) break;
    if (f < (kCTerm * kEps) * x * fp) break;
    if (it >= kMaxIt) { capped = true; break; }
    const double w0 = fma(b2 * abar, r2 * r2 * r2, 1.0);       // omega_0
    const double a = -w0 * r1;                                  // Eq. (5)
    const double b = fma(f, r1, fp);
    const double q = 2.0 * f / b;                               // Eq. (6)
    const double disc = fmax(0.0, fma(2.0 * a / b, q, 1.0));
    const double xn = x - q / (1.0 + sqrt(disc));
    if (!(xn < x)) break;
    x = xn;
  }
  return x;
}

// One matrix.  a: packed (a11,a22,a33,a12,a13,a23); lam ascending; U[i*3+k]
// = component i of eigenvector k.  Returns bit 0 = capped, bit 1 = non-finite.
__device__ __forceinline__ unsigned solve3(const double a_in[6], double lam[3], double U[9]) {
  bool finite = true;
#pragma unroll
  for (int i = 0; i < 6; ++i) finite &= isfinite(a_in[i]);
  if (!finite) {
#pragma unroll
    for (int k = 0; k < 3; ++k) lam[k] = __longlong_as_double(0x7ff8000000000000LL);
#pragma unroll
    for (int k = 0; k < 9; ++k) U[k] = __longlong_as_double(0x7ff8000000000000LL);
    return 2u;
  }
  // Exact power-of-two pre-scale: largest entry in [0.5, 1).
  double amax = 0.0;
#pragma unroll
  for (int i = 0; i < 6; ++i) amax = fmax(amax, fabs(a_in[i]));
  int e = 0;
  if (amax > 0.0) frexp(amax, &e);
  double a[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) a[i] = scalbn(a_in[i], -e);

  // Sec. 1: ordered arrow [[a1,0,b1],[0,a2,b2],[b1,b2,g]].
  const Rot J = ordered_rotation(a[0], a[3], a[1]);
  const double a1 = J.l1, a2 = J.l2, g = a[2];
  const double b1 = fma(J.c, a[4], J.s * a[5]);
  const double b2 = fma(J.c, a[5], -J.s * a[4]);

  double l[3], v[3][3];
  unsigned status = 0;
  const double h = hypot(b1, b2);
  const double abar = a1 - a2;
  const double bb1 = b1 * b1, bb2 = b2 * b2;
  // Sec. 1.1: diagonal when h = 0; deflated when |abar b1 b2| <= C eps |a1+a2| h^2
  // (this "<=" also takes the exact beta- and combo-deflations) or when a
  // squared spike underflows; reduced otherwise.
  const bool diagonal = (h == 0.0);
  const bool deflated = !diagonal && ((fabs(abar * b1 * b2) <= (kCDefl * kEps) * fabs(a1 + a2) * (h * h)) ||
                                      bb1 == 0.0 || bb2 == 0.0);
  if (diagonal) {
    l[0] = a1; l[1] = a2; l[2] = g;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) v[k][i] = (i == k) ? 1.0 : 0.0;
  } else if (deflated) {
    // Sec. 1.1: G = [[b2/h,-b1/h,0],[b1/h,b2/h,0],[0,0,1]]; eigenvalue
    // (a1 b2^2 + a2 b1^2)/h^2 on G^T e1, then the 2x2 [[d2, h], [h, g]].
    const double rh = 1.0 / h;
    const double gs = b1 * rh, gc = b2 * rh;
    l[0] = fma(a1 * gc, gc, a2 * gs * gs);
    v[0][0] = gc; v[0][1] = -gs; v[0][2] = 0.0;
    const double d2 = fma(a1 * gs, gs, a2 * gc * gc);
    const Rot K = ordered_rotation(d2, h, g);
    l[1] = K.l1; l[2] = K.l2;
    v[1][0] = gs * K.c;  v[1][1] = gc * K.c;  v[1][2] = K.s;
    v[2][0] = -gs * K.s; v[2][1] = -gc * K.s; v[2][2] = K.c;
  } else {
    // Sec. 1.2: mu from A - a1 I, nu from P(a2 I - A)P (spikes swapped).
    bool cm, cn;
    const double mu = zero_bg(abar, bb1, bb2, g - a1, cm);
    const double nu = zero_bg(abar, bb2, bb1, a2 - g, cn);
    status |= (cm || cn) ? 1u : 0u;
    l[0] = a1 + mu;
    l[1] = (nu - mu) + g;   // trace identity
    l[2] = a2 - nu;
    const double mpa = mu + abar, npa = nu + abar;
    v[0][0] = b1 * mpa;         v[0][1] = b2 * mu;          v[0][2] = mu * mpa;
    v[1][0] = -(b2 * mu) * npa; v[1][1] = (b1 * nu) * mpa; v[1][2] = (b1 * b2) * abar;
    v[2][0] = b1 * nu;          v[2][1] = b2 * npa;         v[2][2] = -(nu * npa);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double inv = rsqrt(fma(v[k][0], v[k][0], fma(v[k][1], v[k][1], v[k][2] * v[k][2])));
      v[k][0] *= inv; v[k][1] *= inv; v[k][2] *= inv;
    }
  }
  // Back to the input frame: x = J v with J = [[c,-s,0],[s,c,0],[0,0,1]].
  double w[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    w[k][0] = fma(J.c, v[k][0], -J.s * v[k][1]);
    w[k][1] = fma(J.s, v[k][0], J.c * v[k][1]);
    w[k][2] = v[k][2];
  }
  // Ascending, stable (strict comparisons: equal eigenvalues keep the order
  // above), as three compare-and-swap steps on registers.
  double l0 = l[0], l1 = l[1], l2 = l[2];
  double x00 = w[0][0], x01 = w[0][1], x02 = w[0][2];
  double x10 = w[1][0], x11 = w[1][1], x12 = w[1][2];
  double x20 = w[2][0], x21 = w[2][1], x22 = w[2][2];
#define SYEV3_CSWAP(la, a0, a1, a2, lb, b0, b1, b2)      \
  if (lb < la) {                                          \
    double t_;                                            \
    t_ = la; la = lb; lb = t_;                            \
    t_ = a0; a0 = b0; b0 = t_;                            \
    t_ = a1; a1 = b1; b1 = t_;                            \
    t_ = a2; a2 = b2; b2 = t_;                            \
  }
  SYEV3_CSWAP(l0, x00, x01, x02, l1, x10, x11, x12)
  SYEV3_CSWAP(l1, x10, x11, x12, l2, x20, x21, x22)
  SYEV3_CSWAP(l0, x00, x01, x02, l1, x10, x11, x12)
#undef SYEV3_CSWAP
  const double ls[3] = {l0, l1, l2};
  const double xs[3][3] = {{x00, x01, x02}, {x10, x11, x12}, {x20, x21, x22}};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double x0 = xs[k][0], x1 = xs[k][1], x2 = xs[k][2];
    // Largest-magnitude component positive, first one on ties.
    double big = x0;
    if (fabs(x1) > fabs(big)) big = x1;
    if (fabs(x2) > fabs(x0) && fabs(x2) > fabs(x1)) big = x2;
    const double sg = (big < 0.0) ? -1.0 : 1.0;
    lam[k] = scalbn(ls[k], e);
    U[0 * 3 + k] = sg * x0;
    U[1 * 3 + k] = sg * x1;
    U[2 * 3 + k] = sg * x2;
  }
  return status;
}

template <bool kBulkIn>
__global__ void __launch_bounds__(kTPB) k_syev3_f64(const double* __restrict__ A, int64_t n,
                                                    double* __restrict__ lam_out, double* __restrict__ U_out,
                                                    unsigned long long* __restrict__ counters) {
  __shared__ alignas(16) double s_in[2][kTPB * 6];
  __shared__ alignas(16) double s_lam[kTPB * 3];
  __shared__ alignas(16) double s_U[kTPB * 9];
  __shared__ alignas(8) uint64_t s_bar[2];

  const int tid = threadIdx.x;
  const int64_t n_tiles = (n + kTPB - 1) / kTPB;
  const bool want_U = (U_out != nullptr);
  const bool vec_lam = ((reinterpret_cast<uintptr_t>(lam_out) & 15) == 0);
  const bool vec_U = want_U && ((reinterpret_cast<uintptr_t>(U_out) & 15) == 0);

  if (kBulkIn && tid == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();

  auto issue = [&](int64_t tile, int buf) {
    const int64_t base = tile * kTPB;
    const int cnt = (int)((n - base) < kTPB ? (n - base) : kTPB);
    const uint32_t bytes = (uint32_t)cnt * 48u;  // 48 = 3 * 16: always a multiple of 16
    mbar_arrive_expect_tx(&s_bar[buf], bytes);
    bulk_g2s(s_in[buf], A + base * 6, bytes, &s_bar[buf]);
  };

  uint32_t phases = 0u;  // bit b: parity of the next completion of s_bar[b]
  int buf = 0;
  int64_t tile = blockIdx.x;
  if (kBulkIn && tid == 0 && tile < n_tiles) issue(tile, 0);

  for (; tile < n_tiles; tile += gridDim.x, buf ^= 1) {
    const int64_t base = tile * kTPB;
    const int cnt = (int)((n - base) < kTPB ? (n - base) : kTPB);
    const int64_t next = tile + gridDim.x;
    if (kBulkIn) {
      if (tid == 0 && next < n_tiles) issue(next, buf ^ 1);
      const bool ok = mbar_wait(&s_bar[buf], (phases >> buf) & 1u);
      if (__syncthreads_or(!ok)) {
        // Lost wait (CTA-uniform decision): flag it, give the copies in
        // flight a second bounded chance to land so that no write into
        // shared memory outlives the CTA, and stop.
        if (tid == 0) atomicOr(&g_flags, kFlagWaitTimeout);
        mbar_wait(&s_bar[buf], (phases >> buf) & 1u);
        if (next < n_tiles) mbar_wait(&s_bar[buf ^ 1], (phases >> (buf ^ 1)) & 1u);
        return;
      }
      phases ^= 1u << buf;
    } else {
      for (int i = tid; i < cnt * 6; i += kTPB) s_in[buf][i] = A[base * 6 + i];
      __syncthreads();
    }

    double lam[3], U[9];
    unsigned st = 0;
    if (tid < cnt) {
      const double2* src = reinterpret_cast<const double2*>(&s_in[buf][tid * 6]);
      const double2 p0 = src[0], p1 = src[1], p2 = src[2];
      const double a[6] = {p0.x, p0.y, p1.x, p1.y, p2.x, p2.y};
      st = solve3(a, lam, U);
#pragma unroll
      for (int k = 0; k < 3; ++k) s_lam[tid * 3 + k] = lam[k];
#pragma unroll
      for (int k = 0; k < 9; ++k) s_U[tid * 9 + k] = U[k];
    }
    if (counters != nullptr) {
      const unsigned capped = __ballot_sync(0xffffffffu, st & 1u);
      const unsigned nonfin = __ballot_sync(0xffffffffu, st & 2u);
      if ((tid & 31) == 0) {
        if (capped) atomicAdd(&counters[0], (unsigned long long)__popc(capped));
        if (nonfin) atomicAdd(&counters[1], (unsigned long long)__popc(nonfin));
      }
    }
    __syncthreads();

    // Coalesced write-back of the tile: 16-byte stores where aligned.
    {
      double* dst = lam_out + base * 3;
      const int m = cnt * 3;
      if (vec_lam) {
        double2* d2 = reinterpret_cast<double2*>(dst);
        const double2* s2 = reinterpret_cast<const double2*>(s_lam);
        for (int i = tid; i < m / 2; i += kTPB) d2[i] = s2[i];
        if ((m & 1) && tid == 0) dst[m - 1] = s_lam[m - 1];
      } else {
        for (int i = tid; i < m; i += kTPB) dst[i] = s_lam[i];
      }
    }
    if (want_U) {
      double* dst = U_out + base * 9;
      const int m = cnt * 9;
      if (vec_U) {
        double2* d2 = reinterpret_cast<double2*>(dst);
        const double2* s2 = reinterpret_cast<const double2*>(s_U);
        for (int i = tid; i < m / 2; i += kTPB) d2[i] = s2[i];
        if ((m & 1) && tid == 0) dst[m - 1] = s_U[m - 1];
      } else {
        for (int i = tid; i < m; i += kTPB) dst[i] = s_U[i];
      }
    }
    __syncthreads();
  }
}

int blocks_per_sm_f64(bool bulk) {
  static int cached[2] = {-1, -1};
  int& c = cached[bulk ? 1 : 0];
  if (c < 0) {
    int v = 0;
    cudaError_t e = bulk ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_syev3_f64<true>, kTPB, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_syev3_f64<false>, kTPB, 0);
    c = (e == cudaSuccess && v > 0) ? v : 1;
  }
  return c;
}

}  // namespace

cudaError_t launch_f64(const double* A, int64_t n, double* lam, double* U, unsigned long long* counters,
                       cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const bool bulk = (reinterpret_cast<uintptr_t>(A) & 15) == 0;
  const int64_t n_tiles = (n + kTPB - 1) / kTPB;
  const int64_t resident = (int64_t)sms * blocks_per_sm_f64(bulk);
  const int grid = (int)(n_tiles < resident ? n_tiles : resident);
  if (bulk)
    k_syev3_f64<true><<<grid, kTPB, 0, stream>>>(A, n, lam, U, counters);
  else
    k_syev3_f64<false><<<grid, kTPB, 0, stream>>>(A, n, lam, U, counters);
  return cudaGetLastError();
}

cudaError_t take_flags_f64(unsigned* flags) {
  unsigned v = 0, zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_flags, sizeof(v));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(g_flags, &zero, sizeof(zero));
  *flags |= v;
  return e;
}

}  // namespace syev3
