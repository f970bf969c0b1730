// syev3_f64.cu -- FP64 batched 3x3 symmetric eigensolver for sm_103a.
//
// The per-matrix arithmetic is the method of C. F. Borges, "Solving the 3x3
// Real Symmetric Eigenproblem" (arXiv 1806.06698):
//   Sec. 1     ordered Jacobi rotation in the (1,2)-plane -> ordered arrow,
//   Sec. 1.1   h, the deflation test, the deflated 2x2 solve,
//   Sec. 1.2   mu, nu, the trace identity, the closed-form eigenvectors,
//   Sec. 1.4.1 the Borges-Gragg zero finder and its stopping rule.
// Choices the paper leaves open (pre-scaling, tiny spikes, the constants C,
// order and sign of the output, acceptance at the rounding level of f) are
// the readings the CPU oracle makes; the two implementations share no code.
//
// GB300 executes 2 FP64 lanes per SM per clock (1/64 of FP32), so this
// solver is bound by the FP64 pipe, not by HBM.  The kernel is built to spend
// as few FP64 lane-slots per matrix as the method allows:
//  * one matrix per thread; tiles of kTPB packed records arrive by 1-D bulk
//    copy (TMA) into shared memory, double-buffered on two mbarriers, and
//    leave through shared-memory staging with 16-byte stores;
//  * both shifted roots mu and nu are first located in FP32 by the same
//    Borges-Gragg iteration (on the 64x faster pipe), moved right of the root
//    by a bound on the FP32 error, then finished in FP64 by one Borges-Gragg
//    step and the paper's stopping test;
//  * the roots that do not pass (clustered spectra whose root is below FP32
//    resolution, tiny spikes) are compacted with warp ballots into a
//    shared-memory work list and finished by the full FP64 iteration, so that
//    their extra steps occupy ceil(k/32) warps instead of every warp;
//  * reciprocals come from the hardware's 2^-20 estimate and one cubic
//    Newton-Raphson step (<= 1 ulp) instead of IEEE division.

#include <cmath>
#include <cstdint>

#include "common.cuh"
#include "internal.h"

namespace syev3 {
namespace {

constexpr int kTPB = 128;        // matrices (threads) per tile
constexpr int kMaxIt = 64;       // zero-finder step cap
constexpr int kSeedIt = 16;      // FP32 seeding step cap
constexpr double kEps = 0x1p-52;
constexpr double kCDefl = 1.0;   // C of the deflation test (Sec. 1.1)
constexpr double kCTerm = 2.0;   // C of the stopping rule (Sec. 1.4.1)
constexpr double kTinySpike = 0x1p-480;  // spikes below this are zeroed (beta-deflation)
constexpr float kEps32 = 0x1p-23f;

constexpr int kDiagonal = 0, kDeflated = 1, kReduced = 2, kNonFinite = 3, kIdle = 4;

__device__ unsigned g_flags;     // kFlagWaitTimeout when a bulk-copy wait ran out

// ---------------------------------------------------------------------------
// Arithmetic primitives
// ---------------------------------------------------------------------------

// 1/x: hardware estimate (relative error 2^-20) refined by one cubic
// Newton-Raphson step, e = 1 - x y, y <- y (1 + e + e^2) (error e^3 ~ 2^-60);
// within 1 ulp for 2^-1000 < |x| < 2^1000.
__device__ __forceinline__ double rcp64(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

__device__ __forceinline__ float rcp32(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float sqrt32(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 2^k for -1022 <= k <= 1023, built from its exponent field.
__device__ __forceinline__ double pow2(int k) { return __hiloint2double((k + 1023) << 20, 0); }

// ---------------------------------------------------------------------------
// Sec. 1: ordered Jacobi rotation of [[p,q],[q,r]]; l1 >= l2, (c,s) the unit
// eigenvector of l1 and (-s,c) that of l2.  The larger eigenvalue's vector
// is (1,t) or (t,1) with t = q/(|d| + hypot(d,q)), d = (p-r)/2, |t| <= 1.
// ---------------------------------------------------------------------------

struct Rot {
  double c, s, l1, l2;
};

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
  const double D = p - r, q2 = q + q;
  const double rad = sqrt(fma(D, D, q2 * q2));  // 2 hypot(d, q)
  const double den = fabs(D) + rad;
  double t;
  if (den >= 0x1p-1000)
    t = q2 * rcp64(den);
  else
    t = (den > 0.0) ? q2 / den : copysign(1.0, q);
  const bool right = D >= 0.0;
  const double hi = right ? p : r, lo = right ? r : p;
  J.l1 = fma(t, q, hi);  // rounding is monotone: l1 >= hi >= lo >= l2
  J.l2 = fma(-t, q, lo);
  const double k = rsqrt(fma(t, t, 1.0));
  J.c = right ? k : t * k;
  J.s = right ? t * k : k;
  return J;
}

// ---------------------------------------------------------------------------
// Zero finding on a fully reduced arrow (Sec. 1.4): the zero in (0, inf) of
// f(x) = x - g - b1/x - b2/(x + ab), b1 = beta1^2, b2 = beta2^2, ab = abar.
// ---------------------------------------------------------------------------

// For x < ab the spectral function is evaluated as
//   f(x) = x + K - b1/x + c x/(x + ab),   c = b2/ab,  K = -g - c,
// which equals x - g - b1/x - b2/(x + ab) but has no cancellation between
// O(1) terms when the root is small (c and K are formed once in FP64).  For
// x >= ab the printed form is used: there c x/(x + ab) ~ c can be far larger
// than b2/(x + ab), while for x < ab the printed form already carries a term
// b2/(x + ab) > c/2, so the choice is never the less accurate one.
// f'(x) = 1 + b1/x^2 + b2/(x + ab)^2 (Eq. (3)) and omega_0 are unchanged.

// FP32 Borges-Gragg pass for two problems at once (mu and nu), started from
// the zero of the limit model Eq. (7).  Each returned start lies right of
// its root by a bound on the FP32 error (checked again in FP64).
__device__ __forceinline__ void seed32x2(const float ab, const float b1[2], const float b2[2], const float g[2],
                                         const float c[2], const float K[2], float out[2]) {
  float x[2];
  bool live[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float hg = 0.5f * g[k], bs = b1[k] + b2[k];
    const float rt = sqrt32(fmaf(hg, hg, bs));
    x[k] = (g[k] >= 0.f) ? hg + rt : bs * rcp32(rt - hg);
    live[k] = true;
    out[k] = 0.f;
  }
#pragma unroll 1
  for (int it = 0; it <= kSeedIt && (live[0] || live[1]); ++it) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (!live[k]) continue;
      const float r1 = rcp32(x[k]), r2 = rcp32(x[k] + ab);
      const float t1 = b1[k] * r1, t2 = b2[k] * r2;
      const bool small = x[k] < ab;
      const float lead = small ? K[k] : -g[k];
      const float u = small ? c[k] * x[k] * r2 : -t2;
      const float f = ((x[k] + lead) - t1) + u;
      const float fp = fmaf(t2, r2, fmaf(t1, r1, 1.f));
      bool done = !(f > (4.f * kEps32) * x[k] * fp) || it == kSeedIt;
      float xn = x[k];
      if (!done) {
        const float w0 = fmaf(t2 * ab, r2 * r2, 1.f);
        const float rb = rcp32(fmaf(f, r1, fp));
        const float fr = f * rb;
        const float z = (-4.f * w0) * (r1 * rb) * fr;
        const float delta = 2.f * fr * rcp32(1.f + sqrt32(fmaxf(0.f, 1.f + z)));
        if (delta < 0.5f * x[k]) {
          xn = x[k] - delta;
        } else {  // zero of phi_j far below x: solve omega_0 x^2 - sigma x - omega_1 = 0 directly
          const float xr = x[k] * r2;
          const float w1 = fmaf(b2[k] * xr, xr * xr, b1[k]);
          const float sg = fmaf(w0, x[k], -fmaf(w1, r1, f));
          const float rt = sqrt32(fmaf(sg, sg, 4.f * w0 * w1));
          xn = (sg > 0.f) ? (sg + rt) * rcp32(2.f * w0) : (2.f * w1) * rcp32(rt - sg);
        }
        done = !(xn < x[k]);
      }
      if (done) {
        // Distance to the root: |f|/f' plus the FP32 rounding of f and of
        // its data (about 10 eps32 of its terms), doubled.
        const float err = 10.f * kEps32 * (x[k] + fabsf(lead) + t1 + fabsf(u));
        out[k] = x[k] + 2.f * (fabsf(f) + err) * rcp32(fp);
        live[k] = false;
      } else {
        x[k] = xn;
      }
    }
  }
}

// FP64 finish of one root from a start x right of it: one Borges-Gragg step
// (Eqs. (5), (6)) and the stopping rule of Sec. 1.4.1 at the new iterate.
// Returns 0 when x holds the accepted root, 1 when x holds an iterate still
// right of the root (more steps needed), 2 when the start was not right of
// the root.
__device__ __forceinline__ int finish64(const double ab, const double b1, const double b2, const double g,
                                        const double c, const double K, double& x) {
  const bool small = x < ab;  // choice of the evaluation form (see above)
  const double lead = small ? K : -g;
  double r1 = rcp64(x), r2 = rcp64(x + ab);
  double t1 = b1 * r1, t2 = b2 * r2;
  double f = ((x + lead) - t1) + (small ? c * x * r2 : -t2);
  double fp = fma(t2, r2, fma(t1, r1, 1.0));  // Eq. (3)
  if (!(f > 0.0)) return 2;
  const double w0 = fma(t2 * ab, r2 * r2, 1.0);  // omega_0
  const double rb = rcp64(fma(f, r1, fp));       // 1/b, b = f' + f/x
  const double fr = f * rb;                      // q/2 = f/b
  const double z = (-4.0 * w0) * (r1 * rb) * fr; // (2a/b) q, a = -omega_0/x
  // Delta = q/(1 + sqrt(1+z)) = fr * S(z); S = 2/(1+sqrt(1+z)) = 1 - z/4 + z^2/8 - ...
  const double S = (fabs(z) < 0x1p-12) ? fma(z, fma(z, 0.125, -0.25), 1.0)
                                       : 2.0 / (1.0 + sqrt(fmax(0.0, 1.0 + z)));
  const double delta = fr * S;
  if (!(delta < 0.5 * x)) return 1;  // zero of phi_j far below x: leave it to the full iteration
  const double xn = x - delta;
  if (!(xn < x)) return 0;  // the step no longer moves x: rounding level
  x = xn;
  r1 = rcp64(x);
  r2 = rcp64(x + ab);
  t1 = b1 * r1;
  t2 = b2 * r2;
  f = ((x + lead) - t1) + (small ? c * x * r2 : -t2);
  fp = fma(t2, r2, fma(t1, r1, 1.0));
  if (!(f > 0.0)) return 0;                       // at or past the root: rounding level
  if (f < (kCTerm * kEps) * x * fp) return 0;     // f/f' < C eps x
  return 1;
}

// Full FP64 Borges-Gragg iteration (IEEE arithmetic, any data) from x0 > 0
// right of the root, or from the start of Eq. (7) when x0 <= 0.  The next
// iterate is x - Delta (Eq. (6)), or the zero of phi_j taken directly when
// Delta >= x/2.
__device__ double zero_bg_full(double ab, double b1, double b2, double g, double x, bool& capped) {
  if (!(x > 0.0)) {
    const double hg = 0.5 * g, bs = b1 + b2;
    const double rt = sqrt(fma(hg, hg, bs));
    x = (g >= 0.0) ? hg + rt : bs / (rt - hg);
  }
  const double c = b2 / ab, K = -g - c;  // f = x + K - b1/x + c x/(x + ab)
  capped = false;
  for (int it = 0;; ++it) {
    const double r1 = 1.0 / x, r2 = 1.0 / (x + ab);
    const double t1 = b1 * r1, t2 = b2 * r2;
    const bool small = x < ab;
    const double f = ((x + (small ? K : -g)) - t1) + (small ? c * x * r2 : -t2);
    const double fp = fma(t2, r2, fma(t1, r1, 1.0));
    if (!(f > 0.0)) break;
    if (f < (kCTerm * kEps) * x * fp) break;
    if (it >= kMaxIt) {
      capped = true;
      break;
    }
    const double w0 = fma(t2 * ab, r2 * r2, 1.0);
    const double b = fma(f, r1, fp);
    const double q = 2.0 * f / b;
    const double disc = fmax(0.0, fma((-2.0 * w0 * r1) / b, q, 1.0));
    const double delta = q / (1.0 + sqrt(disc));
    double xn;
    if (delta < 0.5 * x) {
      xn = x - delta;
    } else {
      // x_{j+1} is the zero of phi_j; far below x_j the difference x_j - Delta
      // cancels, so take it from omega_0 x^2 - sigma x - omega_1 = 0 directly.
      const double xr = x * r2;
      const double w1 = fma(b2 * xr, xr * xr, b1);
      const double sg = fma(w0, x, -fma(w1, r1, f));
      const double rt = sqrt(fma(sg, sg, 4.0 * w0 * w1));
      xn = (sg > 0.0) ? (sg + rt) / (2.0 * w0) : (2.0 * w1) / (rt - sg);
    }
    if (!(xn < x)) break;
    x = xn;
  }
  return x;
}

// ---------------------------------------------------------------------------
// Per-matrix state between the phases of a tile
// ---------------------------------------------------------------------------

struct Lane {
  double a1, a2, b1, b2, g, c, s;  // ordered arrow and its rotation (pre-scaled frame)
  double unscale;                  // 2^e (fast path), or 0 -> use scalbn(., e)
  int e;
  int cls;
};

// Phase A: pre-scale, Sec. 1 arrow reduction, Sec. 1.1 classification.
__device__ __forceinline__ Lane make_lane(const double a_in[6]) {
  Lane L;
  int E = 0;
  bool finite = true;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const int ex = (__double2hiint(a_in[i]) >> 20) & 0x7ff;
    finite &= (ex != 0x7ff);
    E = max(E, ex);
  }
  if (!finite) {
    L.cls = kNonFinite;
    return L;
  }
  // Exact power-of-two pre-scale: the largest entry lands in [0.5, 1).
  double a[6];
  if (E >= 1 && E <= 2044) {
    L.e = E - 1022;
    const double sc = pow2(-L.e);
#pragma unroll
    for (int i = 0; i < 6; ++i) a[i] = a_in[i] * sc;
    L.unscale = pow2(L.e);
  } else {  // zero, subnormal or huge entries
    double amax = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) amax = fmax(amax, fabs(a_in[i]));
    int e = 0;
    if (amax > 0.0) frexp(amax, &e);
    L.e = e;
#pragma unroll
    for (int i = 0; i < 6; ++i) a[i] = scalbn(a_in[i], -e);
    L.unscale = 0.0;
  }
  const Rot J = ordered_rotation(a[0], a[3], a[1]);
  L.a1 = J.l1;
  L.a2 = J.l2;
  L.c = J.c;
  L.s = J.s;
  L.g = a[2];
  double b1 = fma(J.c, a[4], J.s * a[5]);
  double b2 = fma(J.c, a[5], -J.s * a[4]);
  if (fabs(b1) < kTinySpike) b1 = 0.0;  // exact beta-deflation of a negligible spike
  if (fabs(b2) < kTinySpike) b2 = 0.0;
  L.b1 = b1;
  L.b2 = b2;
  const double abar = L.a1 - L.a2;
  const double h2 = fma(b1, b1, b2 * b2);
  if (h2 == 0.0)
    L.cls = kDiagonal;
  else if (fabs(abar * b1 * b2) <= (kCDefl * kEps) * fabs(L.a1 + L.a2) * h2)
    L.cls = kDeflated;  // also the exact beta- and combo-deflations
  else
    L.cls = kReduced;
  return L;
}

// Phase E: eigenpairs in the arrow frame, back-transform, sort, sign,
// unscale; writes lam[3] and U[9] (U[i*3+k] = component i of vector k).
__device__ __forceinline__ void finish_lane(const Lane& L, double mu, double nu, double lam[3], double U[9]) {
  const double a1 = L.a1, a2 = L.a2, b1 = L.b1, b2 = L.b2, g = L.g;
  double l[3], v[3][3];
  if (L.cls == kDiagonal) {
    l[0] = a1; l[1] = a2; l[2] = g;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) v[k][i] = (i == k) ? 1.0 : 0.0;
  } else if (L.cls == kDeflated) {
    // Sec. 1.1: G = [[b2/h,-b1/h,0],[b1/h,b2/h,0],[0,0,1]]; eigenvalue
    // (a1 b2^2 + a2 b1^2)/h^2 on G^T e1, then the 2x2 [[d2, h], [h, g]].
    const double h2 = fma(b1, b1, b2 * b2);
    const double rh = rsqrt(h2), h = h2 * rh;
    const double gs = b1 * rh, gc = b2 * rh;
    l[0] = fma(a1 * gc, gc, a2 * gs * gs);
    v[0][0] = gc; v[0][1] = -gs; v[0][2] = 0.0;
    const double d2 = fma(a1 * gs, gs, a2 * gc * gc);
    const Rot K = ordered_rotation(d2, h, g);
    l[1] = K.l1; l[2] = K.l2;
    v[1][0] = gs * K.c;  v[1][1] = gc * K.c;  v[1][2] = K.s;
    v[2][0] = -gs * K.s; v[2][1] = -gc * K.s; v[2][2] = K.c;
  } else {
    // Sec. 1.2: lambda1 = a1 + mu, lambda3 = a2 - nu, trace identity for
    // lambda2; closed-form u1, u2, u3, each normalised.
    const double abar = a1 - a2;
    l[0] = a1 + mu;
    l[1] = (nu - mu) + g;
    l[2] = a2 - nu;
    const double mpa = mu + abar, npa = nu + abar;
    v[0][0] = b1 * mpa;         v[0][1] = b2 * mu;         v[0][2] = mu * mpa;
    v[1][0] = -(b2 * mu) * npa; v[1][1] = (b1 * nu) * mpa; v[1][2] = (b1 * b2) * abar;
    v[2][0] = b1 * nu;          v[2][1] = b2 * npa;        v[2][2] = -(nu * npa);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double ss = fma(v[k][0], v[k][0], fma(v[k][1], v[k][1], v[k][2] * v[k][2]));
      if (!(ss >= 0x1p-1000)) {
        // Squares near underflow (u2 ~ beta^3 when mu and nu are both tiny):
        // bring the largest component to [0.5, 1) by an exact power of two.
        int E = 1;
#pragma unroll
        for (int i = 0; i < 3; ++i) E = max(E, (__double2hiint(v[k][i]) >> 20) & 0x7ff);
        const double sc = pow2(1022 - E);
        v[k][0] *= sc; v[k][1] *= sc; v[k][2] *= sc;
        ss = fma(v[k][0], v[k][0], fma(v[k][1], v[k][1], v[k][2] * v[k][2]));
      }
      const double inv = rsqrt(ss);
      v[k][0] *= inv; v[k][1] *= inv; v[k][2] *= inv;
    }
  }
  // Input frame: x = J v with J = [[c,-s,0],[s,c,0],[0,0,1]].
  double x00 = fma(L.c, v[0][0], -L.s * v[0][1]), x01 = fma(L.s, v[0][0], L.c * v[0][1]), x02 = v[0][2];
  double x10 = fma(L.c, v[1][0], -L.s * v[1][1]), x11 = fma(L.s, v[1][0], L.c * v[1][1]), x12 = v[1][2];
  double x20 = fma(L.c, v[2][0], -L.s * v[2][1]), x21 = fma(L.s, v[2][0], L.c * v[2][1]), x22 = v[2][2];
  double l0 = l[0], l1 = l[1], l2 = l[2];
  // Ascending and stable (strict comparisons keep equal eigenvalues in the
  // order above): three compare-and-swap steps on registers.
#define SYEV3_CSWAP(la, a0, a1_, a2_, lb, b0, b1_, b2_) \
  if (lb < la) {                                       \
    double t_;                                         \
    t_ = la; la = lb; lb = t_;                         \
    t_ = a0; a0 = b0; b0 = t_;                         \
    t_ = a1_; a1_ = b1_; b1_ = t_;                     \
    t_ = a2_; a2_ = b2_; b2_ = t_;                     \
  }
  SYEV3_CSWAP(l0, x00, x01, x02, l1, x10, x11, x12)
  SYEV3_CSWAP(l1, x10, x11, x12, l2, x20, x21, x22)
  SYEV3_CSWAP(l0, x00, x01, x02, l1, x10, x11, x12)
#undef SYEV3_CSWAP
  const double ls[3] = {l0, l1, l2};
  const double xs[3][3] = {{x00, x01, x02}, {x10, x11, x12}, {x20, x21, x22}};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double y0 = xs[k][0], y1 = xs[k][1], y2 = xs[k][2];
    // Largest-magnitude component positive, first one on ties.
    double big = y0;
    if (fabs(y1) > fabs(big)) big = y1;
    if (fabs(y2) > fabs(y0) && fabs(y2) > fabs(y1)) big = y2;
    const double sg = (big < 0.0) ? -1.0 : 1.0;
    lam[k] = (L.unscale != 0.0) ? ls[k] * L.unscale : scalbn(ls[k], L.e);
    U[0 * 3 + k] = sg * y0;
    U[1 * 3 + k] = sg * y1;
    U[2 * 3 + k] = sg * y2;
  }
}

// ---------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------

template <bool kBulkIn>
__global__ void __launch_bounds__(kTPB) k_syev3_f64(const double* __restrict__ A, int64_t n,
                                                    double* __restrict__ lam_out, double* __restrict__ U_out,
                                                    unsigned long long* __restrict__ counters) {
  __shared__ alignas(16) double s_in[2][kTPB * 6];
  __shared__ alignas(16) double s_lam[kTPB * 3];
  __shared__ alignas(16) double s_U[kTPB * 9];
  // Work list of roots left for the full FP64 iteration: up to two per lane.
  __shared__ double s_hx[2 * kTPB], s_hab[2 * kTPB], s_hb1[2 * kTPB], s_hb2[2 * kTPB], s_hg[2 * kTPB];
  __shared__ int s_nhard;
  __shared__ alignas(8) uint64_t s_bar[2];

  const int tid = threadIdx.x, lane_id = tid & 31;
  const unsigned lt_mask = (1u << lane_id) - 1u;
  const int64_t n_tiles = (n + kTPB - 1) / kTPB;
  const bool want_U = (U_out != nullptr);
  const bool vec_lam = ((reinterpret_cast<uintptr_t>(lam_out) & 15) == 0);
  const bool vec_U = want_U && ((reinterpret_cast<uintptr_t>(U_out) & 15) == 0);

  if (tid == 0) {
    s_nhard = 0;
    if (kBulkIn) {
      mbar_init(&s_bar[0], 1);
      mbar_init(&s_bar[1], 1);
      fence_mbar_init();
    }
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

    // Phase A: arrow and class.
    Lane L;
    L.cls = kIdle;
    if (tid < cnt) {
      const double2* src = reinterpret_cast<const double2*>(&s_in[buf][tid * 6]);
      const double2 p0 = src[0], p1 = src[1], p2 = src[2];
      const double a[6] = {p0.x, p0.y, p1.x, p1.y, p2.x, p2.y};
      L = make_lane(a);
    }

    // Phases B, C: FP32 seeds, then one FP64 step and the stopping test.
    // Problem 0 is mu (A - a1 I), problem 1 is nu (P(a2 I - A)P: spikes
    // swapped), Sec. 1.2.
    const bool reduced = (L.cls == kReduced);
    double root[2] = {0.0, 0.0};
    bool hard[2] = {false, false};
    double ab = 0.0, pb1[2] = {0.0, 0.0}, pb2[2] = {0.0, 0.0}, pg[2] = {0.0, 0.0};
    if (reduced) {
      ab = L.a1 - L.a2;
      const double bb1 = L.b1 * L.b1, bb2 = L.b2 * L.b2;
      pb1[0] = bb1; pb2[0] = bb2; pg[0] = L.g - L.a1;
      pb1[1] = bb2; pb2[1] = bb1; pg[1] = L.a2 - L.g;
      // FP32 can carry the problem when its data are normal FP32 numbers.
      const bool fp32_ok = bb1 >= 0x1p-100 && bb2 >= 0x1p-100 && ab >= 0x1p-100;
      float sd[2] = {0.f, 0.f};
      double pc[2] = {0.0, 0.0}, pK[2] = {0.0, 0.0};
      if (fp32_ok) {
        const double rab = rcp64(ab);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          pc[k] = pb2[k] * rab;
          pK[k] = -pg[k] - pc[k];
        }
        const float fb1[2] = {(float)pb1[0], (float)pb1[1]}, fb2[2] = {(float)pb2[0], (float)pb2[1]};
        const float fg[2] = {(float)pg[0], (float)pg[1]};
        const float fc[2] = {(float)pc[0], (float)pc[1]}, fK[2] = {(float)pK[0], (float)pK[1]};
        seed32x2((float)ab, fb1, fb2, fg, fc, fK, sd);
      }
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        double x = (double)sd[k];
        int st = 2;
        if (x >= 0x1p-900 && x <= 0x1p+100) st = finish64(ab, pb1[k], pb2[k], pg[k], pc[k], pK[k], x);
        root[k] = (st == 2) ? 0.0 : x;  // 0: restart from Eq. (7)
        hard[k] = (st != 0);
      }
    }

    // Phase D: compact the unfinished roots into the shared work list and
    // finish them with every lane of the CTA available.
    int slot[2] = {-1, -1};
    {
      const unsigned m0 = __ballot_sync(0xffffffffu, hard[0]);
      const unsigned m1 = __ballot_sync(0xffffffffu, hard[1]);
      const int total = __popc(m0) + __popc(m1);
      int wbase = 0;
      if (lane_id == 0 && total) wbase = atomicAdd(&s_nhard, total);
      wbase = __shfl_sync(0xffffffffu, wbase, 0);
      if (hard[0]) slot[0] = wbase + __popc(m0 & lt_mask);
      if (hard[1]) slot[1] = wbase + __popc(m0) + __popc(m1 & lt_mask);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        if (slot[k] >= 0) {
          s_hx[slot[k]] = root[k];
          s_hab[slot[k]] = ab;
          s_hb1[slot[k]] = pb1[k];
          s_hb2[slot[k]] = pb2[k];
          s_hg[slot[k]] = pg[k];
        }
      }
    }
    __syncthreads();
    const int n_hard = s_nhard;
    bool capped = false;
    for (int i = tid; i < n_hard; i += kTPB) {
      bool cp;
      s_hx[i] = zero_bg_full(s_hab[i], s_hb1[i], s_hb2[i], s_hg[i], s_hx[i], cp);
      capped |= cp;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 2; ++k)
      if (slot[k] >= 0) root[k] = s_hx[slot[k]];

    // Phase E: eigenpairs, staged for the write-back.
    bool nonfinite = false;
    if (L.cls != kIdle) {
      double lam[3], U[9];
      if (L.cls == kNonFinite) {
        nonfinite = true;
        const double qnan = __longlong_as_double(0x7ff8000000000000LL);
#pragma unroll
        for (int k = 0; k < 3; ++k) lam[k] = qnan;
#pragma unroll
        for (int k = 0; k < 9; ++k) U[k] = qnan;
      } else {
        finish_lane(L, root[0], root[1], lam, U);
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) s_lam[tid * 3 + k] = lam[k];
#pragma unroll
      for (int k = 0; k < 9; ++k) s_U[tid * 9 + k] = U[k];
    }
    if (counters != nullptr) {
      const unsigned cm = __ballot_sync(0xffffffffu, capped);
      const unsigned nf = __ballot_sync(0xffffffffu, nonfinite);
      if (lane_id == 0) {
        if (cm) atomicAdd(&counters[0], (unsigned long long)__popc(cm));
        if (nf) atomicAdd(&counters[1], (unsigned long long)__popc(nf));
      }
    }
    __syncthreads();
    if (tid == 0) s_nhard = 0;

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
