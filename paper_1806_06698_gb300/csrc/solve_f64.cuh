// solve_f64.cuh -- per-matrix FP64 steps of the method of C. F. Borges,
// "Solving the 3x3 Real Symmetric Eigenproblem" (arXiv 1806.06698), shared
// by the FP64 solve kernel and the FP64 refinement of the FP32 kernels.
//   Sec. 1     ordered Jacobi rotation in the (1,2)-plane -> ordered arrow,
//   Sec. 1.1   h, the deflation test, the deflated 2x2 solve,
//   Sec. 1.2   mu, nu, the trace identity, the closed-form eigenvectors,
//   Sec. 1.4.1 the Borges-Gragg zero finder and its stopping rule.
// Choices the paper leaves open (pre-scaling, tiny spikes, the constants C,
// order and sign of the output, acceptance at the rounding level of f) are
// the readings the CPU oracle makes; the two implementations share no code.
#pragma once

#include <cmath>
#include <cstdint>

#include "arith.cuh"

namespace syev3 {
namespace f64 {
namespace {  // internal linkage: every translation unit gets its own copy
constexpr int kMaxIt = 64;       // zero-finder step cap
constexpr int kSeedIt = 16;      // FP32 seeding step cap
constexpr double kEps = 0x1p-52;
constexpr double kCDefl = 1.0;   // C of the deflation test (Sec. 1.1)
constexpr double kCTerm = 2.0;   // C of the stopping rule (Sec. 1.4.1)
constexpr int kTinySpikeExp = -480;  // spikes below 2^-480 are zeroed (beta-deflation)
constexpr float kEps32 = 0x1p-23f;

constexpr int kDiagonal = 0, kDeflated = 1, kReduced = 2, kNonFinite = 3, kIdle = 4;


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
  if (is_zero(q)) {
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
  if (hi_mag(den) >= hi_pow2(-1000))  // den >= 2^-1000 (den >= 0)
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

// Start of the Borges-Gragg iteration (FP32).  Sec. 1.4.1 starts from the
// zero x7 of the limit model Eq. (7), right of the root.  For a root far
// below abar (clustered spectra, small spikes) x7 can be many orders of
// magnitude too large, and the iteration then needs 5-10 steps to come down.
// Near 0, f(x) = (1 + c/ab) x + K - b1/x - c x^2/(ab (x+ab)) + ..., so the
// zero xm of (1 + c/ab) x^2 + K x - b1 lies just left of the root, by about
// c xm^2 / (ab^2 f'(xm)); twice that (plus 2^-20 xm) moves it right.  That
// start is used when it lies below x7 and xm < ab/16; the caller restarts
// from x7 if f is not positive there.  Returns the start, sets x7.
__device__ __forceinline__ float start32(const float ab, const float b1, const float b2, const float g,
                                        const float c, const float K, float& x7, bool& from_model) {
  const float hg = 0.5f * g, bs = b1 + b2;
  const float rt = sqrt32(fmaf(hg, hg, bs));
  x7 = (g >= 0.f) ? hg + rt : bs * rcp32(rt - hg);
  const float c2 = fmaf(c, rcp32(ab), 1.f);
  const float disc = sqrt32(fmaf(K, K, 4.f * c2 * b1));
  const float xm = (K >= 0.f) ? 2.f * b1 * rcp32(K + disc) : (disc - K) * rcp32(2.f * c2);
  const float r1 = rcp32(xm), r2 = rcp32(xm + ab);
  const float fpm = fmaf(b2 * r2, r2, fmaf(b1 * r1, r1, 1.f));
  const float x0 = xm + fmaf(2.f * c * xm * xm, rcp32(ab * ab * fpm), 0x1p-20f * xm);
  from_model = (xm > 0.f) && (xm < 0.0625f * ab) && (x0 < x7);
  return from_model ? x0 : x7;
}

// FP32 Borges-Gragg pass for two problems at once (mu and nu), started by
// start32 (the zero of the limit model Eq. (7), or the small-root model).  Each returned start lies right of
// its root by a bound on the FP32 error (checked again in FP64).
__device__ __forceinline__ void seed32x2(const float ab, const float b1[2], const float b2[2], const float g[2],
                                         const float c[2], const float K[2], float out[2]) {
  float x[2], x7[2];
  bool live[2], model[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    x[k] = start32(ab, b1[k], b2[k], g[k], c[k], K[k], x7[k], model[k]);
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
      if (model[k]) {  // first evaluation at the small-root start: keep it only if right of the root
        model[k] = false;
        if (!(f > 0.f)) {
          x[k] = x7[k];
          continue;
        }
      }
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
                                        const double c, const double K, const float abf, const float b1f,
                                        const float b2f, double& x) {
  // x >= 2^-900, ab >= 2^-100 and b1, b2 >= 2^-120 (checked by the caller;
  // abf, b1f, b2f are ab, b1, b2 rounded to FP32): every quantity compared below is a normal
  // positive number or a finite f, so the comparisons run on bit patterns
  // (see arith.cuh).
  const bool small = dbits(x) < dbits(ab);  // x < ab: choice of the evaluation form (see above)
  const double lead = small ? K : -g;
  double r1 = rcp64(x), r2 = rcp64(x + ab);
  double t1 = b1 * r1, t2 = b2 * r2;
  double f = ((x + lead) - t1) + (small ? c * x * r2 : -t2);
  const double t1r = t1 * r1, t2r = t2 * r2;  // b1/x^2, b2/(x+ab)^2
  const double fp = (1.0 + t1r) + t2r;        // Eq. (3)
  if (!is_pos(f)) return 2;
  // The step of Eqs. (5), (6): Delta = (f/b) S(z) with b = f' + f/x,
  // z = -4 omega_0 f / (x b^2) and S(z) = 2/(1 + sqrt(1 + z)).  Only f/b is
  // needed to FP64 accuracy: an FP32 reciprocal of b and one correction give
  // it to 2^-46.  From a start within FP32 accuracy of the root |z| is tiny
  // and S - 1 = -z/4 + z^2/8 - ... (about z/4) is formed in FP32; a start
  // with |z| >= 2^-12, or with b beyond FP32 range, is left to the full
  // iteration.
  const double b = fma(f, r1, fp);
  if (hi_mag(b) >= hi_pow2(126)) return 1;  // b >= 2^126 (b >= 1 always)
  const float rbf = rcp32(d2f_rn(b));
  const double rbd = f2d_exact(rbf);
  const double q0 = f * rbd;
  const double fr = fma(fma(-b, q0, f), rbd, q0);  // f/b
  const float xf = d2f_rn(x), r1f = rcp32(xf), r2f = rcp32(xf + abf);
  const float w0f = fmaf(b2f * r2f * abf, r2f * r2f, 1.f);  // omega_0
  const float zf = (-4.f * w0f) * (r1f * rbf) * d2f_rn(fr);
  if (!(fabsf(zf) < 0x1p-12f)) return 1;
  const double delta = fma(fr, f2d_exact(zf * fmaf(zf, 0.125f, -0.25f)), fr);
  // delta >= x/2: the zero of phi_j is far below x; leave it to the full iteration.
  if (dbits(delta) >= dbits(x) - (1ull << 52)) return 1;
  const double xn = x - delta;
  if (!(dbits(xn) < dbits(x))) return 0;  // the step no longer moves x: rounding level
  if (dbits(delta) <= dbits(x) - (16ull << 52)) {
    // delta <= 2^-16 x (every step from an FP32 start in practice): f at
    // the new iterate from Taylor's formula about x to third order,
    //   f(xn) = f - delta f1 + delta^2 f2/2 - delta^3 f3/6 + delta^4 f4(xi)/24,
    // with f1 = f', f2 = -2 (b1/x^3 + b2/(x+ab)^3), f3 = 6 (b1/x^4 +
    // b2/(x+ab)^4) and |f4| <= 24 f1/x^3 (1 + 2^-13) on [xn, x]: the dropped
    // term is below 2^-64 x f1, far under the stopping threshold, and the
    // rounding error of this form is that of f itself (the leading terms
    // cancel to the size of the next).  The threshold uses f1(x) <= f1(xn):
    // at most 2^-15 stricter.
    const double s1 = t1r * r1, s2 = t2r * r2;  // b1/x^3, b2/(x+ab)^3
    const double hc = fma(s1, fma(delta, r1, 1.0), s2 * fma(delta, r2, 1.0));
    const double fn = fma(-(delta * delta), hc, fma(-delta, fp, f));
    x = xn;
    if (!is_pos(fn)) return 0;  // at or past the root: rounding level
    if (dbits(fn) < dbits(x * fp) - (51ull << 52)) return 0;  // f/f1 < 2^-51 x (Sec. 1.4.1)
    return 1;
  }
  x = xn;
  r1 = rcp64(x);
  r2 = rcp64(x + ab);
  t1 = b1 * r1;
  t2 = b2 * r2;
  f = ((x + lead) - t1) + (small ? c * x * r2 : -t2);
  if (!is_pos(f)) return 0;  // at or past the root: rounding level
  // f/f' < C eps x with C eps = 2^-51: f < 2^-51 (x f'), the product normal.
  // f' only scales the threshold: FP32 is enough, capped at 2^120 (an f'
  // under the true one, or an FP32 x that underflowed, only makes the test
  // stricter and leaves the root to the full iteration).
  const float xf2 = d2f_rn(x), q1 = rcp32(xf2), q2 = rcp32(xf2 + abf);
  const float fpf = fminf(fmaf(b2f * q2, q2, fmaf(b1f * q1, q1, 1.f)), 0x1p120f);
  if (dbits(f) < dbits(x * f2d_exact(fpf)) - (51ull << 52)) return 0;
  return 1;
}

// One FP64 Newton step x - f(x)/f'(x) on the spectral function (the
// iteration of Sec. 1.4.2), with the evaluation form chosen as above.
// Returns x unchanged when the step would leave (0, inf).
__device__ __forceinline__ double newton64(const double ab, const double b1, const double b2, const double g,
                                           const double c, const double K, const double x) {
  const bool small = x < ab;
  const double r1 = rcp64(x), r2 = rcp64(x + ab);
  const double t1 = b1 * r1, t2 = b2 * r2;
  const double f = ((x + (small ? K : -g)) - t1) + (small ? c * x * r2 : -t2);
  const double fp = fma(t2, r2, fma(t1, r1, 1.0));
  const double xn = x - f * rcp64(fp);
  return (xn > 0.0 && xn < 0x1p+1000) ? xn : x;
}

// Full FP64 Borges-Gragg iteration (IEEE arithmetic, any data) from x0 > 0
// right of the root, or from the start of Eq. (7) when x0 <= 0.  The next
// iterate is x - Delta (Eq. (6)), or the zero of phi_j taken directly when
// Delta >= x/2.
__device__ double zero_bg_full(double ab, double b1, double b2, double g, double x, bool& capped, int& steps) {
  if (!(x > 0.0)) {
    const double hg = 0.5 * g, bs = b1 + b2;
    const double rt = sqrt(fma(hg, hg, bs));
    x = (g >= 0.0) ? hg + rt : bs / (rt - hg);
  }
  const double c = b2 / ab, K = -g - c;  // f = x + K - b1/x + c x/(x + ab)
  capped = false;
  int it = 0;
  for (;; ++it) {
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
  steps = it;
  return x;
}

// Newton's method of Sec. 1.4.2 in FP64 (IEEE arithmetic, printed form of
// f): started left of the zero at the positive zero of x - g - b1/x (the
// point where f meets -b2/(x + ab); conjugate form when g < 0), stopped when
// |f| < C eps x, when f >= 0 (at or past the zero: rounding level, the
// iteration being monotone from the left) or when a step no longer
// increases x.  Sets steps and capped (kMaxIt steps without a stop).
__device__ double zero_newton_full(double ab, double b1, double b2, double g, bool& capped, int& steps) {
  const double hg = 0.5 * g;
  const double rt = sqrt(fma(hg, hg, b1));
  double x = (g >= 0.0) ? hg + rt : b1 / (rt - hg);
  capped = false;
  int it = 0;
  for (;; ++it) {
    const double r1 = 1.0 / x, r2 = 1.0 / (x + ab);
    const double f = ((x - g) - b1 * r1) - b2 * r2;
    const double fp = fma(b2 * r2, r2, fma(b1 * r1, r1, 1.0));
    if (!(f < 0.0)) break;
    if (-f < (kCTerm * kEps) * x) break;
    if (it >= kMaxIt) {
      capped = true;
      break;
    }
    const double xn = x - f / fp;
    if (!(xn > x)) break;
    x = xn;
  }
  steps = it;
  return x;
}

// ---------------------------------------------------------------------------
// Per-matrix state between the phases of a tile
// ---------------------------------------------------------------------------

struct Lane {
  double a1, a2, b1, b2, g, c, s;  // ordered arrow and its rotation (pre-scaled frame)
  int e;                           // input = 2^e x pre-scaled frame
  int cls;
};

// Phase A: pre-scale, Sec. 1 arrow reduction, Sec. 1.1 classification.
// kEispack selects the EISPACK-style deflation test of Sec. 1.1 (the form
// the paper starts from) instead of the simplified one it adopts.
template <bool kEispack = false>
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
  // Exact power-of-two pre-scale: the largest entry lands in [0.5, 1).  When
  // every entry is zero or stays normal, by exponent arithmetic; otherwise
  // (subnormal results or inputs, huge entries) by scalbn.
  double a[6];
  L.e = E - 1022;
  bool exp_ok = (E >= 1 && E <= 2044);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const int ex = (__double2hiint(a_in[i]) >> 20) & 0x7ff;
    exp_ok &= is_zero(a_in[i]) || (ex >= 1 && ex - L.e >= 1);
  }
  if (exp_ok) {
#pragma unroll
    for (int i = 0; i < 6; ++i)
      a[i] = is_zero(a_in[i]) ? a_in[i]
                              : __hiloint2double(__double2hiint(a_in[i]) - L.e * (1 << 20), __double2loint(a_in[i]));
  } else {
    double amax = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) amax = fmax(amax, fabs(a_in[i]));
    int e = 0;
    if (amax > 0.0) frexp(amax, &e);
    L.e = e;
#pragma unroll
    for (int i = 0; i < 6; ++i) a[i] = scalbn(a_in[i], -e);
  }
  const Rot J = ordered_rotation(a[0], a[3], a[1]);
  L.a1 = J.l1;
  L.a2 = J.l2;
  L.c = J.c;
  L.s = J.s;
  L.g = a[2];
  double b1 = fma(J.c, a[4], J.s * a[5]);
  double b2 = fma(J.c, a[5], -J.s * a[4]);
  // Exact beta-deflation of a negligible spike (|b| < 2^kTinySpikeExp).
  if (hi_mag(b1) < hi_pow2(kTinySpikeExp)) b1 = 0.0;
  if (hi_mag(b2) < hi_pow2(kTinySpikeExp)) b2 = 0.0;
  L.b1 = b1;
  L.b2 = b2;
  const double abar = L.a1 - L.a2;
  const double h2 = fma(b1, b1, b2 * b2);
  // Both sides of the deflation test are >= +0: compared as bit patterns.
  // Simplified: |abar b1 b2| <= C eps |a1 + a2| h^2; EISPACK-style:
  // |abar b1 b2| <= C eps (|a1 b2^2 + a2 b1^2| + |a1 b1^2 + a2 b2^2|).
  const double rhs = kEispack ? (kCDefl * kEps) * (fabs(fma(L.a1 * b2, b2, L.a2 * b1 * b1)) +
                                                    fabs(fma(L.a1 * b1, b1, L.a2 * b2 * b2)))
                              : (kCDefl * kEps) * fabs(L.a1 + L.a2) * h2;
  if (dbits(h2) == 0)
    L.cls = kDiagonal;
  else if (dbits(fabs(abar * b1 * b2)) <= dbits(rhs))
    L.cls = kDeflated;  // also the exact beta- and combo-deflations
  else
    L.cls = kReduced;
  return L;
}

// Phase E for eigenvalues only: the values of finish_lane (the same
// expressions, the same compare-and-swap order and tie rule), unscaled.
__device__ __forceinline__ void finish_values(const Lane& L, double mu, double nu, double lam[3]) {
  const double a1 = L.a1, a2 = L.a2, b1 = L.b1, b2 = L.b2, g = L.g;
  double l0, l1, l2;
  if (L.cls == kDiagonal) {
    l0 = a1; l1 = a2; l2 = g;
  } else if (L.cls == kDeflated) {
    const double h2 = fma(b1, b1, b2 * b2);
    const double rh = rsqrt(h2), h = h2 * rh;
    const double gs = b1 * rh, gc = b2 * rh;
    l0 = fma(a1 * gc, gc, a2 * gs * gs);
    const Rot K = ordered_rotation(fma(a1 * gs, gs, a2 * gc * gc), h, g);
    l1 = K.l1; l2 = K.l2;
  } else {
    l0 = a1 + mu;
    l1 = (nu - mu) + g;
    l2 = a2 - nu;
  }
  double t;
  if (l1 < l0) { t = l0; l0 = l1; l1 = t; }
  if (l2 < l1) { t = l1; l1 = l2; l2 = t; }
  if (l1 < l0) { t = l0; l0 = l1; l1 = t; }
  lam[0] = mul_pow2(l0, L.e);
  lam[1] = mul_pow2(l1, L.e);
  lam[2] = mul_pow2(l2, L.e);
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
    // lambda2; closed-form u1 and u3, normalised (u2 below).
    const double abar = a1 - a2;
    l[0] = a1 + mu;
    l[1] = (nu - mu) + g;
    l[2] = a2 - nu;
    const double mpa = mu + abar, npa = nu + abar;
    v[0][0] = b1 * mpa; v[0][1] = b2 * mu;  v[0][2] = mu * mpa;
    v[2][0] = b1 * nu;  v[2][1] = b2 * npa; v[2][2] = -(nu * npa);
#pragma unroll
    for (int k = 0; k < 3; k += 2) {
      double ss = fma(v[k][0], v[k][0], fma(v[k][1], v[k][1], v[k][2] * v[k][2]));
      if (hi_mag(ss) < hi_pow2(-1000)) {  // ss < 2^-1000 (ss >= 0)
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
  double x20 = fma(L.c, v[2][0], -L.s * v[2][1]), x21 = fma(L.s, v[2][0], L.c * v[2][1]), x22 = v[2][2];
  double x10, x11, x12;
  if (L.cls == kReduced) {
    // u2 is the cross product of u1 and u3 (Sec. 1.3 relies on exactly
    // this for its orthogonality); formed from the normalised u1 and u3,
    // which are unit and orthogonal to rounding, so the product is unit
    // without a normalisation, and its error is at most the sum of theirs,
    // each within eps / gap of its eigenvalue <= eps / (middle gap).  J is a
    // rotation (det 1), so J(u1 x u3) = (J u1) x (J u3): taken in the input
    // frame directly.
    x10 = fma(x01, x22, -x02 * x21);
    x11 = fma(x02, x20, -x00 * x22);
    x12 = fma(x00, x21, -x01 * x20);
  } else {
    x10 = fma(L.c, v[1][0], -L.s * v[1][1]);
    x11 = fma(L.s, v[1][0], L.c * v[1][1]);
    x12 = v[1][2];
  }
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
    lam[k] = mul_pow2(ls[k], L.e);
    // Largest-magnitude component positive, first one on ties: magnitudes
    // compared as integers (|y| orders like its bit pattern with the sign
    // cleared), the sign applied by flipping sign bits (no FP64 work).
    const uint64_t m0 = mag_bits(xs[k][0]), m1 = mag_bits(xs[k][1]), m2 = mag_bits(xs[k][2]);
    const double big = (m2 > m0 && m2 > m1) ? xs[k][2] : ((m1 > m0) ? xs[k][1] : xs[k][0]);
    const int flip = __double2hiint(big) & (int)0x80000000;
    U[0 * 3 + k] = flip_sign(xs[k][0], flip);
    U[1 * 3 + k] = flip_sign(xs[k][1], flip);
    U[2 * 3 + k] = flip_sign(xs[k][2], flip);
  }
}

}  // namespace
}  // namespace f64
}  // namespace syev3
