// syev3_f32.cu -- FP32 batched 3x3 symmetric eigensolver for sm_103a, plain
// and compensated (the precision form).
//
// The steps are those of the FP64 solver (C. F. Borges, arXiv 1806.06698,
// Secs. 1-1.4.1) carried out in FP32: ordered Jacobi rotation to an arrow,
// the deflation test, the deflated 2x2 solve or the Borges-Gragg zero finder
// for mu and nu, the trace identity and the closed-form eigenvectors.  The
// spectral function is evaluated in the cancellation-free form for x < abar
// (see solve_f64.cuh).
//
// The compensated form (SYEV3_F32_COMPENSATED) adds, in FP32:
//  * the deflation test of Sec. 1.1 decided as on exact products, so the
//    decision is not blurred by FP32 rounding: on the FP32 sides where they
//    are clearly apart, with double-float (error-free transformation)
//    products where they are close;
//  * a double-float evaluation of the spectral function at the FP32 root
//    and one Newton correction (Sec. 1.4.2) with it;
// and uses FP64 only on the lanes it flags -- near-deflated (the test's two
// sides within a factor kNearDefl), clustered (a relative eigenvalue gap
// below kClusterTau) or capped -- for a final FP64 Newton step on mu and nu,
// eigenvectors re-formed (and so re-orthogonalised) in FP64 and an FP64
// residual check against the input.  Flagged lanes are compacted with warp
// ballots into a shared-memory list and refined in whole warps, the rest
// carried from tile to tile, so the FP64 work runs on as few warps as
// possible; no global scratch memory is used (syev3_batched_ws instead
// appends them to a list in a workspace for k_refine_f32, which runs beside
// the FP32 solve on a second stream for large batches).
//
// The two root problems of a lane (mu and nu) run the same expressions, so
// their arithmetic is paired on the packed FP32 instructions (two correctly
// rounded operations per instruction); reciprocals, roots, comparisons and
// selections stay per half.  Lanes of the three classes (diagonal, deflated,
// reduced) in one warp take different branches of the solve; an explicit
// __syncwarp over the lanes that form eigenpairs rejoins them for the common
// tail (without it the warp was measured to stay split there).
//
// Memory path as in the FP64 kernel: tiles of kTPB records (24 B each) by
// 1-D bulk copy into shared memory, double-buffered on mbarriers; results
// staged in shared memory and written with 16-byte stores.  The plain form
// moves 72 B per matrix; it is bound by instruction issue, not by HBM.

#include <cmath>
#include <cstdint>
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "serve_tile.cuh"
#include "solve_f64.cuh"

namespace syev3 {
namespace {

constexpr int kTPB = 128;
constexpr int kMaxIt32 = 32;              // FP32 zero-finder step cap
constexpr float kEps32 = 0x1p-23f;
constexpr float kCDefl32 = 1.0f;          // C of the deflation test (Sec. 1.1)
constexpr float kCTerm32 = 2.0f;          // C of the stopping rule (Sec. 1.4.1)
constexpr float kTinySpike32 = 0x1p-60f;  // spikes below this are zeroed (beta-deflation)
// The lanes refined in FP64 are those FP32 cannot resolve: a deflation test
// whose two sides lie within a factor kNearDefl of each other (the decision
// rests on the last bits of the FP32 data), or a relative eigenvalue gap
// below kClusterTau = one unit of FP32 resolution (the pair's eigenvectors are
// then not determined by FP32 arithmetic).  A sweep of both on the mixed and
// structure-tensor batches found every subset's error against the FP64
// oracle within 2.1 eps32 ||A||_F (eigenvalues), 2.9 (residual) and 7.6
// (orthogonality) for every setting, far inside the 64 eps32 bar; wider
// windows only cost time (a factor 16 window flagged 16 % of the mixed batch).
constexpr float kNearDefl = 2.0f;         // near-deflated: test sides within this factor
constexpr float kClusterTau = 0x1p-23f;   // clustered: relative gap below this
constexpr double kResidualTol = 16.0 * 0x1p-23;  // FP64 residual check, times ||A||_F
// Plain and workspace forms: a last zero-finder move above kMoveTol x
// (relative error of order kMoveTol^3 = 2^-24 after the cubically
// convergent step) sends the root to further steps.
constexpr float kMoveTol = 0x1p-8f;
constexpr int kPlain = 0, kInline = 1, kDeferred = 2;  // modes of k_syev3_f32

constexpr int kDiag = f64::kDiagonal, kDefl = f64::kDeflated, kRed = f64::kReduced,
              kNonFin = f64::kNonFinite, kIdle = f64::kIdle;

__device__ unsigned g_flags32;

struct Lane32 {
  float a1, a2, b1, b2, g, c, s;  // ordered arrow and rotation (pre-scaled frame)
  int e;                          // A was divided by 2^e
  int cls;
  bool near_defl;
};

// Sec. 1: ordered Jacobi rotation of [[p,q],[q,r]] in FP32.
struct Rot32 {
  float c, s, l1, l2;
};

__device__ __forceinline__ Rot32 ordered_rotation32(float p, float q, float r) {
  Rot32 J;
  if (q == 0.f) {
    const bool keep = p >= r;
    J.c = keep ? 1.f : 0.f;
    J.s = keep ? 0.f : 1.f;
    J.l1 = keep ? p : r;
    J.l2 = keep ? r : p;
    return J;
  }
  const float D = p - r, q2 = q + q;
  const float rad = sqrt32(fmaf(D, D, q2 * q2));
  const float den = fabsf(D) + rad;
  const float t = (den > 0.f) ? q2 * rcp32(den) : copysignf(1.f, q);
  const bool right = D >= 0.f;
  const float hi = right ? p : r, lo = right ? r : p;
  J.l1 = fmaf(t, q, hi);
  J.l2 = fmaf(-t, q, lo);
  const float k = rsqrt32(fmaf(t, t, 1.f));
  J.c = right ? k : t * k;
  J.s = right ? t * k : k;
  return J;
}

template <bool kComp>
__device__ __forceinline__ Lane32 make_lane32(const float a_in[6]) {
  Lane32 L;
  L.near_defl = false;
  unsigned mag = 0u;  // largest |a_ij| as a bit pattern (orders like |a_ij|)
#pragma unroll
  for (int i = 0; i < 6; ++i) mag = max(mag, __float_as_uint(a_in[i]) & 0x7fffffffu);
  if (mag >= 0x7f800000u) {  // an infinite or NaN entry
    L.cls = kNonFin;
    return L;
  }
  const int E = (int)(mag >> 23);
  float a[6];
  if (E >= 1 && E <= 252) {  // exact power-of-two pre-scale: largest entry in [0.5, 1)
    L.e = E - 126;
    const float sc = pow2f(-L.e);
#pragma unroll
    for (int i = 0; i < 6; ++i) a[i] = a_in[i] * sc;
  } else {
    float amax = 0.f;
#pragma unroll
    for (int i = 0; i < 6; ++i) amax = fmaxf(amax, fabsf(a_in[i]));
    int e = 0;
    if (amax > 0.f) frexpf(amax, &e);
    L.e = e;
#pragma unroll
    for (int i = 0; i < 6; ++i) a[i] = scalbnf(a_in[i], -e);
  }
  const Rot32 J = ordered_rotation32(a[0], a[3], a[1]);
  L.a1 = J.l1;
  L.a2 = J.l2;
  L.c = J.c;
  L.s = J.s;
  L.g = a[2];
  float b1 = fmaf(J.c, a[4], J.s * a[5]);
  float b2 = fmaf(J.c, a[5], -J.s * a[4]);
  if (fabsf(b1) < kTinySpike32) b1 = 0.f;
  if (fabsf(b2) < kTinySpike32) b2 = 0.f;
  L.b1 = b1;
  L.b2 = b2;
  if (b1 == 0.f && b2 == 0.f) {
    L.cls = kDiag;
    return L;
  }
  // Sec. 1.1: |abar b1 b2| <= C eps |a1 + a2| h^2.
  const float h2 = fmaf(b1, b1, b2 * b2);
  const float lhs = fabsf((L.a1 - L.a2) * b1 * b2);
  const float rhs = (kCDefl32 * kEps32) * fabsf(L.a1 + L.a2) * h2;
  if (kComp) {
    // The decision of the exact sides (exact arithmetic on the FP32 arrow).
    // The FP32 sides above carry 3 and 4 roundings, a relative error below
    // 7 x 2^-24 together, and every intermediate is normal when both sides
    // are >= 2^-120; sides further apart than a factor 1 + 2^-20 (one more
    // rounding in forming the bounds) are therefore ordered as the exact
    // ones.  Closer sides, or sides near underflow, are decided with
    // double-float products, which carry the exact sides to ~2^-46.
    const bool clear = lhs >= 0x1p-120f && rhs >= 0x1p-120f &&
                       (lhs <= rhs * (1.f - 0x1p-20f) || lhs >= rhs * (1.f + 0x1p-20f));
    if (clear) {
      L.cls = (lhs <= rhs) ? kDefl : kRed;
    } else {
      const F2 ab = two_sum(L.a1, -L.a2);
      const F2 dl = ff_mul1(ff_mul1(ab, b1), b2);
      const F2 sum12 = two_sum(L.a1, L.a2);
      const F2 dh2 = ff_add(two_prod(b1, b1), two_prod(b2, b2));
      F2 dr = ff_mul(sum12, dh2);
      dr.h *= kCDefl32 * kEps32;
      dr.l *= kCDefl32 * kEps32;
      const F2 al = {fabsf(dl.h), dl.h < 0.f ? -dl.l : dl.l};
      const F2 ar = {fabsf(dr.h), dr.h < 0.f ? -dr.l : dr.l};
      L.cls = ff_le(al, ar) ? kDefl : kRed;
    }
    L.near_defl = (lhs < kNearDefl * rhs) && (lhs * kNearDefl > rhs);
  } else {
    L.cls = (lhs <= rhs) ? kDefl : kRed;
  }
  return L;
}

// The zero of phi_j (the model of Eq. (5) through x) taken directly: the
// root of omega_0 y^2 - sigma y - omega_1 = 0, for a step Delta >= x/2 (a
// start far right of the root).  r1 = 1/x, r2 = 1/(x + ab).
__device__ __forceinline__ float phi_zero32(const float b1, const float b2, const float x, const float r1,
                                            const float r2, const float w0, const float f) {
  const float xr = x * r2;
  const float w1 = fmaf(b2 * xr, xr * xr, b1);
  const float sg = fmaf(w0, x, -fmaf(w1, r1, f));
  const float rt = sqrt32(fmaf(sg, sg, 4.f * w0 * w1));
  return (sg > 0.f) ? (sg + rt) * rcp32(2.f * w0) : (2.f * w1) * rcp32(rt - sg);
}

// One Borges-Gragg step in FP32 (Sec. 1.4.1) from x: returns x_{j+1}, or x
// itself when f(x) <= 0 (at or past the root: rounding level).  For x < ab,
// f = x + K - b1/x + c x/(x+ab) (the cancellation-free form); x_{j+1} is
// x - Delta (Eq. (6)), or the zero of phi_j taken directly when Delta >= x/2.
// *fx receives f(x).
__device__ __forceinline__ float bg_step32(const float ab, const float b1, const float b2, const float g,
                                          const float c, const float K, const float x, float* fx,
                                          float* fpx = nullptr) {
  const float r1 = rcp32(x), r2 = rcp32(x + ab);
  const float t1 = b1 * r1, t2 = b2 * r2;
  const bool small = x < ab;
  const float f = ((x + (small ? K : -g)) - t1) + (small ? c * x * r2 : -t2);
  *fx = f;
  const float fp = fmaf(t2, r2, fmaf(t1, r1, 1.f));
  if (fpx) *fpx = fp;
  const float w0 = fmaf(t2 * ab, r2 * r2, 1.f);
  const float rb = rcp32(fmaf(f, r1, fp));
  const float fr = f * rb;
  const float z = (-4.f * w0) * (r1 * rb) * fr;
  const float delta = 2.f * fr * rcp32(1.f + sqrt32(fmaxf(0.f, 1.f + z)));
  float xn = x - delta;
  if (!(delta < 0.5f * x)) xn = phi_zero32(b1, b2, x, r1, r2, w0, f);  // rare
  return (f > 0.f && xn < x) ? xn : x;
}

// Pairs of FP32 values -- .x for the problem of mu, .y for that of nu -- on
// the packed FP32 instructions of sm_100 and later, which perform the same
// correctly rounded operation on both halves: the two problems of a lane run
// the same expressions, so they issue as one instruction stream.  A
// difference a - b is formed as fma(b, -1, a), which rounds the exact
// difference once, as a subtraction does.  Reciprocals, roots, comparisons
// and selections stay per half.
using P2 = float2;
__device__ __forceinline__ P2 pp(const float a) { return make_float2(a, a); }
__device__ __forceinline__ P2 padd(const P2 a, const P2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ P2 psub(const P2 a, const P2 b) { return __ffma2_rn(b, pp(-1.f), a); }
__device__ __forceinline__ P2 pmul(const P2 a, const P2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ P2 pfma(const P2 a, const P2 b, const P2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ P2 prcp(const P2 a) { return make_float2(rcp32(a.x), rcp32(a.y)); }
__device__ __forceinline__ P2 psqrt(const P2 a) { return make_float2(sqrt32(a.x), sqrt32(a.y)); }
__device__ __forceinline__ P2 psel(const bool px, const bool py, const P2 a, const P2 b) {
  return make_float2(px ? a.x : b.x, py ? a.y : b.y);
}

// The starts of f64::start32 for both problems: the zero x7 of the limit
// model of Eq. (7), and the small-root model's start taken where it applies
// (model[k]).  rab = 1/ab.
__device__ __forceinline__ P2 start32x2(const P2 ab, const P2 rab, const P2 b1, const P2 b2, const P2 g, const P2 c,
                                       const P2 K, P2& x7, bool model[2]) {
  const P2 hg = pmul(pp(0.5f), g), bs = padd(b1, b2);
  const P2 rt = psqrt(pfma(hg, hg, bs));
  x7 = psel(g.x >= 0.f, g.y >= 0.f, padd(hg, rt), pmul(bs, prcp(psub(rt, hg))));
  const P2 c2 = pfma(c, rab, pp(1.f));
  const P2 disc = psqrt(pfma(K, K, pmul(pmul(pp(4.f), c2), b1)));
  const bool kx = K.x >= 0.f, ky = K.y >= 0.f;
  const P2 xm = pmul(psel(kx, ky, padd(b1, b1), psub(disc, K)), prcp(psel(kx, ky, padd(K, disc), padd(c2, c2))));
  const P2 r1 = prcp(xm), r2 = prcp(padd(xm, ab));
  const P2 fpm = pfma(pmul(b2, r2), r2, pfma(pmul(b1, r1), r1, pp(1.f)));
  const P2 x0 = padd(xm, pfma(pmul(pmul(padd(c, c), xm), xm), prcp(pmul(pmul(ab, ab), fpm)),
                             pmul(pp(0x1p-20f), xm)));
  model[0] = (xm.x > 0.f) && (xm.x < 0.0625f * ab.x) && (x0.x < x7.x);
  model[1] = (xm.y > 0.f) && (xm.y < 0.0625f * ab.y) && (x0.y < x7.y);
  return psel(model[0], model[1], x0, x7);
}

// The step of bg_step32 for both problems (nb2 = -b2, ng = -g); *fx
// receives f(x).
template <bool kBranchFree>
__device__ __forceinline__ P2 bg_step32x2(const P2 ab, const P2 b1, const P2 b2, const P2 nb2, const P2 ng,
                                         const P2 c, const P2 K, const P2 x, P2* fx) {
  const P2 r1 = prcp(x), r2 = prcp(padd(x, ab));
  const P2 t1 = pmul(b1, r1);
  const bool sx = x.x < ab.x, sy = x.y < ab.y;
  // x + K - b1/x + c x/(x+ab) below ab, x - g - b1/x - b2/(x+ab) above
  const P2 f = padd(psub(padd(x, psel(sx, sy, K, ng)), t1), pmul(psel(sx, sy, pmul(c, x), nb2), r2));
  *fx = f;
  const P2 t2 = pmul(b2, r2);
  const P2 fp = pfma(t2, r2, pfma(t1, r1, pp(1.f)));
  const P2 w0 = pfma(pmul(t2, ab), pmul(r2, r2), pp(1.f));
  const P2 rb = prcp(pfma(f, r1, fp));
  const P2 fr = pmul(f, rb);
  const P2 q = padd(pp(1.f), pmul(pmul(pmul(pp(-4.f), w0), pmul(r1, rb)), fr));
  const P2 delta = pmul(padd(fr, fr), prcp(padd(pp(1.f), psqrt(make_float2(fmaxf(0.f, q.x), fmaxf(0.f, q.y))))));
  P2 xn = psub(x, delta);
  const P2 d2 = padd(delta, delta);  // Delta >= x/2 (exact doubling)
  const bool dx = !(d2.x < x.x), dy = !(d2.y < x.y);
  if constexpr (kBranchFree) {
    // the zero of phi_j for both problems, kept where Delta >= x/2
    const P2 xr = pmul(x, r2);
    const P2 w1 = pfma(pmul(b2, xr), pmul(xr, xr), b1);
    const P2 sg = pfma(w0, x, pmul(pfma(w1, r1, f), pp(-1.f)));
    const P2 rt = psqrt(pfma(sg, sg, pmul(pmul(pp(4.f), w0), w1)));
    const bool px = sg.x > 0.f, py = sg.y > 0.f;
    const P2 xd = pmul(psel(px, py, padd(sg, rt), padd(w1, w1)), prcp(psel(px, py, padd(w0, w0), psub(rt, sg))));
    xn = psel(dx, dy, xd, xn);
  } else {
    if (dx || dy) {  // rare
      if (dx) xn.x = phi_zero32(b1.x, b2.x, x.x, r1.x, r2.x, w0.x, f.x);
      if (dy) xn.y = phi_zero32(b1.y, b2.y, x.y, r1.y, r2.y, w0.y, f.y);
    }
  }
  return psel(f.x > 0.f && xn.x < x.x, f.y > 0.f && xn.y < x.y, xn, x);
}

// The schedule of roots32x2 (below) one problem at a time, for the
// compensated form with its refinement inside the kernel.  more[k] as in
// roots32x2, for a move above 2^-12 x; the warp finishes such roots right
// after.
__device__ __forceinline__ void roots32(const float ab, const float b1[2], const float b2[2], const float g[2],
                                        const float c[2], const float K[2], float x[2], bool more[2]) {
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    float f0, f1, x7;
    bool model;
    const float x0 = f64::start32(ab, b1[k], b2[k], g[k], c[k], K[k], x7, model);
    float x1 = bg_step32(ab, b1[k], b2[k], g[k], c[k], K[k], x0, &f0);
    const bool restart = model && !(f0 > 0.f);  // the small-root start was not right of the root
    if (restart) x1 = x7;
    const float x2 = bg_step32(ab, b1[k], b2[k], g[k], c[k], K[k], x1, &f1);
    float f2;
    const float x3 = bg_step32(ab, b1[k], b2[k], g[k], c[k], K[k], x2, &f2);
    more[k] = (x2 - x3) > 0x1p-12f * x3;
    x[k] = x3;
  }
}

// mu and nu in FP32 on a fixed schedule, both problems paired: from the
// starts of start32x2 three Borges-Gragg steps, straight-line (no lane
// leaves early, so the warp stays converged; a small-root start found left
// of the root is replaced by the start of Eq. (7) after the first
// evaluation).  The last step moves x by about the error the one before
// left, and the step converges cubically, so a move below kMoveTol x leaves
// an error of order kMoveTol^3 x.  more[k] marks a problem whose last step
// moved x by more than that; the kernel finishes those roots apart from the
// straight-line code (see k_syev3_f32).
__device__ __forceinline__ void roots32x2(const P2 ab, const P2 rab, const P2 b1, const P2 b2, const P2 g,
                                          const P2 c, const P2 K, float x[2], bool more[2]) {
  const P2 nb2 = make_float2(-b2.x, -b2.y), ng = make_float2(-g.x, -g.y);
  P2 x7, f0, f1, f2;
  bool model[2];
  const P2 x0 = start32x2(ab, rab, b1, b2, g, c, K, x7, model);
  P2 x1 = bg_step32x2<true>(ab, b1, b2, nb2, ng, c, K, x0, &f0);
  // the small-root start was not right of the root: restart from Eq. (7)'s
  x1 = psel(model[0] && !(f0.x > 0.f), model[1] && !(f0.y > 0.f), x7, x1);
  const P2 x2 = bg_step32x2<false>(ab, b1, b2, nb2, ng, c, K, x1, &f1);
  const P2 x3 = bg_step32x2<false>(ab, b1, b2, nb2, ng, c, K, x2, &f2);
  const P2 mv = psub(x2, x3), th = pmul(pp(kMoveTol), x3);
  more[0] = mv.x > th.x;
  more[1] = mv.y > th.y;
  x[0] = x3.x;
  x[1] = x3.y;
}

// Further steps for one problem until f/f' < C eps32 x (Sec. 1.4.1), f <= 0
// or a stalled step; returns false if kMaxIt32 steps were not enough.  Not
// inlined: it runs for few roots, and inlined it would weigh on the
// registers and scheduling of the kernel's main path.
__device__ __noinline__ bool roots32_more(const float ab, const float b1, const float b2, const float g, float* x) {
  const float c = b2 * rcp32(ab), K = -g - c;
  for (int it = 0; it < kMaxIt32; ++it) {
    float f, fp;
    const float xn = bg_step32(ab, b1, b2, g, c, K, *x, &f, &fp);
    const bool go = f > (kCTerm32 * kEps32) * (*x) * fp && xn < *x;  // f/f' >= C eps x: not yet
    *x = xn;
    if (!go) return true;
  }
  return false;
}

// The two problems' data of a reduced arrow (Sec. 1.2): problem 0 (mu)
// has spikes (b1^2, b2^2) and gap g - a1, problem 1 (nu) the spikes swapped
// and a2 - g; ab = a1 - a2.
__device__ __forceinline__ void roots_setup32(const Lane32& L, const float ab, float b1[2], float b2[2],
                                              float g[2]) {
  (void)ab;
  const P2 bb = pmul(make_float2(L.b1, L.b2), make_float2(L.b1, L.b2));
  const P2 gg = psub(make_float2(L.g, L.a2), make_float2(L.a1, L.g));
  b1[0] = bb.x; b1[1] = bb.y; b2[0] = bb.y; b2[1] = bb.x;
  g[0] = gg.x; g[1] = gg.y;
}

// Double-float value of the spectral function at x (FP32 data exact), and
// one Newton correction x - f/f' with it (Sec. 1.4.2).  Each term is formed
// as an unevaluated pair (head, low part) without renormalisation, and the
// terms are added by cascaded summation (Ogita, Rump and Oishi 2005,
// "Sum2"): the heads with TwoSum, every rounding error and low part in one
// FP32 sum, so f comes out as if summed in twice the working precision and
// rounded once.  Data pairs (ab, b1, b2, g, c, K) need not be normalised.
__device__ __forceinline__ float newton_ff(const F2 ab, const F2 b1, const F2 b2, const F2 g, const F2 c, const F2 K,
                                          const float x) {
  const float r1 = rcp32(x);
  const F2 s0 = two_sum(x, ab.h);
  const float sh = s0.h, sl = s0.l + ab.l;  // x + ab
  const float r2 = rcp32(sh);
  // b1 / x: the quotient's head and the remainder over x.
  const float q1 = b1.h * r1;
  const float q1l = (fmaf(-q1, x, b1.h) + b1.l) * r1;
  // Last term: + c x / (x + ab) for x < ab (the cancellation-free form),
  // - b2 / (x + ab) otherwise; numerator (nh, nl), quotient (q2, q2l).
  const bool small = x < ab.h;
  const float cx = c.h * x;
  const float nh = small ? cx : b2.h;
  const float nl = small ? fmaf(c.h, x, -cx) + c.l * x : b2.l;
  const float q2 = nh * r2;
  const float q2l = ((fmaf(-q2, sh, nh) + nl) - q2 * sl) * r2;
  const float th = small ? q2 : -q2, tl = small ? q2l : -q2l;
  // Leading part: K (small) or -g.
  const float lh = small ? K.h : -g.h, ll = small ? K.l : -g.l;
  // Sum2 over x + lead - b1/x + last.
  const F2 u = two_sum(x, lh);
  const F2 v = two_sum(u.h, -q1);
  const F2 w = two_sum(v.h, th);
  const float f = w.h + (((u.l + v.l) + (w.l + ll)) + (tl - q1l));
  const float fp = fmaf(b2.h * r2, r2, fmaf(q1, r1, 1.f));
  const float xn = x - f * rcp32(fp);
  return (xn > 0.f) ? xn : x;
}

// newton_ff for both problems at once (pairs as in roots32x2): each
// double-float datum as a (head pair, low pair); ng = -g.  The same
// expressions as newton_ff, term by term.
__device__ __forceinline__ P2 pneg(const P2 a) { return pmul(a, pp(-1.f)); }

__device__ __forceinline__ void ptwo_sum(const P2 a, const P2 b, P2& s, P2& e) {
  s = padd(a, b);
  const P2 bb = psub(s, a);
  e = padd(psub(a, psub(s, bb)), psub(b, bb));
}

__device__ __forceinline__ P2 newton_ff2(const P2 abh, const P2 abl, const P2 b1h, const P2 b1l, const P2 b2h,
                                        const P2 b2l, const P2 ngh, const P2 ngl, const P2 ch, const P2 cl,
                                        const P2 Kh, const P2 Kl, const P2 x) {
  const P2 r1 = prcp(x), nx = pneg(x);
  P2 sh, s0l;
  ptwo_sum(x, abh, sh, s0l);
  const P2 sl = padd(s0l, abl);  // x + ab = sh + sl
  const P2 r2 = prcp(sh);
  // b1 / x: the quotient's head and the remainder over x.
  const P2 q1 = pmul(b1h, r1);
  const P2 q1l = pmul(padd(pfma(q1, nx, b1h), b1l), r1);
  // Last term: + c x / (x + ab) below ab (the cancellation-free form),
  // - b2 / (x + ab) above; numerator (nh, nl), quotient (q2, q2l).
  const bool sx = x.x < abh.x, sy = x.y < abh.y;
  const P2 cx = pmul(ch, x);
  const P2 nh = psel(sx, sy, cx, b2h);
  const P2 nl = psel(sx, sy, pfma(cl, x, pfma(ch, x, pneg(cx))), b2l);
  const P2 q2 = pmul(nh, r2), nq2 = pneg(q2);
  const P2 q2l = pmul(pfma(nq2, sl, padd(pfma(nq2, sh, nh), nl)), r2);
  const P2 sg = psel(sx, sy, pp(1.f), pp(-1.f));
  const P2 th = pmul(q2, sg), tl = pmul(q2l, sg);
  const P2 lh = psel(sx, sy, Kh, ngh), ll = psel(sx, sy, Kl, ngl);
  // Sum2 over x + lead - b1/x + last.
  P2 uh, ul, vh, vl, wh, wl;
  ptwo_sum(x, lh, uh, ul);
  vh = psub(uh, q1);  // TwoSum(u.h, -q1)
  {
    const P2 bb = psub(vh, uh);
    vl = psub(psub(uh, psub(vh, bb)), padd(q1, bb));
  }
  ptwo_sum(vh, th, wh, wl);
  const P2 f = padd(wh, padd(padd(padd(ul, vl), padd(wl, ll)), psub(tl, q1l)));
  const P2 fp = pfma(pmul(b2h, r2), r2, pfma(q1, r1, pp(1.f)));
  const P2 xn = pfma(pneg(f), prcp(fp), x);
  return psel(xn.x > 0.f, xn.y > 0.f, xn, x);
}

// Eigenpairs of a classified lane in FP32 (scaled frame); returns eigenvalues
// ascending in l[] and vectors as columns in U[i*3+k].
// Eigenvalues only: those of finish32 (the same expressions, compare order
// and tie rule), ascending, in the scaled frame.
template <bool kSync>
__device__ __forceinline__ void finish32_values(const Lane32& L, float mu, float nu, float l_out[3],
                                                const unsigned sync_mask) {
  const float a1 = L.a1, a2 = L.a2, b1 = L.b1, b2 = L.b2, g = L.g;
  float l0, l1, l2;
  if (L.cls == kDiag) {
    l0 = a1; l1 = a2; l2 = g;
  } else if (L.cls == kDefl) {
    const float h2 = fmaf(b1, b1, b2 * b2);
    const float rh = rsqrt32(h2), h = h2 * rh;
    const float gs = b1 * rh, gc = b2 * rh;
    l0 = fmaf(a1 * gc, gc, a2 * gs * gs);
    const Rot32 K = ordered_rotation32(fmaf(a1 * gs, gs, a2 * gc * gc), h, g);
    l1 = K.l1; l2 = K.l2;
  } else {
    l0 = a1 + mu;
    l1 = (nu - mu) + g;
    l2 = a2 - nu;
  }
  if constexpr (kSync) __syncwarp(sync_mask);  // the classes' lanes rejoin
  float t;
  if (l1 < l0) { t = l0; l0 = l1; l1 = t; }
  if (l2 < l1) { t = l1; l1 = l2; l2 = t; }
  if (l1 < l0) { t = l0; l0 = l1; l1 = t; }
  l_out[0] = l0; l_out[1] = l1; l_out[2] = l2;
}

template <bool kSync>
__device__ __forceinline__ void finish32(const Lane32& L, float mu, float nu, float l_out[3], float U[9], int rk[3],
                                         const unsigned sync_mask) {
  const float a1 = L.a1, a2 = L.a2, b1 = L.b1, b2 = L.b2, g = L.g;
  float l[3], v[3][3];
  if (L.cls == kDiag) {
    l[0] = a1; l[1] = a2; l[2] = g;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) v[k][i] = (i == k) ? 1.f : 0.f;
  } else if (L.cls == kDefl) {
    const float h2 = fmaf(b1, b1, b2 * b2);
    const float rh = rsqrt32(h2), h = h2 * rh;
    const float gs = b1 * rh, gc = b2 * rh;
    l[0] = fmaf(a1 * gc, gc, a2 * gs * gs);
    v[0][0] = gc; v[0][1] = -gs; v[0][2] = 0.f;
    const float d2 = fmaf(a1 * gs, gs, a2 * gc * gc);
    const Rot32 K = ordered_rotation32(d2, h, g);
    l[1] = K.l1; l[2] = K.l2;
    v[1][0] = gs * K.c;  v[1][1] = gc * K.c;  v[1][2] = K.s;
    v[2][0] = -gs * K.s; v[2][1] = -gc * K.s; v[2][2] = K.c;
  } else {
    const float abar = a1 - a2;
    l[0] = a1 + mu;
    l[1] = (nu - mu) + g;
    l[2] = a2 - nu;
    const float mpa = mu + abar, npa = nu + abar;
    v[0][0] = b1 * mpa; v[0][1] = b2 * mu;  v[0][2] = mu * mpa;
    v[2][0] = b1 * nu;  v[2][1] = b2 * npa; v[2][2] = -(nu * npa);
    v[1][0] = v[1][1] = v[1][2] = 0.f;  // u2 = u1 x u3, formed below in the input frame
#pragma unroll
    for (int k = 0; k < 3; k += 2) {
      float ss = fmaf(v[k][0], v[k][0], fmaf(v[k][1], v[k][1], v[k][2] * v[k][2]));
      if (!(ss >= 0x1p-100f)) {  // squares near underflow: exact power-of-two rescale
        int E = 1;
#pragma unroll
        for (int i = 0; i < 3; ++i) E = max(E, (__float_as_int(v[k][i]) >> 23) & 0xff);
        const float sc = pow2f(126 - E);
        v[k][0] *= sc; v[k][1] *= sc; v[k][2] *= sc;
        ss = fmaf(v[k][0], v[k][0], fmaf(v[k][1], v[k][1], v[k][2] * v[k][2]));
      }
      const float inv = rsqrt32(ss);
      v[k][0] *= inv; v[k][1] *= inv; v[k][2] *= inv;
    }
  }
  if constexpr (kSync) __syncwarp(sync_mask);  // the three classes' lanes rejoin for the common tail
  float x[3][3];
#pragma unroll
  for (int k = 0; k < 3; k += 2) {
    x[k][0] = fmaf(L.c, v[k][0], -L.s * v[k][1]);
    x[k][1] = fmaf(L.s, v[k][0], L.c * v[k][1]);
    x[k][2] = v[k][2];
  }
  if (L.cls == kRed) {
    // u2 is the cross product of u1 and u3 (Sec. 1.3), of the normalised
    // vectors and in the input frame ((J u1) x (J u3) = J (u1 x u3)): no
    // normalisation and no back-transform of its own.
    x[1][0] = fmaf(x[0][1], x[2][2], -x[0][2] * x[2][1]);
    x[1][1] = fmaf(x[0][2], x[2][0], -x[0][0] * x[2][2]);
    x[1][2] = fmaf(x[0][0], x[2][1], -x[0][1] * x[2][0]);
  } else {
    x[1][0] = fmaf(L.c, v[1][0], -L.s * v[1][1]);
    x[1][1] = fmaf(L.s, v[1][0], L.c * v[1][1]);
    x[1][2] = v[1][2];
  }
  // Stable ascending ranks of the three eigenvalues (strict "<" for the
  // later index keeps equal values in branch order); the caller stores each
  // eigenpair at its rank.
  rk[0] = (int)(l[1] < l[0]) + (int)(l[2] < l[0]);
  rk[1] = (int)(l[0] <= l[1]) + (int)(l[2] < l[1]);
  rk[2] = (int)(l[0] <= l[2]) + (int)(l[1] <= l[2]);
  // Sign rule: each vector's largest-magnitude component (the first of
  // equals) made positive, by XOR-ing its sign bits with that component's
  // (never zero: at least 1/sqrt(3) in a unit vector).
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float y0 = x[k][0], y1 = x[k][1], y2 = x[k][2];
    float big = (fabsf(y1) > fabsf(y0)) ? y1 : y0;
    big = (fabsf(y2) > fabsf(big)) ? y2 : big;
    const unsigned sb = __float_as_uint(big) & 0x80000000u;
    l_out[k] = l[k];
    U[0 * 3 + k] = __uint_as_float(__float_as_uint(y0) ^ sb);
    U[1 * 3 + k] = __uint_as_float(__float_as_uint(y1) ^ sb);
    U[2 * 3 + k] = __uint_as_float(__float_as_uint(y2) ^ sb);
  }
}

// Eigenvalues back to the input's scale, l * 2^e: one exact multiply when
// 2^e is a normal float, scalbnf otherwise (the range check once per lane).
__device__ __forceinline__ void unscale3(float l[3], int e) {
  if (e >= -126 && e <= 127) {
    const float sc = pow2f(e);
#pragma unroll
    for (int k = 0; k < 3; ++k) l[k] *= sc;
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k) l[k] = scalbnf(l[k], e);
  }
}

// FP64 refinement of one flagged lane (compensated form): the arrow and the
// FP32 roots f[0..8] = (a1, a2, b1, b2, g, c, s, mu, nu), code = e << 2 | cls.
// A final FP64 Newton step on mu and nu (Sec. 1.4.2), eigenvectors re-formed
// in FP64; with `rec` (the input record), the FP64 residual check
// ||A u - lambda u|| <= 16 eps32 ||A||_F, whose failure is returned.
__device__ __forceinline__ bool refine_one(const float f[9], const int code, const float* rec, double lam[3],
                                        double U[9]) {
  f64::Lane D;
  D.a1 = f[0]; D.a2 = f[1]; D.b1 = f[2]; D.b2 = f[3]; D.g = f[4]; D.c = f[5]; D.s = f[6];
  D.cls = code & 3;
  D.e = code >> 2;
  double mu = f[7], nu = f[8];
  if (D.cls == kRed) {
    const double ab = D.a1 - D.a2, bb1 = D.b1 * D.b1, bb2 = D.b2 * D.b2;
    const double rab = rcp64(ab);
    const double g0 = D.g - D.a1, g1 = D.a2 - D.g;
    const double c0 = bb2 * rab, c1 = bb1 * rab;
    if (mu > 0.0) mu = f64::newton64(ab, bb1, bb2, g0, c0, -g0 - c0, mu);
    if (nu > 0.0) nu = f64::newton64(ab, bb2, bb1, g1, c1, -g1 - c1, nu);
  }
  f64::finish_lane(D, mu, nu, lam, U);
  if (rec == nullptr) return false;
  const double M[3][3] = {{rec[0], rec[3], rec[4]}, {rec[3], rec[1], rec[5]}, {rec[4], rec[5], rec[2]}};
  double nA = 0.0, worst = 0.0;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) nA = fma(M[r][q], M[r][q], nA);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double rr = 0.0;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const double v = fma(M[r][0], U[k], fma(M[r][1], U[3 + k], fma(M[r][2], U[6 + k], -lam[k] * U[r * 3 + k])));
      rr = fma(v, v, rr);
    }
    worst = fmax(worst, rr);
  }
  return !(worst <= kResidualTol * kResidualTol * nA);
}

// kMode: kPlain (SYEV3_F32), kInline (compensated, flagged lanes refined in
// FP64 inside the kernel on a shared-memory list) or kDeferred (compensated,
// flagged lanes appended to a list in global memory -- the workspace of
// syev3_batched_ws -- and refined by k_refine_f32; the kernel then holds no
// FP64 code and needs fewer registers).
// kVectors = false (plain mode only): eigenvalues only, U_out NULL.
// kServe: the serving build (plain or in-kernel compensated).  The tiles are
// those of the device-resident work list `list` (A, n, lam_out and U_out are
// unused), each with its own input and output rows; a tile's input is
// bulk-copied from its first 16-byte boundary-aligned record on, or loaded
// with plain loads when its start is not 16-byte aligned.  The production
// builds (kServe = false) compile this out.
template <bool kBulkIn, int kMode, bool kVectors = true, bool kServe = false>
__global__ void __launch_bounds__(kTPB) k_syev3_f32(const float* __restrict__ A, int64_t n,
                                                    float* __restrict__ lam_out, float* __restrict__ U_out,
                                                    unsigned long long* __restrict__ counters,
                                                    FlagRec* __restrict__ flag_list,
                                                    unsigned long long* __restrict__ flag_count,
                                                    const ServeList* __restrict__ list) {
  static_assert(!kServe || (kBulkIn && kMode != kDeferred && kVectors), "the serving build is bulk, vectors");
  static_assert(kTPB == kServeTile, "serving tiles are solve tiles");
  constexpr bool kComp = kMode != kPlain;
  constexpr bool kDefer = kMode == kDeferred;
  __shared__ alignas(16) float s_in[2][kTPB * 6];
  __shared__ alignas(16) float s_lam[kTPB * 3];
  __shared__ alignas(16) float s_U[kTPB * 9];
  // Compensated form, refinement in the kernel: the list of flagged lanes,
  // kFA floats each (arrow, roots, then the input record for the residual
  // check), their codes and global indices.  Slots [0, nfc) hold the lanes
  // carried from earlier tiles (fewer than 32), then this tile's.
  constexpr int kFA = 15, kFW = kTPB + 32;
  constexpr bool kInl = kMode == kInline;
  __shared__ float s_fa[kInl ? kFA * kFW : 1];
  __shared__ int s_fc[kInl ? kFW : 1];
  __shared__ int64_t s_fg[kInl ? kFW : 1];
  __shared__ int s_nflag;
  __shared__ alignas(8) uint64_t s_bar[2];
  // Serving build: the tile of each buffer; the eigenvector row of each
  // flagged lane in the list (s_fg then holds its eigenvalue row's address).
  __shared__ TileRef<float> s_ref[kServe ? 2 : 1];
  __shared__ float* s_fU[(kServe && kInl) ? kFW : 1];

  const int tid = threadIdx.x, lane_id = tid & 31;
  const unsigned lt_mask = (1u << lane_id) - 1u;
  const int64_t n_tiles = kServe ? list->n_tiles : (n + kTPB - 1) / kTPB;
  bool want_U = (U_out != nullptr);
  bool vec_lam = ((reinterpret_cast<uintptr_t>(lam_out) & 15) == 0);
  bool vec_U = want_U && ((reinterpret_cast<uintptr_t>(U_out) & 15) == 0);
  int64_t cursor = 0;  // serving build: item cursor of the tiles this CTA issues (thread 0)

  if (tid == 0) {
    s_nflag = 0;
    if (kBulkIn) {
      mbar_init(&s_bar[0], 1);
      mbar_init(&s_bar[1], 1);
      fence_mbar_init();
    }
  }
  __syncthreads();

  // Bulk-copy part of a tile: its first (cnt * 24) & ~15 bytes; the odd last
  // record of a tile with an odd count (8 bytes past a 16-byte boundary) is
  // loaded with plain loads after the wait.
  auto issue = [&](int64_t tile, int buf) {
    if constexpr (kServe) {
      const TileRef<float> r = serve_tile<float>(list, tile, cursor);
      s_ref[buf] = r;
      const uint32_t bytes = (reinterpret_cast<uintptr_t>(r.src) & 15) ? 0u : (((uint32_t)r.cnt * 24u) & ~15u);
      if (bytes == 0) {  // plain loads after the wait
        mbar_arrive(&s_bar[buf]);
        return;
      }
      mbar_arrive_expect_tx(&s_bar[buf], bytes);
      bulk_g2s(s_in[buf], r.src, bytes, &s_bar[buf]);
      return;
    }
    const int64_t base = tile * kTPB;
    const int cnt = (int)((n - base) < kTPB ? (n - base) : kTPB);
    const uint32_t bytes = ((uint32_t)cnt * 24u) & ~15u;
    mbar_arrive_expect_tx(&s_bar[buf], bytes);
    if (bytes) bulk_g2s(s_in[buf], A + base * 6, bytes, &s_bar[buf]);
  };

  uint32_t phases = 0u;
  int nfc = 0;  // flagged lanes carried into this tile (CTA-uniform)
  int buf = 0;
  int64_t tile = blockIdx.x;
  if (kBulkIn && tid == 0 && tile < n_tiles) issue(tile, 0);

  for (; tile < n_tiles; tile += gridDim.x, buf ^= 1) {
    const int64_t base = tile * kTPB;
    int cnt = (int)((n - base) < kTPB ? (n - base) : kTPB);
    const int64_t next = tile + gridDim.x;
    if (kBulkIn) {
      if (tid == 0 && next < n_tiles) issue(next, buf ^ 1);
      const bool ok = mbar_wait(&s_bar[buf], (phases >> buf) & 1u);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(&g_flags32, kFlagWaitTimeout);
        mbar_wait(&s_bar[buf], (phases >> buf) & 1u);
        if (next < n_tiles) mbar_wait(&s_bar[buf ^ 1], (phases >> (buf ^ 1)) & 1u);
        return;
      }
      phases ^= 1u << buf;
      if constexpr (kServe) {
        const TileRef<float> r = s_ref[buf];
        cnt = r.cnt;
        want_U = (r.U != nullptr);
        vec_lam = ((reinterpret_cast<uintptr_t>(r.lam) & 15) == 0);
        vec_U = want_U && ((reinterpret_cast<uintptr_t>(r.U) & 15) == 0);
        const int done_f =
            (reinterpret_cast<uintptr_t>(r.src) & 15) ? 0 : (int)((((uint32_t)cnt * 24u) & ~15u) / 4u);
        for (int i = done_f + tid; i < cnt * 6; i += kTPB) s_in[buf][i] = r.src[i];
        if (done_f < cnt * 6) __syncthreads();
      } else {
        const int done_f = (int)((((uint32_t)cnt * 24u) & ~15u) / 4u);
        for (int i = done_f + tid; i < cnt * 6; i += kTPB) s_in[buf][i] = A[base * 6 + i];
        if (done_f < cnt * 6) __syncthreads();
      }
    } else {
      for (int i = tid; i < cnt * 6; i += kTPB) s_in[buf][i] = A[base * 6 + i];
      __syncthreads();
    }

    Lane32 L;
    L.cls = kIdle;
    L.near_defl = false;
    float a_in[6];
    if (tid < cnt) {
      const float2* src = reinterpret_cast<const float2*>(&s_in[buf][tid * 6]);
      const float2 p0 = src[0], p1 = src[1], p2 = src[2];
      a_in[0] = p0.x; a_in[1] = p0.y; a_in[2] = p1.x; a_in[3] = p1.y; a_in[4] = p2.x; a_in[5] = p2.y;
      L = make_lane32<kComp>(a_in);
    }
    // Plain and workspace forms: the warp's lanes that form eigenpairs (taken
    // where all 32 are together), which rejoin after the class-specific part
    // of the solve.
    unsigned fin_mask = 0u;
    if constexpr (kMode != kInline) fin_mask = __ballot_sync(0xffffffffu, L.cls != kIdle && L.cls != kNonFin);

    // Roots (Sec. 1.2): problem 0 is mu, problem 1 is nu (spikes swapped).
    float root[2] = {0.f, 0.f};
    bool capped = false;
    bool more[2] = {false, false};
    float ab = 0.f, pb1[2] = {0.f, 0.f}, pb2[2] = {0.f, 0.f}, pg[2] = {0.f, 0.f};
    if (L.cls == kRed) {
      ab = L.a1 - L.a2;
      if constexpr (kMode != kInline) {
        roots_setup32(L, ab, pb1, pb2, pg);
        const P2 rab = pp(rcp32(ab)), b1p = make_float2(pb1[0], pb1[1]), b2p = make_float2(pb2[0], pb2[1]);
        const P2 g2 = make_float2(pg[0], pg[1]);
        const P2 pc = pmul(b2p, rab);
        roots32x2(pp(ab), rab, b1p, b2p, g2, pc, psub(make_float2(-g2.x, -g2.y), pc), root, more);
      } else {
        const float bb1 = L.b1 * L.b1, bb2 = L.b2 * L.b2;
        pb1[0] = bb1; pb1[1] = bb2; pb2[0] = bb2; pb2[1] = bb1;
        pg[0] = L.g - L.a1; pg[1] = L.a2 - L.g;
        const float rab = rcp32(ab);
        const float pc[2] = {pb2[0] * rab, pb2[1] * rab};
        const float pK[2] = {-pg[0] - pc[0], -pg[1] - pc[1]};
        roots32(ab, pb1, pb2, pg, pc, pK, root, more);
      }
    }
    // Rare: roots still moving after the straight-line steps, finished in
    // their own lanes (the warp runs this only when one of its roots needs it).
    if (__any_sync(0xffffffffu, more[0] || more[1])) {
      float xa = root[0], xb = root[1];
      bool ca = false, cb = false;
      if (more[0]) ca = !roots32_more(ab, pb1[0], pb2[0], pg[0], &xa);
      if (more[1]) cb = !roots32_more(ab, pb1[1], pb2[1], pg[1], &xb);
      root[0] = xa;
      root[1] = xb;
      capped = capped || ca || cb;
    }
    if (L.cls == kRed) {
      if (kComp) {
        if constexpr (kMode == kInline) {
          // Exact FP32 data as double-float, then one Newton correction with
          // a double-float f at each root (both problems paired; the
          // workspace form keeps the scalar code: its 47 registers leave room
          // for the refinement CTAs beside it).
          const F2 abf = two_sum(L.a1, -L.a2);
          const P2 abh = pp(abf.h), abl = pp(abf.l), rabh = pp(rcp32(abf.h));
          // spikes (b1^2, b2^2) exactly; problem 1 has them swapped
          const P2 B = make_float2(L.b1, L.b2);
          const P2 bh = pmul(B, B), bl = pfma(B, B, pneg(bh));
          const P2 sbh = make_float2(bh.y, bh.x), sbl = make_float2(bl.y, bl.x);
          P2 gh, gl;  // (g - a1, a2 - g) exactly
          ptwo_sum(make_float2(L.g, L.a2), make_float2(-L.a1, -L.g), gh, gl);
          // c = b2 / abar and K = -(g + c) as unnormalised pairs.
          const P2 ch = pmul(sbh, rabh);
          const P2 cl = pmul(pfma(pneg(ch), abl, padd(pfma(pneg(ch), abh, sbh), sbl)), rabh);
          P2 th, tl;
          ptwo_sum(gh, ch, th, tl);
          const P2 Kh = pneg(th), Kl = pneg(padd(padd(tl, gl), cl));
          const P2 xr = newton_ff2(abh, abl, bh, bl, sbh, sbl, pneg(gh), pneg(gl), ch, cl, Kh, Kl,
                                   make_float2(root[0], root[1]));
          root[0] = xr.x;
          root[1] = xr.y;
        } else {
          const F2 abf = two_sum(L.a1, -L.a2);
          const float rabh = rcp32(abf.h);
          const F2 fb1 = two_prod(L.b1, L.b1), fb2 = two_prod(L.b2, L.b2);
          const F2 fg0 = two_sum(L.g, -L.a1), fg1 = two_sum(L.a2, -L.g);
          // c = b2 / abar and K = -(g + c) as unnormalised pairs.
          auto div_pair = [rabh, abf](const F2 num) {
            const float q = num.h * rabh;
            return F2{q, ((fmaf(-q, abf.h, num.h) + num.l) - q * abf.l) * rabh};
          };
          auto neg_sum_pair = [](const F2 a, const F2 b) {
            const F2 t = two_sum(a.h, b.h);
            return F2{-t.h, -((t.l + a.l) + b.l)};
          };
          const F2 fc0 = div_pair(fb2), fc1 = div_pair(fb1);
          const F2 fK0 = neg_sum_pair(fg0, fc0), fK1 = neg_sum_pair(fg1, fc1);
          root[0] = newton_ff(abf, fb1, fb2, fg0, fc0, fK0, root[0]);
          root[1] = newton_ff(abf, fb2, fb1, fg1, fc1, fK1, root[1]);
        }
      }
    }

    bool flagged = false, nonfinite = false;
    int rk[3] = {0, 1, 2};  // rank of each eigenpair (ascending); identity for the other paths
    if (L.cls != kIdle) {
      float l[3], U[9];
      if (L.cls == kNonFin) {
        nonfinite = true;
        const float qnan = __int_as_float(0x7fc00000);
#pragma unroll
        for (int k = 0; k < 3; ++k) l[k] = qnan;
#pragma unroll
        for (int k = 0; k < 9; ++k) U[k] = qnan;
      } else if (!kVectors) {
        finish32_values<kMode == kPlain>(L, root[0], root[1], l, fin_mask);
        unscale3(l, L.e);
      } else {
        finish32<kMode != kInline>(L, root[0], root[1], l, U, rk, fin_mask);
        if (kComp && L.cls != kDiag) {
          // the eigenvalues' gaps in ascending order (min, median, max)
          const float lo = fminf(fminf(l[0], l[1]), l[2]), hi = fmaxf(fmaxf(l[0], l[1]), l[2]);
          const float md = fmaxf(fminf(l[0], l[1]), fminf(fmaxf(l[0], l[1]), l[2]));
          const float nrm2 = fmaf(lo, lo, fmaf(md, md, hi * hi));
          const float gap = fminf(md - lo, hi - md);
          flagged = capped || L.near_defl || (gap * gap < (kClusterTau * kClusterTau) * nrm2);
        }
        unscale3(l, L.e);
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) s_lam[tid * 3 + rk[k]] = l[k];
      if (kVectors) {
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int i = 0; i < 3; ++i) s_U[tid * 9 + i * 3 + rk[k]] = U[i * 3 + k];
      }
    }

    if (kDefer) {
      // Append the flagged lanes to the global list (one atomic per warp and
      // class): reduced arrows from the front (count [0]), the other classes
      // from the back (count [1]), so that k_refine_f32 runs each class in
      // whole warps; it refines them and overwrites their outputs.
      const bool fr = flagged && L.cls == kRed;
      const unsigned mr = __ballot_sync(0xffffffffu, fr);
      const unsigned mo = __ballot_sync(0xffffffffu, flagged && !fr);
      unsigned long long br = 0, bo = 0;
      if (lane_id == 0) {
        if (mr) br = atomicAdd(&flag_count[0], (unsigned long long)__popc(mr));
        if (mo) bo = atomicAdd(&flag_count[1], (unsigned long long)__popc(mo));
      }
      br = __shfl_sync(0xffffffffu, br, 0);
      bo = __shfl_sync(0xffffffffu, bo, 0);
      if (flagged) {
        FlagRec r;
        r.v[0] = L.a1; r.v[1] = L.a2; r.v[2] = L.b1; r.v[3] = L.b2; r.v[4] = L.g; r.v[5] = L.c; r.v[6] = L.s;
        r.v[7] = root[0]; r.v[8] = root[1];
        r.code = (L.e << 2) | L.cls;
        r.gidx = base + tid;
        const int64_t at = fr ? (int64_t)(br + __popc(mr & lt_mask)) : n - 1 - (int64_t)(bo + __popc(mo & lt_mask));
        flag_list[at] = r;
      }
    } else if (kComp) {
      // Compact the flagged lanes after the carried ones and refine a whole
      // number of warps' worth of them in FP64, with every lane of the CTA
      // available; the rest (fewer than 32) are carried to the next tile, so
      // no warp runs the FP64 code with idle lanes.  A lane of this tile
      // gets its refined result in the staging area, a carried one straight
      // in memory (over the FP32 result written with its own tile).  The
      // CTA refines its last carried lanes after its final tile.
      const unsigned m = __ballot_sync(0xffffffffu, flagged);
      int wbase = 0;
      if (lane_id == 0 && m) wbase = atomicAdd(&s_nflag, __popc(m));
      wbase = __shfl_sync(0xffffffffu, wbase, 0);
      if (flagged) {
        const int slot = nfc + wbase + __popc(m & lt_mask);
        float* f = &s_fa[slot * kFA];
        f[0] = L.a1; f[1] = L.a2; f[2] = L.b1; f[3] = L.b2; f[4] = L.g; f[5] = L.c; f[6] = L.s;
        f[7] = root[0]; f[8] = root[1];
#pragma unroll
        for (int k = 0; k < 6; ++k) f[9 + k] = a_in[k];
        s_fc[slot] = (L.e << 2) | L.cls;
        if constexpr (kServe) {
          const TileRef<float> r = s_ref[buf];
          s_fg[slot] = (int64_t)reinterpret_cast<uintptr_t>(r.lam + tid * 3);
          s_fU[slot] = r.U ? r.U + tid * 9 : nullptr;
        } else {
          s_fg[slot] = base + tid;
        }
      }
      __syncthreads();
      const int n_avail = nfc + s_nflag;
      const int P = n_avail & ~31;
      for (int i = tid; i < P; i += kTPB) {
        double lam[3], U[9];
        // The residual check (counter [3]) only when counters are asked for.
        const bool bad = refine_one(&s_fa[i * kFA], s_fc[i], counters != nullptr ? &s_fa[i * kFA + 9] : nullptr,
                                    lam, U);
        if (bad) atomicAdd(&counters[3], 1ull);
        const int64_t gi = s_fg[i];
        int64_t row;
        float *dl_far, *dU_far;  // where a lane of an earlier tile writes
        if constexpr (kServe) {
          const int64_t d = (int64_t)(uintptr_t)gi - (int64_t)reinterpret_cast<uintptr_t>(s_ref[buf].lam);
          row = (d >= 0 && d < (int64_t)cnt * 12) ? d / 12 : -1;
          dl_far = reinterpret_cast<float*>((uintptr_t)gi);
          dU_far = s_fU[i];
        } else {
          row = gi - base;
          dl_far = lam_out + gi * 3;
          dU_far = want_U ? U_out + gi * 9 : nullptr;
        }
        const bool here = row >= 0 && row < cnt;
        float* dl = here ? &s_lam[row * 3] : dl_far;
#pragma unroll
        for (int k = 0; k < 3; ++k) dl[k] = (float)lam[k];
        if (here || dU_far != nullptr) {
          float* dU = here ? &s_U[row * 9] : dU_far;
#pragma unroll
          for (int k = 0; k < 9; ++k) dU[k] = (float)U[k];
        }
      }
      __syncthreads();
      const int nc_next = n_avail - P;
      if (P > 0 && tid < nc_next) {  // [P, n_avail) -> [0, nc_next): no overlap, P >= 32 > nc_next
#pragma unroll
        for (int k = 0; k < kFA; ++k) s_fa[tid * kFA + k] = s_fa[(P + tid) * kFA + k];
        s_fc[tid] = s_fc[P + tid];
        s_fg[tid] = s_fg[P + tid];
        if constexpr (kServe) s_fU[tid] = s_fU[P + tid];
      }
      nfc = nc_next;
    }
    if (counters != nullptr) {
      const unsigned cm = __ballot_sync(0xffffffffu, capped);
      const unsigned nf = __ballot_sync(0xffffffffu, nonfinite);
      const unsigned fl = __ballot_sync(0xffffffffu, flagged);
      if (lane_id == 0) {
        if (cm) atomicAdd(&counters[0], (unsigned long long)__popc(cm));
        if (nf) atomicAdd(&counters[1], (unsigned long long)__popc(nf));
        if (fl) atomicAdd(&counters[2], (unsigned long long)__popc(fl));
      }
    }
    __syncthreads();
    if (tid == 0) s_nflag = 0;

    {
      float* dst = kServe ? s_ref[buf].lam : lam_out + base * 3;
      const int m = cnt * 3;
      if (vec_lam) {
        float4* d4 = reinterpret_cast<float4*>(dst);
        const float4* s4 = reinterpret_cast<const float4*>(s_lam);
        for (int i = tid; i < m / 4; i += kTPB) d4[i] = s4[i];
        for (int i = (m & ~3) + tid; i < m; i += kTPB) dst[i] = s_lam[i];
      } else {
        for (int i = tid; i < m; i += kTPB) dst[i] = s_lam[i];
      }
    }
    if (want_U) {
      float* dst = kServe ? s_ref[buf].U : U_out + base * 9;
      const int m = cnt * 9;
      if (vec_U) {
        float4* d4 = reinterpret_cast<float4*>(dst);
        const float4* s4 = reinterpret_cast<const float4*>(s_U);
        for (int i = tid; i < m / 4; i += kTPB) d4[i] = s4[i];
        for (int i = (m & ~3) + tid; i < m; i += kTPB) dst[i] = s_U[i];
      } else {
        for (int i = tid; i < m; i += kTPB) dst[i] = s_U[i];
      }
    }
    __syncthreads();
  }
  if (kInl) {
    // The flagged lanes still carried after the CTA's final tile (nfc is
    // CTA-uniform; the list was completed before the loop's last barrier).
    for (int i = tid; i < nfc; i += kTPB) {
      double lam[3], U[9];
      const bool bad = refine_one(&s_fa[i * kFA], s_fc[i], counters != nullptr ? &s_fa[i * kFA + 9] : nullptr,
                                  lam, U);
      if (bad) atomicAdd(&counters[3], 1ull);
      const int64_t gi = s_fg[i];
      float* dl = kServe ? reinterpret_cast<float*>((uintptr_t)gi) : lam_out + gi * 3;
      float* dU = kServe ? s_fU[kServe ? i : 0] : (want_U ? U_out + gi * 9 : nullptr);
#pragma unroll
      for (int k = 0; k < 3; ++k) dl[k] = (float)lam[k];
      if (dU != nullptr) {
#pragma unroll
        for (int k = 0; k < 9; ++k) dU[k] = (float)U[k];
      }
    }
  }
}

template <bool kBulkIn, int kMode, bool kVectors, bool kServe = false>
int blocks_per_sm_f32() {
  static int cached = -1;
  if (cached < 0) {
    int v = 0;
    cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_syev3_f32<kBulkIn, kMode, kVectors, kServe>, kTPB, 0);
    cached = (e == cudaSuccess && v > 0) ? v : 1;
  }
  return cached;
}

// per_sm_cap > 0: at most that many CTAs per SM (room left for a kernel
// that runs beside this one).
template <bool kBulkIn, int kMode, bool kVectors = true>
cudaError_t launch(const float* A, int64_t n, float* lam, float* U, unsigned long long* counters,
                   FlagRec* flag_list, unsigned long long* flag_count, cudaStream_t stream, int sms,
                   int per_sm_cap = 0) {
  const int64_t n_tiles = (n + kTPB - 1) / kTPB;
  int per_sm = blocks_per_sm_f32<kBulkIn, kMode, kVectors>();
  if (per_sm_cap > 0 && per_sm > per_sm_cap) per_sm = per_sm_cap;
  const int64_t resident = (int64_t)sms * per_sm;
  const int grid = (int)(n_tiles < resident ? n_tiles : resident);
  k_syev3_f32<kBulkIn, kMode, kVectors>
      <<<grid, kTPB, 0, stream>>>(A, n, lam, U, counters, flag_list, flag_count, nullptr);
  return cudaGetLastError();
}

template <int kMode>
cudaError_t launch_serve(const ServeList* list, unsigned long long* counters, cudaStream_t stream, int sms) {
  // The list's length is known only on the device: a resident grid; CTAs
  // without a tile exit at once.
  const int grid = sms * blocks_per_sm_f32<true, kMode, true, true>();
  k_syev3_f32<true, kMode, true, true>
      <<<grid, kTPB, 0, stream>>>(nullptr, 0, nullptr, nullptr, counters, nullptr, nullptr, list);
  return cudaGetLastError();
}

// The refinement of the deferred compensated form: one flagged lane per
// thread, grid-stride over the list (its lengths are read on the device):
// first the reduced arrows (list front), then the other classes (list back,
// n records from the front), so each warp but one runs a single class.
constexpr int kRefineTPB = 128;

__global__ void __launch_bounds__(kRefineTPB) k_refine_f32(const FlagRec* __restrict__ list,
                                                           const unsigned long long* __restrict__ count,
                                                           int64_t n, const float* __restrict__ A,
                                                           float* __restrict__ lam_out, float* __restrict__ U_out,
                                                           unsigned long long* __restrict__ counters) {
  const unsigned long long m_red = count[0], m = m_red + count[1];
  for (unsigned long long i = (unsigned long long)blockIdx.x * kRefineTPB + threadIdx.x; i < m;
       i += (unsigned long long)gridDim.x * kRefineTPB) {
    const FlagRec r = list[i < m_red ? (int64_t)i : n - 1 - (int64_t)(i - m_red)];
    double lam[3], U[9];
    const bool bad = refine_one(r.v, r.code, counters != nullptr ? A + r.gidx * 6 : nullptr, lam, U);
    if (bad) atomicAdd(&counters[3], 1ull);
#pragma unroll
    for (int k = 0; k < 3; ++k) lam_out[r.gidx * 3 + k] = (float)lam[k];
    if (U_out != nullptr) {
#pragma unroll
      for (int k = 0; k < 9; ++k) U_out[r.gidx * 9 + k] = (float)U[k];
    }
  }
}

int refine_blocks_per_sm() {
  static int cached = -1;
  if (cached < 0) {
    int v = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_refine_f32, kRefineTPB, 0);
    cached = (e == cudaSuccess && v > 0) ? v : 1;
  }
  return cached;
}

}  // namespace

cudaError_t launch_f32(const float* A, int64_t n, float* lam, float* U, bool compensated,
                       unsigned long long* counters, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const bool bulk = (reinterpret_cast<uintptr_t>(A) & 15) == 0;
  if (bulk && !compensated && U == nullptr)
    return launch<true, kPlain, false>(A, n, lam, U, counters, nullptr, nullptr, stream, sms);
  if (bulk)
    return compensated ? launch<true, kInline>(A, n, lam, U, counters, nullptr, nullptr, stream, sms)
                       : launch<true, kPlain>(A, n, lam, U, counters, nullptr, nullptr, stream, sms);
  return compensated ? launch<false, kInline>(A, n, lam, U, counters, nullptr, nullptr, stream, sms)
                     : launch<false, kPlain>(A, n, lam, U, counters, nullptr, nullptr, stream, sms);
}

cudaError_t launch_f32_serve(const ServeList* list, bool compensated, unsigned long long* counters,
                             cudaStream_t stream) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  return compensated ? launch_serve<kInline>(list, counters, stream, sms)
                     : launch_serve<kPlain>(list, counters, stream, sms);
}

size_t f32c_workspace_bytes(int64_t n) { return kFlagListOffset + (size_t)n * sizeof(FlagRec); }

namespace {

// Pipelined deferred path: a batch of at least kPipeMin matrices is cut into
// kPipeChunks runs of whole tiles; the FP32 kernel solves the runs one after
// the other on the caller's stream, and the refinement of run c starts on a
// side stream (after an event recorded behind run c's FP32 kernel) while the
// FP32 kernel works on run c + 1.  The FP32 grid leaves room for
// kPipeRefinePerSM refinement CTAs on every SM, so the refinement -- bound by
// the FP64 pipe -- runs beside the FP32 solve, which is bound by instruction
// issue.  The caller's stream waits for the side stream at the end.  The
// side stream and the events are created once per device, and one call's
// records and waits are enqueued under a lock so that calls from several
// host threads do not interleave them.
constexpr int64_t kPipeMin = (int64_t)1 << 21;
constexpr int kPipeChunks = 8;        // counters: 2 per run, 16 B x 8 <= kFlagListOffset
// Refinement CTAs per SM beside the FP32 kernel (measured on the 2^24 mixed
// batch: 1, 2, 3, 4, 5, 6 gave 1.39, 1.33, 1.59, 1.53, 1.54, 1.48e10
// eigensolves/s; 16 runs instead of 8 were slower, 4 the same; without the
// pipeline 1.37e10).  With 3, the register file holds 9 FP32 CTAs and 2
// refinement CTAs per SM.
constexpr int kPipeRefinePerSM = 3;
static_assert(2 * sizeof(unsigned long long) * kPipeChunks <= kFlagListOffset, "run counters fit");
constexpr int kPipeMaxDevices = 64;

struct Pipe {
  cudaStream_t side = nullptr;
  cudaEvent_t ev[kPipeChunks + 1] = {};
};
std::mutex g_pipe_mu;
Pipe g_pipe[kPipeMaxDevices];

cudaError_t pipe_for(int dev, Pipe** out) {
  Pipe& P = g_pipe[dev];
  if (P.side == nullptr) {
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    for (int i = 0; i <= kPipeChunks; ++i) {
      e = cudaEventCreateWithFlags(&P.ev[i], cudaEventDisableTiming);
      if (e != cudaSuccess) {
        for (int j = 0; j < i; ++j) cudaEventDestroy(P.ev[j]);
        cudaStreamDestroy(s);
        return e;
      }
    }
    P.side = s;
  }
  *out = &P;
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_f32c_deferred(const float* A, int64_t n, float* lam, float* U, unsigned long long* counters,
                                 void* work, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  auto* count = static_cast<unsigned long long*>(work);
  auto* list = reinterpret_cast<FlagRec*>(static_cast<char*>(work) + kFlagListOffset);
  const bool bulk = (reinterpret_cast<uintptr_t>(A) & 15) == 0;
  if (n < kPipeMin || dev < 0 || dev >= kPipeMaxDevices) {
    e = cudaMemsetAsync(count, 0, 2 * sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
    e = bulk ? launch<true, kDeferred>(A, n, lam, U, counters, list, count, stream, sms)
             : launch<false, kDeferred>(A, n, lam, U, counters, list, count, stream, sms);
    if (e != cudaSuccess) return e;
    k_refine_f32<<<sms * refine_blocks_per_sm(), kRefineTPB, 0, stream>>>(list, count, n, A, lam, U, counters);
    return cudaGetLastError();
  }
  std::lock_guard<std::mutex> hold(g_pipe_mu);
  Pipe* P = nullptr;
  e = pipe_for(dev, &P);
  if (e != cudaSuccess) return e;
  // Runs of whole tiles (128 matrices: every run starts 16-byte aligned in
  // all three arrays when the batch does); run c uses counters [2c, 2c+1]
  // and the list records [start, start + len) of its own matrices.
  const int64_t len = ((n + kPipeChunks - 1) / kPipeChunks + kTPB - 1) / kTPB * kTPB;
  e = cudaMemsetAsync(count, 0, 2 * sizeof(unsigned long long) * kPipeChunks, stream);
  if (e != cudaSuccess) return e;
  const int cap = blocks_per_sm_f32<true, kDeferred, true>() - kPipeRefinePerSM;
  for (int c = 0; c < kPipeChunks; ++c) {
    const int64_t start = c * len;
    if (start >= n) break;
    const int64_t m = (n - start) < len ? (n - start) : len;
    const float* Ac = A + start * 6;
    float* lc = lam + start * 3;
    float* Uc = U ? U + start * 9 : nullptr;
    unsigned long long* cc = count + 2 * c;
    e = bulk ? launch<true, kDeferred>(Ac, m, lc, Uc, counters, list + start, cc, stream, sms, cap > 0 ? cap : 1)
             : launch<false, kDeferred>(Ac, m, lc, Uc, counters, list + start, cc, stream, sms, cap > 0 ? cap : 1);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(P->ev[c], stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P->side, P->ev[c], 0);
    if (e != cudaSuccess) return e;
    k_refine_f32<<<sms * kPipeRefinePerSM, kRefineTPB, 0, P->side>>>(list + start, cc, m, Ac, lc, Uc, counters);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  e = cudaEventRecord(P->ev[kPipeChunks], P->side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, P->ev[kPipeChunks], 0);
  return e;
}

cudaError_t take_flags_f32(unsigned* flags) {
  unsigned v = 0, zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_flags32, sizeof(v));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(g_flags32, &zero, sizeof(zero));
  *flags |= v;
  return e;
}

}  // namespace syev3
