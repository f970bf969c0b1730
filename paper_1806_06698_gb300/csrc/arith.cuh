// arith.cuh -- arithmetic primitives of the eigensolver kernels (sm_103a).
#pragma once

#include <cmath>
#include <cstdint>

namespace syev3 {
namespace {  // internal linkage: every translation unit gets its own copy

// 1/x: the hardware's reciprocal estimate y (relative error below 2^-20,
// subnormal results flushed) refined by one step of the third-order
// Newton-Raphson iteration for the reciprocal: with e = 1 - x y (one FMA,
// exact to rounding), 1/x = y / (1 - e) = y (1 + e + e^2 + e^3 + ...), and
// truncating after e^2 leaves a relative error of order e^3 ~ 2^-60 (the
// classical iteration for division, e.g. Muller et al., Handbook of
// Floating-Point Arithmetic, 2nd ed. 2018, on Newton-Raphson-based division).
// The final FMA rounds once, so the result is within 1 ulp of 1/x for
// 2^-1000 < |x| < 2^1000; syev3_selftest_arith exposes it to the tests that
// check this against IEEE division.
__device__ __forceinline__ double rcp64(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

// FP32 hardware approximations (flush-to-zero): 1/x, sqrt(x) and 1/sqrt(x).
// The FP32 zero finder's error allowances assume each within a few units of
// 2^-23 relative; syev3_selftest_arith exposes them to the tests of that.
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

__device__ __forceinline__ float rsqrt32(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 2^k for -1022 <= k <= 1023, built from its exponent field.
__device__ __forceinline__ double pow2(int k) { return __hiloint2double((k + 1023) << 20, 0); }

// Comparisons of doubles whose signs are known, on the integer pipes (the
// FP64 pipe is the scarce one).  For x, y >= +0, not NaN, x < y exactly when
// their bit patterns compare so as unsigned integers; against 2^k (low word
// zero) the high words alone decide.  x > 0 for a non-NaN x is a signed
// comparison of the pattern with 0.
__device__ __forceinline__ uint64_t dbits(double x) { return (uint64_t)__double_as_longlong(x); }

// High word of 2^k, -1022 <= k <= 1023.
__host__ __device__ constexpr unsigned hi_pow2(int k) { return (unsigned)(k + 1023) << 20; }

// High word of |x|.
__device__ __forceinline__ unsigned hi_mag(double x) { return (unsigned)__double2hiint(x) & 0x7fffffffu; }

// x > 0 (x not NaN).
__device__ __forceinline__ bool is_pos(double x) { return __double_as_longlong(x) > 0; }

// x == +0 or -0.
__device__ __forceinline__ bool is_zero(double x) { return (dbits(x) << 1) == 0; }

// x * 2^k by exponent arithmetic for x >= 2^-1022 in magnitude (normal) when
// the result is normal too; otherwise scalbn.  Zero stays zero.
__device__ __forceinline__ double mul_pow2(double x, int k) {
  const int h = __double2hiint(x);
  const int ne = ((h >> 20) & 0x7ff) + k;
  if (((h >> 20) & 0x7ff) != 0 && ne >= 1 && ne <= 2046) return __hiloint2double(h + k * (1 << 20), __double2loint(x));
  if (is_zero(x)) return x;
  return scalbn(x, k);
}

// |x| as an unsigned integer that orders like |x| (any non-NaN x).
__device__ __forceinline__ uint64_t mag_bits(double x) {
  return (uint64_t)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// x with its sign bit XOR-ed with bit 31 of `flip` (0 or 0x80000000).
__device__ __forceinline__ double flip_sign(double x, int flip) {
  return __hiloint2double(__double2hiint(x) ^ flip, __double2loint(x));
}

// 2^k as a float for -126 <= k <= 127.
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

// FP32 <-> FP64 conversions on the integer pipes.  On this GPU a conversion
// instruction between the two formats issues to the FP64 pipe, the scarce
// one (2 lanes per clock per SM), while the integer pipes have room to
// spare in the FP64-bound kernels.  Zero and normal numbers -- everything
// the kernels convert in practice -- are converted on 32-bit words; the
// rest (subnormal results or operands, infinities, NaN) take the hardware
// conversion in a branch.  The results are the IEEE ones bit for bit
// (checked against the hardware conversions by syev3_selftest_arith).
//
// float -> double, exact: a normal float's exponent is rebiased by
// 1023 - 127 = 896 and its 23-bit fraction split over the two words.
__device__ __forceinline__ double f2d_exact(const float x) {
  const unsigned u = __float_as_uint(x), a = u & 0x7fffffffu;
  if (a - 0x00800000u < 0x7f000000u)  // normal
    return __hiloint2double((int)((u & 0x80000000u) | ((a >> 3) + (896u << 20))), (int)(a << 29));
  if (a == 0u) return __hiloint2double((int)u, 0);
  return (double)x;
}

// double -> float, rounded to nearest, ties to even (the IEEE default): in
// the float normal range the top 23 fraction bits are kept and the 29 below
// decide the rounding; a carry out of the fraction steps the exponent (up to
// infinity, the correctly rounded overflow).
__device__ __forceinline__ float d2f_rn(const double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned E = (hi >> 20) & 0x7ffu;
  if (E - 897u <= 253u) {  // float exponent 1..254
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29), rem = lo & 0x1fffffffu;
    unsigned f = ((E - 896u) << 23) + m;
    f += (unsigned)(rem > 0x10000000u) | ((unsigned)(rem == 0x10000000u) & (f & 1u));
    return __uint_as_float((hi & 0x80000000u) | f);
  }
  if (((hi & 0x7fffffffu) | lo) == 0u) return __uint_as_float(hi);  // +-0
  return __double2float_rn(x);
}

// ---------------------------------------------------------------------------
// Double-float arithmetic: an unevaluated sum h + l of two floats, built on
// the error-free transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2),
// FastTwoSum (Dekker 1971, |a| >= |b|) and TwoProd via FMA.  These carry
// about 48 bits, enough to evaluate a secular function or a deflation test
// without the rounding of its FP32 products.
// ---------------------------------------------------------------------------

struct F2 {
  float h, l;
};

__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ F2 two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ F2 ff_add(F2 x, F2 y) {
  const F2 s = two_sum(x.h, y.h);
  return fast_two_sum(s.h, s.l + (x.l + y.l));
}

__device__ __forceinline__ F2 ff_mul(F2 x, F2 y) {
  const F2 p = two_prod(x.h, y.h);
  return fast_two_sum(p.h, fmaf(x.h, y.l, fmaf(x.l, y.h, p.l)));
}

__device__ __forceinline__ F2 ff_mul1(F2 x, float y) {
  const F2 p = two_prod(x.h, y);
  return fast_two_sum(p.h, fmaf(x.l, y, p.l));
}

__device__ __forceinline__ bool ff_le(F2 x, F2 y) { return x.h < y.h || (x.h == y.h && x.l <= y.l); }

}  // namespace
}  // namespace syev3
