// ddjacobi.cpp -- brute-force reference eigensolver for 3x3 symmetric
// matrices: cyclic Jacobi in double-double arithmetic.
//
// TEST INFRASTRUCTURE.  It pins the Borges oracle (syev3_oracle.cpp) from the
// outside: a different algorithm in roughly twice the working precision, so
// its eigenvalues are exact to about 1e-30 ||A|| and any dropped term, wrong
// sign or swapped index in the oracle shows up as a mismatch far above the
// oracle's 8 eps ||A||_F budget.  Shares no code with the oracle or the CUDA
// path.
//
// Double-double arithmetic follows the published error-free transformations:
//   TwoSum        (Knuth, TAOCP vol. 2, Sec. 4.2.2): a + b = s + e exactly;
//   FastTwoSum    (Dekker 1971), valid when |a| >= |b|;
//   TwoProd       via a fused multiply-add: a * b = p + e exactly;
// and the usual double-double add / mul / div / sqrt built on them (Dekker
// 1971; Hida, Li and Bailey 2001), written here from those definitions.
// Cyclic Jacobi follows Golub and Van Loan, Matrix Computations, Sec. 8.5
// (symmetric Schur decomposition of each 2x2 pivot block, row-cyclic sweeps).
//
// Build with -ffp-contract=off (the transformations need unfused a*b and a+b).

#include <cmath>
#include <cstdint>
#include <utility>

namespace {

struct dd {
  double hi, lo;
};

inline dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
inline dd fast_two_sum(double a, double b) {
  double s = a + b;
  double e = b - (s - a);
  return {s, e};
}
inline dd two_prod(double a, double b) {
  double p = a * b;
  double e = std::fma(a, b, -p);
  return {p, e};
}
inline dd mk(double x) { return {x, 0.0}; }
inline dd add(dd x, dd y) {
  dd s = two_sum(x.hi, y.hi);
  dd t = two_sum(x.lo, y.lo);
  double e = s.lo + t.hi;
  dd u = fast_two_sum(s.hi, e);
  e = u.lo + t.lo;
  return fast_two_sum(u.hi, e);
}
inline dd neg(dd x) { return {-x.hi, -x.lo}; }
inline dd sub(dd x, dd y) { return add(x, neg(y)); }
inline dd mul(dd x, dd y) {
  dd p = two_prod(x.hi, y.hi);
  double e = p.lo + (x.hi * y.lo + x.lo * y.hi);
  return fast_two_sum(p.hi, e);
}
inline dd div(dd x, dd y) {
  double q1 = x.hi / y.hi;
  dd r = sub(x, mul(mk(q1), y));
  double q2 = r.hi / y.hi;
  r = sub(r, mul(mk(q2), y));
  double q3 = r.hi / y.hi;
  dd q = fast_two_sum(q1, q2);
  return add(q, mk(q3));
}
inline dd sqrt_dd(dd x) {
  if (x.hi <= 0.0) return mk(0.0);
  // One Newton step on y^2 = x from the double square root doubles the
  // number of correct bits: y + (x - y^2) / (2 y).
  double y = std::sqrt(x.hi);
  dd yy = mk(y);
  dd r = sub(x, mul(yy, yy));
  dd corr = div(r, mk(2.0 * y));
  return add(yy, corr);
}
inline double absd(dd x) { return std::fabs(x.hi); }
inline bool lt(dd x, dd y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }

}  // namespace

extern "C" {

// Eigen-decomposition of the packed symmetric (a11,a22,a33,a12,a13,a23) by
// cyclic Jacobi in double-double.  Outputs, ascending: lam_hi[3] + lam_lo[3]
// (the double-double eigenvalues), V[9] row-major with eigenvector k in
// column k (rounded to double).  Returns the number of sweeps used.
int dd_jacobi3(const double a[6], double lam_hi[3], double lam_lo[3], double V[9]) {
  dd A[3][3] = {{mk(a[0]), mk(a[3]), mk(a[4])},
                {mk(a[3]), mk(a[1]), mk(a[5])},
                {mk(a[4]), mk(a[5]), mk(a[2])}};
  dd Q[3][3] = {{mk(1), mk(0), mk(0)}, {mk(0), mk(1), mk(0)}, {mk(0), mk(0), mk(1)}};
  double scale = 0.0;
  for (int i = 0; i < 6; ++i) scale = std::fmax(scale, std::fabs(a[i]));
  int sweep = 0;
  for (; sweep < 60; ++sweep) {
    double off = absd(A[0][1]) + absd(A[0][2]) + absd(A[1][2]);
    if (off <= 1e-34 * scale || off == 0.0) break;
    for (int p = 0; p < 2; ++p) {
      for (int q = p + 1; q < 3; ++q) {
        if (A[p][q].hi == 0.0) continue;
        // Symmetric Schur decomposition of [[A_pp, A_pq], [A_pq, A_qq]]:
        // tau = (A_qq - A_pp) / (2 A_pq), t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
        // c = 1/sqrt(1 + t^2), s = t c.
        dd tau = div(sub(A[q][q], A[p][p]), mul(mk(2.0), A[p][q]));
        dd t;
        if (std::fabs(tau.hi) > 1e150) {
          t = div(mk(0.5), tau);  // t ~ 1/(2 tau) for huge tau
        } else {
          dd rt = sqrt_dd(add(mk(1.0), mul(tau, tau)));
          dd den = add(tau.hi >= 0 ? tau : neg(tau), rt);
          t = div(mk(tau.hi >= 0 ? 1.0 : -1.0), den);
        }
        dd c = div(mk(1.0), sqrt_dd(add(mk(1.0), mul(t, t))));
        dd s = mul(t, c);
        // A <- R^T A R with R = I except R_pp = c, R_pq = s, R_qp = -s, R_qq = c.
        for (int k = 0; k < 3; ++k) {  // columns: A <- A R
          dd akp = A[k][p], akq = A[k][q];
          A[k][p] = sub(mul(c, akp), mul(s, akq));
          A[k][q] = add(mul(s, akp), mul(c, akq));
        }
        for (int k = 0; k < 3; ++k) {  // rows: A <- R^T A
          dd apk = A[p][k], aqk = A[q][k];
          A[p][k] = sub(mul(c, apk), mul(s, aqk));
          A[q][k] = add(mul(s, apk), mul(c, aqk));
        }
        A[p][q] = mk(0.0);
        A[q][p] = mk(0.0);
        for (int k = 0; k < 3; ++k) {  // Q <- Q R
          dd qkp = Q[k][p], qkq = Q[k][q];
          Q[k][p] = sub(mul(c, qkp), mul(s, qkq));
          Q[k][q] = add(mul(s, qkp), mul(c, qkq));
        }
      }
    }
  }
  int ord[3] = {0, 1, 2};
  for (int i = 1; i < 3; ++i)
    for (int j = i; j > 0 && lt(A[ord[j]][ord[j]], A[ord[j - 1]][ord[j - 1]]); --j)
      std::swap(ord[j], ord[j - 1]);
  for (int k = 0; k < 3; ++k) {
    lam_hi[k] = A[ord[k]][ord[k]].hi;
    lam_lo[k] = A[ord[k]][ord[k]].lo;
    for (int i = 0; i < 3; ++i) V[i * 3 + k] = Q[i][ord[k]].hi + Q[i][ord[k]].lo;
  }
  return sweep;
}

void dd_jacobi3_batch(const double* A, int64_t n, double* lam_hi, double* lam_lo, double* V) {
  for (int64_t m = 0; m < n; ++m) dd_jacobi3(A + 6 * m, lam_hi + 3 * m, lam_lo + 3 * m, V + 9 * m);
}

// Double-double primitives exposed for their own tests:
// op 0 add, 1 mul, 2 div, 3 sqrt (y ignored); result in out[2] = {hi, lo}.
void dd_op(int op, double xh, double xl, double yh, double yl, double out[2]) {
  dd x = {xh, xl}, y = {yh, yl}, r;
  switch (op) {
    case 0: r = add(x, y); break;
    case 1: r = mul(x, y); break;
    case 2: r = div(x, y); break;
    default: r = sqrt_dd(x); break;
  }
  out[0] = r.hi;
  out[1] = r.lo;
}

}  // extern "C"
