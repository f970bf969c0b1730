// syev3_oracle.cpp -- CPU FP64 oracle for the batched 3x3 real symmetric
// eigensolver of C. F. Borges, "Solving the 3x3 Real Symmetric Eigenproblem"
// (arXiv 1806.06698).
//
// TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
// CPU-baseline leg load this library.  It shares no code, header, table or
// helper with the CUDA path and must never be called from the product path.
//
// It is deliberately plain and slow: one matrix at a time, scalar FP64, the
// steps in the paper's order and notation.  Every function names the passage
// it follows.  Where the paper is silent the code says "reading:" and states
// the choice made (the same list is kept in the design notes).
//
// The arithmetic is written once, templated on the scalar type.  With
// T = double it is the oracle; with T = Counted it counts the algorithmic
// floating-point operations (add/sub, mul, div, sqrt) per matrix.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared (no fast-math,
// no contraction, so x86-64 and aarch64 hosts give bit-identical results).

#include <algorithm>
#include <cfloat>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Scalar types
// ---------------------------------------------------------------------------

struct OpCounts {
  uint64_t add = 0, mul = 0, div = 0, sqrt = 0;
};
thread_local OpCounts* tl_ops = nullptr;

// A double that counts the operations applied to it (flop accounting only).
struct Counted {
  double v;
  Counted(double x = 0.0) : v(x) {}
};
inline Counted operator+(Counted a, Counted b) { if (tl_ops) tl_ops->add++; return Counted(a.v + b.v); }
inline Counted operator-(Counted a, Counted b) { if (tl_ops) tl_ops->add++; return Counted(a.v - b.v); }
inline Counted operator*(Counted a, Counted b) { if (tl_ops) tl_ops->mul++; return Counted(a.v * b.v); }
inline Counted operator/(Counted a, Counted b) { if (tl_ops) tl_ops->div++; return Counted(a.v / b.v); }
inline Counted operator-(Counted a) { return Counted(-a.v); }
inline bool operator<(Counted a, Counted b) { return a.v < b.v; }
inline bool operator>(Counted a, Counted b) { return a.v > b.v; }
inline bool operator<=(Counted a, Counted b) { return a.v <= b.v; }
inline bool operator>=(Counted a, Counted b) { return a.v >= b.v; }
inline bool operator==(Counted a, Counted b) { return a.v == b.v; }
inline Counted sqrt(Counted a) { if (tl_ops) tl_ops->sqrt++; return Counted(std::sqrt(a.v)); }
inline Counted fabs(Counted a) { return Counted(std::fabs(a.v)); }
// hypot is counted as its defining formula sqrt(x*x + y*y).
inline Counted hypot(Counted a, Counted b) {
  if (tl_ops) { tl_ops->mul += 2; tl_ops->add += 1; tl_ops->sqrt += 1; }
  return Counted(std::hypot(a.v, b.v));
}
inline double val(double x) { return x; }
inline double val(Counted x) { return x.v; }

// ---------------------------------------------------------------------------
// Parameters ("for some constant C", Sec. 1.1 and Sec. 1.4.1)
// ---------------------------------------------------------------------------

constexpr double EPS = DBL_EPSILON;  // reading: epsilon = 2^-52
constexpr double kTinySpike = 0x1p-480; // reading: spikes below this are zeroed (see solve_one)

struct Params {
  double c_defl = 1.0;    // reading: C in the deflation test of Sec. 1.1
  double c_term = 2.0;    // reading: C in the stopping rule of Sec. 1.4.1 / 1.4.2
  int maxit = 64;         // reading: iteration cap (the paper proves convergence)
  int deflation_test = 0; // 0: simplified test of Sec. 1.1; 1: the EISPACK-style test it starts from
  int zero_finder = 0;    // 0: Borges-Gragg (Sec. 1.4.1); 1: Newton (Sec. 1.4.2)
};

// ---------------------------------------------------------------------------
// Sec. 1: ordered Jacobi rotation of the leading 2x2 [[p, q], [q, r]].
//
// The paper cites an unavailable construction.  Reading: the eigenvector of
// the larger eigenvalue is formed without cancellation as (1, t) when
// p >= r or (t, 1) when p < r, with t = q / (|d| + hypot(d, q)) and
// d = (p - r)/2, so |t| <= 1.  Returns l1 >= l2, (c, s) the unit eigenvector
// of l1; (-s, c) is the eigenvector of l2.  The ordering l1 >= l2 holds in
// floating point because rounding is monotone: l1 = p + t*q >= p >= r >=
// r - t*q = l2 when p >= r (t*q >= 0), and symmetrically otherwise.
// ---------------------------------------------------------------------------

template <class T>
struct Rot2 {
  T c, s, l1, l2;
};

template <class T>
Rot2<T> ordered_jacobi(T p, T q, T r) {
  using std::hypot;
  using std::sqrt;
  Rot2<T> J;
  if (q == T(0.0)) {
    if (p >= r) {
      J.c = 1.0; J.s = 0.0; J.l1 = p; J.l2 = r;
    } else {
      J.c = 0.0; J.s = 1.0; J.l1 = r; J.l2 = p;
    }
    return J;
  }
  T d = (p - r) * T(0.5);
  T rad = hypot(d, q);
  if (d >= T(0.0)) {
    T t = q / (d + rad);
    J.l1 = p + t * q;
    J.l2 = r - t * q;
    T k = T(1.0) / sqrt(T(1.0) + t * t);
    J.c = k;
    J.s = t * k;
  } else {
    T t = q / (rad - d);
    J.l1 = r + t * q;
    J.l2 = p - t * q;
    T k = T(1.0) / sqrt(T(1.0) + t * t);
    J.c = t * k;
    J.s = k;
  }
  return J;
}

// ---------------------------------------------------------------------------
// Sec. 1: the similarity by J = [[c,-s,0],[s,c,0],[0,0,1]] turns the packed
// matrix (a11,a22,a33,a12,a13,a23) into the ordered arrow
// [[alpha1, 0, beta1], [0, alpha2, beta2], [beta1, beta2, gamma]].
// ---------------------------------------------------------------------------

template <class T>
struct ArrowT {
  T a1, a2, b1, b2, g, c, s;
};

template <class T>
ArrowT<T> reduce_to_arrow(const T a[6]) {
  Rot2<T> J = ordered_jacobi(a[0], a[3], a[1]);
  ArrowT<T> w;
  w.a1 = J.l1;
  w.a2 = J.l2;
  w.c = J.c;
  w.s = J.s;
  w.g = a[2];
  w.b1 = J.c * a[4] + J.s * a[5];
  w.b2 = J.c * a[5] - J.s * a[4];
  return w;
}

// ---------------------------------------------------------------------------
// Zero finders for the fully reduced arrow [[0,0,beta1],[0,-abar,beta2],
// [beta1,beta2,gbar]] (Sec. 1.4).  b1 = beta1^2, b2 = beta2^2.  The spectral
// function is f(x) = x - gbar - b1/x - b2/(x + abar) and its derivative is
// Eq. (3); the wanted zero is the unique one in (0, +inf).
// ---------------------------------------------------------------------------

constexpr int kTraceMax = 72;

struct ZfTrace {
  int n = 0;                  // number of evaluated iterates
  double x[kTraceMax];        // iterates x_j
  double f[kTraceMax];        // f(x_j)
  double fp[kTraceMax];       // f'(x_j)
  double w0[kTraceMax];       // omega_0 at x_j (Sec. 1.4.1)
  double w1[kTraceMax];       // omega_1 at x_j (Sec. 1.4.1)
  double direct[kTraceMax];   // 1 where x_{j+1} was taken directly as the zero of phi_j
};

struct ZfResult {
  int iters = 0;      // steps taken
  int converged = 0;  // 1 if a stopping rule fired before the cap
};

// Sec. 1.4.1: Borges-Gragg zero finder, started from +infinity.
template <class T>
T bg_zero(T abar, T b1, T b2, T gbar, const Params& P, ZfResult* res, ZfTrace* tr) {
  using std::sqrt;
  // Start: the zero in (0, inf) of the limit model Eq. (7),
  // x - gbar - (b1 + b2)/x; the conjugate form is used when gbar < 0.
  T hg = gbar * T(0.5);
  T bsum = b1 + b2;
  T rt = sqrt(hg * hg + bsum);
  T x = (gbar >= T(0.0)) ? hg + rt : bsum / (rt - hg);
  int j = 0;
  int converged = 0;
  for (;; ++j) {
    T r1 = T(1.0) / x;
    T r2 = T(1.0) / (x + abar);
    T f = x - gbar - b1 * r1 - b2 * r2;          // spectral function
    T fp = T(1.0) + b1 * r1 * r1 + b2 * r2 * r2; // Eq. (3)
    if (tr && tr->n < kTraceMax) {
      double xr = val(x), ab = val(abar);
      tr->x[tr->n] = xr;
      tr->f[tr->n] = val(f);
      tr->fp[tr->n] = val(fp);
      tr->w0[tr->n] = 1.0 + val(b2) * ab / ((xr + ab) * (xr + ab) * (xr + ab));
      double q = xr / (xr + ab);
      tr->w1[tr->n] = val(b1) + val(b2) * q * q * q;
      tr->direct[tr->n] = 0.0;
      tr->n++;
    }
    // reading: an iterate at or left of the zero (f <= 0 can only come from
    // rounding, the iteration being monotone from the right) is accepted.
    if (!(f > T(0.0))) { converged = 1; break; }
    // Stopping rule of Sec. 1.4.1: f/f' < C eps x, multiplied through by f' > 0.
    if (f < T(P.c_term * EPS) * x * fp) { converged = 1; break; }
    if (j >= P.maxit) break;
    // Osculating model phi_j (Sec. 1.4.1): omega_0 = 1 + b2 abar/(x+abar)^3;
    // increment quadratic Eq. (5) with a = -omega_0/x, b = f' + f/x.
    T w0 = T(1.0) + b2 * abar * r2 * r2 * r2;
    T a = -w0 * r1;
    T b = fp + f * r1;
    // Eq. (6): Delta = (2f/b) / (1 + sqrt(1 + (2a/b)(2f/b))).
    T q = T(2.0) * f / b;
    T disc = T(1.0) + (T(2.0) * a / b) * q;
    if (disc < T(0.0)) disc = T(0.0);  // reading: clamp a rounding-negative radicand
    T delta = q / (T(1.0) + sqrt(disc));
    T xn;
    if (delta < x * T(0.5)) {
      xn = x - delta;
    } else {
      // reading: x_{j+1} is the zero of phi_j in (0, inf) (Sec. 1.4.1).  When
      // it lies far below x_j, Delta agrees with x_j to many digits and
      // x_j - Delta is rounding noise (it can even be negative), so the zero
      // is taken directly from omega_0 x^2 - sigma x - omega_1 = 0, with
      // omega_1 and sigma as in Sec. 1.4.1, in the form free of cancellation.
      T xr = x * r2;
      T w1 = b1 + b2 * xr * xr * xr;
      T sigma = w0 * x - w1 * r1 - f;
      T rt = sqrt(sigma * sigma + T(4.0) * w0 * w1);
      xn = (sigma > T(0.0)) ? (sigma + rt) / (T(2.0) * w0) : (T(2.0) * w1) / (rt - sigma);
      if (tr && tr->n > 0) tr->direct[tr->n - 1] = 1.0;
    }
    // reading: a step that no longer decreases x means the iterate has
    // reached the rounding level of f; it is accepted.
    if (!(xn < x)) { converged = 1; break; }
    x = xn;
  }
  if (res) { res->iters = j; res->converged = converged; }
  return x;
}

// Sec. 1.4.2: Newton's method, started left of the zero.
template <class T>
T newton_zero(T abar, T b1, T b2, T gbar, const Params& P, ZfResult* res, ZfTrace* tr) {
  using std::sqrt;
  // Start: where f meets -b2/(x + abar), i.e. the positive zero of
  // x - gbar - b1/x.  Reading: the conjugate form when gbar < 0, as in Sec. 1.4.1.
  T hg = gbar * T(0.5);
  T rt = sqrt(hg * hg + b1);
  T x = (gbar >= T(0.0)) ? hg + rt : b1 / (rt - hg);
  int j = 0;
  int converged = 0;
  for (;; ++j) {
    T r1 = T(1.0) / x;
    T r2 = T(1.0) / (x + abar);
    T f = x - gbar - b1 * r1 - b2 * r2;
    T fp = T(1.0) + b1 * r1 * r1 + b2 * r2 * r2;
    if (tr && tr->n < kTraceMax) {
      tr->x[tr->n] = val(x);
      tr->f[tr->n] = val(f);
      tr->fp[tr->n] = val(fp);
      tr->w0[tr->n] = 0.0;
      tr->w1[tr->n] = 0.0;
      tr->direct[tr->n] = 0.0;
      tr->n++;
    }
    // reading: an iterate at or right of the zero (f >= 0 can only come from
    // rounding, the iteration being monotone from the left) is accepted.
    if (!(f < T(0.0))) { converged = 1; break; }
    // Stopping rule of Sec. 1.4.2: |f| < C eps x.
    if (T(0.0) - f < T(P.c_term * EPS) * x) { converged = 1; break; }
    if (j >= P.maxit) break;
    T xn = x - f / fp;
    // reading: Sec. 1.4.2's test |f| < C eps x can be out of reach when the
    // rounding error of f (about eps |gbar|) exceeds C eps x; a step that no
    // longer increases x has reached that level and the iterate is accepted.
    if (!(xn > x)) { converged = 1; break; }
    x = xn;
  }
  if (res) { res->iters = j; res->converged = converged; }
  return x;
}

// ---------------------------------------------------------------------------
// The whole method for one matrix.
// ---------------------------------------------------------------------------

enum Cls { CLS_DIAGONAL = 0, CLS_DEFLATED = 1, CLS_REDUCED = 2, CLS_NONFINITE = 3 };

struct Info {
  int cls = 0;
  int it_mu = 0, it_nu = 0;
  int conv = 1;       // 1 if every zero finder call converged
  int exponent = 0;   // pre-scale exponent e, A was divided by 2^e
};

// Internal trace of the arrow-frame quantities, for the invariant tests.
struct Trace {
  double a1, a2, b1, b2, g, c, s, h;
  double mu, nu;
  double u[3][3];  // u1, u2, u3 (reduced branch, unnormalised, arrow frame)
  ZfTrace zmu, znu;
};

template <class T>
void solve_one(const double ain[6], double lam_out[3], double U_out[9], const Params& P,
               Info* info, Trace* tr) {
  using std::sqrt;
  using std::fabs;
  using std::hypot;
  Info inf;

  // reading: a non-finite entry makes every output NaN.
  for (int i = 0; i < 6; ++i) {
    if (!std::isfinite(ain[i])) {
      for (int k = 0; k < 3; ++k) lam_out[k] = NAN;
      for (int k = 0; k < 9; ++k) U_out[k] = NAN;
      inf.cls = CLS_NONFINITE;
      inf.conv = 1;
      if (info) *info = inf;
      return;
    }
  }

  // reading: pre-scale by an exact power of two so the largest entry lies in
  // [0.5, 1); eigenvalues are scaled back at the end.  Keeps the degree-3
  // eigenvector products of Sec. 1.2 in range for entries down to 1e-100.
  double amax = 0.0;
  for (int i = 0; i < 6; ++i) amax = std::max(amax, std::fabs(ain[i]));
  int e = 0;
  if (amax > 0.0) std::frexp(amax, &e);
  inf.exponent = e;
  T a[6];
  for (int i = 0; i < 6; ++i) a[i] = T(std::ldexp(ain[i], -e));

  // Sec. 1: ordered arrow.
  ArrowT<T> w = reduce_to_arrow(a);
  // reading: a spike |beta_j| < 2^-480 of the pre-scaled arrow is set to
  // zero -- an exact beta-deflation (Sec. 1.1) after a perturbation far
  // below eps ||A|| -- so that beta_j^2, the products of the deflation test
  // and those of the zero finder stay clear of underflow.  (Without it two
  // tiny spikes make both sides of the test underflow to 0 <= 0 and
  // "deflate" along an arbitrary direction.)
  if (fabs(w.b1) < T(kTinySpike)) w.b1 = T(0.0);
  if (fabs(w.b2) < T(kTinySpike)) w.b2 = T(0.0);
  const T a1 = w.a1, a2 = w.a2, b1 = w.b1, b2 = w.b2, g = w.g;

  T lamv[3];
  T V[3][3];  // V[k] = eigenvector k in the arrow frame

  // Sec. 1.1: h = sqrt(beta1^2 + beta2^2); h = 0 means the arrow is diagonal.
  T h = hypot(b1, b2);
  T abar = a1 - a2;
  if (tr) {
    *tr = Trace{};
    tr->a1 = val(a1); tr->a2 = val(a2); tr->b1 = val(b1); tr->b2 = val(b2);
    tr->g = val(g); tr->c = val(w.c); tr->s = val(w.s); tr->h = val(h);
  }

  int cls;
  if (h == T(0.0)) {
    cls = CLS_DIAGONAL;
  } else {
    // Sec. 1.1 deflation test |abar beta1 beta2| <= C eps |alpha1 + alpha2| h^2,
    // or (variant) the EISPACK-style test it is derived from.
    T lhs = fabs(abar * b1 * b2);
    T rhs;
    if (P.deflation_test == 1)
      rhs = T(P.c_defl * EPS) * (fabs(a1 * b2 * b2 + a2 * b1 * b1) + fabs(a1 * b1 * b1 + a2 * b2 * b2));
    else
      rhs = T(P.c_defl * EPS) * fabs(a1 + a2) * (h * h);
    // The "<=" takes the exact beta- and combo-deflations of Sec. 1.1
    // (beta_j = 0 or alpha1 = alpha2 make the left side 0).
    if (lhs <= rhs)
      cls = CLS_DEFLATED;
    else
      cls = CLS_REDUCED;
  }
  inf.cls = cls;

  if (cls == CLS_DIAGONAL) {
    // Eigenpairs (alpha1, e1), (alpha2, e2), (gamma, e3) of the arrow.
    lamv[0] = a1; lamv[1] = a2; lamv[2] = g;
    for (int k = 0; k < 3; ++k)
      for (int i = 0; i < 3; ++i) V[k][i] = T(k == i ? 1.0 : 0.0);
  } else if (cls == CLS_DEFLATED) {
    // Sec. 1.1: G = [[beta2/h, -beta1/h, 0], [beta1/h, beta2/h, 0], [0,0,1]].
    // Reading (an equivalent stable form): the entries of G A G^T are formed
    // from the unit vector (beta1/h, beta2/h) instead of dividing by h^2.
    T gs = b1 / h, gc = b2 / h;
    // accepted eigenvalue (alpha1 beta2^2 + alpha2 beta1^2)/h^2, vector G^T e1
    lamv[0] = a1 * gc * gc + a2 * gs * gs;
    V[0][0] = gc; V[0][1] = T(0.0) - gs; V[0][2] = T(0.0);
    // the 2x2 [[(alpha1 beta1^2 + alpha2 beta2^2)/h^2, h], [h, gamma]]
    T d2 = a1 * gs * gs + a2 * gc * gc;
    Rot2<T> K = ordered_jacobi(d2, h, g);
    lamv[1] = K.l1;
    lamv[2] = K.l2;
    // G^T (0, c', s') and G^T (0, -s', c')
    V[1][0] = gs * K.c; V[1][1] = gc * K.c; V[1][2] = K.s;
    V[2][0] = T(0.0) - gs * K.s; V[2][1] = T(0.0) - gc * K.s; V[2][2] = K.c;
  } else {
    // Sec. 1.2: reduced arrow.  mu = lambda1 - alpha1 is the zero of the
    // fully reduced arrow A - alpha1 I (gbar = gamma - alpha1, b1 = beta1^2,
    // b2 = beta2^2); nu = alpha2 - lambda3 is the zero of P(alpha2 I - A)P,
    // whose squared spikes are swapped and gbar = alpha2 - gamma.
    T bb1 = b1 * b1, bb2 = b2 * b2;
    ZfResult rm, rn;
    ZfTrace* tm = tr ? &tr->zmu : nullptr;
    ZfTrace* tn = tr ? &tr->znu : nullptr;
    T mu, nu;
    if (P.zero_finder == 1) {
      mu = newton_zero(abar, bb1, bb2, g - a1, P, &rm, tm);
      nu = newton_zero(abar, bb2, bb1, a2 - g, P, &rn, tn);
    } else {
      mu = bg_zero(abar, bb1, bb2, g - a1, P, &rm, tm);
      nu = bg_zero(abar, bb2, bb1, a2 - g, P, &rn, tn);
    }
    inf.it_mu = rm.iters;
    inf.it_nu = rn.iters;
    inf.conv = rm.converged && rn.converged;
    // Sec. 1.2: lambda1 = alpha1 + mu, lambda3 = alpha2 - nu, and the trace
    // identity lambda2 = nu - mu + gamma.
    lamv[0] = a1 + mu;
    lamv[1] = nu - mu + g;
    lamv[2] = a2 - nu;
    T mpa = mu + abar, npa = nu + abar;
    // u1, u2, u3 of Sec. 1.2.
    V[0][0] = b1 * mpa; V[0][1] = b2 * mu; V[0][2] = mu * mpa;
    V[1][0] = T(0.0) - b2 * mu * npa; V[1][1] = b1 * nu * mpa; V[1][2] = b1 * b2 * abar;
    V[2][0] = b1 * nu; V[2][1] = b2 * npa; V[2][2] = T(0.0) - nu * npa;
    if (tr) {
      tr->mu = val(mu); tr->nu = val(nu);
      for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 3; ++i) tr->u[k][i] = val(V[k][i]);
    }
    // reading: normalise each vector by its 2-norm (Sec. 1.2 leaves them
    // unnormalised; the outputs are to be orthonormal).  The norm is taken
    // of the vector scaled by the power of two that brings its largest
    // component to [0.5, 1): exact, so nothing changes where no underflow
    // occurs, while u2's degree-3 components (beta1 beta2 abar when mu and
    // nu are both tiny) no longer underflow when squared.
    for (int k = 0; k < 3; ++k) {
      double m = std::max(std::fabs(val(V[k][0])), std::max(std::fabs(val(V[k][1])), std::fabs(val(V[k][2]))));
      int ev = 0;
      if (m > 0.0) std::frexp(m, &ev);
      for (int i = 0; i < 3; ++i) V[k][i] = T(std::ldexp(val(V[k][i]), -ev));
      T inv = T(1.0) / sqrt(V[k][0] * V[k][0] + V[k][1] * V[k][1] + V[k][2] * V[k][2]);
      for (int i = 0; i < 3; ++i) V[k][i] = V[k][i] * inv;
    }
  }

  // Back to the original frame: x = J v, J = [[c,-s,0],[s,c,0],[0,0,1]].
  double lam[3], vec[3][3];
  for (int k = 0; k < 3; ++k) {
    T x0 = w.c * V[k][0] - w.s * V[k][1];
    T x1 = w.s * V[k][0] + w.c * V[k][1];
    vec[k][0] = val(x0);
    vec[k][1] = val(x1);
    vec[k][2] = val(V[k][2]);
    lam[k] = val(lamv[k]);
  }

  // reading: eigenvalues ascending (stable: equal values keep the branch
  // order above); each vector's largest-magnitude component made positive
  // (first such component on ties); eigenvalues scaled back by 2^e.
  int ord[3] = {0, 1, 2};
  for (int i = 1; i < 3; ++i)
    for (int j = i; j > 0 && lam[ord[j]] < lam[ord[j - 1]]; --j) std::swap(ord[j], ord[j - 1]);
  for (int k = 0; k < 3; ++k) {
    const double* v = vec[ord[k]];
    int im = 0;
    for (int i = 1; i < 3; ++i)
      if (std::fabs(v[i]) > std::fabs(v[im])) im = i;
    double sg = (v[im] < 0.0) ? -1.0 : 1.0;
    lam_out[k] = std::ldexp(lam[ord[k]], e);
    for (int i = 0; i < 3; ++i) U_out[i * 3 + k] = sg * v[i];
  }
  if (info) *info = inf;
}

// ---------------------------------------------------------------------------
// Eigenvalue/eigenvector derivative (not in the paper; the standard
// first-order perturbation result for simple eigenvalues):
//   dlambda_i = u_i^T dA u_i,  du_i = sum_{j != i} u_j (u_j^T dA u_i)/(lambda_i - lambda_j).
// For a loss with gradients (glam, gU) this gives
//   Abar = U (diag(glam) + F o (U^T gU)) U^T,  F_ij = 1/(lambda_j - lambda_i), i != j,
// with F_ij := 0 where |lambda_i - lambda_j| < tau ||A||_F.  The packed
// gradient sums the two mirrored entries of each off-diagonal.
// ---------------------------------------------------------------------------

void grad_one(const double lam[3], const double U[9], const double glam[3], const double gU[9],
              double tau, double gA[6]) {
  double nrm = std::sqrt(lam[0] * lam[0] + lam[1] * lam[1] + lam[2] * lam[2]);  // ||A||_F
  double M[3][3];  // U^T gU
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += U[k * 3 + i] * gU[k * 3 + j];
      M[i][j] = s;
    }
  double C[3][3];  // diag(glam) + F o M
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      if (i == j) {
        C[i][j] = glam[i];
      } else {
        double gap = lam[j] - lam[i];
        C[i][j] = (std::fabs(gap) < tau * nrm) ? 0.0 : M[i][j] / gap;
      }
    }
  double Ab[3][3];  // U C U^T
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) s += U[r * 3 + i] * C[i][j] * U[c * 3 + j];
      Ab[r][c] = s;
    }
  gA[0] = Ab[0][0];
  gA[1] = Ab[1][1];
  gA[2] = Ab[2][2];
  gA[3] = Ab[0][1] + Ab[1][0];
  gA[4] = Ab[0][2] + Ab[2][0];
  gA[5] = Ab[1][2] + Ab[2][1];
}

Params params_from(const double* p) {
  Params P;
  if (p) {
    P.c_defl = p[0];
    P.c_term = p[1];
    P.maxit = (int)p[2];
    P.deflation_test = (int)p[3];
    P.zero_finder = (int)p[4];
  }
  return P;
}

}  // namespace

// ---------------------------------------------------------------------------
// C entry points (loaded with ctypes by the tests).
//   params: NULL for the defaults, else 5 doubles
//           {C_defl, C_term, maxit, deflation_test, zero_finder}.
//   A: n x 6 packed (a11,a22,a33,a12,a13,a23); lam: n x 3 ascending;
//   U: n x 9 row-major, column k is the eigenvector of lam[k].
//   info (optional): n x 5 int32 {class, it_mu, it_nu, converged, exponent}.
// ---------------------------------------------------------------------------

extern "C" {

int oracle_abi_version(void) { return 1; }

void oracle_syev3(const double* A, int64_t n, double* lam, double* U, int32_t* info,
                  const double* params) {
  Params P = params_from(params);
  for (int64_t m = 0; m < n; ++m) {
    Info inf;
    solve_one<double>(A + 6 * m, lam + 3 * m, U + 9 * m, P, &inf, nullptr);
    if (info) {
      int32_t* o = info + 5 * m;
      o[0] = inf.cls; o[1] = inf.it_mu; o[2] = inf.it_nu; o[3] = inf.conv; o[4] = inf.exponent;
    }
  }
}

// The same over nthreads std::threads on contiguous chunks; returns the wall
// time in seconds (the CPU baseline).
double oracle_syev3_threads(const double* A, int64_t n, double* lam, double* U, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  auto t0 = std::chrono::steady_clock::now();
  std::vector<std::thread> pool;
  int64_t chunk = (n + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    int64_t lo = t * chunk, hi = std::min<int64_t>(n, lo + chunk);
    if (lo >= hi) break;
    pool.emplace_back([=]() {
      Params P;
      for (int64_t m = lo; m < hi; ++m) solve_one<double>(A + 6 * m, lam + 3 * m, U + 9 * m, P, nullptr, nullptr);
    });
  }
  for (auto& th : pool) th.join();
  auto t1 = std::chrono::steady_clock::now();
  return std::chrono::duration<double>(t1 - t0).count();
}

// Algorithmic operation counts per matrix: ops[4m..4m+3] = {add/sub, mul, div, sqrt}.
void oracle_count_ops(const double* A, int64_t n, uint64_t* ops, const double* params) {
  Params P = params_from(params);
  double lam[3], U[9];
  for (int64_t m = 0; m < n; ++m) {
    OpCounts c;
    tl_ops = &c;
    solve_one<Counted>(A + 6 * m, lam, U, P, nullptr, nullptr);
    tl_ops = nullptr;
    ops[4 * m + 0] = c.add;
    ops[4 * m + 1] = c.mul;
    ops[4 * m + 2] = c.div;
    ops[4 * m + 3] = c.sqrt;
  }
}

// Internal quantities of one matrix, for the invariant tests.  Layout of out
// (length >= 32 + 2 * 6 * 72):
//  [0..7]   alpha1, alpha2, beta1, beta2, gamma, c, s, h   (scaled frame)
//  [8..9]   mu, nu
//  [10..18] u1, u2, u3 unnormalised (arrow frame)
//  [19..23] class, it_mu, it_nu, converged, exponent
//  [24]     n_mu (iterates traced), [25] n_nu
//  [32 ...] mu trace: x[72], f[72], fp[72], w0[72], w1[72], direct[72]; then the nu trace.
int oracle_trace(const double a[6], double* out, const double* params) {
  Params P = params_from(params);
  Trace tr;
  Info inf;
  double lam[3], U[9];
  solve_one<double>(a, lam, U, P, &inf, &tr);
  if (inf.cls == CLS_NONFINITE) return -1;
  out[0] = tr.a1; out[1] = tr.a2; out[2] = tr.b1; out[3] = tr.b2;
  out[4] = tr.g; out[5] = tr.c; out[6] = tr.s; out[7] = tr.h;
  out[8] = tr.mu; out[9] = tr.nu;
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i) out[10 + 3 * k + i] = tr.u[k][i];
  out[19] = inf.cls; out[20] = inf.it_mu; out[21] = inf.it_nu; out[22] = inf.conv; out[23] = inf.exponent;
  out[24] = tr.zmu.n; out[25] = tr.znu.n;
  const ZfTrace* zs[2] = {&tr.zmu, &tr.znu};
  for (int z = 0; z < 2; ++z) {
    double* o = out + 32 + z * 6 * kTraceMax;
    for (int j = 0; j < kTraceMax; ++j) {
      bool ok = j < zs[z]->n;
      o[j] = ok ? zs[z]->x[j] : 0.0;
      o[kTraceMax + j] = ok ? zs[z]->f[j] : 0.0;
      o[2 * kTraceMax + j] = ok ? zs[z]->fp[j] : 0.0;
      o[3 * kTraceMax + j] = ok ? zs[z]->w0[j] : 0.0;
      o[4 * kTraceMax + j] = ok ? zs[z]->w1[j] : 0.0;
      o[5 * kTraceMax + j] = ok ? zs[z]->direct[j] : 0.0;
    }
  }
  return inf.cls;
}

// Ordered Jacobi rotation of [[p,q],[q,r]]: out = {c, s, l1, l2}.
void oracle_jacobi2(double p, double q, double r, double out[4]) {
  Rot2<double> J = ordered_jacobi(p, q, r);
  out[0] = J.c; out[1] = J.s; out[2] = J.l1; out[3] = J.l2;
}

// One zero-finder call on a fully reduced arrow: out = {x, iters, converged}.
void oracle_zero(double abar, double b1, double b2, double gbar, int method, double out[3],
                 const double* params) {
  Params P = params_from(params);
  ZfResult r;
  double x = (method == 1) ? newton_zero(abar, b1, b2, gbar, P, &r, nullptr)
                           : bg_zero(abar, b1, b2, gbar, P, &r, nullptr);
  out[0] = x; out[1] = r.iters; out[2] = r.converged;
}

// Packed gradient of a loss through (lambda, U): gA = n x 6.
void oracle_syev3_bwd(const double* lam, const double* U, const double* glam, const double* gU,
                      int64_t n, double tau, double* gA) {
  for (int64_t m = 0; m < n; ++m)
    grad_one(lam + 3 * m, U + 9 * m, glam + 3 * m, gU + 9 * m, tau, gA + 6 * m);
}

}  // extern "C"
