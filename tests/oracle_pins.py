"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each pin is a plain function that raises ``AssertionError`` when the oracle
disagrees with something it cannot be allowed to disagree with: closed-form
spectra, exact special cases, invariants, the properties the paper proves for
its zero finder, an independent double-double brute force and finite
differences.  ``test_oracle.py`` runs each pin; ``test_oracle_mutants.py``
plants plausible mistakes in copies of the oracle and checks that some pin
fails for every one of them.

Citations are to C. F. Borges, "Solving the 3x3 Real Symmetric Eigenproblem"
(arXiv 1806.06698): sections and the numbered equations (1)-(7).
"""

from __future__ import annotations

import os

import numpy as np

import oracle
from paper_1806_06698_gb300 import inputs

EPS = 2.0 ** -52
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

PINS = {}


def pin(fn):
    PINS[fn.__name__] = fn
    return fn


def _mp():
    try:
        import mpmath
    except ImportError:  # pragma: no cover - mpmath ships with sympy here
        import pytest

        pytest.skip("mpmath not installed")
    mpmath.mp.dps = 60
    return mpmath


def fro(A6):
    """||A||_F per matrix, scaled so that 2^+-600 entries neither overflow nor underflow."""
    M = inputs.unpack(np.asarray(A6, np.float64))
    s = np.max(np.abs(M), axis=(1, 2))
    s = np.where(s > 0, s, 1.0)
    return s * np.linalg.norm(M / s[:, None, None], axis=(1, 2))


def residual(A6, lam, U):
    """||A U - U Lambda||_F per matrix, evaluated on A / max|a_ij| and scaled back."""
    M = inputs.unpack(np.asarray(A6, np.float64))
    s = np.max(np.abs(M), axis=(1, 2))
    s = np.where(s > 0, s, 1.0)
    R = (M / s[:, None, None]) @ U - U * (lam / s[:, None])[:, None, :]
    return s * np.linalg.norm(R, axis=(1, 2))


def orthogonality(U):
    return np.linalg.norm(np.swapaxes(U, 1, 2) @ U - np.eye(3), axis=(1, 2))


def load_closed_forms():
    """Parse tests/golden/closed_forms.txt -> list of (name, a6 float, lam mp, source)."""
    mp = _mp()
    ns = {"__builtins__": {}, "sqrt": mp.sqrt}
    cases = []
    with open(os.path.join(GOLDEN, "closed_forms.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, ent, lam, src = [t.strip() for t in line.split(";", 3)]
            a_mp = [mp.mpf(eval(t, ns)) for t in ent.split()]
            a = np.array([float(v) for v in a_mp])
            for v, x in zip(a_mp, a):
                assert mp.mpf(x) == v, f"{name}: entry {v} is not exact in binary64"
            l_mp = [mp.mpf(eval(t, ns)) for t in lam.split(",")]
            cases.append((name, a, l_mp, src))
    return cases


# ---------------------------------------------------------------------------
# Whole-method pins
# ---------------------------------------------------------------------------


@pin
def closed_forms():
    """Textbook spectra (tests/golden/closed_forms.txt) to 8 eps ||A||_F."""
    mp = _mp()
    cases = load_closed_forms()
    A = np.stack([c[1] for c in cases])
    lam, U = oracle.syev3(A)
    nrm = fro(A)
    for i, (name, _, l_mp, _) in enumerate(cases):
        for k in range(3):
            err = abs(mp.mpf(lam[i, k]) - l_mp[k])
            assert err <= 8 * EPS * nrm[i], f"{name}: lambda[{k}] off by {float(err / nrm[i] / EPS):.2f} eps"
    assert np.all(residual(A, lam, U) <= 16 * EPS * nrm)
    assert np.all(orthogonality(U) <= 8 * EPS)


@pin
def rational_eigenvectors():
    """Q diag(9,-18,27) Q^T with Q = (1/3)[[1,2,2],[2,1,-2],[2,-2,1]]: the
    eigenvectors are Q's columns, signed by the largest-component rule."""
    A = np.array([[5.0, 14.0, -1.0, -14.0, 16.0, 2.0]])
    lam, U = oracle.syev3(A)
    Q = np.array([[1, 2, 2], [2, 1, -2], [2, -2, 1]], float) / 3.0
    expect = Q[:, [1, 0, 2]]  # eigenvalues -18, 9, 27
    for k in range(3):
        # (2,-2,1)/3 has a tie between its two largest components, which
        # rounding decides; compare up to sign (the sign rule has its own pin)
        v = expect[:, k]
        d = min(np.max(np.abs(U[0, :, k] - v)), np.max(np.abs(U[0, :, k] + v)))
        assert d <= 8 * EPS, (k, U[0, :, k], v)


@pin
def diagonal_exact():
    """A diagonal matrix is its own spectral factorisation: eigenvalues are the
    sorted diagonal exactly and U is a permutation matrix exactly (h = 0, Sec. 1.1)."""
    rng = np.random.default_rng(11)
    n = 600
    A = np.zeros((n, 6))
    A[:, :3] = rng.standard_normal((n, 3))
    rep = rng.integers(0, 4, n)  # force repeated entries in a share
    A[rep == 0, 1] = A[rep == 0, 0]
    A[rep == 1, 2] = A[rep == 1, 0]
    A[rep == 2, 2] = A[rep == 2, 1]
    A[:5, :3] = 0.0
    lam, U, info = oracle.syev3(A, with_info=True)
    assert np.array_equal(lam, np.sort(A[:, :3], axis=1))
    assert np.all((U == 0.0) | (U == 1.0))
    assert np.array_equal(U.sum(axis=1), np.ones((n, 3))) and np.array_equal(U.sum(axis=2), np.ones((n, 3)))
    assert np.array_equal(inputs.unpack(A) @ U, U * lam[:, None, :])
    assert np.all(info[:, 0] == oracle.CLS_DIAGONAL)


@pin
def zero_and_nonfinite():
    """The zero matrix gives 0 and I; any NaN/Inf entry gives NaN outputs."""
    lam, U = oracle.syev3(np.zeros((1, 6)))
    assert np.array_equal(lam, np.zeros((1, 3))) and np.array_equal(U[0], np.eye(3))
    bad = np.ones((12, 6))
    for i in range(6):
        bad[i, i] = np.nan
        bad[6 + i, i] = np.inf if i % 2 else -np.inf
    lam, U, info = oracle.syev3(bad, with_info=True)
    assert np.all(np.isnan(lam)) and np.all(np.isnan(U))
    assert np.all(info[:, 0] == oracle.CLS_NONFINITE)


@pin
def scale_equivariance():
    """Scaling A by 2^k scales the eigenvalues by 2^k and leaves U unchanged,
    bit for bit (the pre-scale makes the arithmetic scale-free)."""
    A, _ = inputs.mixed(400, seed=5, log10_scale=0.0)
    lam0, U0 = oracle.syev3(A)
    for k in (-600, -37, 3, 600):
        lam, U = oracle.syev3(np.ldexp(A, k))
        assert np.array_equal(lam, np.ldexp(lam0, k)), k
        assert np.array_equal(U, U0), k


@pin
def known_spectrum():
    """Q diag(d) Q^T with Haar Q and known d: |lambda - d| <= 16 eps ||d||_2
    (the rounding made in forming A included)."""
    A, d, _ = inputs.spectral(1500, seed=21, near_degenerate=0.1)
    lam, U = oracle.syev3(A)
    err = np.max(np.abs(lam - d), axis=1) / np.linalg.norm(d, axis=1)
    assert err.max() <= 16 * EPS, err.max() / EPS


@pin
def invariants():
    """tr A = sum(lambda), ||A||_F^2 = sum(lambda^2), det A = prod(lambda)."""
    A, _ = inputs.mixed(1500, seed=6, log10_scale=0.0)
    lam, _ = oracle.syev3(A)
    M = inputs.unpack(A)
    nrm = fro(A)
    assert np.all(np.abs(lam.sum(1) - np.trace(M, axis1=1, axis2=2)) <= 8 * EPS * nrm)
    assert np.all(np.abs((lam ** 2).sum(1) - nrm ** 2) <= 16 * EPS * nrm ** 2)
    assert np.all(np.abs(lam.prod(1) - np.linalg.det(M)) <= 32 * EPS * nrm ** 3)


@pin
def residual_orthogonality():
    """The two measures of Sec. 1.5 on the mixed batch and on matrices with
    entrywise random scales: ||TV - V Lambda||_F <= 1e-14 ||T||_F and
    ||I - V^T V||_F <= 10 eps."""
    A, _ = inputs.mixed(3000, seed=7)
    A = np.concatenate([A, entrywise_scales(3000, seed=29)])
    lam, U = oracle.syev3(A)
    nrm = fro(A)
    assert np.all(residual(A, lam, U) <= 1e-14 * nrm)
    assert np.all(orthogonality(U) <= 10 * EPS)


@pin
def brute_force_dd():
    """An independent double-double cyclic Jacobi agrees to 8 eps ||A||_F on
    eigenvalues; on well separated eigenvalues the eigenvectors agree to
    16 eps ||A||_F / gap."""
    A1, _ = inputs.mixed(1500, seed=8)
    A2 = inputs.gaussian(500, seed=9)
    A = np.concatenate([A1, A2])
    lam, U = oracle.syev3(A)
    hi, lo, V = oracle.dd_jacobi(A)
    nrm = fro(A)
    err = np.max(np.abs((lam - hi) - lo), axis=1) / nrm
    assert err.max() <= 8 * EPS, err.max() / EPS
    gaps = np.stack([hi[:, 1] - hi[:, 0], np.minimum(hi[:, 1] - hi[:, 0], hi[:, 2] - hi[:, 1]),
                     hi[:, 2] - hi[:, 1]], axis=1)
    for k in range(3):
        ok = gaps[:, k] > 1e-6 * nrm
        bound = 16 * EPS * nrm[ok] / gaps[ok, k] + 4 * EPS
        diff = np.min(np.stack([np.linalg.norm(U[ok, :, k] - V[ok, :, k], axis=1),
                                np.linalg.norm(U[ok, :, k] + V[ok, :, k], axis=1)]), axis=0)
        assert np.all(diff <= bound), (k, np.max(diff / bound))


@pin
def numpy_eigh():
    """LAPACK (numpy.linalg.eigvalsh) agrees to 8 eps ||A||_F."""
    A, _ = inputs.mixed(2000, seed=10)
    lam, _ = oracle.syev3(A)
    ref = np.linalg.eigvalsh(inputs.unpack(A))
    err = np.max(np.abs(lam - ref), axis=1) / fro(A)
    assert err.max() <= 8 * EPS, err.max() / EPS


@pin
def ascending_and_signs():
    """Eigenvalues ascending; each vector's largest-magnitude component
    (first on ties) positive."""
    A, _ = inputs.mixed(2000, seed=12)
    lam, U = oracle.syev3(A)
    assert np.all(np.diff(lam, axis=1) >= 0)
    im = np.argmax(np.abs(U), axis=1)  # first maximum per column
    top = np.take_along_axis(U, im[:, None, :], axis=1)[:, 0, :]
    assert np.all(top > 0)


# ---------------------------------------------------------------------------
# Step pins
# ---------------------------------------------------------------------------


@pin
def jacobi2_closed_form():
    """Sec. 1: the ordered Jacobi rotation of [[p,q],[q,r]] gives
    l1,2 = (p+r)/2 +/- sqrt(((p-r)/2)^2 + q^2), l1 >= l2, (c,s) a unit
    eigenvector of l1."""
    mp = _mp()
    rng = np.random.default_rng(13)
    cases = [tuple(rng.standard_normal(3)) for _ in range(150)]
    cases += [(1.0, 0.0, 2.0), (2.0, 0.0, 1.0), (1.0, 1e-200, 1.0), (1.0, 3.0, 1.0), (-1.0, 1e-9, -1.0 + 1e-15)]
    for p, q, r in cases:
        c, s, l1, l2 = oracle.jacobi2(p, q, r)
        m = (mp.mpf(p) + r) / 2
        R = mp.sqrt(((mp.mpf(p) - r) / 2) ** 2 + mp.mpf(q) ** 2)
        sc = max(abs(p), abs(q), abs(r))
        assert l1 >= l2
        assert abs(l1 - (m + R)) <= 2 * EPS * sc and abs(l2 - (m - R)) <= 2 * EPS * sc, (p, q, r)
        assert abs(c * c + s * s - 1.0) <= 4 * EPS
        assert abs(p * c + q * s - l1 * c) <= 4 * EPS * sc and abs(q * c + r * s - l1 * s) <= 4 * EPS * sc


@pin
def beta_deflation_2x2():
    """Sec. 1.1: with a12 = a23 = 0 and a11 > a22 the arrow has beta2 = 0, so
    a22 is an eigenvalue (beta-deflation) and the rest is the 2x2
    [[a11, a13], [a13, a33]] in closed form."""
    mp = _mp()
    rng = np.random.default_rng(14)
    n = 150
    A = np.zeros((n, 6))
    x = rng.standard_normal((n, 3))
    A[:, 0] = np.maximum(x[:, 0], x[:, 1]) + 0.1
    A[:, 1] = np.minimum(x[:, 0], x[:, 1])
    A[:, 2] = x[:, 2]
    A[:, 4] = rng.standard_normal(n)
    lam, U, info = oracle.syev3(A, with_info=True)
    assert np.all(info[:, 0] == oracle.CLS_DEFLATED)
    nrm = fro(A)
    for i in range(n):
        p, q, r = (mp.mpf(v) for v in (A[i, 0], A[i, 4], A[i, 2]))
        R = mp.sqrt(((p - r) / 2) ** 2 + q ** 2)
        exact = sorted([mp.mpf(A[i, 1]), (p + r) / 2 - R, (p + r) / 2 + R])
        for k in range(3):
            assert abs(mp.mpf(lam[i, k]) - exact[k]) <= 4 * EPS * nrm[i], i


@pin
def reduced_arrow_invariants():
    """Sec. 1.2 on reduced arrows: mu, nu > 0; interlacing lambda1 > alpha1 >
    lambda2 > alpha2 > lambda3 (Eq. (2) shifted); u1, u3 satisfy the arrow's
    eigen-equations; u1 x u3 = (mu + nu + abar) u2; u1 and u3 orthogonal to
    about 2 eps (Sec. 1.3)."""
    A = inputs.gaussian(120, seed=15)
    seen = 0
    for a in A:
        t = oracle.trace(a)
        if t["cls"] != oracle.CLS_REDUCED:
            continue
        seen += 1
        a1, a2, b1, b2, g, mu, nu = (t[k] for k in ("alpha1", "alpha2", "beta1", "beta2", "gamma", "mu", "nu"))
        abar = a1 - a2
        sc = max(abs(a1), abs(a2), abs(b1), abs(b2), abs(g))
        assert a1 > a2 and mu > 0 and nu > 0
        lam2 = nu - mu + g
        assert a2 - 4 * EPS * sc < lam2 < a1 + 4 * EPS * sc
        Ar = np.array([[a1, 0, b1], [0, a2, b2], [b1, b2, g]])
        u1, u2, u3 = t["u"]
        for u, lam in ((u1, a1 + mu), (u3, a2 - nu), (u2, lam2)):
            r = np.linalg.norm(Ar @ u - lam * u)
            assert r <= 16 * EPS * sc * np.linalg.norm(u), (r, u)
        cr = np.cross(u1, u3)
        assert np.linalg.norm(cr - (mu + nu + abar) * u2) <= 8 * EPS * np.linalg.norm(u1) * np.linalg.norm(u3)
        assert abs(u1 @ u3) <= 8 * EPS * np.linalg.norm(u1) * np.linalg.norm(u3)
    assert seen >= 100


def _secular_root(abar, b1, b2, g):
    """The zero in (0, inf) of x - g - b1/x - b2/(x+abar) at 60 digits, by
    bisection (f increases from -inf to +inf there, Sec. 1.4)."""
    mp = _mp()
    abar, b1, b2, g = (mp.mpf(v) for v in (abar, b1, b2, g))

    def f(x):
        return x - g - b1 / x - b2 / (x + abar)

    lo = mp.mpf(0)
    hi = abs(g) + mp.sqrt(b1 + b2) + 1
    while f(hi) < 0:
        hi *= 2
    lo = hi
    while f(lo) > 0:
        lo /= 2
    hi = 2 * lo  # f(2 lo) > 0: the bracket [lo, 2 lo] is relative, so 260 halvings give 2^-260
    for _ in range(260):
        mid = (lo + hi) / 2
        if f(mid) > 0:
            hi = mid
        else:
            lo = mid
    return (lo + hi) / 2


def entrywise_scales(n, seed, lo=-120.0):
    """Matrices whose six entries carry independent scales 2^U(lo, 0): roots
    that sit many orders of magnitude below the start of Eq. (7)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, 6)) * 2.0 ** rng.uniform(lo, 0.0, (n, 6))


def _reduced_problems(n_each=40):
    """(abar, b1, b2, gbar, trace) for the mu and nu problems of reduced lanes
    from the Gaussian and the clustered subsets."""
    out = []
    A1 = inputs.gaussian(n_each, seed=16)
    A2, ids = inputs.mixed(8 * n_each, seed=17, log10_scale=0.0)
    A2 = A2[ids == inputs.SUBSET_CLUSTERED][:n_each]
    A3 = entrywise_scales(n_each, seed=28)
    for a in np.concatenate([A1, A2, A3]):
        t = oracle.trace(a)
        if t["cls"] != oracle.CLS_REDUCED:
            continue
        abar = t["alpha1"] - t["alpha2"]
        bb1, bb2 = t["beta1"] * t["beta1"], t["beta2"] * t["beta2"]
        out.append((abar, bb1, bb2, t["gamma"] - t["alpha1"], t["zmu"], t["mu"]))
        out.append((abar, bb2, bb1, t["alpha2"] - t["gamma"], t["znu"], t["nu"]))
    return out


def _f_rounding(x, abar, b1, b2, g):
    """A bound on the rounding error of evaluating f(x) = x - g - b1/x - b2/(x+abar)
    in binary64 (each of the four terms and the three subtractions)."""
    return 8 * EPS * (abs(x) + abs(g) + b1 / x + b2 / (x + abar))


@pin
def borges_gragg_properties():
    """Sec. 1.4.1: started from the zero of Eq. (7) the iterates start right
    of the root, decrease monotonically and stay right of it; omega_0 > 1 and
    omega_1 > beta1^2; at the exit |x - lambda| < f/f' (the mean value
    argument of Sec. 1.4.1) widened by the rounding error of evaluating f,
    which is below C eps x whenever that rounding error allows it; and the
    convergence is cubic (order >= 2.6 where the errors are far above the
    evaluation noise)."""
    mp = _mp()
    for abar, b1, b2, g, z, x_out in _reduced_problems():
        root = _secular_root(abar, b1, b2, g)
        xs = z["x"]
        # x0 is right of the root in exact arithmetic (f(x0) = b2/x0 - b2/(x0+abar) > 0);
        # when b2 is negligible x0 is the root itself, up to its own rounding
        x0_noise = 4 * EPS * xs[0] + _f_rounding(xs[0], abar, b1, b2, g) / z["fp"][0]
        assert mp.mpf(xs[0]) > root - x0_noise
        assert z["f"][0] > 0 or len(xs) == 1
        assert np.all(np.diff(xs) < 0)
        # every iterate lies right of the root, up to the rounding level of f there
        for x, fp in zip(xs, z["fp"]):
            assert mp.mpf(x) > root - _f_rounding(x, abar, b1, b2, g) / fp - 2 * EPS * x
        # omega_0 > 1 and omega_1 > beta1^2 hold strictly; in binary64 the
        # excess rounds away when beta2^2 is negligible, hence >=
        assert np.all(z["w0"] >= 1.0) and np.all(z["w1"] >= b1)
        x = xs[-1]
        assert x == x_out
        err = abs(mp.mpf(x) - root)
        noise = _f_rounding(x, abar, b1, b2, g) / z["fp"][-1]
        bound = max(z["f"][-1] / z["fp"][-1], 0.0) + noise + 2 * EPS * x
        assert err <= bound, (float(err), bound)
        if noise <= EPS * x:
            assert err <= 4 * EPS * x, float(err / x / EPS)
        rel = [float(abs(mp.mpf(v) - root) / root) for v in xs]
        floor = 1e3 * max(noise / float(root), EPS)
        for e0, e1 in zip(rel[:-1], rel[1:]):
            if e0 < 1e-2 and e1 > floor:
                assert np.log(e1) / np.log(e0) >= 2.6, (e0, e1)


@pin
def newton_properties():
    """Sec. 1.4.2: Newton from x0 = gbar/2 + sqrt((gbar/2)^2 + beta1^2) starts
    left of the root (f(x0) < 0), increases monotonically, exits with
    |x - lambda| < |f| and matches Borges-Gragg to rounding."""
    mp = _mp()
    for abar, b1, b2, g, _, x_bg in _reduced_problems(25):
        root = _secular_root(abar, b1, b2, g)
        x, its, conv = oracle.zero(abar, b1, b2, g, method=1)
        assert conv == 1
        noise = _f_rounding(x, abar, b1, b2, g)  # f' >= 1 (Eq. (3))
        assert abs(mp.mpf(x) - root) <= 3 * EPS * x + noise
        assert abs(x - x_bg) <= 6 * EPS * x + 2 * noise
    A = inputs.gaussian(60, seed=18)
    for a in A:
        t = oracle.trace(a, zero_finder=1)
        if t["cls"] != oracle.CLS_REDUCED:
            continue
        for z in (t["zmu"], t["znu"]):
            assert z["f"][0] < 0
            assert np.all(np.diff(z["x"]) > 0)
    lam_bg, _ = oracle.syev3(A)
    lam_nt, _ = oracle.syev3(A, zero_finder=1)
    assert np.all(np.abs(lam_bg - lam_nt) <= 8 * EPS * fro(A)[:, None])


@pin
def deflation_decisions():
    """Sec. 1.1 on hand-made arrows [[alpha1,0,beta1],[0,alpha2,beta2],[beta1,beta2,gamma]]
    (a12 = 0, a11 >= a22 make the Jacobi rotation the identity):
    combo (alpha1 = alpha2) and beta deflations, the threshold
    |abar beta1 beta2| <= C eps |alpha1 + alpha2| h^2 on both sides, and the
    case alpha1 + alpha2 = 0 where only the EISPACK-style test deflates."""
    s = np.sqrt(0.5)
    rows = [  # alpha1, alpha2, gamma, beta1, beta2, expected class (simplified test), expected (EISPACK test)
        (1.0, 1.0, 0.3, 0.6, 0.8, 1, 1),            # combo deflation
        (1.0, 0.5, 0.3, 0.0, 0.8, 1, 1),            # beta1 = 0
        (1.0, 0.5, 0.3, 0.6, 0.0, 1, 1),            # beta2 = 0
        (1.0, 1.0 - 2.0 ** -51, 0.0, s, s, 1, 1),   # |abar b1 b2| = eps < 2 eps |a1+a2| h^2
        (1.0, 1.0 - 2.0 ** -47, 0.0, s, s, 2, 2),   # 16 eps > 2 eps: reduced
        (1.0, 0.5, 0.3, 0.6, 0.8, 2, 2),            # ordinary reduced arrow
        (1.0, -1.0, 0.0, 1e-20, 1.0, 2, 1),         # alpha1 + alpha2 = 0
        (0.7, 0.2, 0.1, 0.0, 0.0, 0, 0),            # h = 0: diagonal
    ]
    A = np.array([[r[0], r[1], r[2], 0.0, r[3], r[4]] for r in rows])
    _, _, info = oracle.syev3(A, with_info=True)
    _, _, info_e = oracle.syev3(A, with_info=True, deflation_test=1)
    assert list(info[:, 0]) == [r[5] for r in rows], list(info[:, 0])
    assert list(info_e[:, 0]) == [r[6] for r in rows], list(info_e[:, 0])
    lam, U = oracle.syev3(A)
    hi, lo, _ = oracle.dd_jacobi(A)
    assert np.all(np.abs(lam - hi - lo) <= 8 * EPS * fro(A)[:, None])


@pin
def eispack_test_is_weaker():
    """Sec. 1.1: by the triangle inequality the simplified test is the more
    restrictive one, so whatever it deflates the EISPACK-style test deflates."""
    rng = np.random.default_rng(19)
    n = 3000
    a1 = rng.standard_normal(n)
    a2 = a1 - np.abs(a1) * 10.0 ** rng.uniform(-17, -12, n)
    ang = rng.uniform(0, np.pi / 2, n) * 10.0 ** rng.uniform(-8, 0, n)
    A = np.stack([a1, a2, rng.standard_normal(n), np.zeros(n), np.cos(ang), np.sin(ang)], axis=1)
    _, _, i0 = oracle.syev3(A, with_info=True)
    _, _, i1 = oracle.syev3(A, with_info=True, deflation_test=1)
    simp = i0[:, 0] == oracle.CLS_DEFLATED
    assert simp.sum() > 100
    assert np.all(i1[simp, 0] == oracle.CLS_DEFLATED)
    assert (i1[:, 0] == oracle.CLS_DEFLATED).sum() >= simp.sum()


@pin
def deflation_constant_sweep():
    """The unstated C of the deflation test (Sec. 1.1) swept over 1, 4, 16:
    deflations only grow with C, and every result stays within the bound the
    test is built on -- the coupling a deflation drops is at most
    C eps |alpha1 + alpha2| <= 2 C eps ||A||_F (Wielandt-Hoffman, as Sec. 1.1
    invokes it), so eigenvalues agree with the double-double brute force to
    (8 + 2C) eps ||A||_F."""
    rng = np.random.default_rng(23)
    n = 3000
    a1 = rng.standard_normal(n)
    a2 = a1 - np.abs(a1) * 10.0 ** rng.uniform(-17, -12, n)
    ang = rng.uniform(0, np.pi / 2, n) * 10.0 ** rng.uniform(-10, 0, n)
    A = np.concatenate([np.stack([a1, a2, rng.standard_normal(n), np.zeros(n), np.cos(ang), np.sin(ang)], axis=1),
                        inputs.trace_free_spiked(1000, seed=24)])
    hi, lo, _ = oracle.dd_jacobi(A)
    nrm = fro(A)
    prev = -1
    for C in (1.0, 4.0, 16.0):
        lam, U, info = oracle.syev3(A, with_info=True, c_defl=C)
        ndefl = int((info[:, 0] == oracle.CLS_DEFLATED).sum())
        assert ndefl >= prev, (C, ndefl, prev)
        prev = ndefl
        err = np.max(np.abs((lam - hi) - lo), axis=1) / nrm
        assert err.max() <= (8 + 2 * C) * EPS, (C, err.max() / EPS)
        assert np.all(residual(A, lam, U) <= (1e-14 + 2 * C * EPS) * nrm)
        assert np.all(orthogonality(U) <= 10 * EPS)
    assert prev > 0


@pin
def iteration_counts():
    """Cubic convergence (Sec. 1.4.1) from the start of Eq. (7): on iid
    N(0,1) matrices the mean is at most 3 steps per root and no root takes
    more than 8; clustered matrices take at most 12."""
    A = inputs.gaussian(2000, seed=20)
    _, _, info = oracle.syev3(A, with_info=True)
    red = info[:, 0] == oracle.CLS_REDUCED
    its = info[red][:, 1:3]
    assert its.mean() <= 3.0 and its.max() <= 8, (its.mean(), its.max())
    A2, ids = inputs.mixed(4000, seed=22)
    _, _, info2 = oracle.syev3(A2, with_info=True)
    assert info2[:, 1:3].max() <= 12
    assert np.all(info2[:, 3] == 1)


@pin
def op_counts():
    """The counting scalar sees the paper's per-step costs: each Borges-Gragg
    step of Sec. 1.4.1 (f, f' of Eq. (3), omega_0, a, b, Delta of Eq. (6))
    costs 11 add/sub, 18 mul (one for the Delta < x/2 choice), 5 div and 1
    sqrt, so on reduced lanes whose steps all use Eq. (6) the counts are
    affine in the number of steps."""
    A = inputs.gaussian(800, seed=23)
    ops = oracle.count_ops(A).astype(np.int64)
    _, _, info = oracle.syev3(A, with_info=True)
    plain = np.array([t is not None and not (t["zmu"]["direct"].any() or t["znu"]["direct"].any())
                      for t in (oracle.trace(a) for a in A)])
    red = (info[:, 0] == oracle.CLS_REDUCED) & plain
    assert red.sum() >= 400
    its = (info[red, 1] + info[red, 2]).astype(np.int64)
    o = ops[red]
    assert len(np.unique(o[:, 0] - 11 * its)) == 1
    assert len(np.unique(o[:, 3] - its)) == 1
    assert len(np.unique(o[:, 2] - 5 * its)) <= 3      # conjugate start adds a division
    assert len(np.unique(o[:, 1] - 18 * its)) <= 3     # an "f <= 0" exit skips the test's 2 mul
    assert np.all(ops.sum(1) > 0)


# ---------------------------------------------------------------------------
# Derivative pins
# ---------------------------------------------------------------------------


def _loss(A6, w, V):
    lam, U = oracle.syev3(A6)
    return (w * lam).sum(1) + (V * U).sum((1, 2))


def _safe_sign(U):
    """True where every column's largest component is clearly the largest
    (finite differences must not flip the sign rule)."""
    a = np.sort(np.abs(U), axis=1)
    return np.all(a[:, 2, :] - a[:, 1, :] > 1e-3, axis=1)


@pin
def gradient_finite_differences():
    """The packed gradient of L = sum w lambda + sum V o U matches central
    differences (h = 1e-6, FP64) on matrices with gaps >= 0.05 ||d||."""
    A, d, _ = inputs.spectral(200, seed=24, near_degenerate=0.0, min_gap=0.05)
    lam, U = oracle.syev3(A)
    keep = _safe_sign(U)
    A, lam, U = A[keep][:40], lam[keep][:40], U[keep][:40]
    n = A.shape[0]
    rng = np.random.default_rng(25)
    w = rng.standard_normal((n, 3))
    V = rng.standard_normal((n, 3, 3))
    g = oracle.syev3_bwd(lam, U, w, V, 1e-6)
    h = 1e-6
    fd = np.empty((n, 6))
    for k in range(6):
        Ap, Am = A.copy(), A.copy()
        Ap[:, k] += h
        Am[:, k] -= h
        fd[:, k] = (_loss(Ap, w, V) - _loss(Am, w, V)) / (2 * h)
    err = np.abs(g - fd) / (1.0 + np.abs(g))
    assert err.max() <= 2e-6, err.max()


@pin
def gradient_mask():
    """Pairs with |lambda_i - lambda_j| < tau ||A||_F get no eigenvector
    coupling: U^T Abar U has a zero (i,j) entry there and keeps every other
    entry of the unmasked gradient."""
    A, d, deg = inputs.spectral(200, seed=26, near_degenerate=0.5)
    lam, U = oracle.syev3(A)
    n = A.shape[0]
    rng = np.random.default_rng(27)
    w = rng.standard_normal((n, 3))
    V = rng.standard_normal((n, 3, 3))
    tau = 1e-6
    g_mask = oracle.syev3_bwd(lam, U, w, V, tau)
    g_full = oracle.syev3_bwd(lam, U, w, V, 0.0)

    def core(g):  # noqa: E306
        # packed off-diagonals hold Abar_ij + Abar_ji: halving them gives the
        # symmetric part S of Abar, and U^T S U = (C + C^T)/2 for Abar = U C U^T
        P = inputs.unpack(g)
        S = 0.5 * (P + P * np.eye(3))
        return np.swapaxes(U, 1, 2) @ S @ U

    Cm, Cf = core(g_mask), core(g_full)
    nrm = np.linalg.norm(lam, axis=1)
    masked = 0
    for i in range(3):
        for j in range(i + 1, 3):
            close = np.abs(lam[:, i] - lam[:, j]) < tau * nrm
            masked += close.sum()
            # reconstructing C from Abar costs a few eps of the largest entry
            tol_m = 64 * EPS * np.abs(Cm).max(axis=(1, 2))
            tol_f = 64 * EPS * np.maximum(np.abs(Cf).max(axis=(1, 2)), np.abs(Cm).max(axis=(1, 2)))
            assert np.all(np.abs(Cm[close, i, j]) <= tol_m[close])
            assert np.all(np.abs(Cm[~close, i, j] - Cf[~close, i, j]) <= tol_f[~close])
    assert masked >= 50
    tol = 64 * EPS * np.abs(Cm).max(axis=(1, 2))[:, None]
    assert np.all(np.abs(np.diagonal(Cm, axis1=1, axis2=2) - w) <= tol)
