"""The kernels' own approximate arithmetic (arith.cuh), through
syev3_selftest_arith, against IEEE results on the host.

rcp64 -- the hardware reciprocal estimate refined by one third-order
Newton-Raphson step -- is claimed within 1 ulp of 1/x for 2^-1000 < |x| <
2^1000; the FP32 approximations rcp32, sqrt32 and rsqrt32 feed the FP32
zero finder, whose error allowances (several eps32 of each term, doubled)
assume each within 2 units of 2^-23 relative.  The exact values come from
extended precision on the host (np.longdouble: 64 or 113 significand bits).

f2d_exact and d2f_rn -- FP32 <-> FP64 conversions on the integer pipes
(normal numbers and zero; the rest through the hardware) -- must give the
IEEE conversions bit for bit: float -> double is exact, double -> float
rounds to nearest, ties to even.  The reference is the host's IEEE
conversion (numpy astype)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def syev3():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_06698_gb300 import build, syev3 as mod

    build.build()
    return mod


def log_uniform(rng, n, lo, hi, dtype):
    x = np.ldexp(1.0 + rng.random(n), rng.integers(lo, hi, n)) * rng.choice([-1.0, 1.0], n)
    return x.astype(dtype)


def ulp_error(y, exact):
    """|y - exact| in units of the spacing of float64 at |exact|."""
    return np.abs(y.astype(np.longdouble) - exact) / np.spacing(np.abs(exact.astype(np.float64)))


def test_rcp64_within_one_ulp(syev3):
    rng = np.random.default_rng(61)
    x = log_uniform(rng, 1 << 21, -1000, 1000, np.float64)
    # edge values: powers of two and their neighbours, the ends of the range,
    # mantissas just below 2 (the largest relative step of the estimate)
    p2 = np.ldexp(1.0, np.arange(-999, 1000))
    edges = np.concatenate([p2, np.nextafter(p2, 0.0), np.nextafter(p2, np.inf), -p2,
                            np.ldexp(np.nextafter(2.0, 0.0), np.arange(-1000, 999)),
                            [np.ldexp(1.0, -1000) * 1.0000001, np.ldexp(1.0, 1000) * 0.9999999, 1.0, 3.0, 7.0]])
    x = np.concatenate([x, edges])
    y = syev3.selftest_arith(syev3.ARITH_RCP64, torch.from_numpy(x).cuda()).cpu().numpy()
    exact = np.longdouble(1) / x.astype(np.longdouble)
    err = ulp_error(y, exact)
    assert np.all(np.sign(y) == np.sign(x))
    assert err.max() <= 1.0, (float(err.max()), float(x[np.argmax(err)]))


@pytest.mark.parametrize("op,f,lo,hi,signed", [
    ("rcp32", lambda v: 1 / v, -125, 125, True),
    ("sqrt32", lambda v: np.sqrt(v), -125, 126, False),
    ("rsqrt32", lambda v: 1 / np.sqrt(v), -125, 126, False),
])
def test_fp32_approximations_within_two_units(syev3, op, f, lo, hi, signed):
    code = {"rcp32": syev3.ARITH_RCP32, "sqrt32": syev3.ARITH_SQRT32, "rsqrt32": syev3.ARITH_RSQRT32}[op]
    rng = np.random.default_rng(62 + code)
    x = log_uniform(rng, 1 << 21, lo, hi, np.float64)
    if not signed:
        x = np.abs(x)
    p2 = np.ldexp(1.0, np.arange(lo, hi))
    x = np.concatenate([x, p2, np.nextafter(p2.astype(np.float32), np.float32(np.inf)).astype(np.float64),
                        np.ldexp(np.float64(np.nextafter(np.float32(2), np.float32(0))), np.arange(lo, hi - 1))])
    x32 = x.astype(np.float32)
    y = syev3.selftest_arith(code, torch.from_numpy(x32).cuda()).cpu().numpy().astype(np.float64)
    exact = f(x32.astype(np.float64))  # float64 is exact to 2^-53 here
    rel = np.abs(y - exact) / np.abs(exact)
    assert rel.max() <= 2.0 * 2.0 ** -23, (op, float(rel.max() / 2.0 ** -23), float(x32[np.argmax(rel)]))


def test_float_to_double_conversion_is_exact(syev3):
    rng = np.random.default_rng(63)
    bits = rng.integers(0, 1 << 32, 1 << 22, dtype=np.uint64).astype(np.uint32)
    edges = np.array([0, 0x80000000, 1, 0x807fffff, 0x007fffff, 0x00800000, 0x80800000, 0x7f7fffff, 0xff7fffff,
                      0x3f800000, 0x7f800000, 0xff800000, 0x7fc00000, 0x33800000, 0x4b800001], dtype=np.uint32)
    # every exponent with the smallest, largest and a random fraction
    e = np.repeat(np.arange(256, dtype=np.uint32) << 23, 3)
    fr = np.tile(np.array([0, 0x7fffff, 0x2aaaab], dtype=np.uint32), 256)
    x = np.concatenate([bits, edges, e | fr, (e | fr) | 0x80000000]).view(np.float32)
    y = syev3.selftest_arith(syev3.ARITH_F2D, torch.from_numpy(x).cuda()).cpu().numpy()
    want = x.astype(np.float64)
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(y), nan)
    assert np.array_equal(y[~nan].view(np.uint64), want[~nan].view(np.uint64))


def test_double_to_float_conversion_rounds_to_nearest_even(syev3):
    rng = np.random.default_rng(64)
    n = 1 << 22
    # exponents across the float subnormal, normal and overflow ranges
    E = rng.integers(820, 1200, n).astype(np.uint64)
    M = rng.integers(0, 1 << 52, n, dtype=np.uint64)
    # halfway and near-halfway fractions below the kept 23 bits
    low = np.array([0x10000000, 0x0fffffff, 0x10000001, 0, 0x1fffffff], dtype=np.uint64)
    M[: 5 * (n // 8)] = (M[: 5 * (n // 8)] & ~np.uint64(0x1fffffff)) | np.repeat(low, n // 8)
    S = rng.integers(0, 2, n).astype(np.uint64) << np.uint64(63)
    rand = (S | (E << np.uint64(52)) | M).view(np.float64)
    edges = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 3.4028234663852886e38, 3.4028235677973366e38,
                      3.402823669209385e38, 1.1754943508222875e-38, 1.1754942807573643e-38, 1.401298464324817e-45,
                      7.006492321624085e-46, 7.006492321624087e-46, 1e-300, -1e300, 1.0, -2.5])
    x = np.concatenate([rand, edges, rng.standard_normal(1 << 20)])
    y = syev3.selftest_arith(syev3.ARITH_D2F, torch.from_numpy(x).cuda()).cpu().numpy()
    with np.errstate(over="ignore"):
        want = x.astype(np.float32)
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(y), nan)
    assert np.array_equal(y[~nan].view(np.uint32), want[~nan].view(np.uint32))
