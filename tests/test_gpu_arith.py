"""The kernels' own approximate arithmetic (arith.cuh), through
syev3_selftest_arith, against IEEE results on the host.

rcp64 -- the hardware reciprocal estimate refined by one third-order
Newton-Raphson step -- is claimed within 1 ulp of 1/x for 2^-1000 < |x| <
2^1000; the FP32 approximations rcp32, sqrt32 and rsqrt32 feed the FP32
zero finder, whose error allowances (several eps32 of each term, doubled)
assume each within 2 units of 2^-23 relative.  The exact values come from
extended precision on the host (np.longdouble: 64 or 113 significand bits)."""

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
