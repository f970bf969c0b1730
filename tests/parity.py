"""Comparison helpers for the GPU parity tests (numpy, float64).

The CUDA results are compared with the CPU oracle element by element:
eigenvalues within a normwise tolerance, eigenvectors up to sign where the
eigenvalue gap makes them unique, and -- everywhere -- the residual and the
orthogonality of the GPU's own factorisation.
"""

from __future__ import annotations

import numpy as np

from paper_1806_06698_gb300 import inputs

EPS64 = 2.0 ** -52
EPS32 = 2.0 ** -23


def fro(A6):
    M = inputs.unpack(np.asarray(A6, np.float64))
    s = np.max(np.abs(M), axis=(1, 2))
    s = np.where(s > 0, s, 1.0)
    return s * np.linalg.norm(M / s[:, None, None], axis=(1, 2))


def residual(A6, lam, U):
    M = inputs.unpack(np.asarray(A6, np.float64))
    s = np.max(np.abs(M), axis=(1, 2))
    s = np.where(s > 0, s, 1.0)
    lam = np.asarray(lam, np.float64)
    U = np.asarray(U, np.float64)
    R = (M / s[:, None, None]) @ U - U * (lam / s[:, None])[:, None, :]
    return s * np.linalg.norm(R, axis=(1, 2))


def orthogonality(U):
    U = np.asarray(U, np.float64)
    return np.linalg.norm(np.swapaxes(U, 1, 2) @ U - np.eye(3), axis=(1, 2))


def sign_rule_holds(U):
    """Each column's first largest-magnitude component is positive."""
    U = np.asarray(U)
    im = np.argmax(np.abs(U), axis=1)
    top = np.take_along_axis(U, im[:, None, :], axis=1)[:, 0, :]
    return np.all(top > 0, axis=1)


def compare(A6, lam, U, lam_o, U_o, *, eps, lam_tol, res_tol, orth_tol, vec_tol):
    """Raise AssertionError with a summary unless the GPU result (lam, U)
    matches the oracle's (lam_o, U_o) on the inputs A6.

    lam_tol:  |lam - lam_o| <= lam_tol * eps * ||A||_F (every eigenvalue)
    res_tol:  ||A U - U Lam||_F <= res_tol * ||A||_F
    orth_tol: ||U^T U - I||_F <= orth_tol * eps
    vec_tol:  where the relative gap g = gap/||A||_F of an eigenvalue to its
              neighbours is >= 1e-6: min(|u - u_o|, |u + u_o|) <= vec_tol * eps / g
    """
    A6 = np.asarray(A6, np.float64)
    lam = np.asarray(lam, np.float64)
    lam_o = np.asarray(lam_o, np.float64)
    nrm = fro(A6)
    ok = nrm > 0
    dl = np.max(np.abs(lam - lam_o), axis=1) / np.where(ok, nrm, 1.0)
    worst = float(np.max(dl) / eps) if dl.size else 0.0
    assert np.all(dl <= lam_tol * eps), f"eigenvalues off by {worst:.2f} eps ||A||_F (tol {lam_tol})"
    if U is None:
        return
    U = np.asarray(U, np.float64)
    U_o = np.asarray(U_o, np.float64)
    res = residual(A6, lam, U) / np.where(ok, nrm, 1.0)
    assert np.all(res <= res_tol), f"residual {res.max():.3e} ||A||_F > {res_tol}"
    orth = orthogonality(U)
    assert np.all(orth <= orth_tol * eps), f"orthogonality {orth.max() / eps:.2f} eps > {orth_tol}"
    assert np.all(sign_rule_holds(U)), "sign rule violated"
    gap = np.stack([lam_o[:, 1] - lam_o[:, 0],
                    np.minimum(lam_o[:, 1] - lam_o[:, 0], lam_o[:, 2] - lam_o[:, 1]),
                    lam_o[:, 2] - lam_o[:, 1]], axis=1) / np.where(ok, nrm, 1.0)[:, None]
    for k in range(3):
        sel = ok & (gap[:, k] >= 1e-6)
        d = np.minimum(np.linalg.norm(U[sel, :, k] - U_o[sel, :, k], axis=1),
                       np.linalg.norm(U[sel, :, k] + U_o[sel, :, k], axis=1))
        bound = vec_tol * eps / gap[sel, k]
        if d.size:
            assert np.all(d <= bound), f"eigenvector {k} off by {np.max(d / bound):.2f} x tolerance"


def compare_f64(A6, lam, U, lam_o, U_o):
    """The FP64 bar: |dlambda| <= 8 eps ||A||_F, residual <= 1e-14 ||A||_F,
    orthogonality <= 16 eps, eigenvectors within 32 eps / relative gap."""
    compare(A6, lam, U, lam_o, U_o, eps=EPS64, lam_tol=8, res_tol=1e-14, orth_tol=16, vec_tol=32)


def compare_f32(A32, lam, U, lam_o, U_o):
    """The FP32 bar: eigenvalues, residual and orthogonality everywhere;
    eigenvectors up to sign where the relative gap is >= 1e-2."""
    A64 = np.asarray(A32, np.float64)
    compare(A64, lam, None, lam_o, None, eps=EPS32, lam_tol=64, res_tol=0, orth_tol=0, vec_tol=0)
    nrm = fro(A64)
    ok = nrm > 0
    res = residual(A64, lam, U) / np.where(ok, nrm, 1.0)
    assert np.all(res <= 64 * EPS32), f"residual {res.max() / EPS32:.1f} eps32 ||A||_F"
    orth = orthogonality(U)
    assert np.all(orth <= 64 * EPS32), f"orthogonality {orth.max() / EPS32:.1f} eps32"
    assert np.all(sign_rule_holds(U)), "sign rule violated"
    gap = np.min(np.diff(lam_o, axis=1), axis=1) / np.where(ok, nrm, 1.0)
    sel = ok & (gap >= 1e-2)
    for k in range(3):
        d = np.minimum(np.linalg.norm(U[sel, :, k] - U_o[sel, :, k], axis=1),
                       np.linalg.norm(U[sel, :, k] + U_o[sel, :, k], axis=1))
        assert np.all(d <= 64 * EPS32 / gap[sel]), (k, float(np.max(d * gap[sel] / EPS32)))


def chunked(check, n: int, chunk: int = 1 << 20, workers: int | None = None):
    """Run check(lo, hi) over [0, n) in chunks on a thread pool (numpy
    releases the interpreter lock inside its array operations); re-raises
    the first failure.  For element-wise comparisons of full-size batches."""
    import concurrent.futures as cf
    import os

    workers = workers or max(1, min(16, os.cpu_count() or 1))
    spans = [(lo, min(n, lo + chunk)) for lo in range(0, n, chunk)]
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        for f in [ex.submit(check, lo, hi) for lo, hi in spans]:
            f.result()


def oracle_all_cores(A6):
    """The CPU oracle over every host core: (lam, U) of the packed batch."""
    import os

    import oracle

    lam, U, _ = oracle.syev3_timed(np.ascontiguousarray(A6, np.float64), os.cpu_count() or 1)
    return lam, U
