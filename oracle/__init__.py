"""Python handle on the CPU FP64 oracle (test infrastructure only).

The oracle is plain C++ (``syev3_oracle.cpp``: the method of C. F. Borges,
"Solving the 3x3 Real Symmetric Eigenproblem", arXiv 1806.06698, step by step;
``ddjacobi.cpp``: an independent double-double cyclic-Jacobi brute force).
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.

Layouts: packed input ``(n, 6)`` float64 in the order (a11, a22, a33, a12,
a13, a23); eigenvalues ``(n, 3)`` ascending; eigenvectors ``(n, 3, 3)`` with
column k the eigenvector of eigenvalue k.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ("syev3_oracle.cpp", "ddjacobi.cpp")
_LIBNAME = "liboracle.so"
_lock = threading.Lock()
_lib = None

# Layout constants of oracle_trace (see syev3_oracle.cpp).
TRACE_MAX = 72
TRACE_LEN = 32 + 2 * 6 * TRACE_MAX

CLS_DIAGONAL, CLS_DEFLATED, CLS_REDUCED, CLS_NONFINITE = 0, 1, 2, 3


def build(force: bool = False, src_dir: str | None = None, out: str | None = None) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (g++, no fast-math,
    no FP contraction, so x86-64 and aarch64 give identical results).
    ``src_dir``/``out`` build a copy elsewhere (the mutation tests use this)."""
    src_dir = src_dir or _HERE
    out = out or os.path.join(_HERE, _LIBNAME)
    srcs = [os.path.join(src_dir, s) for s in _SOURCES]
    if not force and os.path.exists(out):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(out) >= newest:
            return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", *srcs, "-o", tmp, "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _bind(path: str):
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    i64 = ctypes.c_int64
    lib.oracle_syev3.argtypes = [dp, i64, dp, dp, ctypes.POINTER(ctypes.c_int32), dp]
    lib.oracle_syev3.restype = None
    lib.oracle_syev3_threads.argtypes = [dp, i64, dp, dp, ctypes.c_int]
    lib.oracle_syev3_threads.restype = ctypes.c_double
    lib.oracle_count_ops.argtypes = [dp, i64, ctypes.POINTER(ctypes.c_uint64), dp]
    lib.oracle_count_ops.restype = None
    lib.oracle_trace.argtypes = [dp, dp, dp]
    lib.oracle_trace.restype = ctypes.c_int
    lib.oracle_jacobi2.argtypes = [ctypes.c_double] * 3 + [dp]
    lib.oracle_jacobi2.restype = None
    lib.oracle_zero.argtypes = [ctypes.c_double] * 4 + [ctypes.c_int, dp, dp]
    lib.oracle_zero.restype = None
    lib.oracle_syev3_bwd.argtypes = [dp, dp, dp, dp, i64, ctypes.c_double, dp]
    lib.oracle_syev3_bwd.restype = None
    lib.dd_jacobi3_batch.argtypes = [dp, i64, dp, dp, dp]
    lib.dd_jacobi3_batch.restype = None
    lib.dd_op.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4 + [dp]
    lib.dd_op.restype = None
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


def use_library(path: str | None):
    """Point this module at another build of the oracle (``None`` restores
    the default build).  Only the mutation tests use this."""
    global _lib
    with _lock:
        _lib = _bind(path) if path else None


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _params(c_defl=1.0, c_term=2.0, maxit=64, deflation_test=0, zero_finder=0):
    return np.array([c_defl, c_term, maxit, deflation_test, zero_finder], dtype=np.float64)


def _as_packed(A6) -> np.ndarray:
    A6 = np.ascontiguousarray(np.asarray(A6, dtype=np.float64))
    if A6.ndim == 1:
        A6 = A6.reshape(1, 6)
    if A6.ndim != 2 or A6.shape[1] != 6:
        raise ValueError("packed input must have shape (n, 6)")
    return A6


def syev3(A6, *, with_info: bool = False, **params):
    """Eigenvalues (n,3) ascending and eigenvectors (n,3,3) of packed matrices.

    ``params`` overrides the readings of the paper's unstated constants:
    c_defl, c_term, maxit, deflation_test (0 simplified, 1 EISPACK-style),
    zero_finder (0 Borges-Gragg, 1 Newton).  With ``with_info`` also returns an
    (n,5) int32 array {class, it_mu, it_nu, converged, exponent}.
    """
    lib = _load()
    A6 = _as_packed(A6)
    n = A6.shape[0]
    lam = np.empty((n, 3), np.float64)
    U = np.empty((n, 3, 3), np.float64)
    info = np.empty((n, 5), np.int32)
    p = _params(**params)
    lib.oracle_syev3(_dp(A6), n, _dp(lam), _dp(U),
                     info.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(p))
    if with_info:
        return lam, U, info
    return lam, U


def syev3_timed(A6, nthreads: int):
    """Run the oracle over ``nthreads`` host threads; returns (lam, U, seconds)."""
    lib = _load()
    A6 = _as_packed(A6)
    n = A6.shape[0]
    lam = np.empty((n, 3), np.float64)
    U = np.empty((n, 3, 3), np.float64)
    secs = lib.oracle_syev3_threads(_dp(A6), n, _dp(lam), _dp(U), int(nthreads))
    return lam, U, secs


def count_ops(A6, **params) -> np.ndarray:
    """Algorithmic FP64 operation counts per matrix: (n,4) {add/sub, mul, div, sqrt}."""
    lib = _load()
    A6 = _as_packed(A6)
    n = A6.shape[0]
    ops = np.empty((n, 4), np.uint64)
    p = _params(**params)
    lib.oracle_count_ops(_dp(A6), n, ops.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _dp(p))
    return ops


def trace(a6, **params) -> dict | None:
    """Arrow-frame internals of one matrix (None for non-finite input)."""
    lib = _load()
    a = np.ascontiguousarray(np.asarray(a6, dtype=np.float64).reshape(6))
    out = np.zeros(TRACE_LEN, np.float64)
    p = _params(**params)
    cls = lib.oracle_trace(_dp(a), _dp(out), _dp(p))
    if cls < 0:
        return None
    T = TRACE_MAX

    def zf(off, nit):
        blk = out[32 + off * 6 * T: 32 + (off + 1) * 6 * T].reshape(6, T)[:, :nit]
        return dict(x=blk[0].copy(), f=blk[1].copy(), fp=blk[2].copy(),
                    w0=blk[3].copy(), w1=blk[4].copy(), direct=blk[5].astype(bool))

    r = dict(alpha1=out[0], alpha2=out[1], beta1=out[2], beta2=out[3], gamma=out[4],
             c=out[5], s=out[6], h=out[7], mu=out[8], nu=out[9],
             u=out[10:19].reshape(3, 3).copy(), cls=int(out[19]), it_mu=int(out[20]),
             it_nu=int(out[21]), converged=int(out[22]), exponent=int(out[23]))
    r["zmu"] = zf(0, int(out[24]))
    r["znu"] = zf(1, int(out[25]))
    return r


def jacobi2(p: float, q: float, r: float):
    """Ordered Jacobi rotation of [[p,q],[q,r]]: (c, s, l1, l2), l1 >= l2."""
    lib = _load()
    out = np.zeros(4, np.float64)
    lib.oracle_jacobi2(float(p), float(q), float(r), _dp(out))
    return tuple(float(v) for v in out)


def zero(abar, b1, b2, gbar, method: int = 0, **params):
    """Zero of the spectral function of a fully reduced arrow: (x, iters, converged)."""
    lib = _load()
    out = np.zeros(3, np.float64)
    p = _params(**params)
    lib.oracle_zero(float(abar), float(b1), float(b2), float(gbar), int(method), _dp(out), _dp(p))
    return float(out[0]), int(out[1]), int(out[2])


def syev3_bwd(lam, U, glam, gU, tau: float) -> np.ndarray:
    """Packed (n,6) gradient of a loss through (lam, U), gaps below tau*||A||_F masked."""
    lib = _load()
    lam = np.ascontiguousarray(lam, np.float64).reshape(-1, 3)
    n = lam.shape[0]
    U = np.ascontiguousarray(U, np.float64).reshape(n, 9)
    glam = np.ascontiguousarray(glam, np.float64).reshape(n, 3)
    gU = np.ascontiguousarray(gU, np.float64).reshape(n, 9)
    gA = np.empty((n, 6), np.float64)
    lib.oracle_syev3_bwd(_dp(lam), _dp(U), _dp(glam), _dp(gU), n, float(tau), _dp(gA))
    return gA


def dd_jacobi(A6):
    """Double-double cyclic Jacobi: (lam_hi, lam_lo, V), ascending, V columns."""
    lib = _load()
    A6 = _as_packed(A6)
    n = A6.shape[0]
    hi = np.empty((n, 3), np.float64)
    lo = np.empty((n, 3), np.float64)
    V = np.empty((n, 3, 3), np.float64)
    lib.dd_jacobi3_batch(_dp(A6), n, _dp(hi), _dp(lo), _dp(V))
    return hi, lo, V


def dd_op(op: int, x, y=(0.0, 0.0)):
    """Double-double primitive: op 0 add, 1 mul, 2 div, 3 sqrt -> (hi, lo)."""
    lib = _load()
    out = np.zeros(2, np.float64)
    lib.dd_op(int(op), float(x[0]), float(x[1]), float(y[0]), float(y[1]), _dp(out))
    return float(out[0]), float(out[1])
