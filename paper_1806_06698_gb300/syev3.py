"""Thin ctypes binding of ``libsyev3.so`` (include/syev3.h).

Argument marshalling only: tensors are passed to the C ABI as raw device
pointers together with the current CUDA stream; every step of the solve runs
in the library's kernels.  There is no CPU fallback -- a missing library or a
CPU tensor raises.
"""

from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsyev3.so")

SYEV3_F64, SYEV3_F32, SYEV3_F32_COMPENSATED = 0, 1, 2
SYEV3_OK, SYEV3_EINVAL, SYEV3_ECUDA, SYEV3_ENOCONV, SYEV3_ETIMEOUT, SYEV3_EAGAIN = 0, 1, 2, 3, 4, 5
NUM_COUNTERS = 4
# syev3_batched_method: variants of the zero finder and the deflation test,
# and the layout of its statistics (include/syev3.h).
ZF_PRODUCTION, ZF_BORGES_GRAGG, ZF_NEWTON = 0, 1, 2
DEFLATION_SIMPLIFIED, DEFLATION_EISPACK = 0, 1
METHOD_STATS = ("capped", "nonfinite", "diagonal", "deflated", "reduced", "steps", "roots", "warp_slots")

_lock = threading.Lock()
_lib = None


class Syev3Error(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = _load()
        msg = lib.syev3_status_string(status).decode()
        if status == SYEV3_ECUDA:
            msg += f" (cudaError {lib.syev3_last_cuda_error()})"
        super().__init__(f"{where}: {msg}")
        self.status = status


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is not built; run `python -m paper_1806_06698_gb300.build` "
                                   "(or __graft_entry__.build()) -- there is no CPU fallback")
            lib = ctypes.CDLL(LIB_PATH)
            vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
            lib.syev3_abi_version.restype = i32
            lib.syev3_status_string.argtypes = [i32]
            lib.syev3_status_string.restype = ctypes.c_char_p
            lib.syev3_last_cuda_error.restype = i32
            lib.syev3_batched.argtypes = [vp, i64, vp, vp, i32, vp]
            lib.syev3_batched.restype = i32
            lib.syev3_batched_ex.argtypes = [vp, i64, vp, vp, i32, vp, vp]
            lib.syev3_batched_ex.restype = i32
            lib.syev3_batched_method.argtypes = [vp, i64, vp, vp, i32, ctypes.POINTER(_Method), vp, vp]
            lib.syev3_batched_method.restype = i32
            lib.syev3_workspace_bytes.argtypes = [i64, i32]
            lib.syev3_workspace_bytes.restype = ctypes.c_size_t
            lib.syev3_batched_ws.argtypes = [vp, i64, vp, vp, i32, vp, vp, ctypes.c_size_t, vp]
            lib.syev3_batched_ws.restype = i32
            lib.syev3_batched_static_ws.argtypes = [vp, i64, vp, vp, vp, vp]
            lib.syev3_batched_static_ws.restype = i32
            lib.syev3_batched_bwd.argtypes = [vp, vp, vp, vp, i64, vp, ctypes.c_double, i32, vp]
            lib.syev3_batched_bwd.restype = i32
            lib.syev3_batched_host.argtypes = [vp, i64, vp, vp, i32, i64, vp]
            lib.syev3_batched_host.restype = i32
            lib.syev3_selftest_wait_limit.argtypes = [vp]
            lib.syev3_selftest_wait_limit.restype = i32
            lib.syev3_device_flags.argtypes = [ctypes.POINTER(ctypes.c_uint32)]
            lib.syev3_device_flags.restype = i32
            lib.syev3_selftest_arith.argtypes = [i32, vp, vp, i64, vp]
            lib.syev3_selftest_arith.restype = i32
            lib.syev3_probe_dfma.argtypes = [i64, vp, ctypes.POINTER(ctypes.c_int64), vp]
            lib.syev3_probe_dfma.restype = i32
            _lib = lib
    return _lib


def library():
    """The loaded ctypes library (loads it on first use)."""
    return _load()


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _check(status: int, where: str):
    if status != SYEV3_OK:
        raise Syev3Error(status, where)


def dtype_code(dtype: torch.dtype, compensated: bool = False) -> int:
    if dtype == torch.float64:
        if compensated:
            raise ValueError("the compensated path takes float32 inputs")
        return SYEV3_F64
    if dtype == torch.float32:
        return SYEV3_F32_COMPENSATED if compensated else SYEV3_F32
    raise ValueError(f"unsupported dtype {dtype}")


def workspace_bytes(n: int, dtype: torch.dtype, compensated: bool = False) -> int:
    """Bytes of device workspace syev3_batched(..., workspace=...) needs."""
    return int(_load().syev3_workspace_bytes(int(n), dtype_code(dtype, compensated)))


def syev3_batched(A6: torch.Tensor, *, vectors: bool = True, compensated: bool = False,
                  out: tuple[torch.Tensor, torch.Tensor | None] | None = None,
                  counters: torch.Tensor | None = None, workspace: torch.Tensor | None = None, stream=None):
    """Eigenvalues (n,3) ascending and eigenvectors (n,3,3) (columns) of the
    packed symmetric matrices ``A6`` (n,6) on the GPU.  ``counters`` is an
    optional uint64-sized (int64) device tensor of 4 entries the kernels add
    to (see include/syev3.h).  ``workspace`` (a device tensor of at least
    workspace_bytes(...) bytes) selects syev3_batched_ws: for the compensated
    form, the FP64 refinement as a second kernel."""
    if not A6.is_cuda:
        raise ValueError("A6 must be a CUDA tensor (no CPU fallback)")
    if A6.dim() != 2 or A6.shape[1] != 6 or not A6.is_contiguous():
        raise ValueError("A6 must be a contiguous (n, 6) tensor")
    n = A6.shape[0]
    code = dtype_code(A6.dtype, compensated)
    if out is None:
        lam = torch.empty((n, 3), dtype=A6.dtype, device=A6.device)
        U = torch.empty((n, 3, 3), dtype=A6.dtype, device=A6.device) if vectors else None
    else:
        lam, U = out
    lib = _load()
    if workspace is not None:
        st = lib.syev3_batched_ws(_ptr(A6), n, _ptr(lam), _ptr(U), code, _ptr(counters), _ptr(workspace),
                                  workspace.numel() * workspace.element_size(), _stream(stream))
    elif counters is None:
        st = lib.syev3_batched(_ptr(A6), n, _ptr(lam), _ptr(U), code, _stream(stream))
    else:
        st = lib.syev3_batched_ex(_ptr(A6), n, _ptr(lam), _ptr(U), code, _ptr(counters), _stream(stream))
    _check(st, "syev3_batched")
    return lam, U


class _Method(ctypes.Structure):
    _fields_ = [("zero_finder", ctypes.c_int), ("deflation_test", ctypes.c_int)]


def syev3_batched_method(A6: torch.Tensor, *, zero_finder: int = ZF_PRODUCTION,
                         deflation_test: int = DEFLATION_SIMPLIFIED, vectors: bool = True,
                         out: tuple[torch.Tensor, torch.Tensor | None] | None = None,
                         stats: torch.Tensor | None = None, stream=None):
    """FP64 solve with a chosen zero finder and deflation test (the method
    study entry point).  ``stats`` is an optional int64 device tensor of
    len(METHOD_STATS) entries the kernel adds to."""
    if not A6.is_cuda or A6.dtype != torch.float64:
        raise ValueError("A6 must be a float64 CUDA tensor (no CPU fallback)")
    if A6.dim() != 2 or A6.shape[1] != 6 or not A6.is_contiguous():
        raise ValueError("A6 must be a contiguous (n, 6) tensor")
    n = A6.shape[0]
    if out is None:
        lam = torch.empty((n, 3), dtype=A6.dtype, device=A6.device)
        U = torch.empty((n, 3, 3), dtype=A6.dtype, device=A6.device) if vectors else None
    else:
        lam, U = out
    m = _Method(int(zero_finder), int(deflation_test))
    st = _load().syev3_batched_method(_ptr(A6), n, _ptr(lam), _ptr(U), SYEV3_F64, ctypes.byref(m), _ptr(stats),
                                      _stream(stream))
    _check(st, "syev3_batched_method")
    return lam, U


# Largest batch of syev3_batched_static_ws (its scratch is a static array).
STATIC_MAX_N = 262144


def syev3_batched_static_ws(A6: torch.Tensor, *, vectors: bool = True,
                            out: tuple[torch.Tensor, torch.Tensor | None] | None = None,
                            counters: torch.Tensor | None = None, stream=None):
    """The compensated FP32 solve with its refinement list in the library's
    static device memory (no workspace, no allocation); n <= STATIC_MAX_N.
    Calls on one device must not overlap in time."""
    if not A6.is_cuda or A6.dtype != torch.float32:
        raise ValueError("A6 must be a float32 CUDA tensor (no CPU fallback)")
    if A6.dim() != 2 or A6.shape[1] != 6 or not A6.is_contiguous():
        raise ValueError("A6 must be a contiguous (n, 6) tensor")
    n = A6.shape[0]
    if out is None:
        lam = torch.empty((n, 3), dtype=A6.dtype, device=A6.device)
        U = torch.empty((n, 3, 3), dtype=A6.dtype, device=A6.device) if vectors else None
    else:
        lam, U = out
    st = _load().syev3_batched_static_ws(_ptr(A6), n, _ptr(lam), _ptr(U), _ptr(counters), _stream(stream))
    _check(st, "syev3_batched_static_ws")
    return lam, U


def syev3_batched_host(A6: torch.Tensor, lam: torch.Tensor, U: torch.Tensor | None = None, *,
                       compensated: bool = False, chunk: int = 0, stream=None):
    """Blocking solve of host (CPU, ideally pinned) tensors through the C
    ABI's pipelined host entry point; fills lam (n,3) and U (n,3,3).
    ``chunk`` <= 0 takes the library's schedule (2^16 matrices first, each
    next chunk a quarter longer, up to 2^20)."""
    for t in (A6, lam) + ((U,) if U is not None else ()):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError("host buffers must be contiguous CPU tensors")
    lib = _load()
    st = lib.syev3_batched_host(_ptr(A6), A6.shape[0], _ptr(lam), _ptr(U), dtype_code(A6.dtype, compensated),
                                int(chunk), _stream(stream))
    _check(st, "syev3_batched_host")
    return lam, U


def device_flags() -> int:
    """Device-side status bits since the last call (bit 0: a wait timed out)."""
    lib = _load()
    v = ctypes.c_uint32(0)
    _check(lib.syev3_device_flags(ctypes.byref(v)), "syev3_device_flags")
    return int(v.value)


# Operations of syev3_selftest_arith (include/syev3.h).
ARITH_RCP64, ARITH_RCP32, ARITH_SQRT32, ARITH_RSQRT32, ARITH_F2D, ARITH_D2F = 0, 1, 2, 3, 4, 5


def selftest_arith(op: int, x: torch.Tensor, stream=None) -> torch.Tensor:
    """The kernels' arithmetic helpers applied to the device tensor x:
    reciprocal / square root approximations (float64 in and out for
    ARITH_RCP64, float32 otherwise) and the integer-pipe conversions
    (ARITH_F2D: float32 -> float64, ARITH_D2F: float64 -> float32)."""
    want = torch.float64 if op in (ARITH_RCP64, ARITH_D2F) else torch.float32
    out = torch.float64 if op in (ARITH_RCP64, ARITH_F2D) else torch.float32
    if not x.is_cuda or x.dtype != want or not x.is_contiguous():
        raise ValueError(f"x must be a contiguous {want} CUDA tensor")
    y = torch.empty(x.shape, dtype=out, device=x.device)
    _check(_load().syev3_selftest_arith(int(op), _ptr(x), _ptr(y), x.numel(), _stream(stream)),
           "syev3_selftest_arith")
    return y


def probe_dfma(iters: int, sink: torch.Tensor, stream=None) -> int:
    """Launch the FP64 fused multiply-add rate probe on ``stream`` (sink: a
    float64 device tensor of >= 1 element); returns the number of FP64 FMAs
    the launch executes (time it with events on the same stream)."""
    cnt = ctypes.c_int64(0)
    _check(_load().syev3_probe_dfma(int(iters), _ptr(sink), ctypes.byref(cnt), _stream(stream)),
           "syev3_probe_dfma")
    return int(cnt.value)


def syev3_batched_bwd(lam: torch.Tensor, U: torch.Tensor, g_lam: torch.Tensor, g_U: torch.Tensor | None,
                      gap_tau: float = 1e-6, *, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Packed (n, 6) gradient of a loss through (lam, U) of syev3_batched:
    Abar = U (diag(g_lam) + F o (U^T g_U)) U^T with F_ij = 1/(lam_j - lam_i),
    pairs closer than gap_tau * ||A||_F masked; off-diagonal packed entries
    hold Abar_ij + Abar_ji."""
    for t in (lam, U, g_lam) + ((g_U,) if g_U is not None else ()):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("backward inputs must be contiguous CUDA tensors (no CPU fallback)")
    n = lam.shape[0]
    code = SYEV3_F64 if lam.dtype == torch.float64 else SYEV3_F32
    gA = torch.empty((n, 6), dtype=lam.dtype, device=lam.device) if out is None else out
    lib = _load()
    st = lib.syev3_batched_bwd(_ptr(lam), _ptr(U), _ptr(g_lam), _ptr(g_U), n, _ptr(gA), float(gap_tau), code,
                               _stream(stream))
    _check(st, "syev3_batched_bwd")
    return gA


class Syev3Function(torch.autograd.Function):
    """(lam, U) = eigh of packed symmetric 3x3 matrices, differentiable:
    the backward pass is the library's k_syev3_bwd kernel."""

    @staticmethod
    def forward(ctx, A6, compensated: bool = False, gap_tau: float = 1e-6):
        lam, U = syev3_batched(A6, compensated=compensated)
        ctx.save_for_backward(lam, U)
        ctx.gap_tau = gap_tau
        return lam, U

    @staticmethod
    def backward(ctx, g_lam, g_U):
        lam, U = ctx.saved_tensors
        g_lam = torch.zeros_like(lam) if g_lam is None else g_lam.contiguous()
        g_U = None if g_U is None else g_U.contiguous()
        return syev3_batched_bwd(lam, U, g_lam, g_U, ctx.gap_tau), None, None


def eigh3(A6: torch.Tensor, compensated: bool = False, gap_tau: float = 1e-6):
    """Differentiable batched eigendecomposition of packed (n, 6) matrices."""
    return Syev3Function.apply(A6, compensated, gap_tau)


class _ServerConfig(ctypes.Structure):
    _fields_ = [("memory_budget_bytes", ctypes.c_size_t), ("chunk", ctypes.c_int64),
                ("round_matrices", ctypes.c_int64), ("max_rounds_in_flight", ctypes.c_int)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("dtype", ctypes.c_int), ("n", ctypes.c_int64),
                ("d_lambda", ctypes.c_void_p), ("d_U", ctypes.c_void_p), ("t_submit_ns", ctypes.c_int64),
                ("t_admit_ns", ctypes.c_int64), ("t_done_ns", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("matrices", ctypes.c_int64), ("chunks", ctypes.c_int64),
                ("waiting", ctypes.c_int64), ("arena_bytes", ctypes.c_size_t), ("arena_used", ctypes.c_size_t),
                ("arena_peak", ctypes.c_size_t), ("error", ctypes.c_int), ("rounds", ctypes.c_int64),
                ("launches", ctypes.c_int64)]


# Requests outstanding (submitted, not released) at most (include/syev3.h).
SERVER_SLOTS = 16384


def _bind_server(lib):
    if getattr(lib, "_server_bound", False):
        return
    vp = ctypes.c_void_p
    lib.syev3_server_create.argtypes = [ctypes.POINTER(_ServerConfig), ctypes.POINTER(vp)]
    lib.syev3_server_destroy.argtypes = [vp]
    lib.syev3_server_submit.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int64, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_uint64)]
    lib.syev3_server_query.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(RequestInfo)]
    lib.syev3_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_double]
    lib.syev3_server_release.argtypes = [vp, ctypes.c_uint64]
    lib.syev3_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
    lib.syev3_server_inject_failure.argtypes = [vp, ctypes.c_int]
    for f in ("syev3_server_create", "syev3_server_destroy", "syev3_server_submit", "syev3_server_query",
              "syev3_server_wait", "syev3_server_release", "syev3_server_get_stats", "syev3_server_inject_failure"):
        getattr(lib, f).restype = ctypes.c_int
    lib._server_bound = True


class Server:
    """Continuous-batching request server with device-resident queues and
    admission (see include/syev3.h).  Requests are device tensors of packed
    matrices; results stay in the server's device arena until released."""

    def __init__(self, memory_budget_bytes: int = 16 << 30, chunk: int = 1 << 18, round_matrices: int = 1 << 21,
                 max_rounds_in_flight: int = 2):
        self._lib = _load()
        _bind_server(self._lib)
        cfg = _ServerConfig(memory_budget_bytes, chunk, round_matrices, max_rounds_in_flight)
        h = ctypes.c_void_p()
        _check(self._lib.syev3_server_create(ctypes.byref(cfg), ctypes.byref(h)), "syev3_server_create")
        self._h = h
        self._keep = {}

    def submit(self, A6: torch.Tensor, compensated: bool = False, vectors: bool = True) -> int:
        if not A6.is_cuda or not A6.is_contiguous() or A6.dim() != 2 or A6.shape[1] != 6:
            raise ValueError("A6 must be a contiguous (n, 6) CUDA tensor")
        t = ctypes.c_uint64()
        st = self._lib.syev3_server_submit(self._h, dtype_code(A6.dtype, compensated), _ptr(A6), A6.shape[0],
                                           int(vectors), ctypes.byref(t))
        _check(st, "syev3_server_submit")
        self._keep[t.value] = A6  # the input must outlive the request
        return t.value

    def query(self, ticket: int) -> RequestInfo:
        info = RequestInfo()
        _check(self._lib.syev3_server_query(self._h, ticket, ctypes.byref(info)), "syev3_server_query")
        return info

    def wait(self, ticket: int, timeout_s: float = 60.0) -> RequestInfo:
        _check(self._lib.syev3_server_wait(self._h, ticket, float(timeout_s)), "syev3_server_wait")
        return self.query(ticket)

    def results(self, ticket: int):
        """(lambda, U) of a done request: tensors viewing the server's arena
        (no copy); clone them before release if they are to be kept."""
        info = self.query(ticket)
        dt = self._keep[ticket].dtype
        lam = _device_view(info.d_lambda, (info.n, 3), dt)
        U = _device_view(info.d_U, (info.n, 3, 3), dt) if info.d_U else None
        return lam, U

    def release(self, ticket: int):
        _check(self._lib.syev3_server_release(self._h, ticket), "syev3_server_release")
        self._keep.pop(ticket, None)

    def inject_failure(self, status: int = SYEV3_ECUDA):
        """Fail the server as if its next launch returned ``status`` (tests)."""
        _check(self._lib.syev3_server_inject_failure(self._h, int(status)), "syev3_server_inject_failure")

    def stats(self) -> ServerStats:
        st = ServerStats()
        _check(self._lib.syev3_server_get_stats(self._h, ctypes.byref(st)), "syev3_server_get_stats")
        return st

    def close(self):
        if self._h:
            self._lib.syev3_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DeviceArray:
    def __init__(self, ptr: int, shape, dtype):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f8" if dtype == torch.float64 else "<f4",
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def _device_view(ptr: int, shape, dtype) -> torch.Tensor:
    """A tensor viewing library-owned device memory at ``ptr``."""
    return torch.as_tensor(_DeviceArray(ptr, shape, dtype), device="cuda")
