"""FP64 parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar (FP64): |dlambda| <= 8 eps ||A||_F per eigenvalue, residual <= 1e-14
||A||_F, orthogonality <= 16 eps, eigenvectors (where the relative gap is
>= 1e-6) within 32 eps / gap up to sign; exact diagonals bit for bit.
"""

import numpy as np
import pytest

import oracle
import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1806_06698_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def syev3():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_06698_gb300 import build, syev3 as mod

    build.build()
    return mod


def run_gpu(mod, A6_np, vectors=True, counters=None):
    A = torch.from_numpy(np.ascontiguousarray(A6_np)).cuda()
    lam, U = mod.syev3_batched(A, vectors=vectors, counters=counters)
    torch.cuda.synchronize()
    return lam.cpu().numpy(), (U.cpu().numpy() if U is not None else None)


def test_gaussian_4096(syev3):
    """The small parity workload: 4096 matrices with iid N(0,1) entries."""
    A = inputs.gaussian(4096)
    lam, U = run_gpu(syev3, A)
    lam_o, U_o = oracle.syev3(A)
    parity.compare_f64(A, lam, U, lam_o, U_o)


@pytest.mark.parametrize("n", [1, 2, 31, 127, 128, 129, 1000, 3 * 128 + 37, 20011])
def test_mixed_ragged(syev3, n):
    """The mixed-difficulty recipe at sizes spanning several tiles and a ragged tail."""
    A, ids = inputs.mixed(n, seed=1000 + n)
    lam, U = run_gpu(syev3, A)
    lam_o, U_o = oracle.syev3(A)
    parity.compare_f64(A, lam, U, lam_o, U_o)


def test_mixed_subsets_and_exact_diagonals(syev3):
    A, ids = inputs.mixed(1 << 16, seed=77)
    lam, U = run_gpu(syev3, A)
    lam_o, U_o, info = oracle.syev3(A, with_info=True)
    for s in inputs.SUBSET_NAMES:
        m = ids == s
        parity.compare_f64(A[m], lam[m], U[m], lam_o[m], U_o[m])
    d = ids == inputs.SUBSET_DIAGONAL_REPEATED
    assert np.array_equal(lam[d], lam_o[d]) and np.array_equal(U[d], U_o[d])


@pytest.mark.parametrize("n", [1, 129, 5000, 20011])
def test_eigenvalues_only_matches(syev3, n):
    """The eigenvalues-only kernel (no eigenvectors formed) returns the
    eigenvalues of the full solve bit for bit, at sizes that exercise the
    carried arrows and the final pass."""
    A, _ = inputs.mixed(n, seed=78 + n)
    lam_v, _ = run_gpu(syev3, A, vectors=True)
    lam_n, U_n = run_gpu(syev3, A, vectors=False)
    assert U_n is None
    assert np.array_equal(lam_v, lam_n)


def test_scale_equivariance_bitwise(syev3):
    """Power-of-two scaling commutes with the solve bit for bit."""
    A, _ = inputs.mixed(3000, seed=79, log10_scale=0.0)
    lam0, U0 = run_gpu(syev3, A)
    for k in (-500, -11, 7, 500):
        lam, U = run_gpu(syev3, np.ldexp(A, k))
        assert np.array_equal(lam, np.ldexp(lam0, k)) and np.array_equal(U, U0)


def test_special_inputs_and_counters(syev3):
    A = inputs.gaussian(300, seed=80)
    A[0] = 0.0
    A[1, 2] = np.nan
    A[2, 4] = np.inf
    A[3, 0] = -np.inf
    ctr = torch.zeros(syev3.NUM_COUNTERS, dtype=torch.int64, device="cuda")
    lam, U = run_gpu(syev3, A, counters=ctr)
    c = ctr.cpu().numpy()
    assert c[1] == 3 and c[0] == 0
    assert np.array_equal(lam[0], np.zeros(3)) and np.array_equal(U[0], np.eye(3))
    assert np.all(np.isnan(lam[1:4])) and np.all(np.isnan(U[1:4]))
    lam_o, U_o = oracle.syev3(A[4:])
    parity.compare_f64(A[4:], lam[4:], U[4:], lam_o, U_o)


def test_closed_forms(syev3):
    import oracle_pins

    cases = oracle_pins.load_closed_forms()
    A = np.stack([c[1] for c in cases])
    lam, U = run_gpu(syev3, A)
    lam_o, U_o = oracle.syev3(A)
    parity.compare_f64(A, lam, U, lam_o, U_o)


def test_unaligned_buffers(syev3):
    """8-byte but not 16-byte aligned buffers take the plain-load path."""
    A, _ = inputs.mixed(777, seed=81)
    buf = torch.zeros(777 * 6 + 1, dtype=torch.float64, device="cuda")
    buf[1:] = torch.from_numpy(A.reshape(-1)).cuda()
    A_view = buf[1:].view(777, 6)
    lam_buf = torch.zeros(777 * 3 + 1, dtype=torch.float64, device="cuda")
    U_buf = torch.zeros(777 * 9 + 1, dtype=torch.float64, device="cuda")
    lam_v, U_v = lam_buf[1:].view(777, 3), U_buf[1:].view(777, 3, 3)
    syev3.syev3_batched(A_view, out=(lam_v, U_v))
    torch.cuda.synchronize()
    lam_o, U_o = oracle.syev3(A)
    parity.compare_f64(A, lam_v.cpu().numpy(), U_v.cpu().numpy(), lam_o, U_o)
    assert lam_buf[0].item() == 0.0 and U_buf[0].item() == 0.0


def test_rejects_bad_buffers(syev3):
    A = torch.zeros(16, 6, dtype=torch.float64, device="cuda")
    lam = torch.zeros(16, 3, dtype=torch.float64, device="cuda")
    lib = syev3.library()
    import ctypes

    host = np.zeros((16, 6))
    st = lib.syev3_batched(ctypes.c_void_p(host.ctypes.data), 16, ctypes.c_void_p(lam.data_ptr()), None, 0, None)
    assert st == syev3.SYEV3_EINVAL  # pageable host memory
    st = lib.syev3_batched(ctypes.c_void_p(A.data_ptr() + 4), 15, ctypes.c_void_p(lam.data_ptr()), None, 0, None)
    assert st == syev3.SYEV3_EINVAL  # 4-byte misaligned FP64


def test_full_size_mixed(syev3):
    """The 2^24 mixed FP64 batch in the benchmark's launch, every matrix
    against the oracle element by element (the oracle over all host cores,
    the comparison in chunks): the FP64 bar per subset, the exact diagonals
    bit for bit, no capped zero finder and no non-finite lane."""
    n = 1 << 24
    A, ids = inputs.mixed(n)
    At = torch.from_numpy(A).cuda()
    ctr = torch.zeros(syev3.NUM_COUNTERS, dtype=torch.int64, device="cuda")
    lam_t, U_t = syev3.syev3_batched(At, counters=ctr)
    torch.cuda.synchronize()
    assert ctr[0].item() == 0 and ctr[1].item() == 0
    lam, U = lam_t.cpu().numpy(), U_t.cpu().numpy()
    del At, lam_t, U_t
    torch.cuda.empty_cache()
    lam_o, U_o = parity.oracle_all_cores(A)

    def check(lo, hi):
        sl = slice(lo, hi)
        parity.compare_f64(A[sl], lam[sl], U[sl], lam_o[sl], U_o[sl])
        d = ids[sl] == inputs.SUBSET_DIAGONAL_REPEATED
        assert np.array_equal(lam[sl][d], lam_o[sl][d]) and np.array_equal(U[sl][d], U_o[sl][d])

    parity.chunked(check, n)
    assert syev3.device_flags() == 0


@pytest.mark.parametrize("log2_spike", [-30, -60, -200, -400, -470, -490])
def test_small_offdiagonal_scales(syev3, log2_spike):
    """Off-diagonal entries 2^k below the diagonal: FP32 seeds stop being
    usable (k <= -50), roots go to the compacted FP64 work list, and spikes
    below 2^-480 are zeroed (beta-deflation)."""
    A = inputs.gaussian(3000, seed=900 - log2_spike)
    A[:, 3:] *= 2.0 ** log2_spike
    lam, U = run_gpu(syev3, A)
    lam_o, U_o = oracle.syev3(A)
    parity.compare_f64(A, lam, U, lam_o, U_o)


@pytest.mark.parametrize("lo", [-120, -300])
def test_entrywise_random_scales(syev3, lo):
    """Every entry with its own scale 2^U(lo, 0): all branches, both
    zero-finder paths and direct steps to far smaller zeros, mixed in each
    warp."""
    rng = np.random.default_rng(901 - lo)
    A = rng.standard_normal((50000, 6)) * 2.0 ** rng.uniform(lo, 0, (50000, 6))
    lam, U = run_gpu(syev3, A)
    lam_o, U_o = oracle.syev3(A)
    parity.compare_f64(A, lam, U, lam_o, U_o)


def test_clustered_extremes(syev3):
    """Q diag(1, 1+10^-k, -1) Q^T for k up to 15: mu is below FP32
    resolution and is finished by the compacted FP64 iteration."""
    rng = np.random.default_rng(902)
    n = 20000
    k = rng.uniform(6.0, 15.0, n)
    d = np.stack([np.ones(n), 1.0 + 10.0 ** (-k), -np.ones(n)], axis=1)
    A = inputs.conj_diag(inputs.haar(rng, n), d)
    lam, U = run_gpu(syev3, A)
    lam_o, U_o = oracle.syev3(A)
    parity.compare_f64(A, lam, U, lam_o, U_o)


def test_near_combo_arrows(syev3):
    """alpha1 - alpha2 = 10^U(-12,-2) with O(1) spikes (not deflated when
    alpha1 + alpha2 is small): roots far above abar, where the spectral
    function must be evaluated in the paper's printed form."""
    rng = np.random.default_rng(903)
    n = 20000
    a1 = rng.uniform(-0.05, 0.05, n)
    ab = 10.0 ** rng.uniform(-12, -2, n)
    ang = rng.uniform(0.1, 1.4, n)
    A = np.stack([a1, a1 - ab, rng.standard_normal(n), np.zeros(n), np.cos(ang), np.sin(ang)], axis=1)
    lam, U = run_gpu(syev3, A)
    lam_o, U_o, info = oracle.syev3(A, with_info=True)
    assert (info[:, 0] == oracle.CLS_REDUCED).mean() > 0.5
    parity.compare_f64(A, lam, U, lam_o, U_o)


@pytest.mark.parametrize("dtype", ["f64", "f32", "f32c"])
def test_host_entry_point(syev3, dtype):
    """syev3_batched_host on pinned and pageable host buffers, several
    chunks and a ragged last chunk, equals the device entry point bit for bit."""
    n = 50_000
    if dtype == "f64":
        A = inputs.mixed(n, seed=901)[0]
    else:
        A = inputs.mixed_fp32(n, seed=902)[0]
    comp = dtype == "f32c"
    At = torch.from_numpy(A)
    lam_d, U_d = syev3.syev3_batched(At.cuda(), compensated=comp)
    torch.cuda.synchronize()
    for pinned in (True, False):
        Ah = At.pin_memory() if pinned else At.clone()
        lam = torch.empty((n, 3), dtype=At.dtype)
        U = torch.empty((n, 3, 3), dtype=At.dtype)
        if pinned:
            lam, U = lam.pin_memory(), U.pin_memory()
        syev3.syev3_batched_host(Ah, lam, U, compensated=comp, chunk=7_000)
        assert torch.equal(lam, lam_d.cpu()) and torch.equal(U, U_d.cpu())
    lam0 = torch.empty((n, 3), dtype=At.dtype)
    syev3.syev3_batched_host(At, lam0, None, compensated=comp)
    assert torch.equal(lam0, lam_d.cpu())


def test_host_entry_point_default_schedule(syev3):
    """The host entry point's default chunk schedule (2^16 matrices first,
    each next chunk a quarter longer, up to 2^20) over a batch that spans
    several chunks of different lengths and ends in a ragged one: equal to
    the device entry point bit for bit."""
    n = 65536 + 81920 + 102400 + 128000 + 12345
    A = inputs.mixed(n, seed=904)[0]
    At = torch.from_numpy(A)
    lam_d, U_d = syev3.syev3_batched(At.cuda())
    torch.cuda.synchronize()
    Ah = At.pin_memory()
    lam = torch.empty((n, 3), dtype=At.dtype).pin_memory()
    U = torch.empty((n, 3, 3), dtype=At.dtype).pin_memory()
    syev3.syev3_batched_host(Ah, lam, U)
    assert torch.equal(lam, lam_d.cpu()) and torch.equal(U, U_d.cpu())


def test_host_entry_point_full_size(syev3):
    """The end-to-end path at the benchmark's size: 2^24 mixed FP64 matrices
    from pinned host buffers through the default chunk schedule (25 chunks),
    equal bit for bit to the device entry point on the same matrices."""
    n = 1 << 24
    A = inputs.mixed(n)[0]
    Ah = torch.from_numpy(A).pin_memory()
    lam = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    U = torch.empty((n, 3, 3), dtype=torch.float64).pin_memory()
    syev3.syev3_batched_host(Ah, lam, U)
    Ad = Ah.cuda()
    lam_d, U_d = syev3.syev3_batched(Ad)
    torch.cuda.synchronize()
    assert torch.equal(lam, lam_d.cpu())
    assert torch.equal(U, U_d.cpu())


def test_extreme_magnitudes(syev3):
    """The pre-scale and unscale fallbacks (scalbn): largest entries at or
    above 2^1022, wholly subnormal matrices (outputs subnormal), and single
    subnormal entries among normal ones.  Scaling by 2^k commutes with the
    solve, so the first two are compared bit for bit with the scaled results
    of the same matrices at unit scale."""
    rng = np.random.default_rng(903)
    A = rng.standard_normal((4000, 6))
    A *= (0.5 + 0.15 * rng.random(4000))[:, None] / np.max(np.abs(A), axis=1, keepdims=True)  # max in [0.5, 0.65)
    lam1, U1 = run_gpu(syev3, A)
    # largest entry in [2^1022, 0.65 * 2^1023): eigenvalues (<= 3 max) stay finite
    lam, U = run_gpu(syev3, np.ldexp(A, 1023))
    assert np.all(np.isfinite(lam))
    assert np.array_equal(lam, np.ldexp(lam1, 1023)) and np.array_equal(U, U1)
    # wholly subnormal input: compare with the unit-scale solve of the same
    # (exactly representable) matrices, scaled once
    As = np.ldexp(A, -1040)
    Ab = np.ldexp(As, 1040)
    lam2, U2 = run_gpu(syev3, Ab)
    lam, U = run_gpu(syev3, As)
    assert np.array_equal(lam, np.ldexp(lam2, -1040)) and np.array_equal(U, U2)
    # one subnormal entry in an otherwise normal matrix
    B = inputs.gaussian(4000, seed=904)
    B[np.arange(4000), rng.integers(0, 6, 4000)] = np.ldexp(rng.standard_normal(4000), -1060)
    lam, U = run_gpu(syev3, B)
    lam_o, U_o = oracle.syev3(B)
    parity.compare_f64(B, lam, U, lam_o, U_o)
