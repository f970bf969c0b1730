"""Backward kernel (differentiation form) against the oracle's analytic
gradient on the same inputs, against central finite differences of the GPU
forward pass (h = 1e-6, FP64), and through torch.autograd."""

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


def forward(mod, A, dtype=torch.float64):
    At = torch.from_numpy(np.ascontiguousarray(A)).to("cuda", dtype)
    lam, U = mod.syev3_batched(At)
    return At, lam, U


def rel_err(g, ref):
    scale = 1.0 + np.abs(ref).max(axis=1, keepdims=True)
    return np.abs(g - ref) / scale


@pytest.mark.parametrize("with_gU", [True, False])
def test_bwd_matches_oracle_fp64(syev3, with_gU):
    """Same (lambda, U, g_lambda, g_U) into the kernel and the oracle: the
    formulas agree to rounding (gaps >= 1e-3 ||A|| amplify by <= 1e3);
    near-degenerate pairs (5 %) are masked on both sides."""
    A, d, deg = inputs.spectral(1 << 14, seed=3000, near_degenerate=0.05)
    _, lam, U = forward(syev3, A)
    rng = np.random.default_rng(3001)
    w = torch.from_numpy(rng.standard_normal((A.shape[0], 3))).cuda()
    V = torch.from_numpy(rng.standard_normal((A.shape[0], 3, 3))).cuda() if with_gU else None
    g = syev3.syev3_batched_bwd(lam, U, w, V, 1e-6)
    torch.cuda.synchronize()
    lam_c, U_c = lam.cpu().numpy(), U.cpu().numpy()
    V_c = V.cpu().numpy() if with_gU else np.zeros_like(U_c)
    ref = oracle.syev3_bwd(lam_c, U_c, w.cpu().numpy(), V_c, 1e-6)
    assert rel_err(g.cpu().numpy(), ref).max() <= 1e-11


def test_bwd_matches_oracle_fp32(syev3):
    A, d, deg = inputs.spectral(1 << 14, seed=3002, near_degenerate=0.0, min_gap=0.05)
    A32 = A.astype(np.float32)
    _, lam, U = forward(syev3, A32, torch.float32)
    rng = np.random.default_rng(3003)
    w = torch.from_numpy(rng.standard_normal((A.shape[0], 3)).astype(np.float32)).cuda()
    V = torch.from_numpy(rng.standard_normal((A.shape[0], 3, 3)).astype(np.float32)).cuda()
    g = syev3.syev3_batched_bwd(lam, U, w, V, 1e-6)
    torch.cuda.synchronize()
    ref = oracle.syev3_bwd(lam.cpu().numpy().astype(np.float64), U.cpu().numpy().astype(np.float64),
                           w.cpu().numpy().astype(np.float64), V.cpu().numpy().astype(np.float64), 1e-6)
    # gaps >= 0.05 ||d||: rounding amplified by at most ~20 / 0.05
    assert rel_err(g.cpu().numpy().astype(np.float64), ref).max() <= 64 * 400 * parity.EPS32


def test_bwd_finite_differences(syev3):
    """Central differences of L = sum w lambda + sum V o U through the GPU
    forward pass agree with the GPU backward pass."""
    A, d, _ = inputs.spectral(4000, seed=3004, near_degenerate=0.0, min_gap=0.05)
    _, lam, U = forward(syev3, A)
    Uc = U.cpu().numpy()
    srt = np.sort(np.abs(Uc), axis=1)
    keep = np.all(srt[:, 2, :] - srt[:, 1, :] > 1e-3, axis=1)  # sign rule stable under +-h
    A = np.ascontiguousarray(A[keep][:1000])
    n = A.shape[0]
    At, lam, U = forward(syev3, A)
    rng = np.random.default_rng(3005)
    w = torch.from_numpy(rng.standard_normal((n, 3))).cuda()
    V = torch.from_numpy(rng.standard_normal((n, 3, 3))).cuda()
    g = syev3.syev3_batched_bwd(lam, U, w, V, 1e-6).cpu().numpy()

    def loss(Ah):
        l, u = syev3.syev3_batched(Ah)
        return ((w * l).sum(1) + (V * u).sum((1, 2))).cpu().numpy()

    h = 1e-6
    fd = np.empty((n, 6))
    for k in range(6):
        Ap, Am = At.clone(), At.clone()
        Ap[:, k] += h
        Am[:, k] -= h
        fd[:, k] = (loss(Ap) - loss(Am)) / (2 * h)
    assert rel_err(g, fd).max() <= 2e-6


def test_autograd_function(syev3):
    A, d, _ = inputs.spectral(2048, seed=3006, near_degenerate=0.05)
    At = torch.from_numpy(A).cuda().requires_grad_(True)
    rng = np.random.default_rng(3007)
    w = torch.from_numpy(rng.standard_normal((A.shape[0], 3))).cuda()
    V = torch.from_numpy(rng.standard_normal((A.shape[0], 3, 3))).cuda()
    lam, U = syev3.eigh3(At, gap_tau=1e-6)
    loss = (w * lam).sum() + (V * U).sum()
    loss.backward()
    ref = oracle.syev3_bwd(lam.detach().cpu().numpy(), U.detach().cpu().numpy(), w.cpu().numpy(),
                           V.cpu().numpy(), 1e-6)
    assert rel_err(At.grad.cpu().numpy(), ref).max() <= 1e-11
    # eigenvalue-only loss: g_U is None on the C side
    At.grad = None
    lam, U = syev3.eigh3(At)
    (w * lam).sum().backward()
    ref0 = oracle.syev3_bwd(lam.detach().cpu().numpy(), U.detach().cpu().numpy(), w.cpu().numpy(),
                            np.zeros((A.shape[0], 3, 3)), 1e-6)
    assert rel_err(At.grad.cpu().numpy(), ref0).max() <= 1e-13


def test_bwd_ragged_and_unaligned(syev3):
    for n in (1, 63, 64, 65, 129, 1001):
        A, d, _ = inputs.spectral(n, seed=3100 + n, near_degenerate=0.05)
        _, lam, U = forward(syev3, A)
        rng = np.random.default_rng(n)
        w = torch.from_numpy(rng.standard_normal((n, 3))).cuda()
        V = torch.from_numpy(rng.standard_normal((n, 3, 3))).cuda()
        # unaligned copies (8-byte offset) take the plain-load path
        def shift(t):
            b = torch.zeros(t.numel() + 1, dtype=t.dtype, device=t.device)
            b[1:] = t.reshape(-1)
            return b[1:].view(t.shape)
        for conv in (lambda t: t, shift):
            g = syev3.syev3_batched_bwd(conv(lam), conv(U), conv(w), conv(V), 1e-6,
                                        out=conv(torch.zeros((n, 6), dtype=torch.float64, device="cuda")))
            ref = oracle.syev3_bwd(lam.cpu().numpy(), U.cpu().numpy(), w.cpu().numpy(), V.cpu().numpy(), 1e-6)
            assert rel_err(g.cpu().numpy(), ref).max() <= 1e-11, n


def test_bwd_rejects_bad_args(syev3):
    import ctypes

    lib = syev3.library()
    x = torch.zeros(64, 9, dtype=torch.float64, device="cuda")
    p = lambda t, off=0: ctypes.c_void_p(t.data_ptr() + off)  # noqa: E731
    # output overlapping an input
    assert lib.syev3_batched_bwd(p(x), p(x), p(x), None, 4, p(x, 8), 1e-6, 0, None) == syev3.SYEV3_EINVAL
    # negative gap threshold
    y = torch.zeros(64, 6, dtype=torch.float64, device="cuda")
    assert lib.syev3_batched_bwd(p(x), p(x), p(x), None, 4, p(y), -1.0, 0, None) == syev3.SYEV3_EINVAL
    assert lib.syev3_batched_bwd(None, 0, None, None, 0, None, 0.0, 0, None) == syev3.SYEV3_OK


def fp32_bwd_error(g, ref, lam, gl, gU, tau):
    """Per matrix, |g - ref| in units of eps32 times the scale the FP32
    arithmetic of the backward kernel works at: S = max|gl| + max|gU| /
    (smallest unmasked gap).  The kernel forms M_ij - M_ji with 6 FMAs, the
    coupling (M_ij - M_ji) / (2 gap) with one rounded difference and one
    IEEE division, then two 3-term products with U (|U_ij| <= 1); adding up
    these roundings bounds the error by about 200 eps32 S.  Pairs whose gap
    lies within a factor 2 of the mask threshold tau ||lambda|| are
    ambiguous (FP32 and FP64 may decide the mask differently) and returned
    separately."""
    lam = lam.astype(np.float64)
    nl = np.linalg.norm(lam, axis=1)
    gaps = np.stack([lam[:, 1] - lam[:, 0], lam[:, 2] - lam[:, 0], lam[:, 2] - lam[:, 1]], axis=1)
    thr = tau * nl[:, None]
    masked = gaps < thr
    ambiguous = np.any((gaps > 0.5 * thr) & (gaps < 2.0 * thr), axis=1)
    gmin = np.min(np.where(masked, np.inf, gaps), axis=1)
    scale = np.abs(gl).max(axis=1) + np.abs(gU).reshape(len(gU), -1).max(axis=1) / gmin
    err = np.abs(g - ref).max(axis=1) / scale / parity.EPS32
    return err, ambiguous


def test_bwd_full_size(syev3):
    """2^20 matrices (95 % gaps >= 1e-3, 5 % near-degenerate, masked) in
    FP64 and FP32, in the benchmark's launch, every gradient against the
    oracle's analytic gradient on the same (lambda, U, g_lambda, g_U):
    FP64 to 1e-11 relative, FP32 within 256 eps32 of the scale its
    arithmetic works at (fp32_bwd_error)."""
    A, d, deg = inputs.spectral(1 << 20, seed=3008)
    n = A.shape[0]
    rng = np.random.default_rng(3009)
    wn = rng.standard_normal((n, 3))
    Vn = rng.standard_normal((n, 3, 3))
    for dt in (torch.float64, torch.float32):
        _, lam, U = forward(syev3, A.astype(np.float64 if dt == torch.float64 else np.float32), dt)
        w = torch.from_numpy(wn).to("cuda", dt)
        V = torch.from_numpy(Vn).to("cuda", dt)
        g = syev3.syev3_batched_bwd(lam, U, w, V, 1e-6)
        torch.cuda.synchronize()
        lam_c, U_c, w_c, V_c = (t.cpu().numpy() for t in (lam, U, w, V))
        g_c = g.cpu().numpy().astype(np.float64)
        ref = oracle.syev3_bwd(lam_c.astype(np.float64), U_c.astype(np.float64), w_c.astype(np.float64),
                               V_c.astype(np.float64), 1e-6)
        if dt == torch.float64:
            assert rel_err(g_c, ref).max() <= 1e-11
        else:
            err, amb = fp32_bwd_error(g_c, ref, lam_c, w_c.astype(np.float64), V_c.astype(np.float64), 1e-6)
            assert amb.mean() < 1e-3, amb.sum()
            assert err[~amb].max() <= 256, float(err[~amb].max())
