"""FP32 parity of the CUDA path (plain and compensated) with the FP64 oracle.

The oracle solves the FP32 inputs exactly as given (upcast to FP64).  Bar:
|dlambda| <= 64 eps32 ||A||_F per eigenvalue (the precision form's stated
tolerance), residual ||AU - U Lambda||_F <= 64 eps32 ||A||_F and
orthogonality ||U^T U - I||_F <= 64 eps32 (evaluated in FP64 on the FP32
outputs), eigenvectors within 64 eps32 / relative gap up to sign where the
gap is >= 1e-2.
"""

import numpy as np
import pytest

import oracle
import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1806_06698_gb300 import inputs  # noqa: E402

# "workspace": the compensated form through syev3_batched_ws (its FP64
# refinement as a second kernel over a list in a caller-provided workspace).
MODES = ["plain", "compensated", "workspace"]


def solve(mod, A_t, mode, **kw):
    comp = mode in ("compensated", "workspace")
    ws = None
    if mode == "workspace":
        nb = mod.workspace_bytes(A_t.shape[0], A_t.dtype, compensated=True)
        ws = torch.empty(max(nb, 1), dtype=torch.uint8, device=A_t.device)
    return mod.syev3_batched(A_t, compensated=comp, workspace=ws, **kw)


@pytest.fixture(scope="module")
def syev3():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_06698_gb300 import build, syev3 as mod

    build.build()
    return mod


def run32(mod, A32, mode, counters=None, vectors=True):
    A = torch.from_numpy(np.ascontiguousarray(A32, dtype=np.float32)).cuda()
    lam, U = solve(mod, A, mode, vectors=vectors, counters=counters)
    torch.cuda.synchronize()
    return lam.cpu().numpy(), (U.cpu().numpy() if U is not None else None)


def vec_gap_filtered_compare(A32, lam, U, lam_o, U_o):
    """The FP32 bar (parity.compare_f32)."""
    parity.compare_f32(A32, lam, U, lam_o, U_o)


@pytest.mark.parametrize("mode", MODES)
def test_gaussian_4096(syev3, mode):
    A = inputs.gaussian(4096).astype(np.float32)
    lam, U = run32(syev3, A, mode)
    lam_o, U_o = oracle.syev3(A.astype(np.float64))
    vec_gap_filtered_compare(A, lam, U, lam_o, U_o)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n", [1, 3, 127, 128, 129, 255, 3 * 128 + 37, 20011])
def test_mixed_fp32_ragged(syev3, mode, n):
    A, _ = inputs.mixed_fp32(n, seed=2000 + n)
    lam, U = run32(syev3, A, mode)
    lam_o, U_o = oracle.syev3(A.astype(np.float64))
    vec_gap_filtered_compare(A, lam, U, lam_o, U_o)


@pytest.mark.parametrize("mode", MODES)
def test_mixed_fp32_subsets(syev3, mode):
    A, ids = inputs.mixed_fp32(1 << 16, seed=2077)
    ctr = torch.zeros(syev3.NUM_COUNTERS, dtype=torch.int64, device="cuda")
    lam, U = run32(syev3, A, mode, counters=ctr)
    lam_o, U_o = oracle.syev3(A.astype(np.float64))
    for s in inputs.SUBSET_NAMES:
        m = ids == s
        vec_gap_filtered_compare(A[m], lam[m], U[m], lam_o[m], U_o[m])
    c = ctr.cpu().numpy()
    assert c[0] == 0 and c[1] == 0 and c[3] == 0
    if mode != "plain":
        assert c[2] > 0  # the clustered subset is flagged for FP64 refinement
    else:
        assert c[2] == 0


@pytest.mark.parametrize("mode", MODES)
def test_structure_tensors(syev3, mode):
    A = inputs.structure_tensors(50000).astype(np.float32)
    lam, U = run32(syev3, A, mode)
    lam_o, U_o = oracle.syev3(A.astype(np.float64))
    vec_gap_filtered_compare(A, lam, U, lam_o, U_o)
    assert np.all(lam_o[:, 0] >= -64 * parity.EPS32 * parity.fro(A))  # PSD


@pytest.mark.parametrize("mode", MODES)
def test_special_inputs(syev3, mode):
    A = inputs.gaussian(300, seed=81).astype(np.float32)
    A[0] = 0.0
    A[1, 2] = np.nan
    A[2, 4] = np.inf
    A[3] = [3.0, -1.0, 3.0, 0.0, 0.0, 0.0]
    ctr = torch.zeros(syev3.NUM_COUNTERS, dtype=torch.int64, device="cuda")
    lam, U = run32(syev3, A, mode, counters=ctr)
    assert ctr[1].item() == 2
    assert np.array_equal(lam[0], np.zeros(3)) and np.array_equal(U[0], np.eye(3))
    assert np.all(np.isnan(lam[1:3])) and np.all(np.isnan(U[1:3]))
    assert np.array_equal(lam[3], np.array([-1.0, 3.0, 3.0], np.float32))
    lam_o, U_o = oracle.syev3(A[3:].astype(np.float64))
    vec_gap_filtered_compare(A[3:], lam[3:], U[3:], lam_o, U_o)


@pytest.mark.parametrize("mode", MODES)
def test_unaligned_and_eigenvalues_only(syev3, mode):
    A, _ = inputs.mixed_fp32(999, seed=2099)
    buf = torch.zeros(999 * 6 + 1, dtype=torch.float32, device="cuda")
    buf[1:] = torch.from_numpy(A.reshape(-1)).cuda()
    lam_b = torch.zeros(999 * 3 + 1, dtype=torch.float32, device="cuda")
    U_b = torch.zeros(999 * 9 + 1, dtype=torch.float32, device="cuda")
    lam_v, U_v = lam_b[1:].view(999, 3), U_b[1:].view(999, 3, 3)
    solve(syev3, buf[1:].view(999, 6), mode, out=(lam_v, U_v))
    torch.cuda.synchronize()
    lam_o, U_o = oracle.syev3(A.astype(np.float64))
    vec_gap_filtered_compare(A, lam_v.cpu().numpy(), U_v.cpu().numpy(), lam_o, U_o)
    lam_n, U_n = run32(syev3, A, mode, vectors=False)
    assert U_n is None
    assert np.array_equal(lam_n, lam_v.cpu().numpy())


@pytest.fixture(scope="module")
def full_size_sets():
    """The 2^24 mixed FP32 batch and the 2^26 structure tensors with the
    oracle's results on them (upcast exactly to FP64), over all host cores."""
    sets = []
    for name, A in (("mixed_fp32_2^24", inputs.mixed_fp32(1 << 24)[0]),
                    ("structure_tensors_2^26", inputs.structure_tensors(1 << 26).astype(np.float32))):
        lam_o, U_o = parity.oracle_all_cores(A.astype(np.float64))
        sets.append((name, A, lam_o, U_o))
    return sets


@pytest.mark.parametrize("mode", MODES)
def test_full_size_fp32(syev3, mode, full_size_sets):
    """The 2^24 mixed FP32 batch and 2^26 structure tensors in the
    benchmark's launch, every matrix against the oracle element by element
    (the FP32 bar), in chunks on a thread pool; no capped zero finder, no
    non-finite lane, no refined lane failing its residual check."""
    for name, A, lam_o, U_o in full_size_sets:
        n = A.shape[0]
        At = torch.from_numpy(A).cuda()
        ctr = torch.zeros(syev3.NUM_COUNTERS, dtype=torch.int64, device="cuda")
        lam_t, U_t = solve(syev3, At, mode, counters=ctr)
        torch.cuda.synchronize()
        c = ctr.cpu().numpy()
        assert c[0] == 0 and c[1] == 0 and c[3] == 0, (name, c)
        lam, U = lam_t.cpu().numpy(), U_t.cpu().numpy()
        del At, lam_t, U_t
        torch.cuda.empty_cache()

        def check(lo, hi):
            sl = slice(lo, hi)
            vec_gap_filtered_compare(A[sl], lam[sl], U[sl], lam_o[sl], U_o[sl])

        parity.chunked(check, n)


def test_precision_report(syev3, capsys):
    """Per-subset error of the FP32 forms (and of the FP64 solver on the same
    upcast inputs) against the FP64 oracle, in units of eps32 ||A||_F."""
    A_mixed, ids = inputs.mixed_fp32(1 << 17, seed=2100)
    A_st = inputs.structure_tensors(1 << 16, seed=2101).astype(np.float32)
    groups = [(inputs.SUBSET_NAMES[s], A_mixed[ids == s]) for s in inputs.SUBSET_NAMES]
    groups.append(("structure_tensors", A_st))
    lines = ["subset | form | max |dlam|/(eps32 ||A||) | max residual/(eps32 ||A||) | max ||U^T U - I||/eps32"]
    for name, A in groups:
        A64 = A.astype(np.float64)
        lam_o, U_o = oracle.syev3(A64)
        nrm = parity.fro(A64)
        nz = np.where(nrm > 0, nrm, 1.0)
        for form in ("plain", "compensated", "fp64"):
            if form == "fp64":
                At = torch.from_numpy(A64).cuda()
                lam_t, U_t = syev3.syev3_batched(At)
                torch.cuda.synchronize()
                lam, U = lam_t.cpu().numpy(), U_t.cpu().numpy()
            else:
                lam, U = run32(syev3, A, form)
            dl = np.max(np.abs(lam.astype(np.float64) - lam_o), axis=1) / nz / parity.EPS32
            res = parity.residual(A64, lam, U) / nz / parity.EPS32
            orth = parity.orthogonality(U) / parity.EPS32
            lines.append(f"{name} | {form} | {dl.max():.3f} | {res.max():.3f} | {orth.max():.3f}")
            assert dl.max() <= 64 and res.max() <= 64 and orth.max() <= 64
    with capsys.disabled():
        print("\n" + "\n".join(lines))


def test_workspace_path_matches_single_kernel(syev3):
    """syev3_batched_ws (refinement as a second kernel) against syev3_batched
    (refinement inside the kernel) on the same inputs, twice in a row on one
    workspace (the list's counter is cleared by each call): the same
    refinement code, so equal up to the compiler's contraction choices, and
    the same counters; the workspace checks of the C ABI on real buffers."""
    A, _ = inputs.mixed_fp32(1 << 15, seed=2111)
    At = torch.from_numpy(A).cuda()
    c1 = torch.zeros(syev3.NUM_COUNTERS, dtype=torch.int64, device="cuda")
    lam1, U1 = syev3.syev3_batched(At, compensated=True, counters=c1)
    nb = syev3.workspace_bytes(At.shape[0], At.dtype, compensated=True)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    for _ in range(2):
        c2 = torch.zeros(syev3.NUM_COUNTERS, dtype=torch.int64, device="cuda")
        lam2, U2 = syev3.syev3_batched(At, compensated=True, counters=c2, workspace=ws)
        torch.cuda.synchronize()
        assert torch.equal(c1, c2)
        assert float((lam1 - lam2).abs().max()) <= 4 * parity.EPS32 * float(lam1.abs().max())
        lam_o, U_o = oracle.syev3(A.astype(np.float64))
        vec_gap_filtered_compare(A, lam2.cpu().numpy(), U2.cpu().numpy(), lam_o, U_o)
    lib = syev3.library()
    lam3 = torch.empty((At.shape[0], 3), dtype=torch.float32, device="cuda")
    args = (At.data_ptr(), At.shape[0], lam3.data_ptr(), None, syev3.SYEV3_F32_COMPENSATED, None)
    assert lib.syev3_batched_ws(*args, ws.data_ptr(), nb - 1, None) == syev3.SYEV3_EINVAL
    assert lib.syev3_batched_ws(*args, ws.data_ptr() + 16, nb - 256, None) == syev3.SYEV3_EINVAL
    assert lib.syev3_batched_ws(*args, At.data_ptr(), nb, None) == syev3.SYEV3_EINVAL
    assert lib.syev3_batched_ws(*args, ws.data_ptr(), nb, None) == syev3.SYEV3_OK
    torch.cuda.synchronize()


@pytest.mark.parametrize("n", [1, 31, 33, 129, 5_000, 40_001])
@pytest.mark.parametrize("vectors", [True, False])
def test_inline_refinement_carry(syev3, n, vectors):
    """The compensated kernel refines its flagged lanes in whole warps,
    carrying the rest from tile to tile and refining the last group after
    the CTA's final tile.  On batches of the clustered subset only (most
    lanes flagged: carries every tile), at sizes below one warp, across a
    tile boundary and with ragged ends, and with eigenvalues only (a
    carried lane then writes no vector): the same counters and results as
    the workspace path (the refinement as a second kernel), and the FP32
    bar against the oracle."""
    A, ids = inputs.mixed_fp32(6 * n + 200, seed=2112)  # 20 % clustered
    A = np.ascontiguousarray(A[ids == 1][:n])
    assert A.shape[0] == n
    At = torch.from_numpy(A).cuda()
    c1 = torch.zeros(syev3.NUM_COUNTERS, dtype=torch.int64, device="cuda")
    lam1, U1 = syev3.syev3_batched(At, compensated=True, counters=c1, vectors=vectors)
    nb = syev3.workspace_bytes(n, At.dtype, compensated=True)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    c2 = torch.zeros(syev3.NUM_COUNTERS, dtype=torch.int64, device="cuda")
    lam2, U2 = syev3.syev3_batched(At, compensated=True, counters=c2, workspace=ws, vectors=vectors)
    torch.cuda.synchronize()
    assert torch.equal(c1, c2)
    if n >= 129:
        assert int(c1[2]) > n // 4  # many lanes refined in FP64
    scale = float(lam1.abs().max())
    assert float((lam1 - lam2).abs().max()) <= 4 * parity.EPS32 * scale
    lam_o, U_o = oracle.syev3(A.astype(np.float64))
    if vectors:
        # Vectors of (numerically) repeated eigenvalues are not unique: each
        # path against the oracle, with the gap filter.
        vec_gap_filtered_compare(A, lam1.cpu().numpy(), U1.cpu().numpy(), lam_o, U_o)
        vec_gap_filtered_compare(A, lam2.cpu().numpy(), U2.cpu().numpy(), lam_o, U_o)
    else:
        assert U1 is None and U2 is None
        parity.compare(A.astype(np.float64), lam1.cpu().numpy(), None, lam_o, None, eps=parity.EPS32,
                       lam_tol=64, res_tol=0, orth_tol=0, vec_tol=0)


def test_batch_beyond_32_bit_element_indices(syev3):
    """n = 2^29 FP32 matrices (eigenvector elements up to 4.8e9 > 2^32): the
    kernels' 64-bit index arithmetic.  Inputs are generated on the device;
    every output is checked for ordering, orthogonality and the trace, and
    sampled matrices at the far end against the oracle."""
    n = 1 << 29
    free, _ = torch.cuda.mem_get_info()
    if free < 48 << 30:
        pytest.skip("needs about 48 GB of free device memory")
    g = torch.Generator(device="cuda").manual_seed(5)
    A = torch.randn((n, 6), device="cuda", dtype=torch.float32, generator=g)
    lam, U = syev3.syev3_batched(A)
    torch.cuda.synchronize()
    step = 1 << 25
    for b in range(0, n, step):
        l, u, a = lam[b:b + step], U[b:b + step], A[b:b + step]
        assert bool(torch.all(l[:, 1:] >= l[:, :-1]))
        orth = torch.linalg.matrix_norm(u.transpose(1, 2) @ u - torch.eye(3, device="cuda"))
        assert float(orth.max()) <= 64 * parity.EPS32
        tr = a[:, 0].double() + a[:, 1].double() + a[:, 2].double()
        nrm = torch.linalg.vector_norm(a.double(), dim=1)
        assert float(((l.double().sum(dim=1) - tr).abs() / nrm).max()) <= 64 * parity.EPS32
    idx = torch.arange(n - 4096, n, device="cuda")
    As = A[idx].cpu().numpy()
    lam_o, U_o = oracle.syev3(As.astype(np.float64))
    vec_gap_filtered_compare(As, lam[idx].cpu().numpy(), U[idx].cpu().numpy(), lam_o, U_o)
    del A, lam, U
    torch.cuda.empty_cache()


@pytest.mark.parametrize("offset", [0, 1])
def test_workspace_pipeline_ragged(syev3, offset):
    """From 2^21 matrices on, syev3_batched_ws pipelines the FP32 solve and
    the FP64 refinement over 8 runs on two streams.  A ragged batch (the
    last run partial) with the input 16-byte aligned or not: the same
    counters as the single-kernel compensated path, eigenvalues within
    4 eps32 of it, and the FP32 bar against the oracle on every matrix."""
    n = (1 << 21) + 3 * 128 + 77
    A, _ = inputs.mixed_fp32(n + offset, seed=2120)
    buf = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    At = buf[offset:]  # offset 1: 24 bytes from the allocation, not 16-byte aligned
    A = A[offset:]
    c1 = torch.zeros(syev3.NUM_COUNTERS, dtype=torch.int64, device="cuda")
    lam1, U1 = syev3.syev3_batched(At, compensated=True, counters=c1)
    nb = syev3.workspace_bytes(n, At.dtype, compensated=True)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    for _ in range(2):
        c2 = torch.zeros(syev3.NUM_COUNTERS, dtype=torch.int64, device="cuda")
        lam2, U2 = syev3.syev3_batched(At, compensated=True, counters=c2, workspace=ws)
        torch.cuda.synchronize()
        assert torch.equal(c1, c2), (c1, c2)
        assert int(c2[2]) > 0
        nrm = torch.from_numpy(parity.fro(A.astype(np.float64))).cuda()
        dl = ((lam2.double() - lam1.double()).abs().amax(dim=1) / nrm.clamp_min(1e-300)).max().item()
        assert dl <= 4 * parity.EPS32, dl
    lam_o, U_o = parity.oracle_all_cores(A.astype(np.float64))
    lam_h, U_h = lam2.cpu().numpy(), U2.cpu().numpy()

    def check(lo, hi):
        sl = slice(lo, hi)
        parity.compare_f32(A[sl], lam_h[sl], U_h[sl], lam_o[sl], U_o[sl])

    parity.chunked(check, n)
