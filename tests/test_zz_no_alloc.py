"""syev3_batched_static_ws: the compensated FP32 solve whose refinement
list lives in the library's static device memory, so the call allocates
nothing.  Collected last (file name), it must also pass alone: nothing here
depends on what earlier tests did.  Compared with the existing entry point
syev3_batched (compensated) within the FP32 test tolerance, on two calls in a
row, and with the CPU oracle (the FP32 bar)."""

import ctypes

import numpy as np
import pytest

import parity

torch = pytest.importorskip("torch")

from paper_1806_06698_gb300 import inputs  # noqa: E402


def test_header_limit_matches_binding():
    import re
    import os

    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "syev3.h")).read()
    from paper_1806_06698_gb300 import syev3

    m = re.search(r"#define SYEV3_STATIC_MAX_N (\d+)", hdr)
    assert m and int(m.group(1)) == syev3.STATIC_MAX_N


def test_sizes_beyond_the_static_array_are_rejected():
    """n above the array's capacity (or negative) is refused before any CUDA
    call; n == 0 is a no-op (runs without a GPU)."""
    from paper_1806_06698_gb300 import build, syev3

    build.build()
    lib = syev3.library()
    vp = ctypes.c_void_p
    big = syev3.STATIC_MAX_N + 1
    assert lib.syev3_batched_static_ws(vp(1 << 20), big, vp(1 << 30), None, None, None) == syev3.SYEV3_EINVAL
    assert lib.syev3_batched_static_ws(vp(1 << 20), -1, vp(1 << 30), None, None, None) == syev3.SYEV3_EINVAL
    assert lib.syev3_batched_static_ws(None, 0, None, None, None, None) == syev3.SYEV3_OK


@pytest.mark.gpu
@pytest.mark.parametrize("n", [4097, 262144])
def test_matches_existing_entry_point_twice(n):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_06698_gb300 import build, syev3

    build.build()
    A, _ = inputs.mixed_fp32(n, seed=3000 + n)
    At = torch.from_numpy(A).cuda()
    c_ref = torch.zeros(syev3.NUM_COUNTERS, dtype=torch.int64, device="cuda")
    lam_ref, U_ref = syev3.syev3_batched(At, compensated=True, counters=c_ref)
    nrm = torch.from_numpy(parity.fro(A.astype(np.float64))).cuda()
    lam_o, U_o = parity.oracle_all_cores(A.astype(np.float64))
    for _ in range(2):  # the list's counter is cleared by each call
        c = torch.zeros(syev3.NUM_COUNTERS, dtype=torch.int64, device="cuda")
        lam, U = syev3.syev3_batched_static_ws(At, counters=c)
        torch.cuda.synchronize()
        assert torch.equal(c, c_ref)
        dl = ((lam.double() - lam_ref.double()).abs().amax(dim=1) / nrm.clamp_min(1e-300)).max().item()
        assert dl <= 4 * parity.EPS32, dl
        orth = torch.linalg.matrix_norm(U.double().transpose(1, 2) @ U.double()
                                        - torch.eye(3, dtype=torch.float64, device="cuda")).max().item()
        assert orth <= 64 * parity.EPS32, orth
        # eigenvectors agree with the existing entry point's up to sign where
        # the relative gap leaves them determined
        gap = (lam_ref[:, 1:] - lam_ref[:, :-1]).min(dim=1).values.double() / nrm.clamp_min(1e-300)
        sel = gap >= 1e-2
        d = torch.minimum((U - U_ref).abs().amax(dim=1), (U + U_ref).abs().amax(dim=1)).amax(dim=1)
        assert float((d[sel].double() * gap[sel]).max()) <= 64 * parity.EPS32
        parity.compare_f32(A, lam.cpu().numpy(), U.cpu().numpy(), lam_o, U_o)
