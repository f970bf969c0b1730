"""Failure detection without a GPU fault: every device-side wait of the
kernels on a bulk copy is bounded; a wait that runs out sets a status bit
the host reads and the CTA exits, leaving the context usable.  The self-test
kernel makes one such wait run out (an mbarrier that nothing completes)."""

import time

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


def test_wait_limit_sets_timeout_bit_and_context_survives(syev3):
    lib = syev3.library()
    syev3.device_flags()  # read and clear whatever earlier work left
    assert syev3.device_flags() == 0
    t0 = time.perf_counter()
    assert lib.syev3_selftest_wait_limit(None) == syev3.SYEV3_OK
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    # the wait ran out on its 1 s limit: neither instantly nor unbounded
    assert 0.5 <= dt <= 30.0, dt
    assert syev3.device_flags() & 1
    assert syev3.device_flags() == 0  # reading cleared the bit
    # the context is still usable: a normal solve agrees with the oracle and
    # raises no flag
    A = inputs.gaussian(2048, seed=91)
    lam, U = syev3.syev3_batched(torch.from_numpy(A).cuda())
    torch.cuda.synchronize()
    lam_o, U_o = oracle.syev3(A)
    parity.compare_f64(A, lam.cpu().numpy(), U.cpu().numpy(), lam_o, U_o)
    assert syev3.device_flags() == 0
