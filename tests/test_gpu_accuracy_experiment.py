"""The test of Sec. 1.5 on the FP64 kernel: symmetric matrices with iid
entries from U(0,1), N(0,1) and chi^2_1; orthogonality ||I - V^T V||_F and
factorisation residual ||T V - V Lambda||_F against LAPACK's (numpy.linalg.eigh).
The paper reports its method more accurate than LAPACK's in both measures
on most matrices; here each measure must stay within the FP64 bar on every
matrix and be at least as small as LAPACK's on a clear majority."""

import numpy as np
import pytest

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


@pytest.mark.parametrize("dist", ["uniform", "normal", "chisq"])
def test_against_lapack(syev3, dist):
    n = 20000
    T6 = inputs.paper_set(n, dist, seed=inputs.SEED_BASE + 50)
    lam, U = syev3.syev3_batched(torch.from_numpy(T6).cuda())
    torch.cuda.synchronize()
    lam, U = lam.cpu().numpy(), U.cpu().numpy()
    M = inputs.unpack(T6)
    lam_l, U_l = np.linalg.eigh(M)
    nrm = np.linalg.norm(M, axis=(1, 2))

    def orth(V):
        return np.linalg.norm(np.einsum("nki,nkj->nij", V, V) - np.eye(3), axis=(1, 2))

    def resid(L, V):
        return np.linalg.norm(M @ V - V * L[:, None, :], axis=(1, 2))

    o, o_l = orth(U), orth(U_l)
    r, r_l = resid(lam, U), resid(lam_l, U_l)
    assert np.all(o <= 16 * parity.EPS64), o.max()
    assert np.all(r <= 1e-14 * nrm), (r / nrm).max()
    assert np.mean(o <= o_l) >= 0.6, np.mean(o <= o_l)
    assert np.mean(r <= r_l) >= 0.6, np.mean(r <= r_l)
    # eigenvalues agree with LAPACK's within the bar
    assert np.all(np.max(np.abs(lam - lam_l), axis=1) <= 8 * parity.EPS64 * nrm)
