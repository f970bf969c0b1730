"""Serving form: the continuous-batching server returns, for every request,
the same result as a standalone call on the same matrices (bit for bit),
never exceeds its memory budget, admits requests as memory frees up, and
lets requests that arrive while a large one runs finish before it."""

import threading
import time

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


@pytest.fixture(scope="module")
def pools():
    A64 = torch.from_numpy(inputs.mixed(1 << 20, seed=4000)[0]).cuda()
    A32 = torch.from_numpy(inputs.mixed_fp32(1 << 20, seed=4001)[0]).cuda()
    return A64, A32


@pytest.fixture(scope="module")
def pool_oracle(pools):
    """The oracle's (lambda, U) of every matrix of both pools (the FP32 pool
    upcast exactly to FP64)."""
    A64, A32 = pools
    return (parity.oracle_all_cores(A64.cpu().numpy()),
            parity.oracle_all_cores(A32.cpu().numpy().astype(np.float64)))


def check_against_oracle(A, lam, U, ref):
    """A served result against the oracle: the FP64 bar for FP64 requests,
    the FP32 bar (64 eps32) for FP32 ones."""
    A_np = A.cpu().numpy()
    lam_o, U_o = ref
    if A.dtype == torch.float64:
        parity.compare_f64(A_np, lam.cpu().numpy(), U.cpu().numpy(), lam_o, U_o)
    else:
        parity.compare_f32(A_np, lam.cpu().numpy(), U.cpu().numpy(), lam_o, U_o)


def released_stats(srv, timeout_s=10.0):
    """Server statistics once the device has processed the releases made so
    far (it frees released results in its next round)."""
    t0 = time.time()
    st = srv.stats()
    while st.arena_used != 0 and time.time() - t0 < timeout_s:
        time.sleep(0.001)
        st = srv.stats()
    return st


def standalone(syev3, A, comp):
    lam, U = syev3.syev3_batched(A, compensated=comp)
    torch.cuda.synchronize()
    return lam, U


def test_same_alone_and_in_the_mix(syev3, pools, pool_oracle):
    """Requests of uneven sizes and mixed dtypes, submitted from a client
    thread while earlier ones run, through a small budget that makes some
    wait for memory and small chunks that interleave them: every result
    equals a standalone call bit for bit and matches the oracle."""
    A64, A32 = pools
    rng = np.random.default_rng(4002)
    budget = 48 << 20
    srv = syev3.Server(memory_budget_bytes=budget, chunk=1 << 12, round_matrices=1 << 15, max_rounds_in_flight=2)
    reqs = []
    for i in range(160):
        n = int(np.exp(rng.uniform(0, np.log(1 << 17))))
        kind = rng.choice(["f64", "f32", "f32c"], p=[0.6, 0.2, 0.2])
        pool = A64 if kind == "f64" else A32
        off = int(rng.integers(0, pool.shape[0] - n))
        reqs.append((pool[off:off + n], kind == "f32c", kind == "f64", off))
    tickets = [None] * len(reqs)

    def client():
        for i, (A, comp, _, _) in enumerate(reqs):
            tickets[i] = srv.submit(A, compensated=comp)
            if i % 7 == 0:
                time.sleep(0.0005)

    th = threading.Thread(target=client)
    th.start()
    th.join()
    waited = 0
    for i, (A, comp, is64, off) in enumerate(reqs):
        info = srv.wait(tickets[i], 60.0)
        assert info.state == 2 and info.n == A.shape[0]
        waited += info.t_admit_ns > info.t_submit_ns + 200_000
        lam, U = srv.results(tickets[i])
        lam_s, U_s = standalone(syev3, A, comp)
        assert torch.equal(lam, lam_s) and torch.equal(U, U_s), i
        lam_o, U_o = pool_oracle[0 if is64 else 1]
        sl = slice(off, off + A.shape[0])
        check_against_oracle(A, lam, U, (lam_o[sl], U_o[sl]))
        srv.release(tickets[i])
    st = released_stats(srv)
    assert st.completed == len(reqs) and st.waiting == 0 and st.error == 0
    assert st.arena_peak <= budget and st.arena_used == 0
    assert st.chunks > len(reqs)  # large requests were cut into chunks
    srv.close()


def test_small_requests_overtake_a_large_one(syev3, pools):
    """Continuous batching: requests that arrive while a large request is on
    the device are admitted and finish before it does."""
    A64, _ = pools
    # 2^23 matrices in 512 chunks: about 3.4 ms of solving, long against the
    # time the host takes to submit the small requests below.
    A_big = A64.repeat(8, 1)
    srv = syev3.Server(memory_budget_bytes=2 << 30, chunk=1 << 14, round_matrices=1 << 16, max_rounds_in_flight=1)
    big = srv.submit(A_big)
    while srv.query(big).state == 0:
        time.sleep(0.0001)
    small = [srv.submit(A64[i * 97:(i * 97) + 64]) for i in range(16)]
    assert srv.query(big).state == 1  # the small requests arrived while it ran
    done_small = [srv.wait(t, 60.0).t_done_ns for t in small]
    done_big = srv.wait(big, 60.0).t_done_ns
    assert max(done_small) < done_big
    for t in small + [big]:
        srv.release(t)
    srv.close()


def test_budget_is_enforced(syev3, pools):
    A64, _ = pools
    srv = syev3.Server(memory_budget_bytes=1 << 20, chunk=1 << 10)
    with pytest.raises(syev3.Syev3Error):
        srv.submit(A64[:20000])  # 20000 x 96 B > 1 MiB: can never be admitted
    ts = [srv.submit(A64[k * 5000:(k + 1) * 5000]) for k in range(12)]  # each ~0.46 MiB: two at a time
    for t in ts:
        assert srv.wait(t, 60.0).state == 2
        srv.release(t)
    st = released_stats(srv)
    assert st.arena_peak <= (1 << 20) and st.completed == 12 and st.arena_used == 0
    srv.close()


def test_failure_is_reported_and_frees_nothing(syev3, pools):
    """A launch failure made on the host (no device fault): requests not yet
    done fail with the error, waiters wake, later submits are refused, a
    release frees nothing on the device, and the server still shuts down."""
    A64, _ = pools
    srv = syev3.Server(memory_budget_bytes=1 << 30, chunk=1 << 10, round_matrices=1 << 12, max_rounds_in_flight=1)
    done = srv.submit(A64[:1000])
    assert srv.wait(done, 60.0).state == 2
    big = srv.submit(A64[: 1 << 20])  # 1024 rounds of 2^10: still running below
    while srv.query(big).state == 0:
        time.sleep(0.0001)
    srv.inject_failure(syev3.SYEV3_ECUDA)
    with pytest.raises(syev3.Syev3Error) as e:
        srv.wait(big, 60.0)
    assert e.value.status == syev3.SYEV3_ECUDA
    assert srv.query(big).state == 3
    used = srv.stats().arena_used
    assert used > 0
    srv.release(big)
    srv.release(done)
    time.sleep(0.05)
    assert srv.stats().arena_used == used and srv.stats().error == syev3.SYEV3_ECUDA
    with pytest.raises(syev3.Syev3Error):
        srv.submit(A64[:10])
    srv.close()


def test_ring_full_is_refused(syev3, pools):
    """More outstanding (unreleased) requests than the ring's slots: submit
    returns SYEV3_EAGAIN, and succeeds again once one is released."""
    A64, _ = pools
    srv = syev3.Server(memory_budget_bytes=1 << 30)
    ts = [srv.submit(A64[i:i + 1]) for i in range(syev3.SERVER_SLOTS)]
    with pytest.raises(syev3.Syev3Error) as e:
        srv.submit(A64[:1])
    assert e.value.status == syev3.SYEV3_EAGAIN
    for t in ts:
        assert srv.wait(t, 60.0).state == 2
    srv.release(ts[0])
    t = srv.submit(A64[:1])
    assert srv.wait(t, 60.0).state == 2
    for x in ts[1:] + [t]:
        srv.release(x)
    st = srv.stats()
    assert st.completed == syev3.SERVER_SLOTS + 1
    srv.close()


def test_eigenvalues_only_requests(syev3, pools, pool_oracle):
    """Requests without eigenvectors (the arena holds only their eigenvalues;
    the serving solve kernels skip the vector stores of those tiles), mixed
    with requests that want them: eigenvalues equal to a standalone
    eigenvalues-only call bit for bit and within the oracle's bars."""
    A64, A32 = pools
    rng = np.random.default_rng(4010)
    srv = syev3.Server(memory_budget_bytes=256 << 20, chunk=1 << 13, round_matrices=1 << 16)
    reqs = []
    for i in range(40):
        n = int(np.exp(rng.uniform(0, np.log(1 << 16))))
        is64 = bool(rng.uniform() < 0.6)
        pool = A64 if is64 else A32
        off = int(rng.integers(0, pool.shape[0] - n))
        vectors = bool(i % 2)
        comp = (not is64) and bool(rng.uniform() < 0.5)
        t = srv.submit(pool[off:off + n], compensated=comp, vectors=vectors)
        reqs.append((t, pool[off:off + n], comp, is64, off, vectors))
    for t, A, comp, is64, off, vectors in reqs:
        info = srv.wait(t, 60.0)
        assert info.state == 2
        lam, U = srv.results(t)
        assert (U is None) == (not vectors)
        lam_s, _ = syev3.syev3_batched(A, compensated=comp, vectors=False)
        torch.cuda.synchronize()
        assert torch.equal(lam, lam_s)
        lam_o, _ = pool_oracle[0 if is64 else 1]
        sl = slice(off, off + A.shape[0])
        eps, tol = (parity.EPS64, 8) if is64 else (parity.EPS32, 64)
        parity.compare(A.cpu().numpy().astype(np.float64), lam.cpu().numpy(), None, lam_o[sl], None, eps=eps,
                       lam_tol=tol, res_tol=0, orth_tol=0, vec_tol=0)
        srv.release(t)
    assert released_stats(srv).arena_used == 0
    srv.close()
