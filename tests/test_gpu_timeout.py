"""Bounded device-side waits: a look-back wait that runs out is reported, not hung.

Every kernel that waits for another CTA's look-back status word polls it a
bounded number of times, then records a timeout and finishes.  The test hook
lr_test_hold_lookback keeps one cover tile's status word unpublished (a flag
that nothing sets) and shortens the poll limit, so the next tile's wait runs
out without any fault.  The query must report LR_ERR_TIMEOUT within a bounded
time, and the same context must then answer a normal query bit-exactly.
"""
import time

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = None


@pytest.fixture(scope="module")
def ctx():
    global P
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1501_06663_gb300 as lrmod
    lrmod.build_library()
    P = lrmod
    c = lrmod.Context(0)
    yield c
    P.lr_test_hold_lookback(c.handle, -1, 0)
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _outs(n, cap):
    return (torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.int32, device="cuda"),
            torch.empty(n + 1, dtype=torch.int64, device="cuda"), torch.empty(cap, dtype=torch.int32, device="cuda"))


@pytest.mark.parametrize("front", ["sa", "rank"])
def test_lost_wait_reports_timeout_and_the_context_recovers(ctx, front):
    w = W.single("dna_64m", n=200_000)              # 49 cover tiles of 4096 positions
    want = oracle.lr_all_raw(w.rank, w.lcp)
    sa, rank = (_dev(w.sa), None) if front == "sa" else (None, _dev(w.rank))
    lcp = _dev(w.lcp)
    ln, st, off, starts = _outs(w.n, want[3].size)
    assert P.lr_test_hold_lookback(ctx.handle, 5, 1000) == P.LR_OK
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    status, _ = P.lr_query_all(ctx.handle, sa, rank, lcp, ln, st, off, starts)
    dt = time.perf_counter() - t0
    assert status == P.LR_ERR_TIMEOUT
    assert dt < 5.0, dt                             # 1000 polls, not the default limit
    # the error word was read and cleared by the synchronising call
    assert P.lr_device_status(ctx.handle) == P.LR_OK
    # a held tile past the last one: nothing waits on it, nothing times out
    assert P.lr_test_hold_lookback(ctx.handle, 10_000, 1000) == P.LR_OK
    status, total = P.lr_query_all(ctx.handle, sa, rank, lcp, ln, st, off, starts)
    assert status == P.LR_OK and total == want[3].size
    # hook off: the same context answers bit-exactly
    assert P.lr_test_hold_lookback(ctx.handle, -1, 0) == P.LR_OK
    status, total = P.lr_query_all(ctx.handle, sa, rank, lcp, ln, st, off, starts)
    assert status == P.LR_OK and total == want[3].size
    for name, a, b in zip(("lr_len", "lr_start", "offsets", "starts"), (ln, st, off, starts), want):
        assert np.array_equal(a.cpu().numpy(), b), name


def test_asynchronous_timeout_is_reported_by_device_status(ctx):
    w = W.single("english_256m", n=100_000)
    lcp, sa = _dev(w.lcp), _dev(w.sa)
    ln, st, off, starts = _outs(w.n, 4 * w.n)
    assert P.lr_test_hold_lookback(ctx.handle, 0, 500) == P.LR_OK
    status, _ = P.lr_query_all(ctx.handle, sa, None, lcp, ln, st, off, starts, sync=False)
    assert status == P.LR_OK                        # enqueued; the kernels report later
    assert P.lr_device_status(ctx.handle) == P.LR_ERR_TIMEOUT
    assert P.lr_test_hold_lookback(ctx.handle, -1, 0) == P.LR_OK
    status, total = P.lr_query_all(ctx.handle, sa, None, lcp, ln, st, off, starts)
    assert status == P.LR_OK
    want = oracle.lr_all_raw(w.rank, w.lcp)
    assert total == want[3].size and np.array_equal(off.cpu().numpy(), want[2])


def test_hook_arguments(ctx):
    assert P.lr_test_hold_lookback(ctx.handle, 3, 0) == P.LR_ERR_ARG
    assert P.lr_test_hold_lookback(ctx.handle, 3, (1 << 23) + 1) == P.LR_ERR_ARG
    assert P.lr_test_hold_lookback(ctx.handle, -1, 0) == P.LR_OK
