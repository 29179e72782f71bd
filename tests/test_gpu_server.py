"""The serving loop (continuous batching) on the GPU: every job's result equals
the oracle's and the single-string query's on that job alone, whatever else
shares its batch.  Bit-exact.
"""
import threading
import time

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = None


@pytest.fixture(scope="module")
def lrmod():
    global P
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1501_06663_gb300 as m
    m.build_library()
    P = m
    return m


@pytest.fixture(scope="module")
def ctx(lrmod):
    c = lrmod.Context(0)
    yield c
    c.close()


def _jobs(count, seed, median=20000, cap=200000):
    """A serving-shaped mix: lognormal lengths, 70% DNA / 30% protein."""
    text, off, _ = W.serving_mix(count, seed=seed, median=median, sigma=1.0, floor_len=64, cap=cap)
    sa, rank, lcp = W.prep_many(text, off)
    out = []
    for j in range(count):
        a, b = int(off[j]), int(off[j + 1])
        out.append((sa[a:b].copy(), rank[a:b].copy(), lcp[a + j:b + j + 1].copy()))
    return out


def _check_job(res, rank, lcp, what):
    st, ln, start, offs, starts = res
    assert st == P.LR_OK, (what, P.status_str(st))
    want = oracle.lr_all_raw(rank, lcp)
    for name, a, b in zip(("lr_len", "lr_start", "offsets", "starts"), (ln, start, offs, starts), want):
        assert np.array_equal(a, b), (what, name)


def test_mix_equals_oracle_and_alone(lrmod, ctx):
    jobs = _jobs(48, seed=5)
    srv = lrmod.Server(0, max_batch_positions=1 << 21, batch_window_us=3000)
    try:
        ids = [srv.submit(lcp, sa=sa) for sa, _, lcp in jobs]
        results = [srv.wait(i, timeout_ms=120000) for i in ids]
        stats = srv.stats()
    finally:
        srv.close()
    for k, ((sa, rank, lcp), res) in enumerate(zip(jobs, results)):
        _check_job(res, rank, lcp, "job %d" % k)
        alone = [t.cpu().numpy() for t in ctx.query_all(torch.from_numpy(lcp).cuda(), sa=torch.from_numpy(sa).cuda())]
        for a, b in zip(res[1:], alone):
            assert np.array_equal(a, b), "job %d differs from the same query alone" % k
    assert stats["completed"] == len(jobs) and stats["failed"] == 0
    assert 1 <= stats["batches"] < len(jobs)          # jobs shared batches
    assert 0 < stats["p50_us"] <= stats["p99_us"] <= stats["max_us"]


def test_arrivals_while_others_run(lrmod):
    """Jobs submitted from another thread over time, with pinned buffers, sa and rank jobs mixed."""
    jobs = _jobs(40, seed=6, median=50000)
    srv = lrmod.Server(0, max_batch_positions=1 << 20, slots=3, max_inflight=2, batch_window_us=500)
    ids = [None] * len(jobs)
    pinned = [(torch.from_numpy(sa).pin_memory(), torch.from_numpy(rank).pin_memory(),
               torch.from_numpy(lcp).pin_memory()) for sa, rank, lcp in jobs]

    def producer():
        rng = np.random.default_rng(1)
        for k, (sa, rank, lcp) in enumerate(pinned):
            if k % 3 == 2:
                ids[k] = srv.submit(lcp, rank=rank, pinned=True)
            else:
                ids[k] = srv.submit(lcp, sa=sa, pinned=True)
            time.sleep(float(rng.exponential(0.0005)))

    try:
        th = threading.Thread(target=producer)
        th.start()
        th.join()
        results = [srv.wait(i, timeout_ms=120000) for i in ids]
        stats = srv.stats()
    finally:
        srv.close()
    for k, ((_, rank, lcp), res) in enumerate(zip(jobs, results)):
        _check_job(res, rank, lcp, "job %d" % k)
    assert stats["completed"] == len(jobs)


def test_bad_job_fails_alone(lrmod):
    jobs = _jobs(12, seed=7)
    bad = 5
    sa, rank, lcp = jobs[bad]
    lcp = lcp.copy()
    lcp[0] = 3                                         # broken sentinel
    jobs[bad] = (sa, rank, lcp)
    srv = lrmod.Server(0, max_batch_positions=1 << 22, max_inflight=1, batch_window_us=20000)
    try:
        ids = [srv.submit(l, sa=s) for s, _, l in jobs]
        results = [srv.wait(i, timeout_ms=120000) for i in ids]
    finally:
        srv.close()
    for k, ((_, rank, lcp), res) in enumerate(zip(jobs, results)):
        if k == bad:
            assert res[0] == P.LR_ERR_SENTINEL
        else:
            _check_job(res, rank, lcp, "job %d" % k)


def test_capacity_and_starts_growth(lrmod):
    jobs = _jobs(10, seed=8)
    # starts buffers start nearly empty, so batches must grow them
    srv = lrmod.Server(0, max_batch_positions=1 << 21, starts_factor=0.001, batch_window_us=20000, max_inflight=1)
    try:
        sa, rank, lcp = jobs[0]
        want = oracle.lr_all_raw(rank, lcp)
        total = int(want[2][-1])
        small = srv.submit(lcp, sa=sa, capacity=total // 2)
        ids = [srv.submit(l, sa=s) for s, _, l in jobs[1:]]
        res_small = srv.wait(small, timeout_ms=120000)
        results = [srv.wait(i, timeout_ms=120000) for i in ids]
    finally:
        srv.close()
    assert res_small[0] == P.LR_ERR_CAPACITY
    assert np.array_equal(res_small[1], want[0]) and np.array_equal(res_small[3], want[2])
    for k, ((_, rank, lcp), res) in enumerate(zip(jobs[1:], results)):
        _check_job(res, rank, lcp, "job %d" % (k + 1))


def test_admission_limits_cancel_and_stop(lrmod):
    jobs = _jobs(6, seed=9, median=4000, cap=8000)
    srv = lrmod.Server(0, max_batch_positions=8192, slots=1, max_inflight=1, max_queue=3)
    try:
        sa, rank, lcp = jobs[0]
        big = np.zeros(9000, np.int32)
        with pytest.raises(P.LRError) as e:
            srv.submit(np.zeros(9001, np.int32), sa=big)                # can never fit a slot
        assert e.value.status == P.LR_ERR_NOMEM
        ids, busy = [], 0
        for _ in range(2000):
            try:
                ids.append(srv.submit(lcp, sa=sa))
            except P.LRError as ex:
                assert ex.status == P.LR_ERR_BUSY
                busy += 1
                if busy > 3:
                    break
        assert busy > 0                                                  # the queue limit answered
        outcome = srv.cancel(ids[-1])
        assert outcome in (P.LR_OK, P.LR_ERR_BUSY)
        results = [srv.wait(i, timeout_ms=120000) for i in ids]
        for k, res in enumerate(results):
            if k == len(ids) - 1 and outcome == P.LR_OK:
                assert res[0] == P.LR_ERR_BUSY and res[1] is None       # cancelled
            else:
                _check_job(res, rank, lcp, "job %d" % k)
        # stop with work still queued: returns, queued jobs are cancelled
        for _ in range(3):
            try:
                srv.submit(lcp, sa=sa)
            except P.LRError:
                pass
    finally:
        srv.close()


def test_text_jobs_build_their_arrays_on_the_gpu(lrmod, ctx):
    """Jobs that give only their string: the server builds sa / rank / lcp on
    the GPU with the rest of the batch; results equal the oracle's on the
    host-prepped arrays and the query alone; text and array jobs mix."""
    text, off, _ = W.serving_mix(30, seed=41, median=20000, floor_len=64, cap=200000)
    strings = [text[int(off[j]):int(off[j + 1])].copy() for j in range(30)]
    srv = lrmod.Server(0, max_batch_positions=1 << 21, batch_window_us=3000, text_jobs=1)
    try:
        ids = []
        for k, s in enumerate(strings):
            if k % 5 == 4:                                   # every fifth job brings host-prepped arrays
                sa, rank, lcp = W.prep(s)
                ids.append(srv.submit(lcp, sa=sa))
            else:
                ids.append(srv.submit(text=s))
        results = [srv.wait(i, timeout_ms=120000) for i in ids]
        stats = srv.stats()
    finally:
        srv.close()
    for k, (s, res) in enumerate(zip(strings, results)):
        sa, rank, lcp = W.prep(s)
        _check_job(res, rank, lcp, "text job %d" % k)
    assert stats["completed"] == len(strings)


def test_text_jobs_need_a_text_server(lrmod):
    srv = lrmod.Server(0, max_batch_positions=1 << 16)
    try:
        with pytest.raises(lrmod.LRError) as e:
            srv.submit(text=np.frombuffer(b"abcabc", np.uint8).copy())
        assert e.value.status == lrmod.LR_ERR_ARG
    finally:
        srv.close()
