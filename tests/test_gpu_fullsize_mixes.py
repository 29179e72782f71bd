"""The batched and serving paths at the sizes bench.py times, checked against
the oracle (Algorithm 3) on complete strings, plus properties over the whole
output.  Bit-exact.

  * the batched mix of the benchmark: 4096 strings, log-uniform lengths
    1 Ki - 4 Mi (seed 4), about 1.99 G symbols.  Its sa / rank / lcp are built
    on the GPU (lr_batch_build_arrays), as the benchmark does, and compared
    with the host prep on every checked string; one batched query; 64
    complete strings (the 8 longest and 56 drawn at random) against the
    oracle, which is fed the host prep's arrays;
  * the serving pool of the benchmark: 2000 jobs, lognormal lengths
    (median 100 Ki, sigma 1), through the serving loop; 200 complete jobs
    (the 10 longest and 190 drawn at random) against the oracle.
"""
import os

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def lrmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1501_06663_gb300 as m
    m.build_library()
    return m


def _check_string(rank, lcp, ln, st, offs, starts, shift, what):
    """Every position of one string (host prep arrays rank, lcp) against the
    oracle; the GPU results are this string's slices, with positions shifted
    by `shift` and offsets relative to offs[0]."""
    w_ln, w_st, w_off, w_starts = oracle.lr_at_range(rank, lcp, 0, rank.size, threads=THREADS)
    assert np.array_equal(ln, w_ln), what
    assert np.array_equal(np.where(st >= 0, st - shift, st), w_st), what
    assert np.array_equal(offs - offs[0], w_off), what
    assert np.array_equal(starts - shift, w_starts), what


def test_batched_mix_of_the_benchmark(lrmod):
    count = 4096
    text, off, _ = W.batched_mix(count=count, lo=1024, hi=4 * W.MI, seed=4)
    total = int(off[-1])
    free, _ = torch.cuda.mem_get_info()
    need = total * 95                                    # text, arrays and the build's work memory
    if free < need:
        pytest.skip("needs %.0f GB free" % (need / 1e9))
    d_off = torch.from_numpy(off).cuda()
    d_text = torch.from_numpy(text).cuda()
    builder = lrmod.Context(0)
    try:
        sa, rank, lcp = builder.build_arrays_batch(d_off, d_text)
    finally:
        builder.close()                                  # frees the build's work memory
    del d_text
    torch.cuda.empty_cache()
    lens = np.diff(off)
    rng = np.random.default_rng(404)
    rest = np.setdiff1d(np.arange(count), np.argsort(lens)[-8:])
    check = np.concatenate([np.argsort(lens)[-8:], rng.choice(rest, 56, replace=False)])
    ctx = lrmod.Context(0)
    try:
        ln, st, offs, starts = ctx.query_batch(d_off, lcp, sa=sa)
        # properties over the whole batch: complete and non-decreasing CSR,
        # a position has LR's iff its length is positive, leftmost = first start
        assert int(offs[0]) == 0 and int(offs[-1]) == starts.numel()
        step = 1 << 27
        for c0 in range(0, total, step):
            c1 = min(total, c0 + step)
            cnt = offs[c0 + 1:c1 + 1] - offs[c0:c1]
            assert bool((cnt >= 0).all())
            assert bool(((cnt > 0) == (ln[c0:c1] > 0)).all())
            has = torch.nonzero(cnt > 0).squeeze(1) + c0
            assert bool((st[has] == starts[offs[has]]).all())
            assert bool((st[c0:c1][ln[c0:c1] == 0] == -1).all())
            del cnt, has
        for j in check:
            a, b = int(off[j]), int(off[j + 1])
            h_sa, h_rank, h_lcp = W.prep(text[a:b])
            assert np.array_equal(sa[a:b].cpu().numpy(), h_sa), "GPU sa of string %d" % j
            assert np.array_equal(rank[a:b].cpu().numpy(), h_rank), "GPU rank of string %d" % j
            assert np.array_equal(lcp[a + j:b + j + 1].cpu().numpy(), h_lcp), "GPU lcp of string %d" % j
            o = offs[a:b + 1].cpu().numpy()
            _check_string(h_rank, h_lcp, ln[a:b].cpu().numpy(), st[a:b].cpu().numpy(), o,
                          starts[int(o[0]):int(o[-1])].cpu().numpy(), a, "string %d" % j)
    finally:
        ctx.close()


def test_serving_pool_of_the_benchmark(lrmod):
    count = 2000
    text, off, _ = W.serving_mix(count, seed=5)
    sa, rank, lcp = W.prep_many(text, off)
    del text
    srv = lrmod.Server(0, max_batch_positions=1 << 25, slots=4, max_inflight=2, batch_window_us=1000)
    try:
        ids = []
        for j in range(count):
            a, b = int(off[j]), int(off[j + 1])
            ids.append(srv.submit(lcp[a + j:b + j + 1], sa=sa[a:b], capacity=3 * (b - a) + 1024))
        results = [srv.wait(i, timeout_ms=600000) for i in ids]
        stats = srv.stats()
    finally:
        srv.close()
    assert stats["completed"] == count and stats["failed"] == 0
    lens = np.diff(off)
    rng = np.random.default_rng(505)
    rest = np.setdiff1d(np.arange(count), np.argsort(lens)[-10:])
    for j in np.concatenate([np.argsort(lens)[-10:], rng.choice(rest, 190, replace=False)]):
        a, b = int(off[j]), int(off[j + 1])
        res, ln, st, offs, starts = results[j]
        assert res == lrmod.LR_OK
        _check_string(rank[a:b], lcp[a + j:b + j + 1], ln, st, offs, starts, 0, "job %d" % j)
