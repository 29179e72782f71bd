"""The batched and serving paths at the sizes bench.py times, on sampled
positions checked against the oracle (Algorithm 3 per position), plus
properties that hold at any size.  Bit-exact.

  * the batched mix of the benchmark: 512 strings, log-uniform lengths
    1 Ki - 4 Mi (seed 4), one batched query;
  * the serving pool of the benchmark: 2000 jobs, lognormal lengths
    (median 100 Ki, sigma 1), through the serving loop.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lrmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1501_06663_gb300 as m
    m.build_library()
    return m


def _check_sample(rank, lcp, ks, ln, st, offs, starts, shift, what):
    """Positions ks (string-local) of one string against the oracle; the GPU
    arrays are indexed by ks and hold positions shifted by `shift`."""
    w_ln, w_st, w_off, w_starts = oracle.lr_at(rank, lcp, ks)
    assert np.array_equal(ln, w_ln), what
    assert np.array_equal(np.where(st >= 0, st - shift, st), w_st), what
    for q in range(len(ks)):
        got = starts[offs[q]:offs[q + 1]] - shift
        assert np.array_equal(got, w_starts[w_off[q]:w_off[q + 1]]), (what, int(ks[q]))


def test_batched_mix_of_the_benchmark(lrmod):
    text, off, _ = W.batched_mix(count=512, lo=1024, hi=4 * W.MI, seed=4)
    sa, rank, lcp = W.prep_many(text, off)
    del text
    ctx = lrmod.Context(0)
    try:
        out = ctx.query_batch(torch.from_numpy(off).cuda(), torch.from_numpy(lcp).cuda(),
                              sa=torch.from_numpy(sa).cuda())
        ln, st, offs, starts = out
        total = int(off[-1])
        # properties at full size: CSR offsets non-decreasing and complete,
        # no LR's of length 0, leftmost = first listed start
        o = offs.cpu().numpy()
        assert o[0] == 0 and o[-1] == starts.numel() and np.all(np.diff(o) >= 0)
        h_ln = ln.cpu().numpy()
        h_st = st.cpu().numpy()
        h_starts = starts.cpu().numpy()
        has = np.nonzero(np.diff(o) > 0)[0]
        assert np.array_equal(h_ln[has] > 0, np.ones(has.size, bool))
        assert np.array_equal(h_st[has], h_starts[o[has]])
        rng = np.random.default_rng(404)
        for j in rng.choice(512, 24, replace=False):
            a, b = int(off[j]), int(off[j + 1])
            ks = np.unique(np.concatenate([[0, b - a - 1], rng.integers(0, b - a, 64)])).astype(np.int64)
            g = a + ks
            sub_off = np.zeros(len(ks) + 1, np.int64)
            np.cumsum(o[g + 1] - o[g], out=sub_off[1:])
            sub_starts = np.concatenate([h_starts[o[x]:o[x + 1]] for x in g]) if sub_off[-1] else np.zeros(0, np.int32)
            _check_sample(rank[a:b], lcp[a + j:b + j + 1], ks, h_ln[g], h_st[g], sub_off, sub_starts, a,
                          "string %d" % j)
        assert total == h_ln.size
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
    rng = np.random.default_rng(505)
    for j in rng.choice(count, 40, replace=False):
        a, b = int(off[j]), int(off[j + 1])
        res, ln, st, offs, starts = results[j]
        assert res == lrmod.LR_OK
        assert offs[0] == 0 and offs[-1] == len(starts) and np.all(np.diff(offs) >= 0)
        ks = np.unique(np.concatenate([[0, b - a - 1], rng.integers(0, b - a, 64)])).astype(np.int64)
        sub_off = np.zeros(len(ks) + 1, np.int64)
        np.cumsum(offs[ks + 1] - offs[ks], out=sub_off[1:])
        sub_starts = np.concatenate([starts[offs[k]:offs[k + 1]] for k in ks]) if sub_off[-1] else np.zeros(0, np.int32)
        _check_sample(rank[a:b], lcp[a + j:b + j + 1], ks, ln[ks], st[ks], sub_off, sub_starts, 0, "job %d" % j)
