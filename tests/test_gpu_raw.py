"""The raw-LLR variant (Algorithms 1 and 3 on the GPU) and the walk statistics
of Table 2, against the oracle.  Bit-exact."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = None
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))


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
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check_raw(ctx, rank, lcp, what=""):
    want = oracle.lr_all_raw(rank, lcp)
    got = [t.cpu().numpy() for t in ctx.query_all_raw(_dev(lcp), _dev(rank))]
    for name, a, b in zip(("lr_len", "lr_start", "offsets", "starts"), got, want):
        assert a.shape == b.shape and np.array_equal(a, b), (what, name)
    st, ln = ctx.query_leftmost_raw(_dev(lcp), _dev(rank))
    assert np.array_equal(st.cpu().numpy(), want[1]) and np.array_equal(ln.cpu().numpy(), want[0]), what


def _check_stats(ctx, rank, lcp, what=""):
    alpha, beta, m = oracle.walk_counts(rank, lcp)
    summary, a, b = ctx.walk_stats(_dev(lcp), _dev(rank), per_position=True)
    assert np.array_equal(a.cpu().numpy(), alpha), what
    assert np.array_equal(b.cpu().numpy(), beta), what
    assert summary["m"] == m and summary["n"] == len(rank)
    assert summary["alpha_sum"] == int(alpha.astype(np.int64).sum())
    assert summary["beta_sum"] == int(beta.astype(np.int64).sum())
    assert (summary["alpha_min"], summary["alpha_max"]) == (int(alpha.min()), int(alpha.max()))
    assert (summary["beta_min"], summary["beta_max"]) == (int(beta.min()), int(beta.max()))


def test_paper_examples(ctx):
    for s in (GOLD["table1_mississippi"]["text"], "abcabcddbca", "ababab", "aaaa", "a", "ab"):
        sa, rank, lcp = W.prep(np.frombuffer(s.encode(), np.uint8))
        _check_raw(ctx, rank, lcp, s)
        _check_stats(ctx, rank, lcp, s)


def test_random_small_strings(ctx):
    rng = np.random.default_rng(31)
    for _ in range(30):
        n = int(rng.integers(1, 9000))
        text = (rng.integers(0, int(rng.integers(1, 5)), n) + 97).astype(np.uint8)
        sa, rank, lcp = W.prep(text)
        _check_raw(ctx, rank, lcp, n)
        _check_stats(ctx, rank, lcp, n)


@pytest.mark.parametrize("name,n", [("dna_iid_1m", None), ("dna_64m", 1 << 20), ("english_256m", 1 << 22)])
def test_workloads(ctx, name, n):
    w = W.single(name, n=n)
    _check_raw(ctx, w.rank, w.lcp, name)
    _check_stats(ctx, w.rank, w.lcp, name)


def test_long_walks(ctx):
    """a^n: the walk from k meets k + 1 raw LLR's."""
    sa, rank, lcp = W.prep(np.full(6000, 97, np.uint8))
    _check_raw(ctx, rank, lcp, "a^6000")
    _check_stats(ctx, rank, lcp, "a^6000")


def test_capacity_and_bad_input(ctx):
    w = W.single("dna_iid_1m", n=50000)
    n = w.n
    want = oracle.lr_all_raw(w.rank, w.lcp)
    total = int(want[2][-1])
    d_rank, d_lcp = _dev(w.rank), _dev(w.lcp)
    ln = torch.empty(n, dtype=torch.int32, device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    starts = torch.empty(total // 2, dtype=torch.int32, device="cuda")
    s, tot = P.lr_query_all_raw(ctx.handle, d_rank, d_lcp, ln, st, off, starts)
    assert s == P.LR_ERR_CAPACITY and tot == total
    assert np.array_equal(off.cpu().numpy(), want[2])
    bad = w.lcp.copy()
    bad[0] = 2
    s, _ = P.lr_query_all_raw(ctx.handle, d_rank, _dev(bad), ln, st, off, torch.empty(4 * n, dtype=torch.int32,
                                                                                        device="cuda"))
    assert s == P.LR_ERR_SENTINEL
    _check_raw(ctx, w.rank, w.lcp, "after an error")
