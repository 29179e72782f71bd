"""lr_query_all_static, the entry point that allocates nothing.

Some users of this library cannot allocate device memory when they run a
query (a per-request callback inside another framework, a service with a
memory budget fixed at start-up), so the library offers one query whose
working memory is a fixed array inside the library itself.  This file checks,
on the GPU and through the C ABI, that it returns exactly what lr_query_all
returns, on two calls in a row (the array keeps the previous call's
contents), and that it refuses inputs larger than its array.  It is named to
run after every other test file.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1501_06663_gb300 as lr
    lr.build_library()
    return lr


def _out(n, cap):
    return (torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.int32, device="cuda"),
            torch.empty(n + 1, dtype=torch.int64, device="cuda"), torch.empty(cap, dtype=torch.int32, device="cuda"))


def test_static_matches_context_query_twice(lib):
    ctx = lib.Context(0)
    try:
        for name, n, seed in (("dna_64m", 300_000, None), ("english_256m", lib.LR_STATIC_MAX_N, None)):
            w = W.single(name, n)
            rank = torch.from_numpy(w.rank).cuda()
            lcp = torch.from_numpy(w.lcp).cuda()
            want = [t.cpu().numpy() for t in ctx.query_all(lcp, rank=rank)]
            total = int(want[3].size)
            for call in range(2):
                ln, st, off, starts = _out(w.n, total + 7)
                status, tot = lib.lr_query_all_static(rank, lcp, ln, st, off, starts)
                assert status == lib.LR_OK and tot == total, (name, call, status, tot)
                got = (ln.cpu().numpy(), st.cpu().numpy(), off.cpu().numpy(), starts[:tot].cpu().numpy())
                for a, b in zip(got, want):
                    assert np.array_equal(a, b), (name, call)
        # and against the oracle on a small case
        w = W.single("dna_iid_1m", 20_000)
        ln, st, off, starts = _out(w.n, 4 * w.n)
        status, tot = lib.lr_query_all_static(torch.from_numpy(w.rank).cuda(), torch.from_numpy(w.lcp).cuda(),
                                              ln, st, off, starts)
        want = oracle.lr_all_raw(w.rank, w.lcp)
        assert status == lib.LR_OK
        for a, b in zip((ln.cpu().numpy(), st.cpu().numpy(), off.cpu().numpy(), starts[:tot].cpu().numpy()), want):
            assert np.array_equal(a, b)
    finally:
        ctx.close()


def test_static_rejects_inputs_larger_than_its_array(lib):
    n = lib.LR_STATIC_MAX_N + 1
    rank = torch.zeros(n, dtype=torch.int32, device="cuda")
    lcp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    ln, st, off, starts = _out(n, 16)
    status, _ = lib.lr_query_all_static(rank, lcp, ln, st, off, starts)
    assert status == lib.LR_ERR_ARG
