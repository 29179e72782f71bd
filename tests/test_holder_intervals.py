"""A structural property of the all-LR result, checked on the oracle.

Entry t of LLRc (start s_t, end e_t, length l_t) is a longest repeat of k
exactly when it covers k and no strictly longer entry covers k (Algorithm 2's
window maximum, Algorithm 4's ties).  Starts and ends of LLRc increase
(Sec. 3.2), so with PG(t) and NG(t) the nearest strictly longer entries left
and right of t, t holds exactly the positions

    H_t = [max(s_t, e_PG(t) + 1), min(e_t, s_NG(t) - 1)]

and, over the entries with a non-empty H_t, both ends of H_t are
non-decreasing (the holders of a position are a contiguous run of them).
Every position's list of LR starts from the oracle (Algorithm 3, which walks
the raw LLR array and never forms intervals) is inverted into the set of
positions each entry holds and compared with H_t from a brute-force
nearest-longer search: a dropped tie, a wrong window end or a wrong order
in the oracle breaks the equality.
"""
import numpy as np
import pytest

import oracle
import workloads as W


def _holder_intervals(cs, cl):
    m = cs.size
    ce = cs + cl - 1
    a = np.empty(m, np.int64)
    b = np.empty(m, np.int64)
    for t in range(m):
        lt = cl[t]
        pg = next((u for u in range(t - 1, -1, -1) if cl[u] > lt), None)
        ng = next((u for u in range(t + 1, m) if cl[u] > lt), None)
        a[t] = max(cs[t], ce[pg] + 1) if pg is not None else cs[t]
        b[t] = min(ce[t], cs[ng] - 1) if ng is not None else ce[t]
    return a, b


def _held_positions(cs, off, starts, n):
    """Positions whose LR list contains each entry (entries found by start)."""
    held = [[] for _ in range(cs.size)]
    for k in range(n):
        for s in starts[off[k]:off[k + 1]]:
            t = int(np.searchsorted(cs, s))
            assert t < cs.size and cs[t] == s, "an LR start that is not an LLRc start"
            held[t].append(k)
    return held


def _check(text):
    sa, rank, lcp = W.prep(text)
    cs, cl = oracle.compact(rank, lcp)
    cs = cs.astype(np.int64)
    cl = cl.astype(np.int64)
    _, _, off, starts = oracle.lr_all_raw(rank, lcp)
    a, b = _holder_intervals(cs, cl)
    held = _held_positions(cs, off, starts, text.size)
    for t in range(cs.size):
        want = list(range(a[t], b[t] + 1)) if a[t] <= b[t] else []
        assert held[t] == want, (t, cs[t], cl[t], held[t][:8], a[t], b[t])
    ne = a <= b
    assert np.all(np.diff(a[ne]) >= 0) and np.all(np.diff(b[ne]) >= 0)


def test_paper_examples():
    for s in (b"mississippi", b"abcabcddbca", b"ababab", b"aaaa", b"a", b"abcd"):
        _check(np.frombuffer(s, np.uint8))


def test_random_strings():
    import tests.test_oracle as T
    rng = np.random.default_rng(21)
    for _ in range(120):
        n = int(rng.integers(1, 700))
        _check(np.frombuffer(T._random_string(rng, n), np.uint8))


@pytest.mark.parametrize("kind", ["dna_iid", "dna", "english", "protein"])
def test_workload_kinds(kind):
    _check(W.make_text(kind, 4000, 31))


def test_ties_and_periods():
    _check(W.iid(3000, b"ab", 5))                                   # binary: frequent ties
    _check(np.frombuffer(b"ab" * 700, np.uint8))
    _check(np.frombuffer((b"abcab" * 300)[:1499], np.uint8))
