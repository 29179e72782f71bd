"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself: values printed in the
paper (tests/golden/paper_examples.json), the literal Definition 1 enumerated
in pure Python, an O(n^2) brute force from the string alone, mathematical
invariants the paper proves (Lemma 1, Lemma 2, Sec. 3.2 monotonicity), and
direct substring counting on sampled positions.
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import definition

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))


def _prep(s: bytes):
    return W.prep(np.frombuffer(s, np.uint8))


def _rows(csr):
    """CSR -> list of (length, [starts]) per position."""
    ln, st, off, starts = csr
    return [(int(ln[k]), [int(x) for x in starts[off[k]:off[k + 1]]]) for k in range(len(ln))]


def _check_csr_shape(csr):
    ln, st, off, starts = csr
    n = len(ln)
    assert off[0] == 0 and off[n] == len(starts)
    assert np.all(np.diff(off) >= 0)
    for k in range(n):
        row = starts[off[k]:off[k + 1]]
        if ln[k] == 0:
            assert len(row) == 0 and st[k] == -1
        else:
            assert len(row) >= 1 and st[k] == row[0]
            assert np.all(np.diff(row) > 0)


# ---------------------------------------------------------------- paper values

def test_table1_mississippi_prep():
    g = GOLD["table1_mississippi"]
    sa, rank, lcp = _prep(g["text"].encode())
    assert list(sa + 1) == g["sa_1based"]
    assert list(lcp) == g["lcp_1based_n_plus_1"]
    assert np.array_equal(rank[sa], np.arange(len(sa)))


def test_abcabcddbca_lr2_all_variants():
    g = GOLD["abcabcddbca_lr2"]
    s = g["text"].encode()
    k = g["k_1based"] - 1
    want = (g["lr_length"], [x - 1 for x in g["lr_starts_1based"]])
    sa, rank, lcp = _prep(s)
    for csr in (oracle.brute(s), oracle.lr_all_raw(rank, lcp), oracle.lr_all_compact(rank, lcp)):
        assert _rows(csr)[k] == want
    assert definition.lr_all(s)[k] == want
    for st, ln in (oracle.lr_leftmost_raw(rank, lcp), oracle.lr_leftmost_compact(rank, lcp)):
        assert (ln[k], st[k]) == (want[0], want[1][0])


def test_ababab_llr_and_useless():
    g = GOLD["ababab_llr"]
    s = g["text"].encode()
    sa, rank, lcp = _prep(s)
    L = oracle.llr_raw(rank, lcp)
    for i1, (a, b) in g["llr"].items():
        i = int(i1) - 1
        assert a - 1 == i and L[i] == b - a + 1
    cs, cl = oracle.compact(rank, lcp)
    for u in g["useless_1based"]:
        assert (u - 1) not in set(cs.tolist())


def test_fig3_compaction():
    g = GOLD["fig3_compaction"]
    flag, ps, cs, cl = oracle.flag_prefix_scatter(np.array(g["raw_llr"], np.int32))
    assert flag.tolist() == g["flag"]
    assert ps.tolist() == g["prefix_sum"]
    assert [[int(a) + 1, int(b)] for a, b in zip(cs, cl)] == g["llrc_1based"]


# ---------------------------------------------------------------- special cases

@pytest.mark.parametrize("s,want", [
    (b"a", [(0, [])]),
    (b"abcd", [(0, [])] * 4),
    (b"aaaa", [(3, [0]), (3, [0, 1]), (3, [0, 1]), (3, [1])]),  # overlapping occurrences count
    (b"aa", [(1, [0]), (1, [1])]),
    (b"abab", [(2, [0]), (2, [0]), (2, [2]), (2, [2])]),          # ba is unique
])
def test_special_cases(s, want):
    assert definition.lr_all(s) == want
    assert _rows(oracle.brute(s)) == want
    sa, rank, lcp = _prep(s)
    assert _rows(oracle.lr_all_raw(rank, lcp)) == want
    assert _rows(oracle.lr_all_compact(rank, lcp)) == want


def test_aaaa_llr_values():
    sa, rank, lcp = _prep(b"aaaa")
    assert oracle.llr_raw(rank, lcp).tolist() == [3, 3, 2, 1]


# ---------------------------------------------------------------- brute force pins

def _all_strings(alpha: bytes, n: int):
    if n == 0:
        yield b""
        return
    for p in _all_strings(alpha, n - 1):
        for c in alpha:
            yield p + bytes([c])


def test_brute_matches_literal_definition_exhaustive():
    count = 0
    for n in range(1, 9):
        for s in _all_strings(b"ab", n):
            assert _rows(oracle.brute(s)) == definition.lr_all(s), s
            count += 1
    for n in range(1, 6):
        for s in _all_strings(b"abc", n):
            assert _rows(oracle.brute(s)) == definition.lr_all(s), s
    assert count == 510


def test_brute_matches_literal_definition_random():
    rng = np.random.default_rng(11)
    for _ in range(60):
        n = int(rng.integers(1, 22))
        sig = int(rng.choice([1, 2, 3, 4, 8]))
        s = bytes(rng.integers(97, 97 + sig, n).astype(np.uint8))
        assert _rows(oracle.brute(s)) == definition.lr_all(s), s


def _random_string(rng, n):
    kind = int(rng.integers(0, 5))
    if kind == 0:                                   # small alphabet i.i.d.
        sig = int(rng.choice([1, 2, 4, 20, 96]))
        return bytes(rng.integers(32, 32 + sig, n).astype(np.uint8))
    if kind == 1:                                   # periodic
        p = int(rng.integers(1, 9))
        unit = rng.integers(97, 101, p).astype(np.uint8)
        return bytes(np.resize(unit, n))
    if kind == 2:                                   # tandem insert
        base = rng.integers(65, 69, n).astype(np.uint8)
        u = int(rng.integers(1, 6))
        unit = rng.integers(65, 69, u).astype(np.uint8)
        a = int(rng.integers(0, n))
        ln = min(n - a, u * int(rng.integers(2, 8)))
        base[a:a + ln] = np.resize(unit, ln)
        return bytes(base)
    if kind == 3:                                   # planted copy with mutations
        base = rng.integers(65, 69, n).astype(np.uint8)
        if n >= 8:
            ln = int(rng.integers(2, n // 2 + 1))
            src = int(rng.integers(0, n - ln + 1))
            dst = int(rng.integers(0, n - ln + 1))
            seg = base[src:src + ln].copy()
            mut = rng.random(ln) < 0.05
            seg[mut] = rng.integers(65, 69, int(mut.sum()))
            base[dst:dst + ln] = seg
        return bytes(base)
    return bytes(W.english(n, int(rng.integers(1, 1 << 30)), vocab=50))


def test_walk_oracles_match_brute_force():
    rng = np.random.default_rng(2024)
    for trial in range(400):
        n = int(rng.integers(1, 160)) if trial < 300 else int(rng.integers(160, 2001))
        s = _random_string(rng, n)
        want = oracle.brute(s)
        sa, rank, lcp = _prep(s)
        for got in (oracle.lr_all_raw(rank, lcp), oracle.lr_all_compact(rank, lcp)):
            for a, b in zip(got, want):
                assert np.array_equal(a, b), s
        for st, ln in (oracle.lr_leftmost_raw(rank, lcp), oracle.lr_leftmost_compact(rank, lcp)):
            assert np.array_equal(st, want[1]) and np.array_equal(ln, want[0])


def test_lr_at_matches_full_run():
    """The per-position Algorithm 3 (used for sampled checks at full size)
    equals the full run at every position of inputs with many ties."""
    texts = [W.make_text("dna", 1 << 15, 6), W.iid(6000, b"ab", 8), W.iid(6000, b"abc", 9),
             np.frombuffer(b"abcabcddbca" * 40, np.uint8)]
    ties = 0
    for text in texts:
        sa, rank, lcp = W.prep(text)
        full = oracle.lr_all_raw(rank, lcp)
        ks = np.arange(text.size, dtype=np.int64)
        got = oracle.lr_at(rank, lcp, ks)
        for a, b in zip(got, full):
            assert np.array_equal(a, b)
        ties += int(np.sum(np.diff(full[2]) > 1))
    assert ties > 1000


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("name,n", [("dna_iid_1m", 1 << 16), ("dna_64m", 1 << 17), ("english_256m", 1 << 17)])
def test_invariants_on_workloads(name, n):
    w = W.single(name, n=n)
    s = w.text.tobytes()
    L = oracle.llr_raw(w.rank, w.lcp)
    idx = np.arange(n)
    # Lemma 1: L_i = 0 iff S[i] is a singleton
    counts = np.bincount(w.text, minlength=256)
    assert np.array_equal(L == 0, counts[w.text] == 1)
    # Lemma 2: |LLR_i| <= |LLR_{i+1}| + 1, i.e. ends i + L_i - 1 never decrease
    assert np.all(L[:-1] <= L[1:] + 1)
    # Sec. 3.2: compact LLR starts and ends strictly increase
    cs, cl = oracle.compact(w.rank, w.lcp)
    ce = cs.astype(np.int64) + cl - 1
    assert np.all(np.diff(cs) > 0) and np.all(np.diff(ce) > 0)
    # the one-pass rule of Algorithm 2 equals the Flag / Prefix_Sum scatter of Sec. 4.2.1
    flag, ps, cs2, cl2 = oracle.flag_prefix_scatter(L)
    assert np.array_equal(cs, cs2) and np.array_equal(cl, cl2)
    csr = oracle.lr_all_raw(w.rank, w.lcp)
    _check_csr_shape(csr)
    ln, st, off, starts = csr
    assert np.array_equal(ln == 0, counts[w.text] == 1)
    comp = oracle.lr_all_compact(w.rank, w.lcp)
    for a, b in zip(csr, comp):
        assert np.array_equal(a, b)
    # sampled positions: the LR occurs at least twice, and no longer substring covering k repeats
    rng = np.random.default_rng(n)
    for k in rng.choice(idx, 40, replace=False):
        k = int(k)
        if ln[k] == 0:
            continue
        ell = int(ln[k])
        for a in starts[off[k]:off[k + 1]]:
            a = int(a)
            assert a <= k <= a + ell - 1
            sub = s[a:a + ell]
            assert s.find(sub) != -1 and s.find(sub, s.find(sub) + 1) != -1
        for a in range(max(0, k - ell), min(k, n - ell - 1) + 1):
            sub = s[a:a + ell + 1]
            if len(sub) == ell + 1:
                first = s.find(sub)
                assert s.find(sub, first + 1) == -1


# ---------------------------------------------------------------- walk statistics (Table 2)

def test_walk_counts_match_definition():
    """alpha / beta per position against intervals built from the string alone."""
    rng = np.random.default_rng(77)
    for trial in range(120):
        n = int(rng.integers(1, 36))
        s = _random_string(rng, n)
        sa, rank, lcp = _prep(s)
        alpha, beta, m = oracle.walk_counts(rank, lcp)
        a2, b2 = definition.covering_counts(s)
        assert alpha.tolist() == a2, s
        assert beta.tolist() == b2, s
        assert m == len(oracle.compact(rank, lcp)[0])


@pytest.mark.parametrize("n", [1, 2, 7, 300])
def test_walk_counts_closed_forms(n):
    # a^n (n >= 2): LLR_0 = S[0..n-2] and, for i >= 1, LLR_i = S[i..n-1] (the
    # whole suffix recurs one position to the left); the useful ones are
    # LLR_0 and LLR_1
    sa, rank, lcp = _prep(b"a" * n)
    alpha, beta, m = oracle.walk_counts(rank, lcp)
    if n == 1:
        want_a, want_b, want_m = [0], [0], 0
    else:
        want_a = [1] + [k + 1 for k in range(1, n - 1)] + [n - 1]
        want_b = [1] + [2] * (n - 2) + [1]
        want_m = 2
    assert alpha.tolist() == want_a and beta.tolist() == want_b
    assert m == want_m
    # all symbols distinct: no repeat, no LLR
    s = bytes(range(1, min(n, 250) + 1))
    sa, rank, lcp = _prep(s)
    alpha, beta, m = oracle.walk_counts(rank, lcp)
    assert not alpha.any() and not beta.any() and m == 0


@pytest.mark.parametrize("name,n", [("dna_64m", 1 << 16), ("english_256m", 1 << 16)])
def test_walk_count_sums(name, n):
    """Every LLR covers exactly its length in positions: sum(alpha) = sum of
    |LLR_i|, sum(beta) = sum of the compact lengths."""
    w = W.single(name, n=n)
    alpha, beta, m = oracle.walk_counts(w.rank, w.lcp)
    L = oracle.llr_raw(w.rank, w.lcp)
    cs, cl = oracle.compact(w.rank, w.lcp)
    assert int(alpha.sum()) == int(L.astype(np.int64).sum())
    assert int(beta.sum()) == int(cl.astype(np.int64).sum())
    assert m == len(cs)
    assert np.all(beta <= alpha) and np.array_equal(beta == 0, alpha == 0)


# ---------------------------------------------------------------- the prep (SA, rank, lcp) itself

def test_prep_matches_naive_suffix_sort():
    """The host prep's sa / rank / lcp (the inputs every test feeds both
    sides, and the expected arrays of the GPU builder) against sorting the
    suffixes as byte strings and comparing neighbours symbol by symbol."""
    rng = np.random.default_rng(5)
    cases = [b"mississippi", b"a", b"aaaaaaa", b"\x00\x00\x01\x00\xff\xff\x00"]
    for _ in range(200):
        n = int(rng.integers(1, 80))
        sigma = int(rng.integers(1, 5))
        alphabet = rng.choice(256, size=sigma, replace=False)
        cases.append(bytes(alphabet[rng.integers(0, sigma, n)].astype(np.uint8)))
    for s in cases:
        sa, rank, lcp = W.prep(np.frombuffer(s, np.uint8))
        n = len(s)
        want_sa = sorted(range(n), key=lambda i: s[i:])
        assert sa.tolist() == want_sa, s
        assert np.array_equal(rank[sa], np.arange(n))
        want_lcp = [0] * (n + 1)
        for r in range(1, n):
            a, b = s[want_sa[r - 1]:], s[want_sa[r]:]
            m = 0
            while m < min(len(a), len(b)) and a[m] == b[m]:
                m += 1
            want_lcp[r] = m
        assert lcp.tolist() == want_lcp, s


def test_prep_many_matches_per_string_prep():
    """The batched prep (the input of every batched and serving test) is the
    per-string prep laid out back to back: string j's local sa and rank at
    off[j], its lcp (n_j + 1 entries) at off[j] + j; empty strings included."""
    rng = np.random.default_rng(6)
    lens = [0, 1, 5, 0, 300, 2, 1000, 0, 77, 3000, 1]
    pieces = [W.make_text("dna", m, 40 + j) if m >= 64 else rng.integers(97, 100, m).astype(np.uint8)
              for j, m in enumerate(lens)]
    off = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    text = np.concatenate(pieces).astype(np.uint8)
    sa, rank, lcp = W.prep_many(text, off)
    assert sa.size == text.size and lcp.size == text.size + len(lens)
    for j, m in enumerate(lens):
        a = int(off[j])
        if m == 0:
            assert lcp[a + j] == 0
            continue
        s1, r1, l1 = W.prep(text[a:a + m])
        assert np.array_equal(sa[a:a + m], s1) and np.array_equal(rank[a:a + m], r1)
        assert np.array_equal(lcp[a + j:a + j + m + 1], l1)


def test_lr_at_range_equals_the_full_run():
    """The block-parallel driver of Algorithm 3 (lr_at on disjoint blocks at
    once) gives the full run's CSR, for any split, and a sub-range's CSR."""
    w = W.single("english_256m", n=200_000)
    full = oracle.lr_all_raw(w.rank, w.lcp)
    for threads in (1, 3, 8):
        got = oracle.lr_at_range(w.rank, w.lcp, 0, w.n, threads=threads)
        for a, b in zip(got, full):
            assert np.array_equal(a, b)
    got = oracle.lr_at_range(w.rank, w.lcp, 1234, 5678, threads=4)
    ks = np.arange(1234, 5678)
    for a, b in zip(got, oracle.lr_at(w.rank, w.lcp, ks)):
        assert np.array_equal(a, b)
    empty = oracle.lr_at_range(w.rank, w.lcp, 10, 10, threads=4)
    assert empty[0].size == 0 and empty[2].tolist() == [0]
