"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle.

Integer and index work: every comparison is bit-exact.  Every input,
the full-size workloads included, is compared in full (Algorithm 3 per
position at the largest sizes), plus properties that hold at any size.
"""
import os

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
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


FRONTS = ("sa", "rank")        # rank-order front end (suffix array given); rank alone (rank gather, or rank windows from 2^24 positions on)


def _gpu_all(ctx, sa, rank, lcp, front="sa"):
    if front == "sa":
        out = ctx.query_all(_dev(lcp), sa=_dev(sa))
    else:
        out = ctx.query_all(_dev(lcp), rank=_dev(rank))
    return tuple(t.cpu().numpy() for t in out)


def _assert_csr_equal(got, want, what=""):
    names = ("lr_len", "lr_start", "offsets", "starts")
    for name, a, b in zip(names, got, want):
        assert a.shape == b.shape, (what, name, a.shape, b.shape)
        if not np.array_equal(a, b):
            bad = np.nonzero(a != b)[0][:10]
            raise AssertionError("%s %s differs at %s: got %s want %s" % (what, name, bad, a[bad], b[bad]))


def _full_check(ctx, text):
    sa, rank, lcp = W.prep(text)
    want = oracle.lr_all_raw(rank, lcp)
    for front in FRONTS:
        got = _gpu_all(ctx, sa, rank, lcp, front)
        _assert_csr_equal(got, want, "n=%d front=%s" % (text.size, front))
        kw = {"sa": _dev(sa)} if front == "sa" else {"rank": _dev(rank)}
        st, ln = ctx.query_leftmost(_dev(lcp), **kw)
        assert np.array_equal(st.cpu().numpy(), want[1]) and np.array_equal(ln.cpu().numpy(), want[0])


def _sampled_check(ctx, w, got, nsamples, seed):
    """Sampled positions against Algorithm 3, plus size-independent properties."""
    ln, st, off, starts = got
    n = w.n
    rng = np.random.default_rng(seed)
    ks = np.unique(np.concatenate([rng.integers(0, n, nsamples), [0, 1, n - 2, n - 1],
                                   np.arange(2040, 2060), np.arange(n - 2100, n - 2000)]))
    ks = ks[(ks >= 0) & (ks < n)]
    wl, ws, wo, wst = oracle.lr_at(w.rank, w.lcp, ks)
    for q, k in enumerate(ks):
        assert ln[k] == wl[q] and st[k] == ws[q], (k, ln[k], wl[q], st[k], ws[q])
        assert np.array_equal(starts[off[k]:off[k + 1]], wst[wo[q]:wo[q + 1]]), k
    # properties at every position
    assert off[0] == 0 and off[n] == starts.size and np.all(np.diff(off) >= 0)
    cnt = np.diff(off)
    assert np.array_equal(cnt == 0, ln == 0) and np.all(st[ln == 0] == -1)
    has = ln > 0
    assert np.array_equal(st[has], starts[off[:-1][has]])
    counts = np.bincount(w.text, minlength=256)
    assert np.array_equal(ln == 0, counts[w.text] == 1)         # Lemma 1: none iff singleton


# ------------------------------------------------------------------ small inputs

def test_paper_examples(ctx):
    for s in (b"mississippi", b"abcabcddbca", b"ababab", b"aaaa", b"a", b"ab", b"abcd", b"aa"):
        _full_check(ctx, np.frombuffer(s, np.uint8))


def test_random_small_strings(ctx):
    import tests.test_oracle as T
    rng = np.random.default_rng(99)
    for trial in range(150):
        n = int(rng.integers(1, 300)) if trial < 100 else int(rng.integers(300, 6000))
        _full_check(ctx, np.frombuffer(T._random_string(rng, n), np.uint8))


@pytest.mark.parametrize("n", [31, 32, 33, 2047, 2048, 2049, 4095, 4096, 4097, 6143, 10240, 65536 + 7])
def test_tile_boundaries(ctx, n):
    for kind, seed in (("dna_iid", 5), ("dna", 6), ("english", 7), ("protein", 8)):
        _full_check(ctx, W.make_text(kind, n, seed))


def test_degenerate_strings(ctx):
    _full_check(ctx, np.full(5000, ord("a"), np.uint8))                  # one symbol
    _full_check(ctx, np.arange(256, dtype=np.uint8))                       # all singletons
    _full_check(ctx, np.frombuffer(b"ab" * 3000, np.uint8))                # period 2
    _full_check(ctx, np.frombuffer((b"abcdefghij" * 700)[:6999], np.uint8))


def test_long_repeats_cross_many_tiles(ctx):
    rng = np.random.default_rng(3)
    base = rng.integers(65, 69, 200_000).astype(np.uint8)
    base[150_000:190_000] = base[10_000:50_000]                              # a 40k copy
    base[100_000:100_300] = base[60_000:60_300]
    _full_check(ctx, base)


def test_wide_windows_spill_to_global(ctx):
    """beta(k) > the shared-memory window: W candidates of equal length cover one position."""
    rng = np.random.default_rng(4)
    Wn = 4400
    R = rng.integers(65, 69, 2 * Wn + 2).astype(np.uint8)
    parts = [R]
    for j in range(Wn):
        parts.append(R[j:j + Wn + 1])
        parts.append(np.array([ord("#")], np.uint8))
    text = np.concatenate(parts)
    w = W.Workload("wide", text, *W.prep(text))
    ks = np.arange(Wn - 50, Wn + 50)
    wl, ws, wo, wst = oracle.lr_at(w.rank, w.lcp, ks)
    assert int(np.diff(wo).max()) > 4096                      # wider than the staged window
    for front in FRONTS:
        got = _gpu_all(ctx, w.sa, w.rank, w.lcp, front)
        _sampled_check(ctx, w, got, 3000, 5)
        for q, k in enumerate(ks):
            assert np.array_equal(got[3][got[2][k]:got[2][k + 1]], wst[wo[q]:wo[q + 1]])


# ------------------------------------------------------------------ workloads

@pytest.mark.parametrize("front", FRONTS)
def test_dna_iid_1m_full(ctx, front):
    w = W.single("dna_iid_1m")
    _assert_csr_equal(_gpu_all(ctx, w.sa, w.rank, w.lcp, front), oracle.lr_all_raw(w.rank, w.lcp), w.name)


@pytest.mark.parametrize("front", FRONTS)
def test_binary_iid_full(ctx, front):
    """Binary i.i.d. text: nearly every position starts a useful LLR and
    windows are wide, so runs of 32 positions often span more than 32 compact
    LLR's (the cover's looped path) and ties are frequent and spread."""
    text = W.iid(1 << 24, b"ab", 77)
    sa, rank, lcp = W.prep(text)
    want = oracle.lr_all_raw(rank, lcp)
    _assert_csr_equal(_gpu_all(ctx, sa, rank, lcp, front), want, "binary iid")
    # some positions have holders 18 or more compact LLR's apart (the cover
    # then lists them by walking the window instead of from a bit mask)
    _, _, off, starts = want
    cs, _ = oracle.compact(rank, lcp)
    multi = np.nonzero(np.diff(off) > 1)[0]
    span = np.searchsorted(cs, starts[off[multi + 1] - 1]) - np.searchsorted(cs, starts[off[multi]])
    assert int(span.max()) >= 18


@pytest.mark.parametrize("front", FRONTS)
def test_dna_planted_4m_full(ctx, front):
    w = W.single("dna_64m", n=4 * W.MI)
    _assert_csr_equal(_gpu_all(ctx, w.sa, w.rank, w.lcp, front), oracle.lr_all_raw(w.rank, w.lcp), w.name)


@pytest.mark.parametrize("front", FRONTS)
def test_english_4m_full(ctx, front):
    w = W.single("english_256m", n=4 * W.MI)
    _assert_csr_equal(_gpu_all(ctx, w.sa, w.rank, w.lcp, front), oracle.lr_all_raw(w.rank, w.lcp), w.name)


def test_multi_bucket_sizes(ctx):
    """Sizes around the 65536-position buckets of the rank-order front end."""
    for n in (65535, 65536, 65537, 3 * 65536 + 1):
        _full_check(ctx, W.make_text("dna", n, 11))


def test_long_lengths_escape_16_bits(ctx):
    """LLR lengths >= 65535 take the escape path of the packed partition entries."""
    rng = np.random.default_rng(12)
    base = rng.integers(65, 69, 300_000).astype(np.uint8)
    base[200_000:280_000] = base[20_000:100_000]                  # an 80k exact copy
    _full_check(ctx, base)


@pytest.mark.parametrize("name", ["dna_64m", "english_256m"])
def test_full_size_exact(ctx, name, tmp_path):
    """Every position of the full-size workloads (64 Mi planted-repeat DNA,
    256 Mi english) against Algorithm 3, run on all host cores over disjoint
    blocks of positions: the all-LR query with both front ends, the
    leftmost-only query and the raw-LLR variant; plus the size-independent
    properties, and the autotuner's other kernel shapes."""
    w = W.single(name)
    got = _gpu_all(ctx, w.sa, w.rank, w.lcp, "sa")
    want = oracle.lr_at_range(w.rank, w.lcp, 0, w.n, threads=os.cpu_count() or 1)
    _assert_csr_equal(got, want, name)
    # the leftmost-only query (Algorithm 2's output) and the raw-LLR variant
    # (Algorithms 1 and 3, no compaction) against the same oracle run
    st, ln = ctx.query_leftmost(_dev(w.lcp), sa=_dev(w.sa))
    assert np.array_equal(ln.cpu().numpy(), want[0]) and np.array_equal(st.cpu().numpy(), want[1])
    del st, ln
    raw = tuple(t.cpu().numpy() for t in ctx.query_all_raw(_dev(w.lcp), _dev(w.rank)))
    _assert_csr_equal(raw, want, name + " raw")
    del want, raw
    _sampled_check(ctx, w, got, 200, 17)
    got2 = _gpu_all(ctx, w.sa, w.rank, w.lcp, "rank")
    for a, b in zip(got, got2):
        assert np.array_equal(a, b)
    del got2
    # the other shapes the autotuner can pick at this size (warp-segment
    # cover; tile cover with 2048- or 8192-position tiles; the warp-segment
    # cover behind the rank gather), forced through an autotune table
    lg = w.n.bit_length() - 1
    for code in (0, 8, 12, 2):
        path = tmp_path / ("codes%d.txt" % code)
        path.write_text("%d %d\n" % (lg * 64 + lg, code))
        c = P.Context(0)
        try:
            P.lr_autotune_load(c.handle, str(path))
            got3 = tuple(t.cpu().numpy() for t in c.query_all(_dev(w.lcp), sa=_dev(w.sa), rank=_dev(w.rank)))
        finally:
            c.close()
        _assert_csr_equal(got3, got, "%s, shape code %d" % (name, code))
        del got3


def test_513_super_buckets(ctx):
    """n = 2^29 + 12345 planted-repeat DNA: the first partition level spreads
    the rank-order entries over 513 super-buckets of 2^20 positions, the last
    of them (and its last bucket of 2^15) ragged.  Every position against
    Algorithm 3, then the rank-window front end against that result."""
    n = (1 << 29) + 12345
    free, _ = torch.cuda.mem_get_info()
    if free < n * 64:
        pytest.skip("needs %.0f GB free" % (n * 64 / 1e9))
    text = W.make_text("dna", n, 21)
    sa, rank, lcp = W.prep(text)
    del text
    got = _gpu_all(ctx, sa, rank, lcp, "sa")
    want = oracle.lr_at_range(rank, lcp, 0, n, threads=os.cpu_count() or 1)
    _assert_csr_equal(got, want, "n = 2^29 + 12345")
    del want
    # rank alone: the rank-window front end over 129 windows of 2^22 ranks, the last ragged
    _assert_csr_equal(_gpu_all(ctx, sa, rank, lcp, "rank"), got, "n = 2^29 + 12345, rank windows")



def test_maximum_size_batch_closed_form(ctx):
    """A batch of three strings a^m whose total is 2^31 - 2, the largest the
    ABI takes, with string boundaries inside partition rounds (the batched
    rank-order front end then copies lcp slices from unaligned starts and
    has 2048 super-buckets).  String j of length m at offset o: every length
    is m - 1 (all beyond the partition entries' length fields and the
    cover's staged key range), LR_k = {o} at k = 0, {o, o + 1} inside and
    {o + 1} at k = m - 1; the total exceeds 2^32."""
    total = 2**31 - 2
    ms = [(1 << 30) + 4099, (1 << 29) + 3]
    ms.append(total - sum(ms))
    free, _ = torch.cuda.mem_get_info()
    need = total * (4 + 4 + 4 + 4 + 8 + 8 + 16 + 8) + (1 << 30)
    if free < need:
        pytest.skip("needs %.0f GB free" % (need / 1e9))
    off = np.zeros(len(ms) + 1, np.int64)
    np.cumsum(ms, out=off[1:])
    sa = torch.empty(total, dtype=torch.int32, device="cuda")
    lcp = torch.empty(total + len(ms), dtype=torch.int32, device="cuda")
    for j, m in enumerate(ms):
        o = int(off[j])
        sa[o:o + m] = torch.arange(m - 1, -1, -1, dtype=torch.int32, device="cuda")
        lcp[o + j:o + j + m + 1] = torch.arange(0, m + 1, dtype=torch.int32, device="cuda")
        lcp[o + j + m] = 0
    ln, st, offs, starts = ctx.query_batch(_dev(off), lcp, sa=sa, capacity=2 * total)
    del sa, lcp
    assert int(offs[total]) == sum(2 * m - 2 for m in ms) == starts.numel()
    step = 1 << 28
    base = 0
    for j, m in enumerate(ms):
        o = int(off[j])
        assert bool((ln[o:o + m] == m - 1).all()), j
        assert bool((st[o:o + m - 1] == o).all()) and int(st[o + m - 1]) == o + 1, j
        for a in range(0, m, step):                    # offsets: base + (0, 1, 3, 5, ..., 2m - 3)
            k = torch.arange(a, min(a + step, m), dtype=torch.int64, device="cuda")
            want = base + torch.where(k == 0, 0, 2 * k - 1)
            assert bool((offs[o + a:o + a + k.numel()] == want).all()), j
        del k, want
        sj = starts[base:base + 2 * m - 2]
        assert int(sj[0]) == o and int(sj[-1]) == o + 1, j
        pair = torch.tensor([o, o + 1], dtype=torch.int32, device="cuda")
        assert bool((sj[1:-1].view(-1, 2) == pair).all()), j
        base += 2 * m - 2


# ------------------------------------------------------------------ API behaviour

def test_capacity_error_keeps_offsets(ctx):
    w = W.single("dna_64m", n=100_000)
    want = oracle.lr_all_raw(w.rank, w.lcp)
    sa, lcp = _dev(w.sa), _dev(w.lcp)
    n = w.n
    ln = torch.empty(n, dtype=torch.int32, device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    small = torch.full((1000,), -7, dtype=torch.int32, device="cuda")
    status, total = P.lr_query_all(ctx.handle, sa, None, lcp, ln, st, off, small)
    assert status == P.LR_ERR_CAPACITY and total == want[3].size
    assert np.array_equal(off.cpu().numpy(), want[2]) and np.array_equal(ln.cpu().numpy(), want[0])
    assert np.array_equal(small.cpu().numpy(), want[3][:1000])


def test_host_buffer_entry_point(ctx):
    w = W.single("english_256m", n=300_000)
    want = oracle.lr_all_raw(w.rank, w.lcp)
    n = w.n
    ln = np.empty(n, np.int32)
    st = np.empty(n, np.int32)
    off = np.empty(n + 1, np.int64)
    starts = np.empty(2 * n, np.int32)
    for sa, rank in ((w.sa, None), (None, w.rank)):
        status, total = P.lr_query_all_host(ctx.handle, sa, rank, w.lcp, ln, st, off, starts)
        assert status == P.LR_OK
        _assert_csr_equal((ln, st, off, starts[:total]), want, "host")


def test_invalid_arguments(ctx):
    t = torch.zeros(4, dtype=torch.int32, device="cuda")
    lib = P.load()
    import ctypes
    null = ctypes.c_void_p(0)
    tot = ctypes.c_int64()
    s = P._stream(None)
    T = P._ptr(t)
    for n in (0, -5, 2**31 - 1):
        assert lib.lr_query_all(ctx.handle, s, T, null, T, n, T, T, T, T, 4, ctypes.byref(tot)) == P.LR_ERR_ARG
    assert lib.lr_query_all(ctx.handle, s, null, null, T, 3, T, T, T, T, 4, ctypes.byref(tot)) == P.LR_ERR_ARG
    assert lib.lr_query_leftmost(ctx.handle, s, null, T, null, 3, T, T) == P.LR_ERR_ARG


def test_bad_sentinel_and_rank_are_reported(ctx):
    w = W.single("dna_iid_1m", n=5000)
    lcp = w.lcp.copy()
    lcp[0] = 3
    for kw in ({"sa": _dev(w.sa)}, {"rank": _dev(w.rank)}):
        with pytest.raises(P.LRError) as e:
            ctx.query_all(_dev(lcp), **kw)
        assert e.value.status == P.LR_ERR_SENTINEL
    rank = w.rank.copy()
    rank[17] = w.n + 100                                       # out of range: clamped, reported
    with pytest.raises(P.LRError) as e:
        ctx.query_all(_dev(w.lcp), rank=_dev(rank))
    assert e.value.status == P.LR_ERR_SENTINEL
    sa = w.sa.copy()
    sa[17] = sa[18]                                            # not a permutation: detected, reported
    with pytest.raises(P.LRError) as e:
        ctx.query_all(_dev(w.lcp), sa=_dev(sa))
    assert e.value.status == P.LR_ERR_SENTINEL
    sa[17] = -4                                                # out of range
    with pytest.raises(P.LRError) as e:
        ctx.query_all(_dev(w.lcp), sa=_dev(sa))
    assert e.value.status == P.LR_ERR_SENTINEL
    # the context stays usable
    for front in FRONTS:
        _assert_csr_equal(_gpu_all(ctx, w.sa, w.rank, w.lcp, front), oracle.lr_all_raw(w.rank, w.lcp))


def test_bad_rank_in_the_rank_window_front(ctx):
    """Rank alone for one string of 2^24 positions or more goes through the
    rank-window front end; a rank that is out of range, a rank given twice
    and a broken lcp sentinel are reported there, and the context stays
    usable."""
    w = W.single("english_256m", n=(1 << 24) + 5)
    for what in ("range", "twice", "sentinel"):
        rank, lcp = w.rank.copy(), w.lcp
        if what == "range":
            rank[17] = w.n + 100
        elif what == "twice":
            rank[17] = rank[(1 << 23) + 3]
        else:
            lcp = w.lcp.copy()
            lcp[w.n] = 2
        with pytest.raises(P.LRError) as e:
            ctx.query_all(_dev(lcp), rank=_dev(rank))
        assert e.value.status == P.LR_ERR_SENTINEL, what
    got = _gpu_all(ctx, w.sa, w.rank, w.lcp, "rank")
    _assert_csr_equal(got, _gpu_all(ctx, w.sa, w.rank, w.lcp, "sa"), "after the errors")
    _sampled_check(ctx, w, got, 200, 23)
    # the leftmost-only query through the same front end
    st, ln = ctx.query_leftmost(_dev(w.lcp), rank=_dev(w.rank))
    assert np.array_equal(ln.cpu().numpy(), got[0]) and np.array_equal(st.cpu().numpy(), got[1])
    # and the host-buffer entry point with rank alone
    n = w.n
    h = (np.empty(n, np.int32), np.empty(n, np.int32), np.empty(n + 1, np.int64), np.empty(got[3].size + 8, np.int32))
    status, total = P.lr_query_all_host(ctx.handle, None, w.rank, w.lcp, *h)
    assert status == P.LR_OK
    _assert_csr_equal((h[0], h[1], h[2], h[3][:total]), got, "host buffers, rank windows")


@pytest.mark.parametrize("front", FRONTS)
def test_maximum_size_closed_form(ctx, front):
    """S = a^n with n = 2^31 - 2, the largest n the ABI takes, through the
    rank-order front end and through rank alone (the rank-window front end,
    512 windows of 2^22 ranks, the last of them partial).

    sa[r] = n-1-r, rank[i] = n-1-i, lcp = [0, 1, ..., n-1, 0]; so L_0 = n-1
    and L_i = n-i (all beyond the 16-bit length field of the partition
    entries), only <0, n-1> and <1, n-1> are useful, and LR_k is {0} for
    k = 0, {0, 1} for 0 < k < n-1 and {1} for k = n-1, all of length n-1.
    The total (2n - 2) exceeds 2^31, exercising the int64 offsets.
    """
    free, _ = torch.cuda.mem_get_info()
    n = 2**31 - 2
    need = n * (4 + 4 + 4 + 4 + 8 + 8 + 16 + 8) + (1 << 30)
    if free < need:
        pytest.skip("needs %.0f GB free" % (need / 1e9))
    sa = torch.arange(n - 1, -1, -1, dtype=torch.int32, device="cuda")     # rank is the same array
    lcp = torch.arange(0, n + 1, dtype=torch.int32, device="cuda")
    lcp[n] = 0
    ln, st, off, starts = ctx.query_all(lcp, capacity=2 * n, **({"sa": sa} if front == "sa" else {"rank": sa}))
    del sa, lcp
    assert int(off[n]) == 2 * n - 2
    assert bool((ln == n - 1).all())
    assert bool((st[:n - 1] == 0).all()) and int(st[n - 1]) == 1
    step = 1 << 28
    for a in range(0, n + 1, step):                       # offsets in chunks: 0, 1, 3, 5, ..., 2n-3, 2n-2
        k = torch.arange(a, min(a + step, n + 1), dtype=torch.int64, device="cuda")
        want = torch.where(k == 0, 0, 2 * k - 1)
        want[k == n] = 2 * n - 2
        assert bool((off[a:a + k.numel()] == want).all())
    del k, want
    assert int(starts[0]) == 0 and int(starts[-1]) == 1
    assert bool((starts[1:-1].view(-1, 2) == torch.tensor([0, 1], dtype=torch.int32, device="cuda")).all())
