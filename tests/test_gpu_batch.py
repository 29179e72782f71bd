"""Batched queries, the autotuner and captured plans on the GPU, against the oracle.

A batch is many strings packed back to back.  Its flattened result must be,
string by string, exactly what the oracle (Algorithm 3) gives for that string
alone, with positions shifted by the string's offset.  Bit-exact.
"""
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


def _expected(off, rank, lcp):
    """Oracle per string, flattened the way the batched query reports it."""
    lens, lstart, counts, starts = [], [], [], []
    for j in range(off.size - 1):
        a, b = int(off[j]), int(off[j + 1])
        if a == b:
            continue
        ln, st, offs, sts = oracle.lr_all_raw(rank[a:b], lcp[a + j:b + j + 1])
        lens.append(ln)
        lstart.append(np.where(st >= 0, st + a, st).astype(np.int32))
        counts.append(np.diff(offs))
        starts.append((sts + a).astype(np.int32))
    cat = lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt)
    c = cat(counts, np.int64)
    offsets = np.zeros(c.size + 1, np.int64)
    np.cumsum(c, out=offsets[1:])
    return cat(lens, np.int32), cat(lstart, np.int32), offsets, cat(starts, np.int32)


def _assert_equal(got, want, what=""):
    for name, a, b in zip(("lr_len", "lr_start", "offsets", "starts"), got, want):
        assert a.shape == b.shape, (what, name, a.shape, b.shape)
        if not np.array_equal(a, b):
            bad = np.nonzero(a != b)[0][:10]
            raise AssertionError("%s %s differs at %s: got %s want %s" % (what, name, bad, a[bad], b[bad]))


def _batch(text, off):
    sa, rank, lcp = W.prep_many(text, off)
    return sa, rank, lcp


def _run(ctx, off, sa, rank, lcp, front):
    kw = {"sa": _dev(sa)} if front == "sa" else {"rank": _dev(rank)}
    out = ctx.query_batch(_dev(off), _dev(lcp), **kw)
    return tuple(t.cpu().numpy() for t in out)


def _check(ctx, text, off, fronts=("sa", "rank")):
    sa, rank, lcp = _batch(text, off)
    want = _expected(off, rank, lcp)
    for front in fronts:
        _assert_equal(_run(ctx, off, sa, rank, lcp, front), want, front)
    return want


def _offsets(lens):
    off = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(np.asarray(lens, np.int64), out=off[1:])
    return off


def _random_text(rng, n, sigma):
    return rng.integers(0, sigma, n, dtype=np.uint8) + ord("a")


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_mix_with_empty_and_tiny_strings(ctx, seed):
    rng = np.random.default_rng(100 + seed)
    lens = rng.choice([0, 1, 2, 3, 7, 50, 300, 2047, 2048, 2049, 5000], size=200)
    lens[0] = 0
    lens[-1] = 0
    off = _offsets(lens)
    text = _random_text(rng, int(off[-1]), int(rng.integers(2, 5)))
    _check(ctx, text, off)


def test_more_strings_per_tile_than_staged(ctx):
    """Thousands of strings of length 0-3 per tile: the string lookup leaves shared memory."""
    rng = np.random.default_rng(7)
    lens = rng.integers(0, 4, size=30000)
    off = _offsets(lens)
    text = _random_text(rng, int(off[-1]), 2)
    _check(ctx, text, off)


def test_long_repeats_next_to_short_strings(ctx):
    """Strings whose LR's cross many cover tiles, packed between tiny ones."""
    parts = [b"ab", b"a" * 20000, b"x", (b"abcde" * 3000), b"", b"q" * 9000 + b"z", b"aa"]
    lens = [len(p) for p in parts]
    off = _offsets(lens)
    text = np.frombuffer(b"".join(parts), np.uint8).copy()
    _check(ctx, text, off)


def test_single_string_batch_matches_lr_query_all(ctx):
    w = W.single("dna_64m", n=300_000)
    off = np.array([0, w.n], np.int64)
    got = _run(ctx, off, w.sa, w.rank, w.lcp, "sa")
    single = tuple(t.cpu().numpy() for t in ctx.query_all(_dev(w.lcp), sa=_dev(w.sa)))
    _assert_equal(got, single, "batch of one")


def test_batched_mix_scaled(ctx):
    """The batched mix (log-uniform lengths, DNA and protein kinds), 96 strings up to 256 Ki."""
    text, off, _ = W.batched_mix(count=96, lo=1024, hi=256 * 1024, seed=11)
    _check(ctx, text, off)


def test_bad_offset_tables_are_reported(ctx):
    rng = np.random.default_rng(3)
    lens = [100, 200, 0, 300]
    off = _offsets(lens)
    text = _random_text(rng, int(off[-1]), 3)
    sa, rank, lcp = _batch(text, off)
    for bad in (np.array([0, 100, 300, 300, 650], np.int64),     # last offset past the total
                np.array([0, 250, 200, 300, 600], np.int64),     # decreasing
                np.array([5, 100, 300, 300, 600], np.int64)):    # does not start at 0
        d = P.batch_desc(_dev(bad), _dev(lcp), sa=_dev(sa))
        n = int(off[-1])
        outs = [torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.int32, device="cuda"),
                torch.empty(n + 1, dtype=torch.int64, device="cuda"),
                torch.empty(4 * n, dtype=torch.int32, device="cuda")]
        st, _ = P.lr_batch_query_all(ctx.handle, d, *outs)
        assert st == P.LR_ERR_SENTINEL, (bad, P.status_str(st))
    # the context still answers correctly afterwards
    _check(ctx, text, off, fronts=("sa",))


def test_broken_sentinels_in_bulk_rounds(ctx):
    """Strings that start on a partition round (4096 ranks) and fill whole
    rounds arrive by bulk copies; a string's first lcp entry that is not 0
    is caught there, and its last one in the round that ends the string."""
    rng = np.random.default_rng(31)
    lens = [8192, 5 * 4096 + 100, 3000]
    off = _offsets(lens)
    text = _random_text(rng, int(off[-1]), 4)
    sa, rank, lcp = _batch(text, off)
    n = int(off[-1])
    for where in (0, int(off[1]) + 1, int(off[2]) + 1):    # first of string 0, first and last of string 1
        bad = lcp.copy()
        bad[where] = 5
        for front in ("sa", "rank"):
            kw = {"sa": _dev(sa)} if front == "sa" else {"rank": _dev(rank)}
            d = P.batch_desc(_dev(off), _dev(bad), **kw)
            st, _ = P.lr_batch_query_all(ctx.handle, d, *_outs(n, 4 * n))
            assert st == P.LR_ERR_SENTINEL, (where, front, P.status_str(st))
    _check(ctx, text, off)


def test_invalid_batch_descriptors(ctx):
    z = torch.zeros(8, dtype=torch.int32, device="cuda")
    o = torch.zeros(8, dtype=torch.int64, device="cuda")
    outs = [z, z, o, z]
    d = P.BatchDesc(0, 5, P._ptr(o), P._ptr(z), None, P._ptr(z))      # num = 0
    assert P.lr_batch_query_all(ctx.handle, d, *outs)[0] == P.LR_ERR_ARG
    d = P.BatchDesc(1, 5, P._ptr(o), None, None, P._ptr(z))           # neither sa nor rank
    assert P.lr_batch_query_all(ctx.handle, d, *outs)[0] == P.LR_ERR_ARG
    d = P.BatchDesc(1, 0, P._ptr(o), P._ptr(z), None, P._ptr(z))      # empty total
    assert P.lr_batch_query_all(ctx.handle, d, *outs)[0] == P.LR_ERR_ARG


def _outs(n, cap):
    return (torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.int32, device="cuda"),
            torch.empty(n + 1, dtype=torch.int64, device="cuda"), torch.empty(cap, dtype=torch.int32, device="cuda"))


def test_autotune_choice_keeps_results_and_round_trips(ctx, tmp_path):
    text, off, _ = W.batched_mix(count=64, lo=1024, hi=128 * 1024, seed=12)
    sa, rank, lcp = _batch(text, off)
    want = _expected(off, rank, lcp)
    n = int(off[-1])
    d_off, d_sa, d_rank, d_lcp = _dev(off), _dev(sa), _dev(rank), _dev(lcp)
    desc = P.batch_desc(d_off, d_lcp, sa=d_sa, rank=d_rank)
    outs = _outs(n, 4 * n)
    code = P.lr_autotune(ctx.handle, desc, *outs)
    assert code in SHAPE_CODES
    # every shape gives the same answer: run the tuned one through the normal entry point
    got = ctx.query_batch(d_off, d_lcp, sa=d_sa, rank=d_rank)
    _assert_equal(tuple(t.cpu().numpy() for t in got), want, "tuned code %d" % code)
    path = str(tmp_path / "tuned.txt")
    P.lr_autotune_save(ctx.handle, path)
    lines = open(path).read().split()
    assert len(lines) >= 2 and int(lines[1]) == code
    other = P.Context(0)
    try:
        P.lr_autotune_load(other.handle, path)
        got = other.query_batch(d_off, d_lcp, sa=d_sa, rank=d_rank)
        _assert_equal(tuple(t.cpu().numpy() for t in got), want, "loaded choice")
    finally:
        other.close()


@pytest.mark.parametrize("front", ["sa", "rank"])
def test_plan_replays_and_follows_refilled_inputs(ctx, front):
    rng = np.random.default_rng(21)
    lens = rng.integers(0, 40000, size=40)
    off = _offsets(lens)
    n = int(off[-1])
    texts = [_random_text(rng, n, 2), _random_text(rng, n, 4)]
    prepped = [_batch(t, off) for t in texts]
    d_off = _dev(off)
    d_sa = torch.empty(n, dtype=torch.int32, device="cuda")
    d_rank = torch.empty(n, dtype=torch.int32, device="cuda")
    d_lcp = torch.empty(n + off.size - 1, dtype=torch.int32, device="cuda")
    desc = P.batch_desc(d_off, d_lcp, sa=d_sa if front == "sa" else None, rank=d_rank if front == "rank" else None)
    outs = _outs(n, 4 * n)
    plan = P.lr_plan_create(ctx.handle, desc, *outs)
    try:
        for rep in range(3):
            sa, rank, lcp = prepped[rep % 2]
            d_sa.copy_(torch.from_numpy(sa))
            d_rank.copy_(torch.from_numpy(rank))
            d_lcp.copy_(torch.from_numpy(lcp))
            P.lr_plan_launch(plan)
            st, total = P.lr_plan_result(plan)
            want = _expected(off, rank, lcp)
            assert st == P.LR_OK, P.status_str(st)
            assert total == int(want[2][-1])
            got = (outs[0].cpu().numpy(), outs[1].cpu().numpy(), outs[2].cpu().numpy(),
                   outs[3][:total].cpu().numpy())
            _assert_equal(got, want, "plan launch %d" % rep)
    finally:
        P.lr_plan_destroy(plan)


def test_plan_reports_capacity(ctx):
    text = np.frombuffer(b"ab" * 3000, np.uint8).copy()
    off = np.array([0, 2000, 6000], np.int64)
    sa, rank, lcp = _batch(text, off)
    want = _expected(off, rank, lcp)
    total = int(want[2][-1])
    desc = P.batch_desc(_dev(off), _dev(lcp), sa=_dev(sa))
    outs = _outs(6000, max(1, total // 2))
    plan = P.lr_plan_create(ctx.handle, desc, *outs)
    try:
        P.lr_plan_launch(plan)
        st, got_total = P.lr_plan_result(plan)
        assert st == P.LR_ERR_CAPACITY and got_total == total
        assert np.array_equal(outs[2].cpu().numpy(), want[2])
    finally:
        P.lr_plan_destroy(plan)


SHAPE_CODES = [0, 2, 8, 9, 12, 10, 11, 14]


@pytest.mark.parametrize("code", SHAPE_CODES)
def test_every_shape_code_matches_the_oracle(ctx, code, tmp_path):
    """Each shape the autotuner can pick (warp-segment cover, or tile cover
    with tiles of 2048 / 4096 / 8192, either front end) gives the oracle's
    answer, single string and batch."""
    w = W.single("dna_64m", n=700_000)
    text, off, _ = W.batched_mix(count=24, lo=1024, hi=64 * 1024, seed=13)
    sa_b, rank_b, lcp_b = _batch(text, off)
    lg = lambda v: int(v).bit_length() - 1
    classes = [lg(w.n) * 64 + lg(w.n), lg(off[-1]) * 64 + lg(int(off[-1]) // (off.size - 1))]
    path = tmp_path / "codes.txt"
    path.write_text("".join("%d %d\n" % (c, code) for c in classes))
    c = P.Context(0)
    try:
        P.lr_autotune_load(c.handle, str(path))
        got = tuple(t.cpu().numpy() for t in c.query_all(_dev(w.lcp), sa=_dev(w.sa), rank=_dev(w.rank)))
        _assert_equal(got, oracle.lr_all_raw(w.rank, w.lcp), "single, code %d" % code)
        got = tuple(t.cpu().numpy() for t in c.query_batch(_dev(off), _dev(lcp_b), sa=_dev(sa_b), rank=_dev(rank_b)))
        _assert_equal(got, _expected(off, rank_b, lcp_b), "batch, code %d" % code)
    finally:
        c.close()


def _dense_compact_text(seed, front, w=40):
    """A random ACGT string R of 3 x 8192 + 200 symbols, then every length-w
    window of R followed by '#', with `front` random bytes before R.  Every
    position of R (but its last w) has L = w (the window copy repeats it and
    the '#' ends the repeat), so it is a compact LLR: whole 8192-position
    cover tiles consist of compact LLR's, plus w - 1 carried from the tile
    before, and the staged window indices run past 8191."""
    rng = np.random.default_rng(seed)
    R = np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, 3 * 8192 + 200)]
    win = np.lib.stride_tricks.sliding_window_view(R, w)
    tail = np.concatenate([win, np.full((win.shape[0], 1), ord("#"), np.uint8)], axis=1).reshape(-1)
    head = rng.integers(0, 256, front).astype(np.uint8)
    return np.concatenate([head, R, tail])


@pytest.mark.parametrize("code", SHAPE_CODES)
def test_every_shape_code_on_tiles_of_compact_llrs(ctx, code, tmp_path):
    """Each shape code on an input whose cover tiles consist entirely of
    compact LLR's (the packed holder index of a staged 8192-position tile
    then needs 14 bits), with the tile grid at two offsets into the dense
    region; single string and batch (the dense string between two others)."""
    lg = lambda v: int(v).bit_length() - 1
    c = P.Context(0)
    try:
        for front in (0, 100):
            text = _dense_compact_text(21, front)
            sa, rank, lcp = W.prep(text)
            rng = np.random.default_rng(5 + front)
            btext = np.concatenate([_random_text(rng, 300, 4), text, _random_text(rng, 5000, 3)])
            off = _offsets([300, text.size, 5000])
            sa_b, rank_b, lcp_b = _batch(btext, off)
            classes = [lg(text.size) * 64 + lg(text.size), lg(off[-1]) * 64 + lg(int(off[-1]) // 3)]
            path = tmp_path / ("codes%d.txt" % front)
            path.write_text("".join("%d %d\n" % (cl, code) for cl in classes))
            P.lr_autotune_load(c.handle, str(path))
            got = tuple(t.cpu().numpy() for t in c.query_all(_dev(lcp), sa=_dev(sa), rank=_dev(rank)))
            _assert_equal(got, oracle.lr_all_raw(rank, lcp), "single, code %d, front %d" % (code, front))
            got = tuple(t.cpu().numpy() for t in
                        c.query_batch(_dev(off), _dev(lcp_b), sa=_dev(sa_b), rank=_dev(rank_b)))
            _assert_equal(got, _expected(off, rank_b, lcp_b), "batch, code %d, front %d" % (code, front))
    finally:
        c.close()
