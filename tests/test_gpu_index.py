"""The GPU prefix-doubling build of sa / rank / lcp against the host prep
(itself pinned to a naive suffix sort in test_oracle.py).  Bit-exact."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1501_06663_gb300 as lrmod
    lrmod.build_library()
    c = lrmod.Context(0)
    yield c
    c.close()


def _check(ctx, text):
    text = np.array(text, dtype=np.uint8)              # a writable copy
    sa, rank, lcp = W.prep(text)
    got = [t.cpu().numpy() for t in ctx.build_arrays(torch.from_numpy(text).cuda())]
    for name, a, b in zip(("sa", "rank", "lcp"), got, (sa, rank, lcp)):
        assert a.shape == b.shape and np.array_equal(a, b), (name, len(text))


def test_small_and_special(ctx):
    for s in (b"mississippi", b"a", b"ab", b"abcabcddbca", b"\x00\x00\x01\x00\xff\xff\x00", b"ababababab"):
        _check(ctx, np.frombuffer(s, np.uint8))
    rng = np.random.default_rng(9)
    for _ in range(20):
        n = int(rng.integers(1, 5000))
        sigma = int(rng.integers(1, 6))
        _check(ctx, rng.integers(0, sigma, n).astype(np.uint8) * 51)


def test_alphabet_sizes(ctx):
    """Round-0 keys code the symbols that occur densely (more of them per key
    for a small alphabet): sizes at the code-width boundaries, all 256 byte
    values included, with a planted repeat so that later rounds run."""
    rng = np.random.default_rng(10)
    for sigma in (1, 2, 3, 4, 7, 8, 15, 16, 127, 128, 255, 256):
        syms = rng.permutation(256)[:sigma].astype(np.uint8)
        n = int(rng.integers(3000, 7000))
        text = syms[rng.integers(0, sigma, n)]
        text[:sigma] = syms                                  # every symbol occurs
        text[n // 2:n // 2 + 700] = text[300:1000]
        _check(ctx, text)


def test_long_repeats(ctx):
    """a^n and a long tandem need many doubling rounds."""
    _check(ctx, np.full(100000, 97, np.uint8))
    unit = np.frombuffer(b"abcdefghij" * 3 + b"k", np.uint8)
    _check(ctx, np.tile(unit, 3000))


@pytest.mark.parametrize("name,n", [("dna_iid_1m", None), ("dna_64m", 1 << 22), ("english_256m", 1 << 22)])
def test_workloads(ctx, name, n):
    kind, n0, seed = W.SINGLE[name]
    _check(ctx, W.make_text(kind, n or n0, seed))


def _check_batch(ctx, text, off):
    import paper_1501_06663_gb300 as lrmod
    text = np.array(text, dtype=np.uint8)
    sa, rank, lcp = W.prep_many(text, off)
    d_text = torch.from_numpy(text).cuda() if text.size else torch.empty(0, dtype=torch.uint8, device="cuda")
    got = [t.cpu().numpy() for t in ctx.build_arrays_batch(torch.from_numpy(off).cuda(), d_text)]
    for name, a, b in zip(("sa", "rank", "lcp"), got, (sa, rank, lcp)):
        assert a.shape == b.shape and np.array_equal(a, b), (name, len(off) - 1)


def test_batch_of_strings(ctx):
    rng = np.random.default_rng(21)
    lens = rng.choice([0, 1, 2, 5, 64, 1000, 3000], size=300)
    off = np.zeros(lens.size + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    text = (rng.integers(0, 3, int(off[-1])) + 97).astype(np.uint8)
    _check_batch(ctx, text, off)
    # thousands of tiny strings (the string index takes most of the round-0 key)
    lens = rng.integers(0, 4, size=40000)
    off = np.zeros(lens.size + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    _check_batch(ctx, (rng.integers(0, 2, int(off[-1])) + 97).astype(np.uint8), off)


def test_batch_of_workload_strings(ctx):
    text, off, _ = W.serving_mix(64, seed=31, median=20000, floor_len=64, cap=200000)
    _check_batch(ctx, text, off)
    _check_batch(ctx, np.zeros(0, np.uint8), np.zeros(3, np.int64))        # only empty strings


def test_bad_text_offsets_are_reported(ctx):
    import paper_1501_06663_gb300 as lrmod
    text = torch.from_numpy(np.frombuffer(b"abcabcabc", np.uint8).copy()).cuda()
    out = [torch.empty(9, dtype=torch.int32, device="cuda"), torch.empty(9, dtype=torch.int32, device="cuda"),
           torch.empty(12, dtype=torch.int32, device="cuda")]
    for bad in ([0, 5, 3, 9], [1, 3, 6, 9], [0, 3, 6, 10]):
        off = torch.tensor(bad, dtype=torch.int64, device="cuda")
        st, _ = lrmod.lr_batch_build_arrays(ctx.handle, off, text, *out)
        assert st == lrmod.LR_ERR_SENTINEL, bad
