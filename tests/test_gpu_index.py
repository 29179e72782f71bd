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


def test_long_repeats(ctx):
    """a^n and a long tandem need many doubling rounds."""
    _check(ctx, np.full(100000, 97, np.uint8))
    unit = np.frombuffer(b"abcdefghij" * 3 + b"k", np.uint8)
    _check(ctx, np.tile(unit, 3000))


@pytest.mark.parametrize("name,n", [("dna_iid_1m", None), ("dna_64m", 1 << 22), ("english_256m", 1 << 22)])
def test_workloads(ctx, name, n):
    kind, n0, seed = W.SINGLE[name]
    _check(ctx, W.make_text(kind, n or n0, seed))
