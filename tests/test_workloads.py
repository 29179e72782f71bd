"""The seeded input generators against the recipes the benchmark's inputs
are stated with (alphabets, English word and separator laws, planted
repeats, the length laws of the batched and serving mixes), and their
determinism.  CPU only."""
import numpy as np

import workloads as W


def test_dna_iid_is_uniform_acgt():
    t = W.dna_iid(1 << 20, 1)
    vals, cnt = np.unique(t, return_counts=True)
    assert bytes(vals.astype(np.uint8)) == b"ACGT"
    assert np.all(np.abs(cnt / t.size - 0.25) < 0.005)


def test_protein_alphabet():
    t = W.protein_tandem(1 << 18, 8)
    assert set(np.unique(t).tolist()) <= set(b"ACDEFGHIKLMNPQRSTVWY")
    assert len(np.unique(t)) == 20


def test_english_recipe():
    t = W.english(1 << 21, 3)
    vals = set(np.unique(t).tolist())
    assert vals <= set(range(32, 127)) | {10} and len(vals) <= 96
    s = t.tobytes()
    words = [w for w in s.replace(b"\n", b" ").split(b" ") if w]
    # a word is a-z only, 2..12 letters; a non-letter symbol is its own token
    letters = [w.rstrip(bytes(range(33, 97)) + bytes(range(123, 127))) for w in words[:-1]]
    lens = np.array([len(w) for w in letters if w.isalpha()])
    assert lens.min() >= 2 and lens.max() <= 12
    # separators after a word: newline 1 %, a space 85 %, a symbol then a space 14 %
    nl = s.count(b"\n")
    sym = sum(1 for c in s if 33 <= c <= 126 and not (97 <= c <= 122))
    seps = nl + sym + s.count(b" ") - sym                     # every symbol is followed by a space
    assert abs(nl / seps - 0.01) < 0.002 and abs(sym / seps - 0.14) < 0.01
    # Zipf(1.1) over the vocabulary: frequency falls about 10^1.1 from rank 1 to rank 10
    _, cnt = np.unique(np.array(letters, dtype=object), return_counts=True)
    top = np.sort(cnt)[::-1]
    assert 6 < top[0] / top[9] < 25


def test_dna_planted_repeats():
    t = W.dna_planted(1 << 20, 2)
    assert set(np.unique(t).tolist()) <= set(b"ACGT")
    _, _, lcp = W.prep(t)
    m = np.maximum(lcp[:-1], lcp[1:])
    # long exact repeats come only from the planted copies (i.i.d. DNA of
    # 1 Mi symbols has none of 40 or more); copies mutated at up to 10 %
    # break into shorter exact runs, lightly mutated ones keep long runs
    assert np.mean(m >= 40) > 0.05 and m.max() >= 300
    assert np.mean(W.prep(W.dna_iid(1 << 20, 3))[2] >= 40) == 0


def test_length_laws():
    ln = W.lengths_lognormal(40000, 1e5, 1.0, 1024, 16 << 20, 5)
    assert ln.min() >= 1024 and ln.max() <= 16 << 20
    assert abs(np.median(ln) / 1e5 - 1) < 0.03
    assert abs(np.std(np.log(ln)) - 1.0) < 0.03
    lu = W.lengths_loguniform(40000, 1024, 4 << 20, 4)
    assert lu.min() >= 1024 and lu.max() <= 4 << 20
    lo, hi = np.log(1024), np.log(4 << 20)
    assert abs(np.mean(np.log(lu)) - (lo + hi) / 2) < 0.05 * (hi - lo)
    assert abs(np.mean(np.log(lu) < (lo + hi) / 2) - 0.5) < 0.02


def test_generators_are_seeded():
    for kind in ("dna_iid", "dna", "english", "protein"):
        a, b, c = W.make_text(kind, 50000, 7), W.make_text(kind, 50000, 7), W.make_text(kind, 50000, 8)
        assert np.array_equal(a, b) and not np.array_equal(a, c), kind
