"""Mutation check of the oracle's pins (no GPU).

Each case plants one plausible mistake in a copy of the C oracle (a dropped
term, a wrong comparison, an off-by-one index, a reversed order), builds it
on the CPU, and asserts that the pins of test_oracle.py reject it: the paper's
printed examples, the literal definition and the string-only brute force.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import definition

SRC = os.path.join(os.path.dirname(oracle.__file__), "lr_oracle.c")

MUTANTS = [
    ("lemma1 drops the successor lcp", "int32_t a = lcp[rank[i]], b = lcp[rank[i] + 1];",
     "int32_t a = lcp[rank[i]], b = lcp[rank[i]];"),
    ("lemma1 min instead of max", "return a > b ? a : b;", "return a < b ? a : b;"),
    ("walk break off by one", "if (i + llrr[i] - 1 < k) break;\n            else if (llrr[i] >= best_len)",
     "if (i + llrr[i] < k) break;\n            else if (llrr[i] >= best_len)"),
    ("alg1 tie keeps the rightmost", "else if (llrr[i] >= best_len)", "else if (llrr[i] > best_len)"),
    ("alg3 second walk break off by one", "if (i + llrr[i] - 1 < k) break;\n                else if (llrr[i] == length)",
     "if (i + llrr[i] - 2 < k) break;\n                else if (llrr[i] == length)"),
    ("alg3 keeps descending order", "for (int64_t a = first; a < hi; ++a, --hi) {\n                int32_t t = starts[a]; starts[a] = starts[hi]; starts[hi] = t;\n            }\n        }\n        lr_len[k] = length;\n        lr_start[k] = (length > 0 && first < cap) ? starts[first] : -1;\n        offsets[k + 1] = total;\n    }\n    free(llrr);",
     "(void)hi;\n        }\n        lr_len[k] = length;\n        lr_start[k] = (length > 0 && first < cap) ? starts[first] : -1;\n        offsets[k + 1] = total;\n    }\n    free(llrr);"),
    ("compaction keeps only strict growth", "if (L > 0 && L >= prev)", "if (L > 0 && L > prev)"),
    ("K1 flag strict", "flag[i] = llrr[i] > 0 && llrr[i] >= llrr[i - 1];", "flag[i] = llrr[i] > 0 && llrr[i] > llrr[i - 1];"),
    ("K3 scatter index off by one", "c_start[prefix[i] - 1] = (int32_t)i;", "c_start[prefix[i] - 1] = (int32_t)i + 1;"),
    ("binary search on end > k", "if ((int64_t)c_start[mid] + c_len[mid] - 1 >= k) hi = mid;",
     "if ((int64_t)c_start[mid] + c_len[mid] - 1 > k) hi = mid;"),
    ("compact walk stops on start < k", "if (!(cs[i] <= k && (int64_t)cs[i] + cl[i] - 1 >= k)) break;\n                else if (cl[i] > length) length",
     "if (!(cs[i] < k && (int64_t)cs[i] + cl[i] - 1 >= k)) break;\n                else if (cl[i] > length) length"),
    ("brute diagonal shifted", "run = (s[i] == s[i + d]) ? run + 1 : 0;", "run = (s[i] == s[i + d - 1]) ? run + 1 : 0;"),
    ("brute ignores the later suffix", "if (run > maxrep[i + d]) maxrep[i + d] = run;", "(void)0;"),
    ("alpha counts the breaking step", "if (i + llrr[i] - 1 < k) break;\n            ++a;",
     "if (i + llrr[i] - 1 < k) { ++a; break; }\n            ++a;"),
    ("beta walk stops one early", "if (!(cs[i] <= k && (int64_t)cs[i] + cl[i] - 1 >= k)) break;\n                ++b;",
     "if (!(cs[i] < k && (int64_t)cs[i] + cl[i] - 1 >= k)) break;\n                ++b;"),
    ("alg2 tie keeps the rightmost", "else if (cl[i] > best_len) { best_start = cs[i]; best_len = cl[i]; }",
     "else if (cl[i] >= best_len) { best_start = cs[i]; best_len = cl[i]; }"),
    ("compaction keeps empty LLR's", "if (L > 0 && L >= prev)", "if (L >= prev)"),
    # the per-position Algorithm 3 used for sampled checks at full size
    ("sampled walk break off by one",
     "        for (int64_t i = k; i >= 0; --i) {\n            int32_t L = llr_len(rank, lcp, i);\n"
     "            if (i + L - 1 < k) break;\n            else if (L >= length) length = L;\n        }",
     "        for (int64_t i = k; i >= 0; --i) {\n            int32_t L = llr_len(rank, lcp, i);\n"
     "            if (i + L < k) break;\n            else if (L >= length) length = L;\n        }"),
    ("sampled walk keeps descending order",
     "            for (int64_t a = first; a < hi; ++a, --hi) {\n"
     "                int32_t t = starts[a]; starts[a] = starts[hi]; starts[hi] = t;\n            }\n        }\n"
     "        lr_len[q] = length;",
     "            (void)hi;\n        }\n        lr_len[q] = length;"),
    ("sampled walk lists only the leftmost tie",
     "                else if (L == length) {\n                    if (total < cap) starts[total] = (int32_t)i;",
     "                else if (L == length && total == first) {\n                    if (total < cap) starts[total] = (int32_t)i;"),
]


def _pins_pass() -> bool:
    """Run the paper-value and brute-force pins against whichever oracle build is active."""
    try:
        import tests.test_oracle as T
        T.test_table1_mississippi_prep()
        T.test_abcabcddbca_lr2_all_variants()
        T.test_ababab_llr_and_useless()
        T.test_fig3_compaction()
        for s, want in [(b"aaaa", [(3, [0]), (3, [0, 1]), (3, [0, 1]), (3, [1])])]:
            T.test_special_cases(s, want)
        rng = np.random.default_rng(7)
        for _ in range(40):
            n = int(rng.integers(1, 14))
            s = bytes(rng.integers(97, 100, n).astype(np.uint8))
            assert T._rows(oracle.brute(s)) == definition.lr_all(s)
        rng = np.random.default_rng(8)
        for _ in range(60):
            s = T._random_string(rng, int(rng.integers(1, 300)))
            want = oracle.brute(s)
            sa, rank, lcp = W.prep(np.frombuffer(s, np.uint8))
            for got in (oracle.lr_all_raw(rank, lcp), oracle.lr_all_compact(rank, lcp)):
                for a, b in zip(got, want):
                    assert np.array_equal(a, b)
            for st, ln in (oracle.lr_leftmost_raw(rank, lcp), oracle.lr_leftmost_compact(rank, lcp)):
                assert np.array_equal(st, want[1]) and np.array_equal(ln, want[0])
        T.test_walk_counts_match_definition()
        T.test_lr_at_matches_full_run()
        for n in (2, 7):
            T.test_walk_counts_closed_forms(n)
        return True
    except AssertionError:
        return False


def _build(src_text: str, d: str) -> str:
    c = os.path.join(d, "m.c")
    so = os.path.join(d, "libm.so")
    open(c, "w").write(src_text)
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", "-o", so, c])
    return so


def test_unmutated_copy_passes():
    with tempfile.TemporaryDirectory() as d:
        oracle.use_library(_build(open(SRC).read(), d))
        try:
            assert _pins_pass()
        finally:
            oracle.use_library(None)


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_mutant(name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation site not found: " + name
    with tempfile.TemporaryDirectory() as d:
        oracle.use_library(_build(src.replace(old, new, 1), d))
        try:
            assert not _pins_pass(), "pins did not catch: " + name
        finally:
            oracle.use_library(None)
