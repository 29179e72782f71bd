"""Definition 1 of Tian and Xu (arXiv 1501.06663, Sec. 2), enumerated literally.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

A substring S[i..j] is unique if no other start i' != i carries an equal
substring, and a repeat otherwise; LR_k is a repeat S[i..j] with i <= k <= j
such that no repeat covering k is longer; the problem asks for every such
LR_k.  This module lists all substrings, counts their occurrences by direct
comparison and picks the longest repeats covering each position: pure Python,
O(n^4), for strings of a few dozen symbols.  It uses no suffix array, no
lemma of the paper and no code of the C oracle.
"""
from __future__ import annotations


def is_repeat(s: bytes, i: int, j: int) -> bool:
    """True iff S[i..j] (inclusive, 0-based) occurs at some other start."""
    sub = s[i:j + 1]
    for i2 in range(len(s) - len(sub) + 1):
        if i2 != i and s[i2:i2 + len(sub)] == sub:
            return True
    return False


def lr_all(s: bytes):
    """Per position k: (length, sorted list of starts) of all LR_k; (0, []) if none."""
    n = len(s)
    repeats = [(i, j) for i in range(n) for j in range(i, n) if is_repeat(s, i, j)]
    out = []
    for k in range(n):
        cover = [(i, j) for (i, j) in repeats if i <= k <= j]
        if not cover:
            out.append((0, []))
            continue
        best = max(j - i + 1 for (i, j) in cover)
        out.append((best, sorted(i for (i, j) in cover if j - i + 1 == best)))
    return out


def llr_lengths(s: bytes):
    """|LLR_i| for every i: the length of the longest repeat that starts at i
    (Sec. 3.1), by growing S[i..j] while it still occurs elsewhere."""
    n = len(s)
    out = []
    for i in range(n):
        j = i
        while j < n and is_repeat(s, i, j):
            j += 1
        out.append(j - i)
    return out


def covering_counts(s: bytes):
    """Per position k: (number of LLR's covering k, number of useful ones).

    An LLR is useless when its interval lies inside another LLR's interval
    (Sec. 3.2); the averages of the two counts are the alpha and beta of
    Table 2."""
    L = llr_lengths(s)
    iv = [(i, i + L[i] - 1) for i in range(len(s)) if L[i] > 0]
    useful = [(a, b) for (a, b) in iv if not any((c, d) != (a, b) and c <= a and b <= d for (c, d) in iv)]
    alpha = [sum(1 for (a, b) in iv if a <= k <= b) for k in range(len(s))]
    beta = [sum(1 for (a, b) in useful if a <= k <= b) for k in range(len(s))]
    return alpha, beta
