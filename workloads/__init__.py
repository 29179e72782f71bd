"""Seeded synthetic inputs for the longest-repeat query.

This module makes the strings and their suffix / rank / lcp arrays that both
the CPU oracle and the CUDA library are fed with.  It holds none of the
longest-repeat method's arithmetic: the paper builds SA, Rank and LCP on the
host before the query and leaves that time out of its measurements (Section 4,
Section 5); here the same preparation runs once per input, untimed.

The generators and the preparation (prefix-doubling suffix sort and Kasai's
LCP) are plain C in ``lrgen.c``, compiled on first use with gcc + OpenMP.

The workloads stand in for the paper's 50 MB Pizza&Chili DNA, English and
Protein files (Section 5), which are not available here:

========  ==================================================================
name      recipe
========  ==================================================================
dna_iid   i.i.d. uniform over ACGT (n = 2^20, seed 1)
dna       order-2 Markov DNA with planted repeats, 300-6000 long, 0-10 %
          point mutations, ~30 % of the string covered (n = 64 Mi, seed 2)
english   Zipf(1.1) draws from a 50k-word vocabulary (words 2-12 letters over
          a-z), space / punctuation / newline separators, 96-symbol alphabet
          (n = 256 Mi, seed 3)
protein   i.i.d. over the 20 amino-acid letters with 5 % of positions in
          tandem arrays (unit 3-50, 2-20 copies)
batched   4096 strings, lengths log-uniform in [1 Ki, 4 Mi]; even-indexed
          strings DNA as ``dna``, odd-indexed protein-like (seed 4)
serving   lognormal lengths (median 100k, sigma 1, floor 1 Ki, cap 16 Mi);
          70 % DNA / 30 % protein (seed 5)
========  ==================================================================
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lrgen.c")
_LIB = os.path.join(_HERE, "liblrgen.so")
_lock = threading.Lock()
_lib = None

MI = 1 << 20


def build_library(force: bool = False) -> str:
    """Compile ``lrgen.c`` into ``liblrgen.so`` next to it (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build_library()
            lib = ctypes.CDLL(_LIB)
            i64, u64, dbl, vp, ci = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int
            lib.gen_iid.argtypes = [vp, i64, vp, ci, u64]
            lib.gen_dna_planted.argtypes = [vp, i64, u64, i64, i64, dbl, dbl]
            lib.gen_protein_tandem.argtypes = [vp, i64, u64, dbl, ci, ci, ci, ci]
            lib.gen_english.argtypes = [vp, i64, u64, ci, dbl]
            lib.gen_lengths_loguniform.argtypes = [vp, i64, i64, i64, u64]
            lib.gen_lengths_lognormal.argtypes = [vp, i64, dbl, dbl, i64, i64, u64]
            lib.gen_uniforms.argtypes = [vp, i64, u64]
            lib.prep_sa.argtypes = [vp, i64, vp, vp]
            lib.prep_sa.restype = ci
            lib.prep_lcp.argtypes = [vp, i64, vp, vp, vp]
            lib.prep_all.argtypes = [vp, i64, vp, vp, vp]
            lib.prep_all.restype = ci
            lib.prep_many.argtypes = [vp, vp, i64, vp, vp, vp]
            lib.prep_many.restype = ci
            lib.lrgen_num_threads.restype = ci
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


# --------------------------------------------------------------------------
# strings
# --------------------------------------------------------------------------

def iid(n: int, alphabet: bytes, seed: int) -> np.ndarray:
    out = np.empty(n, np.uint8)
    alpha = np.frombuffer(alphabet, np.uint8).copy()
    _load().gen_iid(_p(out), n, _p(alpha), len(alphabet), seed)
    return out


def dna_iid(n: int = MI, seed: int = 1) -> np.ndarray:
    return iid(n, b"ACGT", seed)


def dna_planted(n: int = 64 * MI, seed: int = 2, seg_min: int = 300, seg_max: int = 6000,
                mut_max: float = 0.10, cover: float = 0.30) -> np.ndarray:
    out = np.empty(n, np.uint8)
    _load().gen_dna_planted(_p(out), n, seed, seg_min, seg_max, mut_max, cover)
    return out


def protein_tandem(n: int, seed: int, tandem_frac: float = 0.05, unit_min: int = 3,
                   unit_max: int = 50, copies_min: int = 2, copies_max: int = 20) -> np.ndarray:
    out = np.empty(n, np.uint8)
    _load().gen_protein_tandem(_p(out), n, seed, tandem_frac, unit_min, unit_max, copies_min, copies_max)
    return out


def english(n: int = 256 * MI, seed: int = 3, vocab: int = 50000, zipf_s: float = 1.1) -> np.ndarray:
    out = np.empty(n, np.uint8)
    _load().gen_english(_p(out), n, seed, vocab, zipf_s)
    return out


def lengths_loguniform(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    out = np.empty(count, np.int64)
    _load().gen_lengths_loguniform(_p(out), count, lo, hi, seed)
    return out


def lengths_lognormal(count: int, median: float, sigma: float, floor_len: int, cap: int,
                      seed: int) -> np.ndarray:
    out = np.empty(count, np.int64)
    _load().gen_lengths_lognormal(_p(out), count, median, sigma, floor_len, cap, seed)
    return out


def uniforms(count: int, seed: int) -> np.ndarray:
    out = np.empty(count, np.float64)
    _load().gen_uniforms(_p(out), count, seed)
    return out


# --------------------------------------------------------------------------
# SA / Rank / LCP preparation
# --------------------------------------------------------------------------

def prep(text: np.ndarray):
    """Return (sa, rank, lcp) as int32 arrays; lcp has n+1 entries, lcp[0]=lcp[n]=0."""
    text = np.ascontiguousarray(text, dtype=np.uint8)
    n = int(text.size)
    if n < 1 or n > 2**31 - 2:
        raise ValueError("n must be in [1, 2^31-2]")
    sa = np.empty(n, np.int32)
    rank = np.empty(n, np.int32)
    lcp = np.empty(n + 1, np.int32)
    rc = _load().prep_all(_p(text), n, _p(sa), _p(rank), _p(lcp))
    if rc != 0:
        raise MemoryError("prep_all failed")
    return sa, rank, lcp


def prep_many(text: np.ndarray, offsets: np.ndarray):
    """Prep for strings packed back to back (string j = text[off[j]:off[j+1]]).

    Returns (sa, rank, lcp): sa / rank local to each string at the string's
    offsets, lcp (n_j + 1 entries) at ``off[j] + j``.
    """
    text = np.ascontiguousarray(text, dtype=np.uint8)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    count = off.size - 1
    total = int(off[-1])
    sa = np.empty(total, np.int32)
    rank = np.empty(total, np.int32)
    lcp = np.empty(total + count, np.int32)
    rc = _load().prep_many(_p(text), _p(off), count, _p(sa), _p(rank), _p(lcp))
    if rc != 0:
        raise MemoryError("prep_many failed")
    return sa, rank, lcp


def host_threads() -> int:
    return int(_load().lrgen_num_threads())


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    text: np.ndarray
    sa: np.ndarray
    rank: np.ndarray
    lcp: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.text.size)


def make_text(kind: str, n: int, seed: int) -> np.ndarray:
    if kind == "dna_iid":
        return dna_iid(n, seed)
    if kind == "dna":
        return dna_planted(n, seed)
    if kind == "english":
        return english(n, seed)
    if kind == "protein":
        return protein_tandem(n, seed)
    raise ValueError(kind)


#: the single-string workloads: (kind, n, seed)
SINGLE = {
    "dna_iid_1m": ("dna_iid", MI, 1),
    "dna_64m": ("dna", 64 * MI, 2),
    "english_256m": ("english", 256 * MI, 3),
}


def single(name: str, n: int | None = None) -> Workload:
    """A named single-string workload, optionally shrunk to n symbols (same seed)."""
    kind, n0, seed = SINGLE[name]
    n = n0 if n is None else n
    text = make_text(kind, n, seed)
    sa, rank, lcp = prep(text)
    return Workload(name if n == n0 else "%s@n=%d" % (name, n), text, sa, rank, lcp,
                    {"kind": kind, "seed": seed, "n": n})


def batched_mix(count: int = 4096, lo: int = 1024, hi: int = 4 * MI, seed: int = 4):
    """The batched mix: returns (text, offsets, kinds) with strings packed back to back."""
    lens = lengths_loguniform(count, lo, hi, seed)
    kinds = ["dna" if j % 2 == 0 else "protein" for j in range(count)]
    return _pack(lens, kinds, seed)


def serving_mix(count: int, seed: int = 5, median: float = 1e5, sigma: float = 1.0,
                floor_len: int = 1024, cap: int = 16 * MI):
    """The serving pool: lognormal lengths, 70 % DNA / 30 % protein."""
    lens = lengths_lognormal(count, median, sigma, floor_len, cap, seed)
    u = uniforms(count, seed + 1000)
    kinds = ["dna" if u[j] < 0.7 else "protein" for j in range(count)]
    return _pack(lens, kinds, seed)


def _pack(lens, kinds, seed):
    off = np.zeros(len(lens) + 1, np.int64)
    off[1:] = np.cumsum(lens)
    text = np.empty(int(off[-1]), np.uint8)
    for j, (ln, kind) in enumerate(zip(lens, kinds)):
        sj = seed * 1_000_003 + j
        text[off[j]:off[j + 1]] = dna_planted(int(ln), sj) if kind == "dna" else protein_tandem(int(ln), sj)
    return text, off, kinds
