"""CPU oracle for the all-longest-repeats query (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it.

The arithmetic is plain sequential C in ``lr_oracle.c`` (compiled on first use
with gcc, no optimisation tricks) and, for very short strings, pure Python in
``definition.py``.  Each function follows one passage of Tian and Xu, "On
Longest Repeat Queries Using GPU" (arXiv 1501.06663):

=====================  ======================================================
function               passage
=====================  ======================================================
llr_raw                Lemma 1 (L_i = max(LCP[Rank[i]], LCP[Rank[i]+1]))
flag_prefix_scatter    Sec. 4.2.1, kernels K1, K2, K3 (Flag, Prefix_Sum, LLRc)
compact                Algorithm 2, first loop (one-pass compaction)
lr_leftmost_raw        Algorithm 1
lr_leftmost_compact    Algorithm 2
lr_all_raw             Algorithm 3 (appendix)
lr_all_compact         Algorithm 4 (appendix)
lr_at                  Algorithm 3 for sampled positions only
lr_at_range            Algorithm 3 for a range of positions (lr_at on disjoint
                       blocks at once, one thread each)
brute                  Definition 1 / the problem statement of Sec. 2, from the
                       string alone (O(n^2) suffix-pair comparison)
definition.lr_all      Definition 1 by enumerating every substring (tiny n)
=====================  ======================================================

All results are 0-based; the all-LR results come as CSR:
``(lr_len[n], lr_start[n], offsets[n+1], starts[total])`` with the starts of
each position listed in ascending order, ``lr_start = -1`` and ``lr_len = 0``
where no repeat covers the position.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build_library(force: bool = False) -> str:
    """Compile ``lr_oracle.c`` into ``liboracle.so`` (gcc -O2, single-threaded)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    lib.oracle_llr_raw.argtypes = [vp, vp, i64, vp]
    lib.oracle_flag_prefix_scatter.argtypes = [vp, i64, vp, vp, vp, vp]
    lib.oracle_flag_prefix_scatter.restype = i64
    lib.oracle_compact.argtypes = [vp, vp, i64, vp, vp]
    lib.oracle_compact.restype = i64
    lib.oracle_lr_leftmost_raw.argtypes = [vp, vp, i64, vp, vp]
    lib.oracle_lr_leftmost_compact.argtypes = [vp, vp, i64, vp, vp]
    for f in (lib.oracle_lr_all_raw, lib.oracle_lr_all_compact):
        f.argtypes = [vp, vp, i64, vp, vp, vp, vp, i64]
        f.restype = i64
    lib.oracle_lr_at.argtypes = [vp, vp, i64, vp, i64, vp, vp, vp, vp, i64]
    lib.oracle_lr_at.restype = i64
    lib.oracle_brute.argtypes = [vp, i64, vp, vp, vp, vp, i64]
    lib.oracle_brute.restype = i64
    lib.oracle_walk_counts.argtypes = [vp, vp, i64, vp, vp]
    lib.oracle_walk_counts.restype = i64
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build_library()
            _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


_active = None   # set by use_library() in mutation tests only


def use_library(path):
    """Point this module at another build of the oracle (mutation tests); None restores."""
    global _active
    _active = None if path is None else _bind(ctypes.CDLL(path))


def _L():
    return _active if _active is not None else _load()


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _check_inputs(rank, lcp):
    rank, lcp = _i32(rank), _i32(lcp)
    if lcp.size != rank.size + 1:
        raise ValueError("lcp must have n+1 entries")
    return rank, lcp, int(rank.size)


def llr_raw(rank, lcp) -> np.ndarray:
    """Lemma 1: the raw LLR array LLRr[i] = max(lcp[rank[i]], lcp[rank[i]+1])."""
    rank, lcp, n = _check_inputs(rank, lcp)
    out = np.empty(n, np.int32)
    _L().oracle_llr_raw(_p(rank), _p(lcp), n, _p(out))
    return out


def flag_prefix_scatter(llrr):
    """Sec. 4.2.1, K1-K3: (Flag, Prefix_Sum, LLRc starts, LLRc lengths) from a raw LLR array."""
    llrr = _i32(llrr)
    n = int(llrr.size)
    flag = np.empty(n, np.int32)
    prefix = np.empty(n, np.int64)
    cs = np.empty(n, np.int32)
    cl = np.empty(n, np.int32)
    m = _L().oracle_flag_prefix_scatter(_p(llrr), n, _p(flag), _p(prefix), _p(cs), _p(cl))
    return flag, prefix, cs[:m].copy(), cl[:m].copy()


def compact(rank, lcp):
    """Algorithm 2's one-pass compaction: (LLRc starts, LLRc lengths)."""
    rank, lcp, n = _check_inputs(rank, lcp)
    cs = np.empty(n, np.int32)
    cl = np.empty(n, np.int32)
    m = _L().oracle_compact(_p(rank), _p(lcp), n, _p(cs), _p(cl))
    return cs[:m].copy(), cl[:m].copy()


def lr_leftmost_raw(rank, lcp):
    """Algorithm 1: (lr_start, lr_len), leftmost LR per position."""
    rank, lcp, n = _check_inputs(rank, lcp)
    st = np.empty(n, np.int32)
    ln = np.empty(n, np.int32)
    _L().oracle_lr_leftmost_raw(_p(rank), _p(lcp), n, _p(st), _p(ln))
    return st, ln


def lr_leftmost_compact(rank, lcp):
    """Algorithm 2: (lr_start, lr_len), leftmost LR per position."""
    rank, lcp, n = _check_inputs(rank, lcp)
    st = np.empty(n, np.int32)
    ln = np.empty(n, np.int32)
    _L().oracle_lr_leftmost_compact(_p(rank), _p(lcp), n, _p(st), _p(ln))
    return st, ln


def _csr_call(fn, n, args, cap_hint):
    lr_len = np.empty(n, np.int32)
    lr_start = np.empty(n, np.int32)
    offsets = np.empty(n + 1, np.int64)
    cap = max(16, cap_hint)
    while True:
        starts = np.empty(cap, np.int32)
        total = fn(*args, _p(lr_len), _p(lr_start), _p(offsets), _p(starts), cap)
        if total <= cap:
            return lr_len, lr_start, offsets, starts[:total].copy()
        cap = int(total)


def lr_all_raw(rank, lcp):
    """Algorithm 3: all LR's per position as CSR (lr_len, lr_start, offsets, starts)."""
    rank, lcp, n = _check_inputs(rank, lcp)
    return _csr_call(_L().oracle_lr_all_raw, n, (_p(rank), _p(lcp), n), 2 * n)


def lr_all_compact(rank, lcp):
    """Algorithm 4: all LR's per position as CSR (lr_len, lr_start, offsets, starts)."""
    rank, lcp, n = _check_inputs(rank, lcp)
    return _csr_call(_L().oracle_lr_all_compact, n, (_p(rank), _p(lcp), n), 2 * n)


def lr_at(rank, lcp, ks):
    """Algorithm 3 restricted to the positions ks: CSR over the samples."""
    rank, lcp, n = _check_inputs(rank, lcp)
    ks = np.ascontiguousarray(ks, dtype=np.int64)
    if ks.size and (ks.min() < 0 or ks.max() >= n):
        raise ValueError("sample position out of range")
    nk = int(ks.size)
    return _csr_call(_L().oracle_lr_at, nk, (_p(rank), _p(lcp), n, _p(ks), nk), 4 * nk)


def lr_at_range(rank, lcp, a: int, b: int, threads: int = 1):
    """Algorithm 3 for every position of [a, b), as CSR over those positions.

    Each position's two walks are independent of every other position's
    (Sec. 3), so the range is split into `threads` contiguous blocks that
    run ``lr_at`` at the same time in threads (the C call releases the
    interpreter lock); the blocks' results are concatenated in order.  The
    arithmetic is ``lr_at``'s, unchanged.
    """
    import concurrent.futures as cf
    rank, lcp, n = _check_inputs(rank, lcp)
    a, b = max(0, int(a)), min(n, int(b))
    if b <= a:
        return (np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(1, np.int64), np.zeros(0, np.int32))
    threads = max(1, min(int(threads), b - a))
    cuts = np.linspace(a, b, threads + 1).astype(np.int64)
    blocks = [(int(cuts[i]), int(cuts[i + 1])) for i in range(threads) if cuts[i + 1] > cuts[i]]
    with cf.ThreadPoolExecutor(len(blocks)) as ex:
        parts = list(ex.map(lambda ab: lr_at(rank, lcp, np.arange(ab[0], ab[1], dtype=np.int64)), blocks))
    ln = np.concatenate([q[0] for q in parts])
    st = np.concatenate([q[1] for q in parts])
    sizes = [q[3].size for q in parts]
    base = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    off = np.concatenate([[0]] + [q[2][1:] + base[i] for i, q in enumerate(parts)]).astype(np.int64)
    starts = np.concatenate([q[3] for q in parts]).astype(np.int32)
    return ln, st, off, starts


def walk_counts(rank, lcp):
    """Table 2's walk statistics per position: (alpha, beta, m) with alpha[k]
    the raw LLR's and beta[k] the compact LLR's covering k (the steps of the
    walks of Algorithms 1 and 2 that meet a covering LLR), m = |LLRc|."""
    rank, lcp, n = _check_inputs(rank, lcp)
    alpha = np.empty(n, np.int32)
    beta = np.empty(n, np.int32)
    m = _L().oracle_walk_counts(_p(rank), _p(lcp), n, _p(alpha), _p(beta))
    return alpha, beta, int(m)


def brute(text):
    """Definition 1 from the string alone: CSR (lr_len, lr_start, offsets, starts)."""
    s = np.ascontiguousarray(np.frombuffer(text, np.uint8) if isinstance(text, (bytes, bytearray))
                             else text, dtype=np.uint8)
    n = int(s.size)
    return _csr_call(_L().oracle_brute, n, (_p(s), n), 2 * n)
