"""Python binding of liblr, the GB300 longest-repeat query library.

Argument marshalling only: every step of the query runs in the CUDA kernels
of ``liblr.so`` (sources in ``csrc/``, C ABI in ``include/lr.h``).  PyTorch
supplies device memory and streams.  There is no CPU fallback: if the
library is missing or cannot load, importing the functions below raises.

The names follow the C ABI (``lr_create``, ``lr_query_all`` ...); ``Context``
wraps a context handle with tensor-friendly methods that allocate outputs.
"""
from __future__ import annotations

import ctypes
import os

from ._build import LIB_PATH, build_library  # noqa: F401

_lib = None

LR_OK = 0
LR_ERR_ARG = 1
LR_ERR_SENTINEL = 2
LR_ERR_CAPACITY = 3
LR_ERR_NOMEM = 4
LR_ERR_CUDA = 5
LR_ERR_TIMEOUT = 6
LR_ERR_BUSY = 7

#: every symbol include/lr.h declares
EXPORTED = (
    "lr_create", "lr_destroy", "lr_status_str", "lr_last_cuda_error", "lr_device_status",
    "lr_query_leftmost", "lr_query_all", "lr_query_all_host", "lr_last_launch_count",
    "lr_set_phase_timing", "lr_phase_times", "lr_last_compact_size", "lr_query_all_static",
    "lr_batch_query_all", "lr_autotune", "lr_autotune_save", "lr_autotune_load",
    "lr_plan_create", "lr_plan_launch", "lr_plan_result", "lr_plan_destroy",
    "lr_server_start", "lr_server_submit", "lr_server_poll", "lr_server_wait", "lr_server_cancel",
    "lr_server_stats_get", "lr_server_stop",
    "lr_query_all_raw", "lr_query_leftmost_raw", "lr_walk_stats", "lr_build_arrays", "lr_batch_build_arrays",
    "lr_test_hold_lookback",
)

LR_JOB_QUEUED, LR_JOB_ADMITTED, LR_JOB_RUNNING, LR_JOB_DONE, LR_JOB_CANCELLED = range(5)

#: largest n lr_query_all_static takes (LR_STATIC_MAX_N in include/lr.h)
LR_STATIC_MAX_N = 1 << 20


class BatchDesc(ctypes.Structure):
    """lr_batch_desc: a flattened table of strings (see include/lr.h)."""
    _fields_ = [("num", ctypes.c_int64), ("total", ctypes.c_int64), ("d_off", ctypes.c_void_p),
                ("d_sa", ctypes.c_void_p), ("d_rank", ctypes.c_void_p), ("d_lcp", ctypes.c_void_p)]


class ServerConfig(ctypes.Structure):
    """lr_server_config (zeros mean defaults, see include/lr.h)."""
    _fields_ = [("device", ctypes.c_int32), ("slots", ctypes.c_int32), ("max_inflight", ctypes.c_int32),
                ("max_batch_positions", ctypes.c_int64), ("max_batch_jobs", ctypes.c_int32),
                ("max_queue", ctypes.c_int32), ("batch_window_us", ctypes.c_int32), ("hbm_fraction", ctypes.c_double),
                ("starts_factor", ctypes.c_double), ("text_jobs", ctypes.c_int32)]


class Job(ctypes.Structure):
    """lr_job: one query job with host buffers."""
    _fields_ = [("h_sa", ctypes.c_void_p), ("h_rank", ctypes.c_void_p), ("h_lcp", ctypes.c_void_p),
                ("n", ctypes.c_int32), ("h_lr_len", ctypes.c_void_p), ("h_lr_start", ctypes.c_void_p),
                ("h_offsets", ctypes.c_void_p), ("h_starts", ctypes.c_void_p), ("starts_capacity", ctypes.c_int64),
                ("h_text", ctypes.c_void_p)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("cancelled", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("batches", ctypes.c_int64), ("positions", ctypes.c_int64),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("max_us", ctypes.c_double), ("slots", ctypes.c_int32), ("slot_positions", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64)]


class TextBatch(ctypes.Structure):
    """lr_text_batch: texts packed back to back (see include/lr.h)."""
    _fields_ = [("num", ctypes.c_int64), ("total", ctypes.c_int64), ("d_off", ctypes.c_void_p),
                ("d_text", ctypes.c_void_p)]


class WalkSummary(ctypes.Structure):
    """lr_walk_summary: Table 2's walk statistics of one string."""
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("alpha_sum", ctypes.c_int64),
                ("beta_sum", ctypes.c_int64), ("alpha_min", ctypes.c_int32), ("alpha_max", ctypes.c_int32),
                ("beta_min", ctypes.c_int32), ("beta_max", ctypes.c_int32)]


class LRError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__("%s: %s" % (what, status_str(status)))


def load(path: str | None = None):
    """Load liblr.so (raises OSError if it is missing: build it with build_library())."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError("liblr.so not found at %s; run paper_1501_06663_gb300.build_library()" % p)
    lib = ctypes.CDLL(p)
    vp, i32, i64, ci = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int
    lib.lr_create.argtypes = [ctypes.POINTER(vp), ci]
    lib.lr_destroy.argtypes = [vp]
    lib.lr_status_str.argtypes = [ci]
    lib.lr_status_str.restype = ctypes.c_char_p
    lib.lr_last_cuda_error.argtypes = [vp, ctypes.POINTER(ci)]
    lib.lr_device_status.argtypes = [vp, vp]
    lib.lr_query_leftmost.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp]
    lib.lr_query_all.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp, vp, vp, i64, ctypes.POINTER(i64)]
    lib.lr_query_all_host.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp, vp, vp, i64, ctypes.POINTER(i64)]
    lib.lr_last_launch_count.argtypes = [vp]
    lib.lr_last_launch_count.restype = i32
    lib.lr_test_hold_lookback.argtypes = [vp, i64, i32]
    lib.lr_set_phase_timing.argtypes = [vp, i32]
    lib.lr_phase_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float), i32]
    lib.lr_phase_times.restype = i32
    lib.lr_last_compact_size.argtypes = [vp, vp, ctypes.POINTER(i64)]
    lib.lr_query_all_static.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp, i64, ctypes.POINTER(i64)]
    bd = ctypes.POINTER(BatchDesc)
    lib.lr_batch_query_all.argtypes = [vp, vp, bd, vp, vp, vp, vp, i64, ctypes.POINTER(i64)]
    lib.lr_autotune.argtypes = [vp, vp, bd, vp, vp, vp, vp, i64, ctypes.POINTER(i32)]
    lib.lr_autotune_save.argtypes = [vp, ctypes.c_char_p]
    lib.lr_autotune_load.argtypes = [vp, ctypes.c_char_p]
    lib.lr_plan_create.argtypes = [vp, bd, vp, vp, vp, vp, i64, ctypes.POINTER(vp)]
    lib.lr_plan_launch.argtypes = [vp, vp]
    lib.lr_plan_result.argtypes = [vp, vp, ctypes.POINTER(i64)]
    lib.lr_plan_destroy.argtypes = [vp]
    lib.lr_server_start.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    lib.lr_server_submit.argtypes = [vp, ctypes.POINTER(Job), ctypes.POINTER(i64)]
    lib.lr_server_poll.argtypes = [vp, i64, ctypes.POINTER(i32), ctypes.POINTER(ci), ctypes.POINTER(i64)]
    lib.lr_server_wait.argtypes = [vp, i64, i32, ctypes.POINTER(i32), ctypes.POINTER(ci), ctypes.POINTER(i64)]
    lib.lr_server_cancel.argtypes = [vp, i64]
    lib.lr_server_stats_get.argtypes = [vp, i32, ctypes.POINTER(ServerStats)]
    lib.lr_server_stop.argtypes = [vp]
    lib.lr_query_all_raw.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp, vp, i64, ctypes.POINTER(i64)]
    lib.lr_query_leftmost_raw.argtypes = [vp, vp, vp, vp, i32, vp, vp]
    lib.lr_walk_stats.argtypes = [vp, vp, vp, vp, i32, vp, vp, ctypes.POINTER(WalkSummary)]
    lib.lr_build_arrays.argtypes = [vp, vp, vp, i32, vp, vp, vp, ctypes.POINTER(i32)]
    lib.lr_batch_build_arrays.argtypes = [vp, vp, ctypes.POINTER(TextBatch), vp, vp, vp, ctypes.POINTER(i32)]
    for name in EXPORTED:
        f = getattr(lib, name)
        if name not in ("lr_status_str", "lr_last_launch_count", "lr_phase_times"):
            f.restype = ci
    if path is None:
        _lib = lib
    return lib


def status_str(status: int) -> str:
    return load().lr_status_str(int(status)).decode()


def _check(status: int, what: str, ok=(LR_OK,)):
    if status not in ok:
        raise LRError(status, what)
    return status


def _ptr(t) -> ctypes.c_void_p:
    """Device (or host) address of a tensor / numpy array, or NULL."""
    if t is None:
        return ctypes.c_void_p(0)
    if hasattr(t, "data_ptr"):
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(t.ctypes.data)


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


# ---------------------------------------------------------------- C-ABI mirrors

def lr_create(device: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().lr_create(ctypes.byref(h), int(device)), "lr_create")
    return h


def lr_destroy(ctx) -> None:
    _check(load().lr_destroy(ctx), "lr_destroy")


def lr_device_status(ctx, stream=None) -> int:
    return load().lr_device_status(ctx, _stream(stream))


def lr_last_cuda_error(ctx) -> int:
    code = ctypes.c_int()
    _check(load().lr_last_cuda_error(ctx, ctypes.byref(code)), "lr_last_cuda_error")
    return code.value


def lr_last_launch_count(ctx) -> int:
    return int(load().lr_last_launch_count(ctx))


def lr_test_hold_lookback(ctx, tile: int, spin_limit: int = 1000) -> int:
    """Test hook: cover tile `tile` keeps its look-back word unpublished and
    waits give up after `spin_limit` polls (tile < 0: off).  Returns the status."""
    return int(load().lr_test_hold_lookback(ctx, int(tile), int(spin_limit)))


def lr_set_phase_timing(ctx, enable: bool) -> None:
    _check(load().lr_set_phase_timing(ctx, 1 if enable else 0), "lr_set_phase_timing")


def lr_phase_times(ctx, cap: int = 8):
    """Milliseconds of each kernel of the last query (launch order), or None."""
    buf = (ctypes.c_float * cap)()
    k = load().lr_phase_times(ctx, buf, cap)
    return None if k < 0 else [float(buf[i]) for i in range(min(k, cap))]


def _n_of(sa, rank):
    t = sa if sa is not None else rank
    if hasattr(t, "numel"):
        return int(t.numel())
    return int(t.size)


def lr_last_compact_size(ctx, stream=None) -> int:
    """Number of useful LLR's (compact LLR array size) of the context's last query."""
    m = ctypes.c_int64(-1)
    _check(load().lr_last_compact_size(ctx, _stream(stream), ctypes.byref(m)), "lr_last_compact_size")
    return m.value


def lr_query_leftmost(ctx, sa, rank, lcp, lr_start, lr_len, stream=None) -> int:
    """sa or rank may be None (not both); sa is used when given."""
    n = _n_of(sa, rank)
    return load().lr_query_leftmost(ctx, _stream(stream), _ptr(sa), _ptr(rank), _ptr(lcp), n,
                                    _ptr(lr_start), _ptr(lr_len))


def lr_query_all(ctx, sa, rank, lcp, lr_len, lr_start, offsets, starts, stream=None, sync=True):
    """Device buffers; sa or rank may be None (not both).  Returns (status, total or None)."""
    n = _n_of(sa, rank)
    cap = int(starts.numel()) if starts is not None else 0
    tot = ctypes.c_int64(-1)
    st = load().lr_query_all(ctx, _stream(stream), _ptr(sa), _ptr(rank), _ptr(lcp), n, _ptr(lr_len),
                             _ptr(lr_start), _ptr(offsets), _ptr(starts), cap,
                             ctypes.byref(tot) if sync else None)
    return st, (tot.value if sync else None)


def lr_query_all_host(ctx, sa, rank, lcp, lr_len, lr_start, offsets, starts, stream=None):
    """Host (numpy or CPU tensor) buffers; sa or rank may be None.  Returns (status, total)."""
    n = _n_of(sa, rank)
    cap = int(len(starts)) if starts is not None else 0
    tot = ctypes.c_int64(-1)
    st = load().lr_query_all_host(ctx, _stream(stream), _ptr(sa), _ptr(rank), _ptr(lcp), n, _ptr(lr_len),
                                  _ptr(lr_start), _ptr(offsets), _ptr(starts), cap, ctypes.byref(tot))
    return st, tot.value


def lr_query_all_static(rank, lcp, lr_len, lr_start, offsets, starts, stream=None, sync=True):
    """The all-LR query without any device allocation (no context; n <= LR_STATIC_MAX_N).

    For callers that may not allocate at query time; see include/lr.h.  The
    outputs are caller-provided device tensors.  Returns (status, total or None).
    """
    n = int(rank.numel())
    cap = int(starts.numel()) if starts is not None else 0
    tot = ctypes.c_int64(-1)
    st = load().lr_query_all_static(_stream(stream), _ptr(rank), _ptr(lcp), n, _ptr(lr_len), _ptr(lr_start),
                                    _ptr(offsets), _ptr(starts), cap, ctypes.byref(tot) if sync else None)
    return st, (tot.value if sync else None)


def batch_desc(off, lcp, sa=None, rank=None) -> BatchDesc:
    """lr_batch_desc over device tensors: off (int64, num + 1), lcp (int32,
    total + num), sa / rank (int32, total; at least one)."""
    num = int(off.numel()) - 1
    total = int((sa if sa is not None else rank).numel())
    return BatchDesc(num, total, _ptr(off), _ptr(sa), _ptr(rank), _ptr(lcp))


def lr_batch_query_all(ctx, desc, lr_len, lr_start, offsets, starts, stream=None, sync=True):
    """Batched all-LR query (flattened outputs).  Returns (status, total or None)."""
    cap = int(starts.numel()) if starts is not None else 0
    tot = ctypes.c_int64(-1)
    st = load().lr_batch_query_all(ctx, _stream(stream), ctypes.byref(desc), _ptr(lr_len), _ptr(lr_start),
                                   _ptr(offsets), _ptr(starts), cap, ctypes.byref(tot) if sync else None)
    return st, (tot.value if sync else None)


def lr_autotune(ctx, desc, lr_len, lr_start, offsets, starts, stream=None) -> int:
    """Times the shape choices on this batch; remembers and returns the fastest shape code."""
    cap = int(starts.numel()) if starts is not None else 0
    choice = ctypes.c_int32(-1)
    _check(load().lr_autotune(ctx, _stream(stream), ctypes.byref(desc), _ptr(lr_len), _ptr(lr_start),
                              _ptr(offsets), _ptr(starts), cap, ctypes.byref(choice)), "lr_autotune")
    return choice.value


def lr_autotune_save(ctx, path: str) -> None:
    _check(load().lr_autotune_save(ctx, os.fsencode(path)), "lr_autotune_save")


def lr_autotune_load(ctx, path: str) -> None:
    _check(load().lr_autotune_load(ctx, os.fsencode(path)), "lr_autotune_load")


def lr_plan_create(ctx, desc, lr_len, lr_start, offsets, starts):
    """Captures one batched query into a replayable plan (a CUDA graph with its own scratch)."""
    cap = int(starts.numel()) if starts is not None else 0
    h = ctypes.c_void_p()
    _check(load().lr_plan_create(ctx, ctypes.byref(desc), _ptr(lr_len), _ptr(lr_start), _ptr(offsets),
                                 _ptr(starts), cap, ctypes.byref(h)), "lr_plan_create")
    return h


def lr_plan_launch(plan, stream=None) -> None:
    _check(load().lr_plan_launch(plan, _stream(stream)), "lr_plan_launch")


def lr_plan_result(plan, stream=None):
    """Waits for the stream; returns (status, total LR starts of the last launch)."""
    tot = ctypes.c_int64(-1)
    st = load().lr_plan_result(plan, _stream(stream), ctypes.byref(tot))
    return st, tot.value


def lr_plan_destroy(plan) -> None:
    _check(load().lr_plan_destroy(plan), "lr_plan_destroy")


def lr_build_arrays(ctx, text, sa, rank, lcp, stream=None):
    """sa, rank, lcp of a device uint8 text, built on the GPU.  Returns (status, rounds)."""
    r = ctypes.c_int32(0)
    st = load().lr_build_arrays(ctx, _stream(stream), _ptr(text), int(text.numel()), _ptr(sa), _ptr(rank),
                                _ptr(lcp), ctypes.byref(r))
    return st, r.value


def lr_batch_build_arrays(ctx, off, text, sa, rank, lcp, stream=None):
    """sa, rank, lcp of device uint8 texts packed back to back (off: int64, num + 1).  Returns (status, rounds)."""
    desc = TextBatch(int(off.numel()) - 1, int(text.numel()), _ptr(off), _ptr(text))
    r = ctypes.c_int32(0)
    st = load().lr_batch_build_arrays(ctx, _stream(stream), ctypes.byref(desc), _ptr(sa), _ptr(rank), _ptr(lcp),
                                      ctypes.byref(r))
    return st, r.value


def lr_query_all_raw(ctx, rank, lcp, lr_len, lr_start, offsets, starts, stream=None, sync=True):
    """The raw-LLR variant (no compaction) of lr_query_all.  Returns (status, total or None)."""
    n = int(rank.numel())
    cap = int(starts.numel()) if starts is not None else 0
    tot = ctypes.c_int64(-1)
    st = load().lr_query_all_raw(ctx, _stream(stream), _ptr(rank), _ptr(lcp), n, _ptr(lr_len), _ptr(lr_start),
                                 _ptr(offsets), _ptr(starts), cap, ctypes.byref(tot) if sync else None)
    return st, (tot.value if sync else None)


def lr_query_leftmost_raw(ctx, rank, lcp, lr_start, lr_len, stream=None) -> int:
    return load().lr_query_leftmost_raw(ctx, _stream(stream), _ptr(rank), _ptr(lcp), int(rank.numel()),
                                        _ptr(lr_start), _ptr(lr_len))


def lr_walk_stats(ctx, rank, lcp, alpha=None, beta=None, stream=None) -> dict:
    """Table 2's alpha / beta statistics (per position into alpha / beta when given)."""
    out = WalkSummary()
    _check(load().lr_walk_stats(ctx, _stream(stream), _ptr(rank), _ptr(lcp), int(rank.numel()), _ptr(alpha),
                                _ptr(beta), ctypes.byref(out)), "lr_walk_stats")
    return {name: getattr(out, name) for name, _ in WalkSummary._fields_}


def lr_server_start(cfg: ServerConfig | None = None):
    h = ctypes.c_void_p()
    _check(load().lr_server_start(ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(h)),
           "lr_server_start")
    return h


def lr_server_submit(server, job: Job):
    """Returns (status, job id)."""
    jid = ctypes.c_int64(-1)
    st = load().lr_server_submit(server, ctypes.byref(job), ctypes.byref(jid))
    return st, jid.value


def lr_server_poll(server, job_id: int):
    """Returns (status, state, result, total)."""
    state, res, tot = ctypes.c_int32(-1), ctypes.c_int(-1), ctypes.c_int64(-1)
    st = load().lr_server_poll(server, job_id, ctypes.byref(state), ctypes.byref(res), ctypes.byref(tot))
    return st, state.value, res.value, tot.value


def lr_server_wait(server, job_id: int, timeout_ms: int = -1):
    """Returns (status, state, result, total)."""
    state, res, tot = ctypes.c_int32(-1), ctypes.c_int(-1), ctypes.c_int64(-1)
    st = load().lr_server_wait(server, job_id, timeout_ms, ctypes.byref(state), ctypes.byref(res),
                               ctypes.byref(tot))
    return st, state.value, res.value, tot.value


def lr_server_cancel(server, job_id: int) -> int:
    return load().lr_server_cancel(server, job_id)


def lr_server_stats_get(server, reset: bool = False) -> dict:
    s = ServerStats()
    _check(load().lr_server_stats_get(server, 1 if reset else 0, ctypes.byref(s)), "lr_server_stats_get")
    return {name: getattr(s, name) for name, _ in ServerStats._fields_}


def lr_server_stop(server) -> None:
    _check(load().lr_server_stop(server), "lr_server_stop")


# ---------------------------------------------------------------- convenience

class Context:
    """A liblr context on one CUDA device, with output-allocating query methods."""

    def __init__(self, device: int = 0):
        import torch
        self.device = torch.device("cuda", device)
        self.handle = lr_create(device)

    def close(self):
        if self.handle is not None:
            lr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def query_leftmost(self, lcp, sa=None, rank=None, stream=None):
        """Leftmost LR per position: (lr_start, lr_len).  Give sa or rank (device tensors)."""
        import torch
        t = sa if sa is not None else rank
        n = int(t.numel())
        lr_start = torch.empty(n, dtype=torch.int32, device=t.device)
        lr_len = torch.empty(n, dtype=torch.int32, device=t.device)
        _check(lr_query_leftmost(self.handle, sa, rank, lcp, lr_start, lr_len, stream), "lr_query_leftmost")
        _check(lr_device_status(self.handle, stream), "lr_query_leftmost (device)")
        return lr_start, lr_len

    def query_all(self, lcp, sa=None, rank=None, capacity: int | None = None, stream=None):
        """All LR's as CSR: (lr_len, lr_start, offsets, starts[:total]).  Give sa or rank."""
        import torch
        t = sa if sa is not None else rank
        n = int(t.numel())
        dev = t.device
        lr_len = torch.empty(n, dtype=torch.int32, device=dev)
        lr_start = torch.empty(n, dtype=torch.int32, device=dev)
        offsets = torch.empty(n + 1, dtype=torch.int64, device=dev)
        cap = 2 * n + 1024 if capacity is None else int(capacity)
        starts = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        st, total = lr_query_all(self.handle, sa, rank, lcp, lr_len, lr_start, offsets, starts, stream)
        if st == LR_ERR_CAPACITY:
            starts = torch.empty(total, dtype=torch.int32, device=dev)
            st, total = lr_query_all(self.handle, sa, rank, lcp, lr_len, lr_start, offsets, starts, stream)
        _check(st, "lr_query_all")
        return lr_len, lr_start, offsets, starts[:total]

    def build_arrays(self, text, stream=None):
        """(sa, rank, lcp) of a device uint8 text, built on the GPU by prefix doubling."""
        import torch
        n = int(text.numel())
        sa = torch.empty(n, dtype=torch.int32, device=text.device)
        rank = torch.empty(n, dtype=torch.int32, device=text.device)
        lcp = torch.empty(n + 1, dtype=torch.int32, device=text.device)
        st, _ = lr_build_arrays(self.handle, text, sa, rank, lcp, stream)
        _check(st, "lr_build_arrays")
        return sa, rank, lcp

    def build_arrays_batch(self, off, text, stream=None):
        """(sa, rank, lcp) of device uint8 texts packed back to back, in the batched-query layout."""
        import torch
        total = int(text.numel())
        num = int(off.numel()) - 1
        sa = torch.empty(max(total, 1), dtype=torch.int32, device=text.device)
        rank = torch.empty(max(total, 1), dtype=torch.int32, device=text.device)
        lcp = torch.empty(total + num, dtype=torch.int32, device=text.device)
        st, _ = lr_batch_build_arrays(self.handle, off, text, sa, rank, lcp, stream)
        _check(st, "lr_batch_build_arrays")
        return sa[:total], rank[:total], lcp

    def query_all_raw(self, lcp, rank, capacity: int | None = None, stream=None):
        """The raw-LLR variant: (lr_len, lr_start, offsets, starts[:total]) from rank and lcp."""
        import torch
        n = int(rank.numel())
        dev = rank.device
        lr_len = torch.empty(n, dtype=torch.int32, device=dev)
        lr_start = torch.empty(n, dtype=torch.int32, device=dev)
        offsets = torch.empty(n + 1, dtype=torch.int64, device=dev)
        cap = 2 * n + 1024 if capacity is None else int(capacity)
        starts = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        st, total = lr_query_all_raw(self.handle, rank, lcp, lr_len, lr_start, offsets, starts, stream)
        if st == LR_ERR_CAPACITY:
            starts = torch.empty(total, dtype=torch.int32, device=dev)
            st, total = lr_query_all_raw(self.handle, rank, lcp, lr_len, lr_start, offsets, starts, stream)
        _check(st, "lr_query_all_raw")
        return lr_len, lr_start, offsets, starts[:total]

    def query_leftmost_raw(self, lcp, rank, stream=None):
        import torch
        n = int(rank.numel())
        lr_start = torch.empty(n, dtype=torch.int32, device=rank.device)
        lr_len = torch.empty(n, dtype=torch.int32, device=rank.device)
        _check(lr_query_leftmost_raw(self.handle, rank, lcp, lr_start, lr_len, stream), "lr_query_leftmost_raw")
        _check(lr_device_status(self.handle, stream), "lr_query_leftmost_raw (device)")
        return lr_start, lr_len

    def walk_stats(self, lcp, rank, per_position: bool = False, stream=None):
        """Table 2's statistics; with per_position also the alpha and beta arrays."""
        import torch
        n = int(rank.numel())
        a = torch.empty(n, dtype=torch.int32, device=rank.device) if per_position else None
        b = torch.empty(n, dtype=torch.int32, device=rank.device) if per_position else None
        summary = lr_walk_stats(self.handle, rank, lcp, a, b, stream)
        return (summary, a, b) if per_position else summary

    def query_batch(self, off, lcp, sa=None, rank=None, capacity: int | None = None, stream=None):
        """Batched all-LR query over a flattened string table (device tensors).

        Returns flattened (lr_len, lr_start, offsets, starts[:total]); lr_start
        and starts are flattened positions.
        """
        import torch
        desc = batch_desc(off, lcp, sa=sa, rank=rank)
        n = desc.total
        dev = lcp.device
        lr_len = torch.empty(n, dtype=torch.int32, device=dev)
        lr_start = torch.empty(n, dtype=torch.int32, device=dev)
        offsets = torch.empty(n + 1, dtype=torch.int64, device=dev)
        cap = 2 * n + 1024 if capacity is None else int(capacity)
        starts = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        st, total = lr_batch_query_all(self.handle, desc, lr_len, lr_start, offsets, starts, stream)
        if st == LR_ERR_CAPACITY:
            starts = torch.empty(total, dtype=torch.int32, device=dev)
            st, total = lr_batch_query_all(self.handle, desc, lr_len, lr_start, offsets, starts, stream)
        _check(st, "lr_batch_query_all")
        return lr_len, lr_start, offsets, starts[:total]


class Server:
    """A liblr serving loop (continuous batching) with host-buffer jobs.

    submit() takes host arrays (numpy or CPU tensors; page-locked ones let
    the copies run asynchronously) and allocates the job's host outputs
    (starts: 4n + 1024 entries unless `capacity` is given; a job that needs
    more finishes with LR_ERR_CAPACITY and its total); the arrays are kept
    alive until the job's result is taken with wait().
    """

    def __init__(self, device: int = 0, **cfg):
        c = ServerConfig(device=device)
        for k, v in cfg.items():
            setattr(c, k, v)
        self.handle = lr_server_start(c)
        self._jobs = {}

    def submit(self, lcp=None, sa=None, rank=None, capacity: int | None = None, pinned: bool = False, out=None,
               text=None):
        """Queues one job; returns its id (raises LRError on LR_ERR_BUSY / NOMEM / ARG).

        Give lcp with sa or rank, or `text` alone (uint8; its arrays are built
        on the GPU; the server must be started with text_jobs=1).  `out` =
        (lr_len, lr_start, offsets, starts) host arrays to fill instead of
        newly allocated ones (capacity = len(starts)).
        """
        import numpy as np
        n = int(len(text) if text is not None else (len(sa) if sa is not None else len(rank)))
        if out is not None:
            outs = tuple(out)
            cap = int(len(outs[3]))
        else:
            cap = 4 * n + 1024 if capacity is None else int(capacity)
            if pinned:
                import torch
                outs = (torch.empty(n, dtype=torch.int32, pin_memory=True),
                        torch.empty(n, dtype=torch.int32, pin_memory=True),
                        torch.empty(n + 1, dtype=torch.int64, pin_memory=True),
                        torch.empty(max(cap, 1), dtype=torch.int32, pin_memory=True))
            else:
                outs = (np.empty(n, np.int32), np.empty(n, np.int32), np.empty(n + 1, np.int64),
                        np.empty(max(cap, 1), np.int32))
        job = Job(_ptr(sa), _ptr(rank), _ptr(lcp), n, _ptr(outs[0]), _ptr(outs[1]), _ptr(outs[2]), _ptr(outs[3]),
                  cap, _ptr(text))
        st, jid = lr_server_submit(self.handle, job)
        _check(st, "lr_server_submit")
        self._jobs[jid] = (sa if text is None else text, rank, lcp, outs)
        return jid

    def wait(self, job_id: int, timeout_ms: int = -1):
        """(result status, lr_len, lr_start, offsets, starts[:total]) of a finished job (host arrays)."""
        st, state, res, total = lr_server_wait(self.handle, job_id, timeout_ms)
        _check(st, "lr_server_wait")
        _, _, _, outs = self._jobs.pop(job_id)
        if state == LR_JOB_CANCELLED:
            return LR_ERR_BUSY, None, None, None, None
        conv = [o.numpy() if hasattr(o, "numpy") else o for o in outs]
        k = total if res == LR_OK else 0
        return res, conv[0], conv[1], conv[2], conv[3][:k]

    def cancel(self, job_id: int) -> int:
        return lr_server_cancel(self.handle, job_id)

    def stats(self, reset: bool = False) -> dict:
        return lr_server_stats_get(self.handle, reset)

    def close(self):
        if self.handle is not None:
            lr_server_stop(self.handle)
            self.handle = None
            self._jobs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
