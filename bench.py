#!/usr/bin/env python
"""Benchmark of the all-longest-repeats (all-LR) query on GB300.

One step = one lr_query_all over the whole n = 256 Mi English-like workload
(Zipf(1.1) words over a 50k vocabulary, 96-symbol alphabet, seed 3), with
rank and lcp resident in HBM: the Lemma 1 gather, the compaction, the
covering-max sweep and the CSR writer, all in the library's CUDA kernels.
The inputs (2 GiB) are larger than the 129 MB L2, so no flush is needed
between steps.

Prints one JSON line (rank 0).  Besides the device-resident throughput it
reports: e2e (the same query through the host-buffer entry point, pinned
host memory, H2D and D2H inside the timed region), the roofline of the
dominant kernel and of the whole path against the measured HBM copy
bandwidth, the CPU oracle timed on a bounded sample on the host cores, and
the SM clocks sampled during the timed region.

--impl reference times the CPU oracle (Algorithm 3 of the paper) on the same
workload, a bounded block of positions per step.

With torchrun (N > 1) each rank runs an independent replica of the query on
its own GPU (the query of one string does not shard); value is the positions
of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "all-LR query Gpositions/s and % of HBM roofline at n=256M; serving p50/p99"
UNIT = "Gpositions/s"
WORKLOAD = "english_256m"


# --------------------------------------------------------------------------- helpers

def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def source_hash(files) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1501_06663_gb300", "csrc")
    for f in sorted(files):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(phase: str, workload: str, n: int):
    """DRAM bytes per launch of a phase from the committed ncu summary, or
    None if its kernel sources changed since the capture."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    ent = json.load(open(p)).get("phases", {}).get(phase)
    if not ent or ent.get("workload") != workload or ent.get("n") != n \
            or ent.get("source_hash") != source_hash(ent["files"]):
        return None
    return ent.get("dram_bytes_per_launch")


def load_workload(name: str, n: int | None, ws: int, rank: int):
    """Rank 0 generates and preps; other ranks load its arrays from a shared temp dir."""
    import workloads as W
    if ws == 1:
        return W.single(name, n)
    import torch.distributed as dist
    tag = "lr_bench_%s_%s" % (name, n or "full")
    d = os.path.join("/dev/shm" if os.path.isdir("/dev/shm") else tempfile.gettempdir(), tag)
    if rank == 0:
        w = W.single(name, n)
        os.makedirs(d, exist_ok=True)
        for k in ("text", "sa", "rank", "lcp"):
            np.save(os.path.join(d, k + ".npy"), getattr(w, k))
    dist.barrier()
    if rank != 0:
        arrs = {k: np.load(os.path.join(d, k + ".npy")) for k in ("text", "sa", "rank", "lcp")}
        w = W.Workload(name, arrs["text"], arrs["sa"], arrs["rank"], arrs["lcp"])
    dist.barrier()
    if rank == 0:
        import shutil
        shutil.rmtree(d, ignore_errors=True)
    return w


def max_over_ranks(x: float, device=None) -> float:
    """The largest x over all ranks (x itself with one rank).  The tensor lives
    on `device` (CUDA for NCCL, CPU for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws: int, n: int, ms: float) -> float:
    """Gpositions/s of ws replicas of an n-position query whose slowest rank took ms."""
    return ws * n / (ms * 1e-3) / 1e9


def host_cores() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_oracle_rate(w, target_s: float, seed: int = 0, threads: int = 1):
    """Algorithm 3 (the oracle as it stands) over a contiguous block of
    positions, split into `threads` disjoint sub-blocks run at the same time
    (one host core each)."""
    import oracle
    n = w.n
    rng = np.random.default_rng(seed)
    probe = 20000 * threads
    a = int(rng.integers(0, max(1, n - probe)))
    t0 = time.perf_counter()
    oracle.lr_at_range(w.rank, w.lcp, a, min(n, a + probe), threads=threads)
    dt = max(time.perf_counter() - t0, 1e-4)
    block = int(min(n, max(probe, probe * target_s / dt)))
    a = int(rng.integers(0, max(1, n - block)))
    t0 = time.perf_counter()
    oracle.lr_at_range(w.rank, w.lcp, a, a + block, threads=threads)
    dt = time.perf_counter() - t0
    return block / dt / 1e9, block, a, dt


# --------------------------------------------------------------------------- batched and serving legs

def _event_ms(stream, fn, reps, warm=2):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def host_link(dev, stream, h_in, d_in, h_out, d_out, reps: int = 3):
    """Host link bandwidth (GB/s) of plain pinned copies on `stream`: host to
    device (h_in -> d_in), device to host (d_out -> h_out) and both at once on
    two streams.  The e2e figure cannot beat the slowest of the three for its
    bytes per step."""
    import torch
    s2 = torch.cuda.Stream(dev)

    def h2d():
        with torch.cuda.stream(stream):
            d_in.copy_(h_in, non_blocking=True)

    def d2h():
        with torch.cuda.stream(stream):
            h_out.copy_(d_out, non_blocking=True)

    def both():
        ev = torch.cuda.Event()
        ev.record(stream)
        s2.wait_event(ev)
        with torch.cuda.stream(stream):
            d_in.copy_(h_in, non_blocking=True)
        with torch.cuda.stream(s2):
            h_out.copy_(d_out, non_blocking=True)
        done = torch.cuda.Event()
        done.record(s2)
        stream.wait_event(done)

    b_in = h_in.numel() * h_in.element_size()
    b_out = h_out.numel() * h_out.element_size()
    out = {"h2d_gbs": round(b_in / (_event_ms(stream, h2d, reps, warm=1) * 1e6), 1),
           "d2h_gbs": round(b_out / (_event_ms(stream, d2h, reps, warm=1) * 1e6), 1),
           "duplex_gbs": round((b_in + b_out) / (_event_ms(stream, both, reps, warm=1) * 1e6), 1)}
    torch.cuda.synchronize(dev)
    return out


def batched_leg(lr, dev, stream, count: int, reps: int):
    """The batched mix (log-uniform lengths 1 Ki - 4 Mi, half DNA with planted
    repeats, half protein with tandem repeats) in one batched query, tuned and
    as a captured plan, against one lr_query_all launch per string."""
    import torch

    import workloads as W
    text, off, _ = W.batched_mix(count=count, lo=1024, hi=4 * W.MI, seed=4)
    total = int(off[-1])
    # sa / rank / lcp of every string built on the GPU (the host prep of
    # about 2 G symbols would take minutes), checked against the host prep
    # on a sample of strings
    d_off = torch.from_numpy(off).to(dev)
    d_text = torch.from_numpy(text).to(dev)
    builder = lr.Context(dev.index)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    d_sa, d_rank, d_lcp = builder.build_arrays_batch(d_off, d_text, stream=stream)
    build_ms = (time.perf_counter() - t0) * 1e3
    builder.close()
    del d_text
    torch.cuda.empty_cache()
    sample = np.random.default_rng(44).choice(count, min(16, count), replace=False)
    build_ok = True
    for j in sample:
        a, b = int(off[j]), int(off[j + 1])
        if b > a:
            h_sa, h_rank, h_lcp = W.prep(text[a:b])
            build_ok &= bool(np.array_equal(d_sa[a:b].cpu().numpy(), h_sa)
                             and np.array_equal(d_rank[a:b].cpu().numpy(), h_rank)
                             and np.array_equal(d_lcp[a + j:b + j + 1].cpu().numpy(), h_lcp))
    del text
    if not build_ok:
        raise RuntimeError("batched leg: GPU-built arrays differ from the host prep")
    ln = torch.empty(total, dtype=torch.int32, device=dev)
    st = torch.empty(total, dtype=torch.int32, device=dev)
    offs = torch.empty(total + 1, dtype=torch.int64, device=dev)
    ctx = lr.lr_create(dev.index)
    desc = lr.batch_desc(d_off, d_lcp, sa=d_sa)
    s, tot = lr.lr_batch_query_all(ctx, desc, ln, st, offs, torch.empty(1, dtype=torch.int32, device=dev), stream)
    if s not in (lr.LR_OK, lr.LR_ERR_CAPACITY):
        raise lr.LRError(s, "lr_batch_query_all")
    starts = torch.empty(max(tot, 1), dtype=torch.int32, device=dev)

    def batched(d=desc):
        r, _ = lr.lr_batch_query_all(ctx, d, ln, st, offs, starts, stream, sync=False)
        if r != lr.LR_OK:
            raise lr.LRError(r, "lr_batch_query_all")

    batched_ms = _event_ms(stream, batched, reps)
    both = lr.batch_desc(d_off, d_lcp, sa=d_sa, rank=d_rank)
    code = lr.lr_autotune(ctx, both, ln, st, offs, starts, stream)
    tuned_ms = _event_ms(stream, lambda: batched(both), reps)
    plan = lr.lr_plan_create(ctx, both, ln, st, offs, starts)
    plan_ms = _event_ms(stream, lambda: lr.lr_plan_launch(plan, stream), reps)
    lr.lr_plan_destroy(plan)
    if lr.lr_device_status(ctx, stream) != lr.LR_OK:
        raise RuntimeError("batched leg: device error")

    # one lr_query_all per string, on views of the same device arrays
    h_off = off.tolist()
    flat_off = offs.cpu().numpy()
    offs2 = torch.empty(total + count, dtype=torch.int64, device=dev)
    views = []
    for j in range(count):
        a, b = h_off[j], h_off[j + 1]
        o0, o1 = int(flat_off[a]), int(flat_off[b])
        views.append((d_sa[a:b], d_lcp[a + j:b + j + 1], ln[a:b], st[a:b], offs2[a + j:b + j + 1],
                      starts[o0:max(o1, o0 + 1)]))

    def per_string():
        for v_sa, v_lcp, v_ln, v_st, v_off, v_starts in views:
            r, _ = lr.lr_query_all(ctx, v_sa, None, v_lcp, v_ln, v_st, v_off, v_starts, stream, sync=False)
            if r != lr.LR_OK:
                raise lr.LRError(r, "lr_query_all")

    loop_ms = _event_ms(stream, per_string, max(1, reps // 2), warm=1)
    if lr.lr_device_status(ctx, stream) != lr.LR_OK:
        raise RuntimeError("batched leg: device error in the per-string loop")
    lr.lr_destroy(ctx)
    g = lambda ms: round(total / (ms * 1e-3) / 1e9, 3)
    peak, peak_kind = measured_peaks()
    path_bytes = 4.0 * total + 4.0 * (total + count) + 16.0 * total + 8.0 * (total + 1) + 4.0 * tot
    frac = lambda ms: round(path_bytes / (ms * 1e-3) / 1e9 / peak, 4)
    return {"workload": "batched mix: %d strings, log-uniform lengths 1Ki-4Mi (seed 4)" % count,
            "positions": total, "lr_starts": tot, "reps": reps,
            "arrays": {"built_on": "GPU (lr_batch_build_arrays)", "ms": round(build_ms, 1),
                       "equal_to_host_prep": "checked on %d strings" % len(sample)},
            "path_roofline_frac": {"batched": frac(batched_ms), "autotuned": frac(tuned_ms), "peak_kind": peak_kind},
            "batched": {"ms": round(batched_ms, 3), "value": g(batched_ms)},
            "autotuned": {"ms": round(tuned_ms, 3), "value": g(tuned_ms), "shape_code": code},
            "captured_plan": {"ms": round(plan_ms, 3), "value": g(plan_ms)},
            "one_string_per_launch": {"ms": round(loop_ms, 3), "value": g(loop_ms)},
            "unit": UNIT}


def serving_leg(lr, dev, count: int, loads, seed: int = 5):
    """Poisson arrivals of jobs from the serving pool (lognormal lengths,
    median 100 Ki, sigma 1, 70% DNA / 30% protein) into the library's serving
    loop, host buffers in pinned memory, at offered loads that are fractions
    of the loop's measured saturation throughput; the same arrival traces
    through a plain loop of one lr_query_all_host per job."""
    import torch

    import workloads as W
    text_all, off, _ = W.serving_mix(count, seed=seed)
    sa, rank, lcp = W.prep_many(text_all, off)
    del rank
    lens = np.diff(off)
    total = int(off[-1])
    caps = 3 * lens + 1024
    coff = np.zeros(count + 1, np.int64)
    np.cumsum(caps, out=coff[1:])
    h_sa = torch.from_numpy(sa).pin_memory()
    h_lcp = torch.from_numpy(lcp).pin_memory()
    del sa, lcp
    o_ln = torch.empty(total, dtype=torch.int32).pin_memory()
    o_st = torch.empty(total, dtype=torch.int32).pin_memory()
    o_off = torch.empty(total + count, dtype=torch.int64).pin_memory()
    o_starts = torch.empty(int(coff[-1]), dtype=torch.int32).pin_memory()
    jobs = []
    for j in range(count):
        a, b = int(off[j]), int(off[j + 1])
        jobs.append((h_sa[a:b], h_lcp[a + j:b + j + 1],
                     (o_ln[a:b], o_st[a:b], o_off[a + j:b + j + 1], o_starts[int(coff[j]):int(coff[j + 1])])))
    mean_len = total / count
    srv = lr.Server(dev.index, max_batch_positions=1 << 25, slots=4, max_inflight=2, batch_window_us=1000)

    def run_ours(arrivals):
        srv.stats(reset=True)
        t0 = time.perf_counter()
        ids = []
        for (j_sa, j_lcp, out), t in zip(jobs, arrivals):
            while True:
                dt = t0 + t - time.perf_counter()
                if dt <= 0:
                    break
                if dt > 2e-4:
                    time.sleep(dt - 1e-4)
            ids.append(srv.submit(j_lcp, sa=j_sa, out=out))
        bad = 0
        for i in ids:
            r = srv.wait(i, timeout_ms=600000)[0]
            bad += r != lr.LR_OK
        wall = time.perf_counter() - t0
        st = srv.stats()
        if bad:
            raise RuntimeError("serving leg: %d jobs failed" % bad)
        return {"p50_ms": round(st["p50_us"] / 1e3, 3), "p99_ms": round(st["p99_us"] / 1e3, 3),
                "value": round(total / wall / 1e9, 3), "batches": st["batches"], "jobs": count}

    ctx = lr.lr_create(dev.index)
    stream = torch.cuda.current_stream(dev)

    def run_plain(arrivals):
        lat = []
        t0 = time.perf_counter()
        for (j_sa, j_lcp, out), t in zip(jobs, arrivals):
            while True:
                dt = t0 + t - time.perf_counter()
                if dt <= 0:
                    break
                if dt > 2e-4:
                    time.sleep(dt - 1e-4)
            r, _ = lr.lr_query_all_host(ctx, j_sa, None, j_lcp, out[0], out[1], out[2], out[3], stream)
            if r != lr.LR_OK:
                raise lr.LRError(r, "lr_query_all_host")
            lat.append(time.perf_counter() - (t0 + t))
        wall = time.perf_counter() - t0
        lat = np.array(lat) * 1e3
        return {"p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
                "value": round(total / wall / 1e9, 3)}

    zero = np.zeros(count)
    run_ours(zero)                                   # warm-up: slots, starts buffers
    sat = run_ours(zero)
    run_plain(zero[:8])
    plain_sat = run_plain(zero)
    rng = np.random.default_rng(seed)
    sweep = []
    for load in loads:
        lam = load * sat["value"] * 1e9 / mean_len   # jobs per second
        arrivals = np.cumsum(rng.exponential(1.0 / lam, size=count))
        sweep.append({"offered_load": load, "ours": run_ours(arrivals), "one_job_per_call": run_plain(arrivals)})
    srv.close()
    lr.lr_destroy(ctx)
    # text jobs: the same strings without host prep; their arrays are built
    # on the GPU in the serving loop (saturation and one offered load)
    h_text = torch.from_numpy(text_all).pin_memory()
    tjobs = [(h_text[int(off[j]):int(off[j + 1])], jobs[j][2]) for j in range(count)]
    tsrv = lr.Server(dev.index, max_batch_positions=1 << 25, slots=4, max_inflight=2, batch_window_us=1000,
                     text_jobs=1)

    def run_text(arrivals):
        tsrv.stats(reset=True)
        t0 = time.perf_counter()
        ids = []
        for (j_text, out), t in zip(tjobs, arrivals):
            while True:
                dt = t0 + t - time.perf_counter()
                if dt <= 0:
                    break
                if dt > 2e-4:
                    time.sleep(dt - 1e-4)
            ids.append(tsrv.submit(text=j_text, out=out))
        bad = sum(tsrv.wait(i, timeout_ms=600000)[0] != lr.LR_OK for i in ids)
        wall = time.perf_counter() - t0
        st = tsrv.stats()
        if bad:
            raise RuntimeError("serving leg (text jobs): %d jobs failed" % bad)
        return {"p50_ms": round(st["p50_us"] / 1e3, 3), "p99_ms": round(st["p99_us"] / 1e3, 3),
                "value": round(total / wall / 1e9, 3), "batches": st["batches"]}

    run_text(zero)
    tsat = run_text(zero)
    lam = 0.6 * tsat["value"] * 1e9 / mean_len
    text_jobs = {"saturation": tsat["value"],
                 "at_0.6_saturation": run_text(np.cumsum(rng.exponential(1.0 / lam, size=count))),
                 "note": "jobs carry only their string; sa / rank / lcp are built on the GPU in the loop"}
    tsrv.close()
    mid = min(sweep, key=lambda e: abs(e["offered_load"] - 0.6))
    return {"workload": "serving pool: %d jobs, lognormal lengths (median 100Ki, sigma 1, 1Ki-16Mi), "
                        "70%% DNA / 30%% protein (seed %d), Poisson arrivals" % (count, seed),
            "positions": total, "unit": UNIT, "timing": "wall clock, submit to results in pinned host memory",
            "saturation": sat["value"], "one_job_per_call_saturation": plain_sat["value"],
            "p50_ms": mid["ours"]["p50_ms"], "p99_ms": mid["ours"]["p99_ms"], "at_offered_load": mid["offered_load"],
            "sweep": sweep, "text_jobs": text_jobs}


def single_leg(lr, dev, stream, name: str, steps: int, warmup: int):
    """One lr_query_all per step on another single-string workload (sa + lcp
    resident), with its whole-path roofline."""
    import torch

    import workloads as W
    w = W.single(name)
    n = w.n
    d_sa = torch.from_numpy(w.sa).to(dev)
    d_lcp = torch.from_numpy(w.lcp).to(dev)
    ln = torch.empty(n, dtype=torch.int32, device=dev)
    st = torch.empty(n, dtype=torch.int32, device=dev)
    off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    ctx = lr.lr_create(dev.index)
    s0, total = lr.lr_query_all(ctx, d_sa, None, d_lcp, ln, st, off, torch.empty(1, dtype=torch.int32, device=dev),
                                stream)
    if s0 not in (lr.LR_OK, lr.LR_ERR_CAPACITY):
        raise lr.LRError(s0, "lr_query_all (%s)" % name)
    starts = torch.empty(max(total, 1), dtype=torch.int32, device=dev)

    def step():
        r, _ = lr.lr_query_all(ctx, d_sa, None, d_lcp, ln, st, off, starts, stream, sync=False)
        if r != lr.LR_OK:
            raise lr.LRError(r, "lr_query_all (%s)" % name)

    ms = _event_ms(stream, step, steps, warm=warmup)
    lr.lr_set_phase_timing(ctx, True)
    step()
    phases = lr.lr_phase_times(ctx)
    lr.lr_set_phase_timing(ctx, False)
    if lr.lr_device_status(ctx, stream) != lr.LR_OK:
        raise RuntimeError("%s: device error" % name)
    lr.lr_destroy(ctx)
    peak, peak_kind = measured_peaks()
    path_bytes = 4.0 * n + 4.0 * (n + 1) + 4.0 * n + 4.0 * n + 8.0 * (n + 1) + 4.0 * total
    inputs_mb = (8 * n + 4) / 1e6
    return {"workload": name, "n": n, "ms_per_step": round(ms, 4), "value": round(n / (ms * 1e-3) / 1e9, 3),
            "unit": UNIT, "steps": steps, "total_lr_starts": total,
            "kernel_ms": {nm: round(p, 4) for nm, p in zip(["partition", "bucket_llr", "cover"], phases or [])},
            "path_roofline": {"achieved": round(path_bytes / (ms * 1e-3) / 1e9, 1), "peak": peak, "unit": "GB/s",
                              "frac": round(path_bytes / (ms * 1e-3) / 1e9 / peak, 4), "peak_kind": peak_kind},
            "l2": "inputs %.0f MB: %s" % (inputs_mb, "larger than the 129 MB L2" if inputs_mb > 129 else
                                          "fit in the 129 MB L2 (warm between steps)")}


# --------------------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1501_06663_gb300 as lr

    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lr.build_library() if rank == 0 else None
    if ws > 1:
        dist.barrier()
    w = load_workload(args.workload, args.n, ws, rank)
    n = w.n
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ctx = lr.lr_create(local)
    d_sa = torch.from_numpy(w.sa).to(dev)
    d_rank = torch.from_numpy(w.rank).to(dev)
    d_lcp = torch.from_numpy(w.lcp).to(dev)
    ln = torch.empty(n, dtype=torch.int32, device=dev)
    st = torch.empty(n, dtype=torch.int32, device=dev)
    off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    starts = torch.empty(1, dtype=torch.int32, device=dev)
    status, total = lr.lr_query_all(ctx, d_sa, None, d_lcp, ln, st, off, starts, stream)
    if status not in (lr.LR_OK, lr.LR_ERR_CAPACITY):
        raise lr.LRError(status, "lr_query_all")
    starts = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
    m = lr.lr_last_compact_size(ctx, stream)

    def step(sa=d_sa, rank=None):
        s, _ = lr.lr_query_all(ctx, sa, rank, d_lcp, ln, st, off, starts, stream, sync=False)
        if s != lr.LR_OK:
            raise lr.LRError(s, "lr_query_all")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    launches = lr.lr_last_launch_count(ctx) * args.steps
    dstat = lr.lr_device_status(ctx, stream)
    if dstat != lr.LR_OK:
        raise lr.LRError(dstat, "device status after the timed steps")
    ms = max_over_ranks(ms, dev)

    # per-phase durations (CUDA events on the launching stream, recorded by the library)
    def phase_avg(**kw):
        lr.lr_set_phase_timing(ctx, True)
        acc = None
        reps = max(3, min(args.steps, 20))
        for _ in range(reps):
            step(**kw)
            t = lr.lr_phase_times(ctx)
            acc = list(t) if acc is None else [a + b for a, b in zip(acc, t)]
        lr.lr_set_phase_timing(ctx, False)
        return [a / reps for a in acc]

    per = phase_avg()
    # rank alone (the paper's inputs): the rank-window front end from 2^24
    # positions on, else the rank gather; same cover kernel
    for _ in range(2):
        step(sa=None, rank=d_rank)
    torch.cuda.synchronize(dev)
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    gsteps = max(3, min(args.steps, 10))
    for _ in range(gsteps):
        step(sa=None, rank=d_rank)
    g1.record(stream)
    torch.cuda.synchronize(dev)
    gather_ms = g0.elapsed_time(g1) / gsteps
    per_gather = phase_avg(sa=None, rank=d_rank)
    rank_front = "rank windows" if len(per_gather) == 3 else "rank gather"
    rank_names = ["rank_windows_partition", "bucket_llr", "cover"] if len(per_gather) == 3 else ["gather_llr", "cover"]
    # the paper's data flow itself (rank + a random gather of lcp), run as a
    # batch of one string, which always takes the gather
    paper_gather = None
    if rank_front == "rank windows":
        d_off1 = torch.tensor([0, n], dtype=torch.int64, device=dev)
        desc1 = lr.batch_desc(d_off1, d_lcp, rank=d_rank)

        def gather_step():
            r, _ = lr.lr_batch_query_all(ctx, desc1, ln, st, off, starts, stream, sync=False)
            if r != lr.LR_OK:
                raise lr.LRError(r, "lr_batch_query_all (rank gather)")

        pg_ms = _event_ms(stream, gather_step, max(3, min(args.steps, 10)), warm=2)
        lr.lr_set_phase_timing(ctx, True)
        gather_step()
        pg = lr.lr_phase_times(ctx)
        lr.lr_set_phase_timing(ctx, False)
        paper_gather = {"ms_per_step": round(pg_ms, 4), "value": round(whole_job_rate(ws, n, pg_ms), 3),
                        "kernel_ms": {nm: round(t, 4) for nm, t in zip(["gather_llr", "cover"], pg)},
                        "how": "one-string batch (lr_batch_query_all), rank only"}

    # the leftmost-only query (Algorithm 2's output, no CSR pass), same front end
    def leftmost():
        s_l = lr.lr_query_leftmost(ctx, d_sa, None, d_lcp, st, ln, stream)
        if s_l != lr.LR_OK:
            raise lr.LRError(s_l, "lr_query_leftmost")

    left_ms = _event_ms(stream, leftmost, max(3, min(args.steps, 20)), warm=2)
    lr.lr_set_phase_timing(ctx, True)
    left_acc = None
    for _ in range(3):
        leftmost()
        t = lr.lr_phase_times(ctx)
        left_acc = list(t) if left_acc is None else [a + b for a, b in zip(left_acc, t)]
    lr.lr_set_phase_timing(ctx, False)
    if lr.lr_device_status(ctx, stream) != lr.LR_OK:
        raise RuntimeError("leftmost query: device error")
    leftmost_query = {"ms_per_step": round(left_ms, 4), "value": round(whole_job_rate(ws, n, left_ms), 3),
                      "kernel_ms": {nm: round(a / 3, 4) for nm, a in zip(["partition", "bucket_llr", "cover"],
                                                                         left_acc)}}

    # Table 2's walk statistics and the raw-LLR variant (no compaction), for comparison
    walk = lr.lr_walk_stats(ctx, d_rank, d_lcp, stream=stream)
    raw = None
    if walk["alpha_sum"] <= 64 * n:                  # the raw walks cost about alpha per position
        raw_ms = _event_ms(stream, lambda: lr.lr_query_all_raw(ctx, d_rank, d_lcp, ln, st, off, starts, stream,
                                                               sync=False), 3, warm=1)
        if lr.lr_device_status(ctx, stream) != lr.LR_OK:
            raise RuntimeError("raw-LLR variant: device error")
        raw = {"ms_per_step": round(raw_ms, 4), "value": round(whole_job_rate(ws, n, raw_ms), 3)}

    # the step before the query: sa / rank / lcp built on the GPU from the text
    # (prefix doubling), checked against the host prep
    d_text = torch.from_numpy(w.text).to(dev)
    b_sa = torch.empty(n, dtype=torch.int32, device=dev)
    b_rank = torch.empty(n, dtype=torch.int32, device=dev)
    b_lcp = torch.empty(n + 1, dtype=torch.int32, device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    s_b, rounds = lr.lr_build_arrays(ctx, d_text, b_sa, b_rank, b_lcp, stream)
    build_ms = (time.perf_counter() - t0) * 1e3
    if s_b != lr.LR_OK:
        raise lr.LRError(s_b, "lr_build_arrays")
    index_build = {"ms": round(build_ms, 1), "value": round(n / (build_ms * 1e-3) / 1e9, 3), "unit": UNIT,
                   "doubling_rounds": rounds,
                   "equal_to_host_prep": bool(torch.equal(b_sa, d_sa) and torch.equal(b_rank, d_rank)
                                              and torch.equal(b_lcp, d_lcp))}
    del d_text, b_sa, b_rank, b_lcp
    torch.cuda.empty_cache()

    # e2e through the host-buffer entry point, pinned host memory
    h_sa = torch.from_numpy(w.sa).pin_memory()
    h_lcp = torch.from_numpy(w.lcp).pin_memory()
    h_ln = torch.empty(n, dtype=torch.int32).pin_memory()
    h_st = torch.empty(n, dtype=torch.int32).pin_memory()
    h_off = torch.empty(n + 1, dtype=torch.int64).pin_memory()
    h_starts = torch.empty(max(total, 1), dtype=torch.int32).pin_memory()
    e2e_steps = max(2, min(args.steps, 5))
    lr.lr_query_all_host(ctx, h_sa, None, h_lcp, h_ln, h_st, h_off, h_starts, stream)   # warm the buffers
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s, tot2 = lr.lr_query_all_host(ctx, h_sa, None, h_lcp, h_ln, h_st, h_off, h_starts, stream)
        if s != lr.LR_OK or tot2 != total:
            raise lr.LRError(s, "lr_query_all_host")
    e2e_single_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    e2e_single_ms = max_over_ranks(e2e_single_ms, dev)
    link = host_link(dev, stream, h_sa, d_sa, h_ln, ln)
    h2d_step = 4 * n + 4 * (n + 1)                                   # sa + lcp
    d2h_step = 4 * n + 4 * n + 8 * (n + 1) + 4 * total + 8            # lr_len, lr_start, offsets, starts, total
    link_ms = max(h2d_step / link["h2d_gbs"], d2h_step / link["d2h_gbs"],
                  (h2d_step + d2h_step) / link["duplex_gbs"]) * 1e-6
    link["e2e_bound"] = round(whole_job_rate(ws, n, link_ms), 3)
    # the same calls with `inflight` steps at a time (one host thread, context,
    # stream and output buffers each; ctypes releases the GIL), so that one
    # step's device-to-host copies overlap the next one's host-to-device
    # copies and kernels: whole-job throughput of back-to-back queries
    inflight = max(1, args.e2e_inflight)
    e2e_ms = e2e_single_ms
    e2e_multi_ms = None
    if inflight > 1:
        ctxs = [ctx] + [lr.lr_create(local) for _ in range(inflight - 1)]
        streams = [stream] + [torch.cuda.Stream(dev) for _ in range(inflight - 1)]
        outs = [(h_ln, h_st, h_off, h_starts)] + [
            (torch.empty(n, dtype=torch.int32).pin_memory(), torch.empty(n, dtype=torch.int32).pin_memory(),
             torch.empty(n + 1, dtype=torch.int64).pin_memory(),
             torch.empty(max(total, 1), dtype=torch.int32).pin_memory()) for _ in range(inflight - 1)]
        errors = []

        def worker(i, nsteps):
            for _ in range(nsteps):
                r, t2 = lr.lr_query_all_host(ctxs[i], h_sa, None, h_lcp, *outs[i], streams[i])
                if r != lr.LR_OK or t2 != total:
                    errors.append(r)
                    return

        threads = [threading.Thread(target=worker, args=(i, 1)) for i in range(inflight)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        torch.cuda.synchronize(dev)
        threads = [threading.Thread(target=worker, args=(i, e2e_steps)) for i in range(inflight)]
        t0 = time.perf_counter()
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        e2e_multi_ms = (time.perf_counter() - t0) * 1e3 / (e2e_steps * inflight)
        if errors:
            raise lr.LRError(errors[0], "lr_query_all_host (concurrent)")
        e2e_multi_ms = max_over_ranks(e2e_multi_ms, dev)
        e2e_ms = min(e2e_ms, e2e_multi_ms)           # the faster way to drive the same call
        for c in ctxs[1:]:
            lr.lr_destroy(c)
    lr.lr_destroy(ctx)
    step = phase_avg = None
    del d_sa, d_rank, d_lcp, ln, st, off, starts
    torch.cuda.empty_cache()
    batched = serving = None
    others = []
    if rank == 0:
        for name in [x for x in args.extra_workloads.split(",") if x]:
            others.append(single_leg(lr, dev, stream, name, max(3, min(args.steps, 20)), 3))
            torch.cuda.empty_cache()
    if rank == 0 and args.batched_count > 0:
        batched = batched_leg(lr, dev, stream, args.batched_count, max(3, min(args.steps, 10)))
        torch.cuda.empty_cache()
    if rank == 0 and args.serving_jobs > 0:
        serving = serving_leg(lr, dev, args.serving_jobs, [float(x) for x in args.serving_loads.split(",")])

    if rank == 0:
        peak, peak_kind = measured_peaks()
        names = ["partition", "bucket_llr", "cover"]
        # bytes each phase has to move in this design: partition: sa + lcp read,
        # level-1 entries written and read, level-2 entries written; bucket:
        # entries read, compact LLR's written; cover: compact LLR's read, every
        # output written once
        algo = {
            "partition": 4.0 * n + 4.0 * (n + 1) + 12.0 * n,
            "bucket_llr": 4.0 * n + 8.0 * m,
            "cover": 8.0 * m + 4.0 * n + 4.0 * n + 8.0 * (n + 1) + 4.0 * total,
        }
        dom = int(np.argmax(per))
        kname = names[dom]
        achieved = algo[kname] / (per[dom] * 1e-3) / 1e9
        # compulsory bytes of the whole query: inputs read once, outputs written once
        path_bytes = 4.0 * n + 4.0 * (n + 1) + 4.0 * n + 4.0 * n + 8.0 * (n + 1) + 4.0 * total
        path_achieved = path_bytes / (ms * 1e-3) / 1e9
        value = whole_job_rate(ws, n, ms)
        cores = host_cores()
        rate, block, a0, dt = cpu_oracle_rate(w, args.cpu_seconds, threads=cores)
        rate1, block1, a1, dt1 = cpu_oracle_rate(w, args.cpu_seconds / 4, seed=1, threads=1)
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "parallelism": "replicas" if ws > 1 else "single",
                       "inputs": "sa+lcp resident in HBM (%.2f GiB, larger than the 129 MB L2: no flush)"
                                 % ((8 * n + 4) / 2**30),
                       "input": "sa+lcp (rank-order front end)",
                       "total_lr_starts": total, "compact_llr": m},
            "roofline": {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                         "traffic": recorded_traffic(kname, args.workload, n),
                         "algorithmic_bytes_per_launch": algo[kname], "avg_launch_ms": round(per[dom], 4)},
            "path_roofline": {"bound": "hbm", "achieved": round(path_achieved, 1), "peak": peak, "unit": "GB/s",
                              "frac": round(path_achieved / peak, 4), "peak_kind": peak_kind,
                              "algorithmic_bytes_per_step": path_bytes},
            "kernel_ms": {nm: round(p, 4) for nm, p in zip(names, per)},
            "walk_steps": {"alpha": round(walk["alpha_sum"] / n, 3), "alpha_max": walk["alpha_max"],
                           "beta": round(walk["beta_sum"] / n, 3), "beta_max": walk["beta_max"],
                           "definition": "LLR's covering a position, raw (alpha) and useful (beta), Table 2"},
            "raw_llr_variant": raw,
            "index_build": index_build,
            "leftmost_query": leftmost_query,
            "rank_only_query": {"ms_per_step": round(gather_ms, 4),
                                "value": round(whole_job_rate(ws, n, gather_ms), 3), "front": rank_front,
                                "kernel_ms": {nm: round(p, 4) for nm, p in zip(rank_names, per_gather)}},
            "rank_gather_front": paper_gather,
            "cpu_baseline": {"value": round(rate, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "Algorithm 3 (two leftward raw-LLR walks per position) on positions "
                                       "[%d, %d) of the same workload, split into %d blocks run at once on the "
                                       "host cores, %.1f s" % (a0, a0 + block, cores, dt)},
            "cpu_baseline_single_core": {"value": round(rate1, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                                         "sample": "Algorithm 3 on positions [%d, %d), one thread, %.1f s"
                                                   % (a1, a1 + block1, dt1)},
            "other_workloads": others,
            "e2e": {"value": round(whole_job_rate(ws, n, e2e_ms), 3), "unit": UNIT,
                    "h2d_bytes_per_step": h2d_step,
                    "d2h_bytes_per_step": d2h_step,
                    "steps_in_flight": inflight if e2e_multi_ms is not None and e2e_ms == e2e_multi_ms else 1,
                    "one_in_flight": round(whole_job_rate(ws, n, e2e_single_ms), 3),
                    "%d_in_flight" % inflight: (round(whole_job_rate(ws, n, e2e_multi_ms), 3)
                                               if e2e_multi_ms is not None else None),
                    "host_link": link,
                    "api": "lr_query_all_host (pinned host buffers; copies and kernels inside the call)"},
            "gpu_launches": launches,
            "clocks": clk,
            "batched": batched,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


# --------------------------------------------------------------------------- reference arm

def run_reference(args):
    ws, rank, local = dist_info()
    if rank != 0:
        return
    import workloads as W
    w = W.single(args.workload, args.n)
    cores = host_cores()
    for _ in range(args.warmup):
        cpu_oracle_rate(w, 0.5, seed=1, threads=cores)
    rates, blocks, secs = [], 0, 0.0
    for k in range(args.steps):
        rate, block, a0, dt = cpu_oracle_rate(w, args.ref_step_seconds, seed=100 + k, threads=cores)
        blocks += block
        secs += dt
    value = blocks / secs / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(secs * 1e3 / args.steps, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "n": w.n, "parallelism": "single"},
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "Algorithm 3 on %d random contiguous blocks, %d positions in total, each block "
                                   "split into %d sub-blocks run at once on the host cores" % (args.steps, blocks, cores)},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--n", type=int, default=None, help="shrink the workload (same seed); default full size")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-step-seconds", type=float, default=2.0)
    ap.add_argument("--e2e-inflight", type=int, default=3,
                    help="host-buffer queries in flight at once in the e2e measurement")
    ap.add_argument("--batched-count", type=int, default=4096,
                    help="strings of the batched leg (4096 = the full batched mix; 0 = skip)")
    ap.add_argument("--extra-workloads", default="dna_iid_1m,dna_64m",
                    help="other single-string workloads timed after the main one (comma-separated; empty = none)")
    ap.add_argument("--serving-jobs", type=int, default=2000, help="jobs in the serving pool (0 = skip)")
    ap.add_argument("--serving-loads", default="0.2,0.4,0.6,0.8,1.0,1.2",
                    help="offered loads, as fractions of the serving loop's saturation throughput")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
