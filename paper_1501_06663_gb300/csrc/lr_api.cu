// C ABI of liblr (declared in include/lr.h): contexts, argument checks,
// scratch management and the host-buffer entry point.  All arithmetic of
// the query runs in the kernels of lr_query.cu.
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <new>
#include <vector>
#include "lr.h"
#include "lr_internal.h"
#include "lr_device.cuh"

struct lr_ctx {
    int device = 0;
    int last_cuda_error = 0;
    int last_launches = 0;
    unsigned* d_err = nullptr;            // sticky device error bits
    unsigned char* scratch = nullptr;     // lr::Scratch storage
    size_t scratch_bytes = 0;
    long long scratch_n = 0;              // positions the scratch is laid out for
    long long* h_pinned = nullptr;        // [0] total, [1] error bits
    unsigned char* hostpath = nullptr;    // device buffers of lr_query_all_host
    size_t hostpath_bytes = 0;
    int sms = 0;                          // SM count of the device
    long long last_n = 0;                 // size of the last query (its tile_cbase[ntiles] is m)
    lr::PhaseEvents events;               // per-kernel timing (off by default)
    bool events_created = false;
    std::map<int, int> tuned;             // shape class -> shape code (lr_autotune)
    lr::IndexWork index_work;             // work memory of lr_build_arrays / lr_batch_build_arrays
    int64_t* d_off2 = nullptr;            // {0, n} for single-string builds
    int64_t* d_chunk_off = nullptr;       // rebased offsets of one chunk of a large batched build
    long long chunk_off_cap = 0;          // entries d_chunk_off holds
    int spin_limit = lr::kSpinLimit;      // look-back poll limit of this context's queries
    long long hold_tile = -1;             // test hook (lr_test_hold_lookback): cover tile kept unpublished
};

struct lr_plan {
    int device = 0;
    unsigned char* scratch = nullptr;     // the plan's own scratch
    unsigned* d_err = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const int64_t* d_total = nullptr;     // d_offsets + total
    int64_t capacity = 0;
    long long* h_pinned = nullptr;        // 2 words: total, error bits
};

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
constexpr long long kMaxN = 2147483646LL;  // lcp needs n+1 int32 entries
constexpr long long kBuildChunk = 1LL << 29; // positions per chunk of a large batched array build

// Makes ctx->device current for the scope and restores the caller's device.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

lr_status cuda_fail(lr_ctx* ctx, cudaError_t e) {
    ctx->last_cuda_error = (int)e;
    return e == cudaErrorMemoryAllocation ? LR_ERR_NOMEM : LR_ERR_CUDA;
}

struct Layout {
    size_t off_status_g, off_status_b, off_status_o, off_status_w, off_cursor1, off_cursor2, off_cursor_w, zero_end;
    size_t off_tile_cbase, off_seg_cbase, off_tile_seg, off_cstart, off_cend, off_ent1, off_ent2, off_lbig, off_halo,
        total;
};

Layout layout_for(long long n) {
    const long long nt = lr::num_tiles(n), nb = lr::num_buckets(n), ns = lr::num_supers(n), ng = lr::num_segs(n);
    Layout L;
    L.off_status_g = kAlign;                       // tickets in [0, 16), per-query error bits at 16
    L.off_status_b = align_up(L.off_status_g + (size_t)nt * 8);
    L.off_status_o = align_up(L.off_status_b + (size_t)nb * 8);
    L.off_status_w = align_up(L.off_status_o + (size_t)nt * 8);
    L.off_cursor1 = align_up(L.off_status_w + (size_t)lr::num_seg_tiles(n) * 8);
    L.off_cursor2 = align_up(L.off_cursor1 + (size_t)ns * 4 * lr::kCursorStride);
    L.off_cursor_w = align_up(L.off_cursor2 + (size_t)nb * 4 * lr::kCursorStride);
    L.zero_end = L.off_cursor_w + (size_t)lr::num_wins(n) * 4 * lr::kCursorStride;
    L.off_tile_cbase = align_up(L.zero_end);
    L.off_seg_cbase = align_up(L.off_tile_cbase + (size_t)(nt + 1) * 4);
    L.off_tile_seg = align_up(L.off_seg_cbase + (size_t)(ng + 1) * 4);
    L.off_cstart = align_up(L.off_tile_seg + (size_t)nt * 4);
    L.off_cend = align_up(L.off_cstart + (size_t)n * 4);
    L.off_ent1 = align_up(L.off_cend + (size_t)n * 4);
    L.off_ent2 = align_up(L.off_ent1 + (size_t)ns * lr::kSuper * 4);
    L.off_lbig = align_up(L.off_ent2 + (size_t)nb * lr::kBucket * 4);
    L.off_halo = align_up(L.off_lbig + (size_t)n * 4);
    L.total = align_up(L.off_halo + (size_t)(nb + 1) * 4);
    return L;
}

// Points `s` at the regions of a scratch block laid out for cap_n positions,
// for a query of n <= cap_n positions.
void carve(unsigned char* b, long long cap_n, long long n, unsigned* d_err, lr::Scratch* s) {
    const Layout L = layout_for(cap_n);
    s->tickets = (unsigned*)b;
    s->qerr = (unsigned*)(b + 16);
    s->err = d_err;
    s->status_g = (unsigned long long*)(b + L.off_status_g);
    s->status_b = (unsigned long long*)(b + L.off_status_b);
    s->status_o = (unsigned long long*)(b + L.off_status_o);
    s->status_w = (unsigned long long*)(b + L.off_status_w);
    s->seg_cbase = (int32_t*)(b + L.off_seg_cbase);
    s->cursor1 = (unsigned*)(b + L.off_cursor1);
    s->cursor2 = (unsigned*)(b + L.off_cursor2);
    s->cursor_w = (unsigned*)(b + L.off_cursor_w);
    s->went = (unsigned long long*)(b + L.off_cstart);     // cstart + cend: 8 bytes per position
    s->tile_cbase = (int32_t*)(b + L.off_tile_cbase);
    s->tile_seg = (int32_t*)(b + L.off_tile_seg);
    s->cstart = (int32_t*)(b + L.off_cstart);
    s->cend = (int32_t*)(b + L.off_cend);
    s->ent1 = (uint32_t*)(b + L.off_ent1);
    s->ent2 = (uint32_t*)(b + L.off_ent2);
    s->lbig = (int32_t*)(b + L.off_lbig);
    s->halo = (int32_t*)(b + L.off_halo);
    s->ntiles = lr::num_tiles(n);
    s->nsegs = lr::num_segs(n);
    s->nbuckets = lr::num_buckets(n);
    s->nsupers = lr::num_supers(n);
    s->nwins = lr::num_wins(n);
    s->zero_base = b;
    s->zero_bytes = L.zero_end;          // covers the status words and cursors of any n <= cap_n
}

// Grows the context's scratch to hold a query of n positions and fills `s`.
lr_status get_scratch(lr_ctx* ctx, long long n, lr::Scratch* s) {
    if (n > ctx->scratch_n) {
        const Layout L = layout_for(n);
        if (ctx->scratch) {
            cudaError_t e = cudaDeviceSynchronize();   // previous queries may still read it
            if (e != cudaSuccess) return cuda_fail(ctx, e);
            cudaFree(ctx->scratch);
            ctx->scratch = nullptr; ctx->scratch_n = 0; ctx->scratch_bytes = 0;
        }
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, L.total);
        if (e != cudaSuccess) { cudaGetLastError(); return cuda_fail(ctx, e); }
        ctx->scratch = (unsigned char*)p;
        ctx->scratch_bytes = L.total;
        ctx->scratch_n = n;
    }
    carve(ctx->scratch, ctx->scratch_n, n, ctx->d_err, s);
    s->spin_limit = ctx->spin_limit;
    s->hold_tile = ctx->hold_tile;
    ctx->last_n = n;
    return LR_OK;
}

}  // namespace

namespace lr {

size_t scratch_size(long long n) { return layout_for(n).total; }

void carve_scratch(unsigned char* base, long long cap_n, long long n, unsigned* d_err, Scratch* s) {
    carve(base, cap_n, n, d_err, s);
}

}  // namespace lr

namespace {

// Shape class of a batch: log2 of the total and of the mean string length.
int shape_class(long long total, long long num) {
    auto lg = [](long long v) { int k = 0; while (v > 1) { v >>= 1; ++k; } return k; };
    const long long mean = num > 0 ? total / num : total;
    return lg(total) * 64 + lg(mean > 0 ? mean : 1);
}

lr::Shape shape_of(int code) {
    lr::Shape sh;
    sh.tile_cover = (code & 8) != 0;
    sh.cover_tiles_per = (code & 4) ? 4 : ((code & 1) ? 2 : 1);
    return sh;
}

// Shape codes lr_autotune tries: the warp-segment cover (bit 3 clear) or the
// tile cover (bit 3) with tiles of 2048, 4096 or 8192 positions (bit 0 /
// bit 2), each with either front end (bit 1).
constexpr int kShapeCodes[] = {0, 2, 8, 9, 12, 10, 11, 14};

bool valid_code(int code) {
    if (code < 0 || code >= 16) return false;
    return (code & 8) ? (code & 5) != 5 : (code & 5) == 0;
}

// The tuned shape code for a batch (default: tile cover with 4096-position
// tiles, rank-order front end).
constexpr int kDefaultCode = 9;
int tuned_code(const lr_ctx* ctx, long long total, long long num) {
    auto it = ctx->tuned.find(shape_class(total, num));
    return it == ctx->tuned.end() ? kDefaultCode : it->second;
}

lr_status check_n(int32_t n) {
    return (n >= 1 && (long long)n <= kMaxN) ? LR_OK : LR_ERR_ARG;
}

lr_status device_bits_to_status(unsigned bits) {
    if (bits & lr::kErrTimeout) return LR_ERR_TIMEOUT;
    if (bits & lr::kErrInput) return LR_ERR_SENTINEL;
    return LR_OK;
}

// Copies the total (offsets[n]) and the error bits to the host, waits, and
// clears the error word.
}  // namespace

namespace lr {
lr_status status_of_bits(unsigned bits) { return device_bits_to_status(bits); }
}  // namespace lr

namespace {

lr_status sync_total(lr_ctx* ctx, cudaStream_t stream, const int64_t* d_total, int64_t* h_total) {
    cudaError_t e = cudaSuccess;
    if (d_total) e = cudaMemcpyAsync(&ctx->h_pinned[0], d_total, 8, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ctx->h_pinned[1], ctx->d_err, 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_err, 0, 4, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    if (h_total && d_total) *h_total = ctx->h_pinned[0];
    return device_bits_to_status((unsigned)(ctx->h_pinned[1] & 0xffffffffu));
}

}  // namespace

extern "C" {

const char* lr_status_str(lr_status s) {
    switch (s) {
        case LR_OK: return "LR_OK";
        case LR_ERR_ARG: return "LR_ERR_ARG";
        case LR_ERR_SENTINEL: return "LR_ERR_SENTINEL";
        case LR_ERR_CAPACITY: return "LR_ERR_CAPACITY";
        case LR_ERR_NOMEM: return "LR_ERR_NOMEM";
        case LR_ERR_CUDA: return "LR_ERR_CUDA";
        case LR_ERR_TIMEOUT: return "LR_ERR_TIMEOUT";
        case LR_ERR_BUSY: return "LR_ERR_BUSY";
    }
    return "LR_ERR_UNKNOWN";
}

lr_status lr_create(lr_ctx** out, int device) {
    if (!out) return LR_ERR_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return device < 0 ? LR_ERR_ARG : LR_ERR_CUDA;
    }
    lr_ctx* ctx = new (std::nothrow) lr_ctx();
    if (!ctx) return LR_ERR_NOMEM;
    ctx->device = device;
    DeviceGuard g(device);
    cudaError_t e = g.ok ? cudaSuccess : cudaErrorInvalidDevice;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = lr::configure_kernels();
    if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_err, 256);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, 256);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->h_pinned, 64);
    if (e != cudaSuccess) {
        if (ctx->d_err) cudaFree(ctx->d_err);
        delete ctx;
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? LR_ERR_NOMEM : LR_ERR_CUDA;
    }
    *out = ctx;
    return LR_OK;
}

lr_status lr_destroy(lr_ctx* ctx) {
    if (!ctx) return LR_ERR_ARG;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->hostpath) cudaFree(ctx->hostpath);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    ctx->index_work.release();
    if (ctx->d_off2) cudaFree(ctx->d_off2);
    if (ctx->d_chunk_off) cudaFree(ctx->d_chunk_off);
    if (ctx->events_created)
        for (int i = 0; i <= lr::kMaxPhases; ++i) cudaEventDestroy(ctx->events.ev[i]);
    delete ctx;
    return LR_OK;
}

lr_status lr_last_cuda_error(lr_ctx* ctx, int* code) {
    if (!ctx || !code) return LR_ERR_ARG;
    *code = ctx->last_cuda_error;
    return LR_OK;
}

int32_t lr_last_launch_count(lr_ctx* ctx) { return ctx ? ctx->last_launches : -1; }

lr_status lr_test_hold_lookback(lr_ctx* ctx, int64_t tile, int32_t spin_limit) {
    if (!ctx) return LR_ERR_ARG;
    if (tile < 0) {
        ctx->hold_tile = -1;
        ctx->spin_limit = lr::kSpinLimit;
        return LR_OK;
    }
    if (spin_limit < 1 || spin_limit > lr::kSpinLimit) return LR_ERR_ARG;
    ctx->hold_tile = tile;
    ctx->spin_limit = spin_limit;
    return LR_OK;
}

lr_status lr_set_phase_timing(lr_ctx* ctx, int32_t enable) {
    if (!ctx) return LR_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return cuda_fail(ctx, cudaErrorInvalidDevice);
    if (enable && !ctx->events_created) {
        for (int i = 0; i <= lr::kMaxPhases; ++i) {
            cudaError_t e = cudaEventCreate(&ctx->events.ev[i]);
            if (e != cudaSuccess) {
                for (int j = 0; j < i; ++j) cudaEventDestroy(ctx->events.ev[j]);
                return cuda_fail(ctx, e);
            }
        }
        ctx->events_created = true;
    }
    ctx->events.enabled = enable != 0;
    return LR_OK;
}

lr_status lr_last_compact_size(lr_ctx* ctx, lr_stream_t stream, int64_t* m) {
    if (!ctx || !m || ctx->last_n <= 0 || !ctx->scratch) return LR_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return cuda_fail(ctx, cudaErrorInvalidDevice);
    const Layout L = layout_for(ctx->scratch_n);
    const int32_t* src = (const int32_t*)(ctx->scratch + L.off_tile_cbase) + lr::num_tiles(ctx->last_n);
    cudaError_t e = cudaMemcpyAsync(&ctx->h_pinned[2], src, 4, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    *m = (int64_t)(*(int32_t*)&ctx->h_pinned[2]);
    return LR_OK;
}

int32_t lr_phase_times(lr_ctx* ctx, float* ms, int32_t cap) {
    if (!ctx || !ctx->events.enabled || ctx->events.count <= 0) return -1;
    DeviceGuard g(ctx->device);
    const int nk = ctx->events.count;
    if (cudaEventSynchronize(ctx->events.ev[nk]) != cudaSuccess) return -1;
    for (int i = 0; i < nk && i < cap; ++i) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, ctx->events.ev[i], ctx->events.ev[i + 1]) != cudaSuccess) return -1;
        ms[i] = t;
    }
    return nk;
}

lr_status lr_device_status(lr_ctx* ctx, lr_stream_t stream) {
    if (!ctx) return LR_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return cuda_fail(ctx, cudaErrorInvalidDevice);
    return sync_total(ctx, (cudaStream_t)stream, nullptr, nullptr);
}

lr_status lr_query_leftmost(lr_ctx* ctx, lr_stream_t stream, const int32_t* d_sa, const int32_t* d_rank,
                            const int32_t* d_lcp, int32_t n, int32_t* d_lr_start, int32_t* d_lr_len) {
    if (!ctx || (!d_sa && !d_rank) || !d_lcp || !d_lr_start || !d_lr_len) return LR_ERR_ARG;
    if (check_n(n) != LR_OK) return LR_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return cuda_fail(ctx, cudaErrorInvalidDevice);
    lr::Scratch s;
    lr_status st = get_scratch(ctx, n, &s);
    if (st != LR_OK) return st;
    const int code = tuned_code(ctx, n, 1);
    const lr::Shape shape = shape_of(code);
    if ((code & 2) && d_rank) d_sa = nullptr;                  // tuned: the rank-gather front end
    cudaError_t e = lr::launch_query(d_sa, d_rank, d_lcp, n, s, d_lr_len, d_lr_start, nullptr, nullptr, 0, false,
                                     (cudaStream_t)stream, &ctx->last_launches, &ctx->events, lr::Segs{nullptr, 0},
                                     shape);
    return e == cudaSuccess ? LR_OK : cuda_fail(ctx, e);
}

lr_status lr_query_all(lr_ctx* ctx, lr_stream_t stream, const int32_t* d_sa, const int32_t* d_rank,
                       const int32_t* d_lcp, int32_t n, int32_t* d_lr_len, int32_t* d_lr_start, int64_t* d_offsets,
                       int32_t* d_starts, int64_t starts_capacity, int64_t* h_total) {
    if (!ctx || (!d_sa && !d_rank) || !d_lcp || !d_lr_len || !d_lr_start || !d_offsets) return LR_ERR_ARG;
    if (starts_capacity < 0 || (starts_capacity > 0 && !d_starts)) return LR_ERR_ARG;
    if (check_n(n) != LR_OK) return LR_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return cuda_fail(ctx, cudaErrorInvalidDevice);
    lr::Scratch s;
    lr_status st = get_scratch(ctx, n, &s);
    if (st != LR_OK) return st;
    const int code = tuned_code(ctx, n, 1);
    const lr::Shape shape = shape_of(code);
    if ((code & 2) && d_rank) d_sa = nullptr;                  // tuned: the rank-gather front end
    cudaError_t e = lr::launch_query(d_sa, d_rank, d_lcp, n, s, d_lr_len, d_lr_start, d_offsets, d_starts,
                                     starts_capacity, true, (cudaStream_t)stream, &ctx->last_launches, &ctx->events,
                                     lr::Segs{nullptr, 0}, shape);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    if (!h_total) return LR_OK;
    st = sync_total(ctx, (cudaStream_t)stream, d_offsets + n, h_total);
    if (st != LR_OK) return st;
    return (*h_total > starts_capacity) ? LR_ERR_CAPACITY : LR_OK;
}

lr_status lr_query_all_host(lr_ctx* ctx, lr_stream_t stream, const int32_t* h_sa, const int32_t* h_rank,
                            const int32_t* h_lcp, int32_t n, int32_t* h_lr_len, int32_t* h_lr_start,
                            int64_t* h_offsets, int32_t* h_starts, int64_t starts_capacity, int64_t* h_total) {
    if (!ctx || (!h_sa && !h_rank) || !h_lcp || !h_lr_len || !h_lr_start || !h_offsets || !h_total) return LR_ERR_ARG;
    if (starts_capacity < 0 || (starts_capacity > 0 && !h_starts)) return LR_ERR_ARG;
    if (check_n(n) != LR_OK) return LR_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return cuda_fail(ctx, cudaErrorInvalidDevice);
    const size_t nn = (size_t)n;
    const size_t o_rank = 0, o_lcp = align_up(o_rank + nn * 4), o_len = align_up(o_lcp + (nn + 1) * 4),
                 o_start = align_up(o_len + nn * 4), o_off = align_up(o_start + nn * 4),
                 o_starts = align_up(o_off + (nn + 1) * 8),
                 need = align_up(o_starts + (size_t)starts_capacity * 4);
    cudaStream_t strm = (cudaStream_t)stream;
    cudaError_t e;
    if (need > ctx->hostpath_bytes) {
        if (ctx->hostpath) {
            e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return cuda_fail(ctx, e);
            cudaFree(ctx->hostpath);
            ctx->hostpath = nullptr; ctx->hostpath_bytes = 0;
        }
        e = cudaMalloc((void**)&ctx->hostpath, need);
        if (e != cudaSuccess) { cudaGetLastError(); return cuda_fail(ctx, e); }
        ctx->hostpath_bytes = need;
    }
    unsigned char* b = ctx->hostpath;
    int32_t* d_in = (int32_t*)(b + o_rank);            // sa, or rank when no sa is given
    int32_t* d_lcp = (int32_t*)(b + o_lcp);
    int32_t* d_len = (int32_t*)(b + o_len);
    int32_t* d_start = (int32_t*)(b + o_start);
    int64_t* d_off = (int64_t*)(b + o_off);
    int32_t* d_starts = (int32_t*)(b + o_starts);
    e = cudaMemcpyAsync(d_in, h_sa ? h_sa : h_rank, nn * 4, cudaMemcpyHostToDevice, strm);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_lcp, h_lcp, (nn + 1) * 4, cudaMemcpyHostToDevice, strm);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    lr::Scratch s;
    lr_status st = get_scratch(ctx, n, &s);
    if (st != LR_OK) return st;
    e = lr::launch_query(h_sa ? d_in : nullptr, h_sa ? nullptr : d_in, d_lcp, n, s, d_len, d_start, d_off, d_starts,
                         starts_capacity, true, strm,
                         &ctx->last_launches, &ctx->events);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_lr_len, d_len, nn * 4, cudaMemcpyDeviceToHost, strm);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_lr_start, d_start, nn * 4, cudaMemcpyDeviceToHost, strm);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_offsets, d_off, (nn + 1) * 8, cudaMemcpyDeviceToHost, strm);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    st = sync_total(ctx, strm, d_off + n, h_total);
    if (st != LR_OK) return st;
    const int64_t tot = *h_total;
    const int64_t copy = tot < starts_capacity ? tot : starts_capacity;
    if (copy > 0) {
        e = cudaMemcpyAsync(h_starts, d_starts, (size_t)copy * 4, cudaMemcpyDeviceToHost, strm);
        if (e == cudaSuccess) e = cudaStreamSynchronize(strm);
        if (e != cudaSuccess) return cuda_fail(ctx, e);
    }
    return tot > starts_capacity ? LR_ERR_CAPACITY : LR_OK;
}

namespace {

// Grows the context's index work memory to `total` positions (waits for the
// device when it has to reallocate).
lr_status index_work_for(lr_ctx* ctx, long long total) {
    if (ctx->index_work.cap_n >= total && ctx->index_work.base) return LR_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    e = ctx->index_work.alloc(total > 0 ? total : 1, 8);
    return e == cudaSuccess ? LR_OK : LR_ERR_NOMEM;
}

lr_status index_status(lr_ctx* ctx, cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return LR_ERR_NOMEM; }
    if (e == cudaErrorInvalidValue) { cudaGetLastError(); return LR_ERR_SENTINEL; }   // bad offset table
    return e == cudaSuccess ? LR_OK : cuda_fail(ctx, e);
}

}  // namespace

lr_status lr_build_arrays(lr_ctx* ctx, lr_stream_t stream, const uint8_t* d_text, int32_t n, int32_t* d_sa,
                          int32_t* d_rank, int32_t* d_lcp, int32_t* rounds) {
    if (!ctx || !d_text || !d_sa || !d_rank || !d_lcp) return LR_ERR_ARG;
    if (check_n(n) != LR_OK) return LR_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return cuda_fail(ctx, cudaErrorInvalidDevice);
    lr_status st = index_work_for(ctx, n);
    if (st != LR_OK) return st;
    if (!ctx->d_off2 && cudaMalloc((void**)&ctx->d_off2, 16) != cudaSuccess) { cudaGetLastError(); return LR_ERR_NOMEM; }
    cudaStream_t strm = (cudaStream_t)stream;
    const int64_t h_off[2] = {0, (int64_t)n};
    cudaError_t e = cudaMemcpyAsync(ctx->d_off2, h_off, sizeof(h_off), cudaMemcpyHostToDevice, strm);
    int r = 0;
    if (e == cudaSuccess)
        e = lr::build_arrays_batch(d_text, n, ctx->d_off2, 1, d_sa, d_rank, d_lcp, ctx->index_work, true, strm, &r);
    if (e == cudaSuccess) e = cudaStreamSynchronize(strm);
    st = index_status(ctx, e);
    if (st == LR_OK && rounds) *rounds = r;
    return st;
}

lr_status lr_batch_build_arrays(lr_ctx* ctx, lr_stream_t stream, const lr_text_batch* batch, int32_t* d_sa,
                                int32_t* d_rank, int32_t* d_lcp, int32_t* rounds) {
    if (!ctx || !batch || !batch->d_off || !d_sa || !d_rank || !d_lcp) return LR_ERR_ARG;
    if (batch->num < 1 || batch->total < 0 || batch->total > kMaxN || (batch->total > 0 && !batch->d_text))
        return LR_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return cuda_fail(ctx, cudaErrorInvalidDevice);
    cudaStream_t strm = (cudaStream_t)stream;
    int r = 0;
    if (batch->total <= kBuildChunk) {
        lr_status st = index_work_for(ctx, batch->total);
        if (st != LR_OK) return st;
        cudaError_t e = lr::build_arrays_batch(batch->d_text, batch->total, batch->d_off, batch->num, d_sa, d_rank,
                                               d_lcp, ctx->index_work, true, strm, &r);
        if (e == cudaSuccess) e = cudaStreamSynchronize(strm);
        st = index_status(ctx, e);
        if (st == LR_OK && rounds) *rounds = r;
        return st;
    }
    // A large batch is built in chunks of whole strings of at most
    // kBuildChunk positions (strings are independent), so that the work
    // memory follows the chunk, not the batch.  The offset table is read
    // back and checked on the host first.
    const long long num = batch->num;
    std::vector<int64_t> h(num + 1);
    cudaError_t e = cudaMemcpyAsync(h.data(), batch->d_off, (size_t)(num + 1) * 8, cudaMemcpyDeviceToHost, strm);
    if (e == cudaSuccess) e = cudaStreamSynchronize(strm);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    if (h[0] != 0 || h[num] != batch->total) return LR_ERR_SENTINEL;
    for (long long j = 0; j < num; ++j)
        if (h[j + 1] < h[j]) return LR_ERR_SENTINEL;
    if (ctx->chunk_off_cap < num + 1) {
        if (ctx->d_chunk_off) { cudaFree(ctx->d_chunk_off); ctx->d_chunk_off = nullptr; ctx->chunk_off_cap = 0; }
        e = cudaMalloc((void**)&ctx->d_chunk_off, (size_t)(num + 1) * 8);
        if (e != cudaSuccess) { cudaGetLastError(); return LR_ERR_NOMEM; }
        ctx->chunk_off_cap = num + 1;
    }
    std::vector<int64_t> rebased(num + 1);
    int max_r = 0;
    for (long long j0 = 0; j0 < num;) {
        long long j1 = j0 + 1;
        while (j1 < num && h[j1 + 1] - h[j0] <= kBuildChunk) ++j1;
        const long long ct = h[j1] - h[j0];
        for (long long j = j0; j <= j1; ++j) rebased[j - j0] = h[j] - h[j0];
        lr_status st = index_work_for(ctx, ct > 0 ? ct : 1);
        if (st != LR_OK) return st;
        e = cudaMemcpyAsync(ctx->d_chunk_off, rebased.data(), (size_t)(j1 - j0 + 1) * 8, cudaMemcpyHostToDevice, strm);
        if (e == cudaSuccess)
            e = lr::build_arrays_batch(batch->d_text + h[j0], ct, ctx->d_chunk_off, j1 - j0, d_sa + h[j0],
                                       d_rank + h[j0], d_lcp + h[j0] + j0, ctx->index_work, true, strm, &r);
        if (e == cudaSuccess) e = cudaStreamSynchronize(strm);   // the host offsets are reused next chunk
        st = index_status(ctx, e);
        if (st != LR_OK) return st;
        max_r = r > max_r ? r : max_r;
        j0 = j1;
    }
    if (rounds) *rounds = max_r;
    return LR_OK;
}

lr_status lr_query_all_raw(lr_ctx* ctx, lr_stream_t stream, const int32_t* d_rank, const int32_t* d_lcp, int32_t n,
                           int32_t* d_lr_len, int32_t* d_lr_start, int64_t* d_offsets, int32_t* d_starts,
                           int64_t starts_capacity, int64_t* h_total) {
    if (!ctx || !d_rank || !d_lcp || !d_lr_len || !d_lr_start || !d_offsets) return LR_ERR_ARG;
    if (starts_capacity < 0 || (starts_capacity > 0 && !d_starts)) return LR_ERR_ARG;
    if (check_n(n) != LR_OK) return LR_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return cuda_fail(ctx, cudaErrorInvalidDevice);
    lr::Scratch s;
    lr_status st = get_scratch(ctx, n, &s);
    if (st != LR_OK) return st;
    cudaError_t e = lr::launch_raw_query(d_rank, d_lcp, n, s, d_lr_len, d_lr_start, d_offsets, d_starts,
                                         starts_capacity, true, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    ctx->last_launches = 2;
    if (!h_total) return LR_OK;
    st = sync_total(ctx, (cudaStream_t)stream, d_offsets + n, h_total);
    if (st != LR_OK) return st;
    return (*h_total > starts_capacity) ? LR_ERR_CAPACITY : LR_OK;
}

lr_status lr_query_leftmost_raw(lr_ctx* ctx, lr_stream_t stream, const int32_t* d_rank, const int32_t* d_lcp,
                                int32_t n, int32_t* d_lr_start, int32_t* d_lr_len) {
    if (!ctx || !d_rank || !d_lcp || !d_lr_start || !d_lr_len) return LR_ERR_ARG;
    if (check_n(n) != LR_OK) return LR_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return cuda_fail(ctx, cudaErrorInvalidDevice);
    lr::Scratch s;
    lr_status st = get_scratch(ctx, n, &s);
    if (st != LR_OK) return st;
    cudaError_t e = lr::launch_raw_query(d_rank, d_lcp, n, s, d_lr_len, d_lr_start, nullptr, nullptr, 0, false,
                                         (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    ctx->last_launches = 2;
    return LR_OK;
}

lr_status lr_walk_stats(lr_ctx* ctx, lr_stream_t stream, const int32_t* d_rank, const int32_t* d_lcp, int32_t n,
                        int32_t* d_alpha, int32_t* d_beta, lr_walk_summary* h_summary) {
    if (!ctx || !d_rank || !d_lcp || !h_summary) return LR_ERR_ARG;
    if (check_n(n) != LR_OK) return LR_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return cuda_fail(ctx, cudaErrorInvalidDevice);
    lr::Scratch s;
    lr_status st = get_scratch(ctx, n, &s);
    if (st != LR_OK) return st;
    // the six result words live in the context's 256-byte error block, after the error word
    unsigned long long* d_stats = reinterpret_cast<unsigned long long*>(reinterpret_cast<unsigned char*>(ctx->d_err) + 64);
    cudaStream_t strm = (cudaStream_t)stream;
    cudaError_t e = lr::launch_walk_stats(d_rank, d_lcp, n, s, d_alpha, d_beta, d_stats, strm);
    unsigned long long hs[4] = {0, 0, 0, 0};
    int32_t m = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs, d_stats, sizeof(hs), cudaMemcpyDeviceToHost, strm);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&m, s.tile_cbase + s.ntiles, 4, cudaMemcpyDeviceToHost, strm);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    ctx->last_launches = 4;
    st = sync_total(ctx, strm, nullptr, nullptr);
    if (st != LR_OK) return st;
    const int32_t* w = reinterpret_cast<const int32_t*>(hs + 2);
    h_summary->n = n;
    h_summary->m = m;
    h_summary->alpha_sum = (int64_t)hs[0];
    h_summary->beta_sum = (int64_t)hs[1];
    h_summary->alpha_min = w[0];
    h_summary->alpha_max = w[1];
    h_summary->beta_min = w[2];
    h_summary->beta_max = w[3];
    return LR_OK;
}

namespace {

lr_status check_batch(const lr_batch_desc* b) {
    if (!b || !b->d_off || !b->d_lcp || (!b->d_sa && !b->d_rank)) return LR_ERR_ARG;
    if (b->num < 1 || b->total < 1 || b->total > kMaxN || b->num > b->total + 1) return LR_ERR_ARG;
    return LR_OK;
}

lr_status batch_launch(lr_ctx* ctx, cudaStream_t stream, const lr_batch_desc* b, int code, int32_t* d_lr_len,
                       int32_t* d_lr_start, int64_t* d_offsets, int32_t* d_starts, int64_t cap) {
    lr::Scratch s;
    lr_status st = get_scratch(ctx, b->total, &s);
    if (st != LR_OK) return st;
    const bool use_rank = (code & 2) && b->d_rank;
    const int32_t* sa = use_rank ? nullptr : b->d_sa;
    const int32_t* rank = sa ? nullptr : b->d_rank;
    cudaError_t e = lr::launch_query(sa, rank, b->d_lcp, (int32_t)b->total, s, d_lr_len, d_lr_start, d_offsets,
                                     d_starts, cap, true, stream, &ctx->last_launches, &ctx->events,
                                     lr::Segs{b->d_off, b->num}, shape_of(code));
    return e == cudaSuccess ? LR_OK : cuda_fail(ctx, e);
}

}  // namespace

lr_status lr_batch_query_all(lr_ctx* ctx, lr_stream_t stream, const lr_batch_desc* batch, int32_t* d_lr_len,
                             int32_t* d_lr_start, int64_t* d_offsets, int32_t* d_starts, int64_t starts_capacity,
                             int64_t* h_total) {
    if (!ctx || !d_lr_len || !d_lr_start || !d_offsets) return LR_ERR_ARG;
    if (starts_capacity < 0 || (starts_capacity > 0 && !d_starts)) return LR_ERR_ARG;
    lr_status st = check_batch(batch);
    if (st != LR_OK) return st;
    DeviceGuard g(ctx->device);
    if (!g.ok) return cuda_fail(ctx, cudaErrorInvalidDevice);
    st = batch_launch(ctx, (cudaStream_t)stream, batch, tuned_code(ctx, batch->total, batch->num), d_lr_len,
                      d_lr_start, d_offsets, d_starts, starts_capacity);
    if (st != LR_OK || !h_total) return st;
    st = sync_total(ctx, (cudaStream_t)stream, d_offsets + batch->total, h_total);
    if (st != LR_OK) return st;
    return (*h_total > starts_capacity) ? LR_ERR_CAPACITY : LR_OK;
}

lr_status lr_autotune(lr_ctx* ctx, lr_stream_t stream, const lr_batch_desc* batch, int32_t* d_lr_len,
                      int32_t* d_lr_start, int64_t* d_offsets, int32_t* d_starts, int64_t starts_capacity,
                      int32_t* choice) {
    if (!ctx || !d_lr_len || !d_lr_start || !d_offsets || !choice) return LR_ERR_ARG;
    lr_status st = check_batch(batch);
    if (st != LR_OK) return st;
    DeviceGuard g(ctx->device);
    if (!g.ok) return cuda_fail(ctx, cudaErrorInvalidDevice);
    cudaStream_t strm = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(ctx, cudaErrorUnknown);
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(ctx, cudaErrorUnknown); }
    int best = -1;
    float best_ms = 0.f;
    for (int code : kShapeCodes) {
        const bool front_rank = code & 2;
        if (front_rank && (!batch->d_rank || !batch->d_sa)) continue;   // only a choice when both are given
        float acc = 0.f;
        for (int rep = 0; rep < 4 && st == LR_OK; ++rep) {
            cudaEventRecord(e0, strm);
            st = batch_launch(ctx, strm, batch, code, d_lr_len, d_lr_start, d_offsets, d_starts, starts_capacity);
            cudaEventRecord(e1, strm);
            if (st != LR_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) { st = cuda_fail(ctx, cudaErrorUnknown); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) acc += ms;                                        // first run warms up
        }
        if (st != LR_OK) break;
        if (best < 0 || acc < best_ms) { best = code; best_ms = acc; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LR_OK) return st;
    st = sync_total(ctx, strm, nullptr, nullptr);
    if (st != LR_OK) return st;
    ctx->tuned[shape_class(batch->total, batch->num)] = best;
    *choice = best;
    return LR_OK;
}

lr_status lr_autotune_save(lr_ctx* ctx, const char* path) {
    if (!ctx || !path) return LR_ERR_ARG;
    FILE* f = std::fopen(path, "w");
    if (!f) return LR_ERR_ARG;
    for (const auto& kv : ctx->tuned) std::fprintf(f, "%d %d\n", kv.first, kv.second);
    std::fclose(f);
    return LR_OK;
}

lr_status lr_autotune_load(lr_ctx* ctx, const char* path) {
    if (!ctx || !path) return LR_ERR_ARG;
    FILE* f = std::fopen(path, "r");
    if (!f) return LR_ERR_ARG;
    int cls = 0, code = 0;
    while (std::fscanf(f, "%d %d", &cls, &code) == 2)
        if (valid_code(code)) ctx->tuned[cls] = code;
    std::fclose(f);
    return LR_OK;
}

lr_status lr_plan_create(lr_ctx* ctx, const lr_batch_desc* batch, int32_t* d_lr_len, int32_t* d_lr_start,
                         int64_t* d_offsets, int32_t* d_starts, int64_t starts_capacity, lr_plan** out) {
    if (!ctx || !out || !d_lr_len || !d_lr_start || !d_offsets) return LR_ERR_ARG;
    if (starts_capacity < 0 || (starts_capacity > 0 && !d_starts)) return LR_ERR_ARG;
    *out = nullptr;
    lr_status st = check_batch(batch);
    if (st != LR_OK) return st;
    DeviceGuard g(ctx->device);
    if (!g.ok) return cuda_fail(ctx, cudaErrorInvalidDevice);
    lr_plan* plan = new (std::nothrow) lr_plan();
    if (!plan) return LR_ERR_NOMEM;
    plan->device = ctx->device;
    plan->d_total = d_offsets + batch->total;
    plan->capacity = starts_capacity;
    const Layout L = layout_for(batch->total);
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaMalloc((void**)&plan->scratch, L.total);
    if (e == cudaSuccess) e = cudaMalloc((void**)&plan->d_err, 256);
    if (e == cudaSuccess) e = cudaMemset(plan->d_err, 0, 256);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&plan->h_pinned, 2 * sizeof(long long));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        lr::Scratch s;
        carve(plan->scratch, batch->total, batch->total, plan->d_err, &s);
        const int code = tuned_code(ctx, batch->total, batch->num);
        const bool use_rank = (code & 2) && batch->d_rank;
        const int32_t* sa = use_rank ? nullptr : batch->d_sa;
        const int32_t* rank = sa ? nullptr : batch->d_rank;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t le = lr::launch_query(sa, rank, batch->d_lcp, (int32_t)batch->total, s, d_lr_len, d_lr_start,
                                              d_offsets, d_starts, starts_capacity, true, cs, nullptr, nullptr,
                                              lr::Segs{batch->d_off, batch->num}, shape_of(code));
            e = cudaStreamEndCapture(cs, &plan->graph);
            if (e == cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&plan->exec, plan->graph, 0);
    }
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        lr_plan_destroy(plan);
        return cuda_fail(ctx, e);
    }
    *out = plan;
    return LR_OK;
}

lr_status lr_plan_launch(lr_plan* plan, lr_stream_t stream) {
    if (!plan || !plan->exec) return LR_ERR_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok) return LR_ERR_CUDA;
    return cudaGraphLaunch(plan->exec, (cudaStream_t)stream) == cudaSuccess ? LR_OK : LR_ERR_CUDA;
}

lr_status lr_plan_result(lr_plan* plan, lr_stream_t stream, int64_t* h_total) {
    if (!plan || !plan->exec) return LR_ERR_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok) return LR_ERR_CUDA;
    cudaStream_t strm = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&plan->h_pinned[0], plan->d_total, 8, cudaMemcpyDeviceToHost, strm);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&plan->h_pinned[1], plan->d_err, 4, cudaMemcpyDeviceToHost, strm);
    if (e == cudaSuccess) e = cudaMemsetAsync(plan->d_err, 0, 4, strm);
    if (e == cudaSuccess) e = cudaStreamSynchronize(strm);
    if (e != cudaSuccess) { cudaGetLastError(); return LR_ERR_CUDA; }
    if (h_total) *h_total = plan->h_pinned[0];
    lr_status st = device_bits_to_status((unsigned)(plan->h_pinned[1] & 0xffffffffu));
    if (st != LR_OK) return st;
    return plan->h_pinned[0] > plan->capacity ? LR_ERR_CAPACITY : LR_OK;
}

lr_status lr_plan_destroy(lr_plan* plan) {
    if (!plan) return LR_ERR_ARG;
    DeviceGuard g(plan->device);
    cudaDeviceSynchronize();
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    if (plan->scratch) cudaFree(plan->scratch);
    if (plan->d_err) cudaFree(plan->d_err);
    if (plan->h_pinned) cudaFreeHost(plan->h_pinned);
    delete plan;
    return LR_OK;
}

}  // extern "C"
