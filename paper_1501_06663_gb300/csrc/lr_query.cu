// Kernels of the longest-repeat query (Tian and Xu, arXiv 1501.06663).
//
// Two single-pass kernels, each over tiles of kTile consecutive positions,
// with tiles handed out in order by an atomic ticket so that the decoupled
// look-back of a tile only ever waits on tiles that are already running:
//
//  k_llr_compact  Lemma 1 gather L_i = max(lcp[rank[i]], lcp[rank[i]+1]),
//                 the usefulness flag of Sec. 4.2.1 / Algorithm 2
//                 (keep i iff L_i > 0 and L_i >= L_{i-1}) and the stream
//                 compaction of the kept LLR's (kernels K1-K3 of Sec. 4.2.1)
//                 into the compact array LLRc, stored as cstart / cend.
//  k_cover        for every position k, the window of compact LLR's covering
//                 k (Algorithms 2 and 4; starts and ends of LLRc strictly
//                 increase, Sec. 3.2, so the window is a contiguous run whose
//                 two ends only move right as k grows), the longest length,
//                 the leftmost start and the number of ties; then, for the
//                 all-LR query, the exclusive scan of the tie counts into
//                 CSR offsets and a second walk that writes every start
//                 (the two walks of Algorithm 4).
#include <cuda_runtime.h>
#include <cstdint>
#include "lr_device.cuh"
#include "lr_internal.h"

namespace lr {

// ---------------------------------------------------------------------------
// k_llr_compact
// ---------------------------------------------------------------------------

// Lemma 1: L_k = max(lcp[rank[k]], lcp[rank[k]+1]).  rank is read
// coalesced; the two lcp words sit next to each other (one 32-byte sector
// for 7 of 8 rank values).
__device__ __forceinline__ int32_t llr_at(const int32_t* __restrict__ rank, const int32_t* __restrict__ lcp,
                                          int32_t n, long long k, unsigned& bad) {
    uint32_t r = (uint32_t)__ldg(rank + k);
    if (r >= (uint32_t)n) { bad = 1; r = 0; }
    const int32_t a = __ldg(lcp + r), b = __ldg(lcp + r + 1);
    int32_t L = a > b ? a : b;
    if (L < 0 || (long long)L > (long long)n - k) { bad = 1; L = 0; }   // no LLR runs past the end
    return L;
}

// Each warp owns runs of 32 consecutive positions, so one ballot gives the
// kept-flags of a run in position order.  Run s of the tile covers positions
// [32 s, 32 s + 32); warp w takes runs w, w + kWarps, ...
__global__ void __launch_bounds__(kThreads)
k_llr_compact(const int32_t* __restrict__ rank, const int32_t* __restrict__ lcp, int32_t n,
              TileScratch s) {
    constexpr int kRuns = kTile / kWarp;          // 64 runs of 32 positions
    constexpr int kWarps = kThreads / kWarp;       // 8 warps
    __shared__ int32_t Ls[kTile + 1];              // Ls[0] = L_{k0-1}, Ls[1+x] = L_{k0+x}
    __shared__ int32_t run_off[kRuns];
    __shared__ int32_t c_s[kTile];                  // staged compact starts (tile-local order)
    __shared__ int32_t c_e[kTile];
    __shared__ long long tile_s, base_s;
    __shared__ int32_t total_s;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) tile_s = atomicAdd(&s.tickets[0], 1u);
    __syncthreads();
    const long long tile = tile_s;
    const long long k0 = tile * kTile;

    // An invalid rank or lcp value is reported and replaced by one that
    // keeps every access in bounds.
    unsigned bad = 0;
#pragma unroll
    for (int j = 0; j < kTile / kThreads; ++j) {
        const int x = j * kThreads + tid;
        Ls[1 + x] = (k0 + x < n) ? llr_at(rank, lcp, n, k0 + x, bad) : 0;
    }
    if (tid == 0) {
        Ls[0] = (k0 > 0) ? llr_at(rank, lcp, n, k0 - 1, bad) : 0;
        if (tile == 0 && (__ldg(lcp) != 0 || __ldg(lcp + n) != 0)) bad = 1;
    }
    if (bad) { atomicOr(s.err, kErrInput); atomicOr(s.qerr, kErrInput); }
    __syncthreads();

    // Usefulness flag (K1): keep i iff L_i > 0 and L_i >= L_{i-1}.
    unsigned masks[kRuns / kWarps];
#pragma unroll
    for (int q = 0; q < kRuns / kWarps; ++q) {
        const int run = q * kWarps + warp;
        const int x = run * kWarp + lane;
        const int32_t L = Ls[1 + x], prev = Ls[x];
        const bool keep = (k0 + x < n) && L > 0 && L >= prev;
        masks[q] = __ballot_sync(kFull, keep);
        if (lane == 0) run_off[run] = __popc(masks[q]);
    }
    __syncthreads();
    // Exclusive scan of the 64 run counts by warp 0 (two per lane), giving
    // the tile-local position of every kept LLR (K2 within the tile).
    if (warp == 0) {
        const int a = run_off[2 * lane], b = run_off[2 * lane + 1];
        const int incl = warp_incl_scan(a + b);
        run_off[2 * lane] = incl - a - b;
        run_off[2 * lane + 1] = incl - b;
        if (lane == 31) total_s = incl;
    }
    __syncthreads();
    // Scatter (K3) into shared memory first.
#pragma unroll
    for (int q = 0; q < kRuns / kWarps; ++q) {
        const int run = q * kWarps + warp;
        const int x = run * kWarp + lane;
        if ((masks[q] >> lane) & 1u) {
            const int o = run_off[run] + __popc(masks[q] & ((1u << lane) - 1u));
            c_s[o] = (int32_t)(k0 + x);
            c_e[o] = (int32_t)(k0 + x + Ls[1 + x] - 1);
        }
    }
    // Global position of this tile's LLRc entries: decoupled look-back over
    // the tiles' counts.
    if (warp == 0) {
        const long long ex = lookback_exclusive(s.status_c, tile, total_s, s.err, s.qerr);
        if (lane == 0) {
            base_s = ex;
            s.cbase[tile] = (int32_t)ex;
            if (tile == s.ntiles - 1) s.cbase[s.ntiles] = (int32_t)(ex + total_s);
        }
    }
    __syncthreads();
    const long long base = base_s;
    const int total = total_s;
    for (int i = tid; i < total; i += kThreads) {
        s.cstart[base + i] = c_s[i];
        s.cend[base + i] = c_e[i];
    }
}

// ---------------------------------------------------------------------------
// k_cover
// ---------------------------------------------------------------------------

// Dynamic shared memory layout of k_cover.
struct CoverSmem {
    int32_t cs[kCoverCap];       // compact LLR window: starts
    int32_t ce[kCoverCap];       //                     ends
    int32_t out_len[kTile];
    int32_t out_start[kTile];
    long long out_off[kTile];
};

template <bool kAll>
__global__ void __launch_bounds__(kThreads)
k_cover(int32_t n, TileScratch s, int32_t* __restrict__ lr_len, int32_t* __restrict__ lr_start,
        int64_t* __restrict__ offsets, int32_t* __restrict__ starts, long long capacity) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CoverSmem& sm = *reinterpret_cast<CoverSmem*>(smem_raw);
    __shared__ long long tile_s, base_s;
    __shared__ int32_t lo_s;
    __shared__ int32_t warp_tot[kThreads / kWarp];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) tile_s = atomicAdd(&s.tickets[1], 1u);
    __syncthreads();
    const long long tile = tile_s;
    const long long k0 = tile * kTile;
    // After a lost wait in k_llr_compact the compact array is not complete:
    // write nothing (the host reports LR_ERR_TIMEOUT).
    if (*(volatile unsigned*)s.qerr & kErrTimeout) return;
    const int32_t cb0 = s.cbase[tile];          // first compact LLR starting in this tile
    const int32_t cb1 = s.cbase[tile + 1];      // one past the last

    // lo = first compact LLR whose end reaches k0.  Ends strictly increase,
    // so those are a suffix of [0, cb0) plus the tile's own; scan back 32 at
    // a time from cb0.
    if (warp == 0) {
        int32_t t = cb0;
        while (true) {
            const long long idx = (long long)t - 1 - lane;
            const bool reach = idx >= 0 && __ldg(s.cend + idx) >= k0;
            const unsigned m = __ballot_sync(kFull, reach);
            if (m == kFull) { t -= kWarp; continue; }
            t -= __ffs(~m) - 1;
            break;
        }
        if (lane == 0) lo_s = t;
    }
    __syncthreads();
    const int32_t lo = lo_s;
    const int32_t M = cb1 - lo;                  // window candidates for the whole tile
    const int32_t* CS;
    const int32_t* CE;
    if (M <= kCoverCap) {
        for (int i = tid; i < M; i += kThreads) {
            sm.cs[i] = __ldg(s.cstart + lo + i);
            sm.ce[i] = __ldg(s.cend + lo + i);
        }
        CS = sm.cs; CE = sm.ce;
    } else {                                     // very long windows: read LLRc in place
        CS = s.cstart + lo; CE = s.cend + lo;
    }
    __syncthreads();

    // kPer consecutive positions per thread; the window [wlo, whi] of
    // position k holds the compact LLR's with start <= k <= end.
    constexpr int kPer = kTile / kThreads;
    const int x0 = tid * kPer;
    const long long kfirst = k0 + x0;
    int32_t wlo = 0, whi = -1;
    if (kfirst < n) {
        int32_t a = 0, b = M;                    // first t with CE[t] >= kfirst
        while (a < b) { int32_t mid = (a + b) >> 1; if (CE[mid] >= kfirst) b = mid; else a = mid + 1; }
        wlo = a;
        a = 0; b = M;                            // first t with CS[t] > kfirst
        while (a < b) { int32_t mid = (a + b) >> 1; if (CS[mid] > kfirst) b = mid; else a = mid + 1; }
        whi = a - 1;
    }
    int32_t best[kPer], cnt[kPer], wl[kPer], wh[kPer];
    int32_t my_count = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const long long k = kfirst + q;
        best[q] = 0; cnt[q] = 0; wl[q] = 0; wh[q] = -1;
        int32_t left = -1;
        if (k < n) {
            while (wlo < M && CE[wlo] < k) ++wlo;
            while (whi + 1 < M && CS[whi + 1] <= k) ++whi;
            for (int32_t t = wlo; t <= whi; ++t) {
                const int32_t len = CE[t] - CS[t] + 1;
                if (len > best[q]) { best[q] = len; left = CS[t]; cnt[q] = 1; }
                else if (len == best[q]) ++cnt[q];
            }
            wl[q] = wlo; wh[q] = whi;
        }
        sm.out_len[x0 + q] = best[q];
        sm.out_start[x0 + q] = left;
        my_count += cnt[q];
    }

    if constexpr (kAll) {
        // Block-wide exclusive scan of the per-thread counts, then the tile's
        // global base by decoupled look-back (int64 offsets).
        int incl = warp_incl_scan(my_count);
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        int warp_ex = 0, tile_total = 0;
#pragma unroll
        for (int w = 0; w < kThreads / kWarp; ++w) {
            const int v = warp_tot[w];
            if (w < warp) warp_ex += v;
            tile_total += v;
        }
        if (warp == 0) {
            const long long ex = lookback_exclusive(s.status_o, tile, tile_total, s.err, s.qerr);
            if (lane == 0) base_s = ex;
        }
        __syncthreads();
        long long off = base_s + warp_ex + incl - my_count;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            sm.out_off[x0 + q] = off;
            // second walk: every compact LLR of the longest length, ascending
            if (best[q] > 0) {
                long long o = off;
                for (int32_t t = wl[q]; t <= wh[q]; ++t) {
                    if (CE[t] - CS[t] + 1 == best[q]) {
                        if (o < capacity) starts[o] = CS[t];
                        ++o;
                    }
                }
            }
            off += cnt[q];
        }
        if (tile == s.ntiles - 1 && tid == kThreads - 1) offsets[n] = off;
    }
    __syncthreads();
    // Coalesced write-out of the staged per-position results.
    const long long kend = (k0 + kTile < n) ? k0 + kTile : n;
    for (long long k = k0 + tid; k < kend; k += kThreads) {
        const int x = (int)(k - k0);
        lr_len[k] = sm.out_len[x];
        lr_start[k] = sm.out_start[x];
        if constexpr (kAll) offsets[k] = sm.out_off[x];
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

size_t cover_smem_bytes() { return sizeof(CoverSmem); }

cudaError_t configure_kernels() {
    cudaError_t e = cudaFuncSetAttribute(k_cover<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(CoverSmem));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_cover<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(CoverSmem));
}

cudaError_t launch_query(const int32_t* rank, const int32_t* lcp, int32_t n, const TileScratch& s,
                         int32_t* lr_len, int32_t* lr_start, int64_t* offsets, int32_t* starts,
                         long long capacity, bool all, cudaStream_t stream, int* launches,
                         PhaseEvents* events) {
    cudaError_t e = cudaMemsetAsync(s.zero_base, 0, s.zero_bytes, stream);
    if (e != cudaSuccess) return e;
    const bool timed = events && events->enabled;
    const unsigned grid = (unsigned)s.ntiles;
    if (timed) cudaEventRecord(events->ev[0], stream);
    k_llr_compact<<<grid, kThreads, 0, stream>>>(rank, lcp, n, s);
    if (timed) cudaEventRecord(events->ev[1], stream);
    if (all)
        k_cover<true><<<grid, kThreads, sizeof(CoverSmem), stream>>>(n, s, lr_len, lr_start, offsets, starts, capacity);
    else
        k_cover<false><<<grid, kThreads, sizeof(CoverSmem), stream>>>(n, s, lr_len, lr_start, nullptr, nullptr, 0);
    if (timed) cudaEventRecord(events->ev[2], stream);
    if (launches) *launches = 2;
    return cudaGetLastError();
}

}  // namespace lr
