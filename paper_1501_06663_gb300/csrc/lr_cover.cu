// The cover kernel of the longest-repeat query (Tian and Xu, arXiv
// 1501.06663, Algorithms 2 and 4, GPU kernel of Sec. 4.2.2): from the compact
// LLR array LLRc to the longest repeats of every position.
//
// Starts and ends of LLRc strictly increase (Sec. 3.2), so the compact LLR's
// covering a position k form a contiguous window of LLRc whose two ends only
// move right as k grows.  Per tile of kTile positions (tiles in order by an
// atomic ticket):
//
//  * the window range of the whole tile is LLRc[lo, cb1): the tile's own
//    entries [cb0, cb1) plus the carry [lo, cb0), the earlier entries whose
//    end reaches the tile; lo is found by a warp scanning back from cb0;
//  * the range is staged in shared memory together with two bitmaps over the
//    tile's positions: where an entry of the range starts and where one ends;
//  * for position k the window is [lo_k, hi_k] with hi_k = (starts <= k) - 1
//    and lo_k = (ends < k) in carry ++ local numbering: two prefix popcounts,
//    no binary search (the paper's per-position binary search);
//  * one walk over the window gives the longest length, the leftmost start
//    and the number of ties (Algorithm 2's walk, with Algorithm 4's count);
//  * for the all-LR query, the tie counts are scanned (block scan plus a
//    decoupled look-back over the tiles) into CSR offsets, and a second walk
//    writes every start of the longest length, ascending (Algorithm 4's
//    second walk).
//
// A lane owns one position of each run of 32, so every per-position store of
// a warp is one contiguous 128- or 256-byte run.
#include <cuda_runtime.h>
#include <cstdint>
#include "lr_device.cuh"
#include "lr_internal.h"

namespace lr {

namespace {

constexpr int kWarps = kThreads / kWarp;          // 8
constexpr int kChunks = kTile / kWarp;             // 64 runs of 32 positions
constexpr int kChunksPerWarp = kChunks / kWarps;   // 8

struct __align__(16) CoverSmem {
    int32_t cs[kCoverCap];           // window range LLRc[lo, cb1): starts
    int32_t cl[kCoverCap];           //                             lengths
    unsigned smap[kChunks];          // bit x: an entry of the tile starts at k0 + x
    unsigned emap[kChunks];          // bit x: an entry of the range ends at k0 + x
    int32_t spre[kChunks];           // exclusive prefix popcounts of the bitmap words
    int32_t epre[kChunks];
    int32_t chunk[kChunks];          // run totals of the tie counts
    long long tile;
    long long obase;
    int32_t lo;
};

__device__ __forceinline__ void popc_prefix64(const unsigned* map, int32_t* pre) {
    const int lane = lane_id();
    const int a = __popc(map[2 * lane]), b = __popc(map[2 * lane + 1]);
    const int incl = warp_incl_scan(a + b);
    pre[2 * lane] = incl - a - b;
    pre[2 * lane + 1] = incl - b;
}

}  // namespace

template <bool kAll>
__global__ void __launch_bounds__(kThreads, 5)
k_cover(int32_t n, Scratch s, int32_t* __restrict__ lr_len, int32_t* __restrict__ lr_start,
        int64_t* __restrict__ offsets, int32_t* __restrict__ starts, long long capacity) {
    __shared__ CoverSmem sm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) sm.tile = atomicAdd(&s.tickets[2], 1u);
    if (tid < kChunks) { sm.smap[tid] = 0; sm.emap[tid] = 0; }
    __syncthreads();
    const long long tile = sm.tile;
    const int32_t k0 = (int32_t)(tile * kTile);              // n < 2^31: positions fit 32 bits
    // LLRc entries [cb0, cb1) start inside this tile; clamped so that a
    // corrupted front end (already reported) cannot send reads out of bounds
    int32_t cb0 = s.tile_cbase[tile], cb1 = s.tile_cbase[tile + 1];
    cb0 = cb0 < 0 ? 0 : (cb0 > n ? n : cb0);
    cb1 = cb1 < cb0 ? cb0 : (cb1 > n ? n : cb1);

    // carry: entries before cb0 whose end reaches k0 (a suffix, ends increase)
    if (warp == 0) {
        int32_t t = cb0;
        while (t > 0) {
            const int32_t idx = t - 1 - lane;
            const bool reach = idx >= 0 && __ldg(s.cend + idx) >= k0;
            const unsigned m = __ballot_sync(kFull, reach);
            if (m == kFull) { t -= kWarp; continue; }
            t -= __ffs(~m) - 1;
            break;
        }
        if (lane == 0) sm.lo = t;
    }
    __syncthreads();
    const int32_t lo = sm.lo;
    const int32_t C = cb0 - lo, M = cb1 - lo;
    const bool staged = M <= kCoverCap;
    for (int i = tid; i < M; i += kThreads) {
        const int32_t cs = __ldg(s.cstart + lo + i), ce = __ldg(s.cend + lo + i);
        if (staged) { sm.cs[i] = cs; sm.cl[i] = ce - cs + 1; }
        const uint32_t xs = (uint32_t)(cs - k0), xe = (uint32_t)(ce - k0);
        if (i >= C && xs < (uint32_t)kTile) atomicOr(&sm.smap[xs >> 5], 1u << (xs & 31));
        if (xe < (uint32_t)kTile) atomicOr(&sm.emap[xe >> 5], 1u << (xe & 31));
    }
    __syncthreads();
    if (warp == 0) popc_prefix64(sm.smap, sm.spre);
    if (warp == 1) popc_prefix64(sm.emap, sm.epre);
    __syncthreads();

    // candidate v of the range: start and length (shared memory, or LLRc in
    // place when the range is too long to stage)
    const int32_t* gcs = s.cstart + lo;
    const int32_t* gce = s.cend + lo;
    auto start_of = [&](int32_t v) -> int32_t { return staged ? sm.cs[v] : __ldg(gcs + v); };
    auto len_of = [&](int32_t v) -> int32_t { return staged ? sm.cl[v] : __ldg(gce + v) - __ldg(gcs + v) + 1; };
    const unsigned below = (1u << lane) - 1u;
    // window [lw, hi] of this lane's position in run c (carry ++ local numbering)
    auto window = [&](int c, int32_t& lw, int32_t& hi) {
        hi = C + sm.spre[c] + __popc(sm.smap[c] & (below | (1u << lane))) - 1;
        lw = sm.epre[c] + __popc(sm.emap[c] & below);
    };
    // per run: longest length, index of its leftmost holder, number of ties
    int32_t best[kChunksPerWarp], vbest[kChunksPerWarp], cnt[kChunksPerWarp];
#pragma unroll
    for (int q = 0; q < kChunksPerWarp; ++q) {
        const int c = q * kWarps + warp;
        const int32_t k = k0 + c * kWarp + lane;
        int32_t lw, hi;
        window(c, lw, hi);
        int32_t b = 0, vb = -1, ct = 0;
        for (int32_t v = lw; v <= hi; ++v) {
            const int32_t len = len_of(v);
            if (len > b) { b = len; vb = v; ct = 1; }
            else if (len == b) ++ct;
        }
        best[q] = b; vbest[q] = vb; cnt[q] = ct;
        if (k < n) { __stcs(lr_len + k, b); __stcs(lr_start + k, vb >= 0 ? start_of(vb) : -1); }
    }

    if constexpr (kAll) {
        // CSR offsets: scan of the tie counts within the tile, then the
        // tile's base by look-back over the tiles' totals
        int pre[kChunksPerWarp];
#pragma unroll
        for (int q = 0; q < kChunksPerWarp; ++q) {
            const int incl = warp_incl_scan(cnt[q]);
            pre[q] = incl - cnt[q];
            if (lane == kWarp - 1) sm.chunk[q * kWarps + warp] = incl;
        }
        __syncthreads();
        if (warp == 0) {
            const int x = sm.chunk[2 * lane], y = sm.chunk[2 * lane + 1];
            const int incl = warp_incl_scan(x + y);
            sm.chunk[2 * lane] = incl - x - y;
            sm.chunk[2 * lane + 1] = incl - y;
            const int tot = __shfl_sync(kFull, incl, kWarp - 1);
            const long long ex = lookback_exclusive(s.status_o, tile, tot, s.err, s.qerr);
            if (lane == 0) {
                sm.obase = ex;
                if (tile == s.ntiles - 1) offsets[n] = ex + tot;
            }
        }
        __syncthreads();
        const long long obase = sm.obase;
#pragma unroll
        for (int q = 0; q < kChunksPerWarp; ++q) {
            const int c = q * kWarps + warp;
            const int32_t k = k0 + c * kWarp + lane;
            long long o = obase + sm.chunk[c] + pre[q];
            if (k < n) __stcs(reinterpret_cast<long long*>(offsets) + k, o);
            if (cnt[q] == 0) continue;
            // second walk of Algorithm 4, from the leftmost holder: every
            // compact LLR of the longest length, ascending; with one holder
            // (the common case) it is already known
            if (o < capacity) __stcs(starts + o, start_of(vbest[q]));
            ++o;
            if (cnt[q] > 1) {
                int32_t lw, hi;
                window(c, lw, hi);
                for (int32_t v = vbest[q] + 1; v <= hi; ++v) {
                    if (len_of(v) == best[q]) {
                        if (o < capacity) __stcs(starts + o, start_of(v));
                        ++o;
                    }
                }
            }
        }
    }
}

void launch_cover(int32_t n, const Scratch& s, int32_t* lr_len, int32_t* lr_start, int64_t* offsets,
                  int32_t* starts, long long capacity, bool all, cudaStream_t stream) {
    const unsigned grid = (unsigned)s.ntiles;
    if (all)
        k_cover<true><<<grid, kThreads, 0, stream>>>(n, s, lr_len, lr_start, offsets, starts, capacity);
    else
        k_cover<false><<<grid, kThreads, 0, stream>>>(n, s, lr_len, lr_start, nullptr, nullptr, 0);
}

}  // namespace lr
