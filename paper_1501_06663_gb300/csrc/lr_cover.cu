// The cover kernel of the longest-repeat query (Tian and Xu, arXiv
// 1501.06663, Algorithms 2 and 4, GPU kernel of Sec. 4.2.2): from the compact
// LLR array LLRc to the longest repeats of every position.
//
// Starts and ends of LLRc strictly increase (Sec. 3.2), so the compact LLR's
// covering a position k form a contiguous window of LLRc whose two ends only
// move right as k grows.  Per tile of 2048, 4096 or 8192 positions (tiles in
// order by an atomic ticket):
//
//  * the window range of the whole tile is LLRc[lo, cb1): the tile's own
//    entries [cb0, cb1) plus the carry [lo, cb0), the earlier entries whose
//    end reaches the tile; lo is found by a warp scanning back from cb0;
//  * the range is staged in shared memory together with two bitmaps over the
//    tile's positions: where an entry of the range starts and where one ends;
//  * for position k the window is [lo_k, hi_k] with hi_k = (starts <= k) - 1
//    and lo_k = (ends < k) in carry ++ local numbering: two prefix popcounts,
//    no binary search (the paper's per-position binary search);
//  * the longest length, the leftmost start and the ties of every window
//    (Algorithm 2's walk, with Algorithm 4's count) come from a range-maximum
//    table built per run of 32 positions over the run's entries (a walk over
//    the window when the run spans more than 32 entries);
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

// Shape of a cover tile of kTile x TP positions run by kThreads x TP threads;
// every warp owns 8 runs of 32 positions.
template <int TP>
struct Cfg {
    static constexpr int kTileC = kTile * TP;
    static constexpr int kThr = kThreads * TP;
    static constexpr int kWarps = kThr / kWarp;
    static constexpr int kChunks = kTileC / kWarp;
    static constexpr int kChunksPerWarp = kChunks / kWarps;
    static constexpr int kMinBlocks = TP == 1 ? 5 : (TP == 2 ? 4 : 2);
    static constexpr int kCap = kTileC + 128;     // staged entries: the tile's own and a carry
    // Width of the holder-index field of the packed per-run word pk (see
    // k_cover): every staged index v < kCap and the "none" value all-ones
    // must fit; the holder mask or count takes the bits above it up to 30.
    static constexpr int kVBits = (kCap <= (1 << 13) - 1) ? 13 : 14;
    static constexpr uint32_t kNone = (1u << kVBits) - 1u;
    static constexpr int kMaskBits = 31 - kVBits;
    static_assert(kCap <= (int)kNone, "staged window indices must fit the holder-index field");
    static_assert(kCap < (1 << kMaskBits), "a tie count must fit the count field");
};

template <int TP>
struct __align__(16) CoverSmem {
    static constexpr int kChunks = Cfg<TP>::kChunks;
    int32_t cs[Cfg<TP>::kCap];       // window range LLRc[lo, cb1): starts
    int32_t cl[Cfg<TP>::kCap];       //                             lengths
    unsigned smap[kChunks];          // bit x: an entry of the tile starts at k0 + x
    unsigned emap[kChunks];          // bit x: an entry of the range ends at k0 + x
    int32_t spre[kChunks];           // exclusive prefix popcounts of the bitmap words
    int32_t epre[kChunks];
    int32_t chunk[kChunks];          // run totals of the tie counts
    unsigned rt[Cfg<TP>::kWarps][Cfg<TP>::kChunksPerWarp][kWarp];   // per warp: range-max levels 0..4 and
                                     // equal-length masks; then the runs' tie-count prefixes
    long long tile;
    long long obase;
    int32_t lo;
    int32_t nlow;                    // staged carry candidates that end before the tile
    int32_t ttot;                    // the tile's total of tie counts
    int32_t longlen;                 // a staged length reaches 2^27 (too long for the range-max keys)
};

// Exclusive prefix popcounts of the kChunks bitmap words, by one warp.
template <int kChunks>
__device__ __forceinline__ void popc_prefix(const unsigned* map, int32_t* pre) {
    constexpr int kPer = kChunks / kWarp;
    const int lane = lane_id();
    int c[kPer], sum = 0;
#pragma unroll
    for (int i = 0; i < kPer; ++i) { c[i] = __popc(map[kPer * lane + i]); sum += c[i]; }
    int run = warp_incl_scan(sum) - sum;
#pragma unroll
    for (int i = 0; i < kPer; ++i) { pre[kPer * lane + i] = run; run += c[i]; }
}

// Exclusive scan of the kChunks ints of a[] by one warp; returns the total.
template <int kChunks>
__device__ __forceinline__ int scan_chunks(int32_t* a) {
    constexpr int kPer = kChunks / kWarp;
    const int lane = lane_id();
    int c[kPer], sum = 0;
#pragma unroll
    for (int i = 0; i < kPer; ++i) { c[i] = a[kPer * lane + i]; sum += c[i]; }
    const int incl = warp_incl_scan(sum);
    int run = incl - sum;
#pragma unroll
    for (int i = 0; i < kPer; ++i) { a[kPer * lane + i] = run; run += c[i]; }
    return __shfl_sync(kFull, incl, kWarp - 1);
}

}  // namespace

template <bool kAll, int TP>
__global__ void __launch_bounds__(Cfg<TP>::kThr, Cfg<TP>::kMinBlocks)
k_cover(int32_t n, Scratch s, int32_t* __restrict__ lr_len, int32_t* __restrict__ lr_start,
        int64_t* __restrict__ offsets, int32_t* __restrict__ starts, long long capacity) {
    constexpr int kCoverTile = Cfg<TP>::kTileC;
    constexpr int kCoverThreads = Cfg<TP>::kThr;
    constexpr int kCoverTilesPer = TP;
    constexpr int kWarps = Cfg<TP>::kWarps;
    constexpr int kChunks = Cfg<TP>::kChunks;
    constexpr int kChunksPerWarp = Cfg<TP>::kChunksPerWarp;
    extern __shared__ __align__(16) unsigned char cover_smem[];
    CoverSmem<TP>& sm = *reinterpret_cast<CoverSmem<TP>*>(cover_smem);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) sm.tile = atomicAdd(&s.tickets[2], 1u);
    if (tid < kChunks) { sm.smap[tid] = 0; sm.emap[tid] = 0; }
    if (tid == 0) { sm.nlow = 0; sm.longlen = 0; }
    __syncthreads();
    const long long tile = sm.tile;
    const int32_t k0 = (int32_t)(tile * kCoverTile);         // n < 2^31: positions fit 32 bits
    // LLRc entries [cb0, cb1) start inside this tile; clamped so that a
    // corrupted front end (already reported) cannot send reads out of bounds
    const long long ft = tile * kCoverTilesPer;               // first front-end tile
    const long long ft1 = (ft + kCoverTilesPer < s.ntiles) ? ft + kCoverTilesPer : s.ntiles;
    int32_t cb0 = s.tile_cbase[ft], cb1 = s.tile_cbase[ft1];
    cb0 = cb0 < 0 ? 0 : (cb0 > n ? n : cb0);
    cb1 = cb1 < cb0 ? cb0 : (cb1 > n ? n : cb1);

    // Stage LLRc[cb0 - kSpec, cb1): the tile's own entries and, in the same
    // round trip, the kSpec entries before them, which hold the carry (the
    // entries whose end reaches k0: a suffix, ends increase) unless it is
    // longer than kSpec.  A longer carry takes the slow path below.
    constexpr int32_t kSpec = 64;
    const int32_t sbase = cb0 > kSpec ? cb0 - kSpec : 0;
    const int32_t MS = cb1 - sbase;
    const bool fits = MS <= Cfg<TP>::kCap;
    // One pass over the staged entries: lengths, the two bitmaps (entries of
    // [sbase, lo) end before k0, so they set no bit), and the number of
    // staged carry candidates that end before k0: ends increase, so they
    // are a prefix and lo = sbase + that number.
    const int32_t nspec = cb0 - sbase;
    if (fits) {
        for (int i0 = 0; i0 < MS; i0 += kCoverThreads) {
            const int i = i0 + tid;
            bool low = false;
            if (i < MS) {
                const int32_t cs = __ldg(s.cstart + sbase + i), ce = __ldg(s.cend + sbase + i);
                sm.cs[i] = cs;
                sm.cl[i] = ce - cs + 1;
                if (ce - cs + 1 >= (1 << 27)) sm.longlen = 1;
                const uint32_t xs = (uint32_t)(cs - k0), xe = (uint32_t)(ce - k0);
                if (i >= nspec && xs < (uint32_t)kCoverTile) atomicOr(&sm.smap[xs >> 5], 1u << (xs & 31));
                if (xe < (uint32_t)kCoverTile) atomicOr(&sm.emap[xe >> 5], 1u << (xe & 31));
                low = i < nspec && ce < k0;
            }
            const unsigned m = __ballot_sync(kFull, low);
            if (lane == 0 && m) atomicAdd(&sm.nlow, __popc(m));
        }
    }
    __syncthreads();
    // staged unless every staged candidate reaches k0 with more LLRc before
    // them: then the carry may be longer, and it is found in LLRc itself
    const int32_t nlow = sm.nlow;
    const bool staged = fits && !(sbase > 0 && nlow == 0) && !sm.longlen;
    int32_t lo = sbase + nlow;
    if (!staged) {
        if (tid < kChunks) { sm.smap[tid] = 0; sm.emap[tid] = 0; }
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
        lo = sm.lo;
        const int32_t Cg = cb0 - lo, Mg = cb1 - lo;
        for (int i = tid; i < Mg; i += kCoverThreads) {
            const int32_t cs = __ldg(s.cstart + lo + i), ce = __ldg(s.cend + lo + i);
            const uint32_t xs = (uint32_t)(cs - k0), xe = (uint32_t)(ce - k0);
            if (i >= Cg && xs < (uint32_t)kCoverTile) atomicOr(&sm.smap[xs >> 5], 1u << (xs & 31));
            if (xe < (uint32_t)kCoverTile) atomicOr(&sm.emap[xe >> 5], 1u << (xe & 31));
        }
        __syncthreads();
    }
    const int32_t C = cb0 - lo;
    // staged: window entry v sits at sm.cs/cl[v + shift]
    const int32_t shift = staged ? lo - sbase : 0;
    if (warp == 0) popc_prefix<kChunks>(sm.smap, sm.spre);
    if (warp == 1) popc_prefix<kChunks>(sm.emap, sm.epre);
    __syncthreads();

    // candidate v of the range: start and length (shared memory, or LLRc in
    // place when the range is too long to stage)
    const int32_t* gcs = s.cstart + lo;
    const int32_t* gce = s.cend + lo;
    const int32_t* SCS = sm.cs + shift;
    const int32_t* SCL = sm.cl + shift;
    auto start_of = [&](int32_t v) -> int32_t { return staged ? SCS[v] : __ldg(gcs + v); };
    const unsigned below = (1u << lane) - 1u;
    // window [lw, hi] of this lane's position in run c (carry ++ local numbering)
    auto window = [&](int c, int32_t& lw, int32_t& hi) {
        hi = C + sm.spre[c] + __popc(sm.smap[c] & (below | (1u << lane))) - 1;
        lw = sm.epre[c] + __popc(sm.emap[c] & below);
    };
    // longest length b over the window, index vb of its leftmost holder and
    // the number of holders ct: the first four entries without branches
    // (nearly every window), a loop for the rest
    auto best_of = [&](int32_t lw, int32_t hi, int32_t& b, int32_t& vb, int32_t& ct) {
        b = 0; vb = -1; ct = 0;
        auto step = [&](int32_t len, int32_t v) {
            const bool gt = len > b;
            ct = gt ? 1 : ct + (len == b);
            vb = gt ? v : vb;
            b = gt ? len : b;
        };
        if (staged) {
            const int32_t* CL = SCL;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int32_t v = lw + u;
                const int32_t len = (v <= hi) ? CL[v] : -1;
                step(len, v);
            }
            for (int32_t v = lw + 4; v <= hi; ++v) step(CL[v], v);
        } else {
            for (int32_t v = lw; v <= hi; ++v) step(__ldg(gce + v) - __ldg(gcs + v) + 1, v);
        }
    };
    // Per run of 32 positions: the windows of its lanes lie inside one range
    // [U0, U1] of at most a few dozen entries (both window ends only move
    // right).  When it has at most 32 entries, lane j holds entry U0 + j and
    // the warp builds a range-maximum table over the keys (length << 5 |
    // 31 - j) in five shuffle levels, plus each lane's mask of equal lengths
    // (match.any); a window's longest length and leftmost holder are then
    // two table reads and its holders one mask, with no per-lane loop (whose
    // cost in a warp would be the longest window of its 32 lanes).  Other
    // runs take the walk of best_of.
    //
    // Per run the lane keeps pk[], packed (the longest length is stored at
    // once, and read back from the leftmost holder when needed again):
    //   staged tiles:  bits 0..B-1 leftmost holder v (all ones: none), B =
    //                  kVBits (13, or 14 for 8192-position tiles, whose
    //                  staged indices reach 8319); bit 31 clear: bits B..30 =
    //                  holders as a mask from v (bit 0 = v); bit 31 set:
    //                  bits B..30 = number of holders;
    //   other tiles:   the number of holders.
    constexpr int kVBits = Cfg<TP>::kVBits;
    constexpr uint32_t kNone = Cfg<TP>::kNone;
    constexpr uint32_t kFieldMask = (1u << Cfg<TP>::kMaskBits) - 1u;
    uint32_t pk[kChunksPerWarp];
    unsigned (*RT)[kWarp] = sm.rt[warp];
    // the longest length and the leftmost holder's start of a position are
    // stored as soon as its run is done (Algorithm 2's output)
    auto store_leftmost = [&](int c, int32_t b, int32_t vb) {
        const int32_t k = k0 + c * kWarp + lane;
        if (k < n) {
            __stcs(lr_len + k, b);
            __stcs(lr_start + k, b > 0 ? start_of(vb) : -1);
        }
    };
#pragma unroll
    for (int q = 0; q < kChunksPerWarp; ++q) {
        const int c = q * kWarps + warp;
        int32_t lw, hi;
        window(c, lw, hi);
        const int32_t U0 = __shfl_sync(kFull, lw, 0);
        const int32_t usz = __shfl_sync(kFull, hi, kWarp - 1) - U0 + 1;
        const bool fast = staged && usz <= kWarp;                 // warp-uniform; staged lengths < 2^27
        if (fast) {
            const int32_t len_l = ((int)lane < usz) ? SCL[U0 + (int)lane] : 0;
            unsigned key = ((int)lane < usz) ? (((unsigned)len_l << 5) | (31u - lane)) : 0u;
            RT[0][lane] = key;
            if constexpr (kAll) RT[5][lane] = __match_any_sync(kFull, len_l);
#pragma unroll
            for (int l = 1; l <= 4; ++l) {
                const unsigned o = __shfl_down_sync(kFull, key, 1u << (l - 1));
                key = key > o ? key : o;
                RT[l][lane] = key;
            }
            __syncwarp();
            // every lane queries (an empty window reads a harmless entry and
            // is then discarded), so the warp does not diverge
            const bool valid = lw <= hi;
            const int l0 = valid ? lw - U0 : 0, h0 = valid ? hi - U0 : 0;
            int lv = 31 - __clz(h0 - l0 + 1);
            lv = lv > 4 ? 4 : lv;
            const unsigned ka = RT[lv][l0], kb = RT[lv][h0 - (1 << lv) + 1];
            const unsigned kk = ka > kb ? ka : kb;
            const int jl = 31 - (int)(kk & 31u);
            const int32_t b = valid ? (int32_t)(kk >> 5) : 0;
            const int32_t sj = SCS[valid ? U0 + jl : 0];
            uint32_t p = kNone;
            if constexpr (kAll) {
                const unsigned range = ((2u << h0) - 1u) & ~((1u << jl) - 1u);
                const unsigned hold = (RT[5][jl] & range) >> jl;
                const uint32_t v = (uint32_t)(U0 + jl);
                const uint32_t pm = hold <= kFieldMask ? (v | (hold << kVBits))
                                                       : (v | ((uint32_t)__popc(hold) << kVBits) | 0x80000000u);
                p = valid ? pm : kNone;
            }
            __syncwarp();                                         // before the next run rewrites RT
            pk[q] = p;
            const int32_t k = k0 + c * kWarp + lane;
            if (k < n) {
                __stcs(lr_len + k, b);
                __stcs(lr_start + k, valid ? sj : -1);
            }
        } else {
            int32_t b, vb, ct;
            best_of(lw, hi, b, vb, ct);
            store_leftmost(c, b, vb);
            if (!staged) pk[q] = (uint32_t)ct;
            else if (ct == 0) pk[q] = kNone;
            else if (ct == 1) pk[q] = (uint32_t)vb | (1u << kVBits);
            else pk[q] = (uint32_t)vb | ((uint32_t)ct << kVBits) | 0x80000000u;
        }
    }
    // holders of run q (the tie count of its position)
    auto count_of = [&](uint32_t p) -> int32_t {
        if (!staged) return (int32_t)p;
        return (p >> 31) ? (int32_t)((p >> kVBits) & kFieldMask) : __popc(p >> kVBits);
    };
    if constexpr (kAll) {
        // CSR offsets: scan of the tie counts within the tile.  Counts are
        // almost always below 4: the run scan is then two ballots (the
        // counts' bit planes).  The tile's total is published before the
        // per-position stores of pass 2, so that later tiles rarely wait for
        // it.
#pragma unroll
        for (int q = 0; q < kChunksPerWarp; ++q) {
            const int32_t cq = count_of(pk[q]);
            int ex, tot;
            const unsigned big = __ballot_sync(kFull, cq > 3);
            if (big == 0u) {                              // two bit planes of counts below 4
                const unsigned b0 = __ballot_sync(kFull, cq & 1), b1 = __ballot_sync(kFull, cq & 2);
                ex = __popc(b0 & below) + 2 * __popc(b1 & below);
                tot = __popc(b0) + 2 * __popc(b1);
            } else {
                const int incl = warp_incl_scan(cq);
                ex = incl - cq;
                tot = __shfl_sync(kFull, incl, kWarp - 1);
            }
            RT[q][lane] = (unsigned)ex;               // exclusive prefix within the run
            if (lane == 0) sm.chunk[q * kWarps + warp] = tot;
        }
        __syncthreads();
        if (warp == 0) {
            const int tot = scan_chunks<kChunks>(sm.chunk);
            if (lane == 0) {
                if (tile != s.hold_tile) publish(s.status_o, tile, tile == 0 ? kPrefix : kAggregate, tot);
                sm.ttot = tot;
            }
        }
    }

    if constexpr (kAll) {
        __syncthreads();
        if (warp == 0) {
            const int tot = sm.ttot;
            const long long ex = (tile == 0) ? 0 : lookback(s.status_o, tile, s.err, s.qerr, s.spin_limit);
            if (lane == 0) {
                if (tile != 0 && tile != s.hold_tile) publish(s.status_o, tile, kPrefix, ex + tot);
                sm.obase = ex;
                if (tile == num_cover_tiles(n, TP) - 1) offsets[n] = ex + tot;
            }
        }
        __syncthreads();
        const long long obase = sm.obase;
#pragma unroll
        for (int q = 0; q < kChunksPerWarp; ++q) {
            const int c = q * kWarps + warp;
            const int32_t k = k0 + c * kWarp + lane;
            long long o = obase + sm.chunk[c] + (int)RT[q][lane];
            if (k < n) __stcs(reinterpret_cast<long long*>(offsets) + k, o);
            const uint32_t p = pk[q];
            const int32_t cq = count_of(p);
            if (cq == 0) continue;
            // the second walk of Algorithm 4: every compact LLR of the
            // longest length, ascending
            if (staged && !(p >> 31)) {
                const int32_t v0 = (int32_t)(p & kNone);
                unsigned m = p >> kVBits;
                while (m) {
                    const int j = __ffs(m) - 1;
                    m &= m - 1u;
                    if (o < capacity) __stcs(starts + o, start_of(v0 + j));
                    ++o;
                }
            } else {
                int32_t lw, hi;
                window(c, lw, hi);
                int32_t bq;                                       // the longest length, again
                if (staged) {
                    bq = SCL[p & kNone];
                } else {
                    int32_t vb_, ct_;
                    best_of(lw, hi, bq, vb_, ct_);
                }
                for (int32_t v = staged ? (int32_t)(p & kNone) : lw; v <= hi; ++v) {
                    const int32_t len = staged ? SCL[v] : __ldg(gce + v) - __ldg(gcs + v) + 1;
                    if (len == bq) {
                        if (o < capacity) __stcs(starts + o, start_of(v));
                        ++o;
                    }
                }
            }
        }
    }
}

namespace {

template <bool kAll, int TP>
void launch_cover_t(int32_t n, const Scratch& s, int32_t* lr_len, int32_t* lr_start, int64_t* offsets,
                    int32_t* starts, long long capacity, cudaStream_t stream) {
    const unsigned grid = (unsigned)num_cover_tiles(n, TP);
    k_cover<kAll, TP><<<grid, Cfg<TP>::kThr, sizeof(CoverSmem<TP>), stream>>>(n, s, lr_len, lr_start, offsets, starts,
                                                                              capacity);
}

template <int TP>
cudaError_t set_cover_smem() {
    cudaError_t e = cudaFuncSetAttribute(k_cover<true, TP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(CoverSmem<TP>));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_cover<false, TP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(CoverSmem<TP>));
    return e;
}

}  // namespace

cudaError_t configure_cover() {
    cudaError_t e = set_cover_smem<1>();
    if (e == cudaSuccess) e = set_cover_smem<2>();
    if (e == cudaSuccess) e = set_cover_smem<4>();
    return e;
}

void launch_cover(int32_t n, const Scratch& s, int32_t* lr_len, int32_t* lr_start, int64_t* offsets,
                  int32_t* starts, long long capacity, bool all, int tiles_per, cudaStream_t stream) {
    if (!all) { offsets = nullptr; starts = nullptr; capacity = 0; }
    switch (tiles_per) {
        case 1:
            if (all) launch_cover_t<true, 1>(n, s, lr_len, lr_start, offsets, starts, capacity, stream);
            else launch_cover_t<false, 1>(n, s, lr_len, lr_start, offsets, starts, capacity, stream);
            break;
        case 4:
            if (all) launch_cover_t<true, 4>(n, s, lr_len, lr_start, offsets, starts, capacity, stream);
            else launch_cover_t<false, 4>(n, s, lr_len, lr_start, offsets, starts, capacity, stream);
            break;
        default:
            if (all) launch_cover_t<true, 2>(n, s, lr_len, lr_start, offsets, starts, capacity, stream);
            else launch_cover_t<false, 2>(n, s, lr_len, lr_start, offsets, starts, capacity, stream);
    }
}

}  // namespace lr
