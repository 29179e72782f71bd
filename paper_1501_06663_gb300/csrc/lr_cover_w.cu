// The warp-segment cover kernel of the longest-repeat query (Tian and Xu,
// arXiv 1501.06663, Algorithms 2 and 4, GPU kernel of Sec. 4.2.2): from the
// compact LLR array LLRc to the longest repeats of every position.
//
// Starts and ends of LLRc strictly increase (Sec. 3.2), so the compact LLR's
// covering a position k form a window [lw_k, hi_k] of LLRc whose two ends
// only move right as k grows:
//   hi_k = (number of entries starting at or before k) - 1,
//   lw_k =  number of entries ending before k.
// Each warp owns one segment of kSeg = 256 consecutive positions and covers
// it on its own:
//
//  * it stages the segment's window range in its own shared memory: the
//    entries starting in the segment (LLRc[c0, c1), c0 = seg_cbase[g]) and
//    the carry before them, the entries whose end reaches the segment (a
//    suffix of LLRc[0, c0), since ends increase), found by one ballot over
//    the 32 entries before c0; in the same pass it sets two bitmaps over
//    the segment's positions: where an entry starts and where one ends;
//  * per run of 32 positions, every lane's lw and hi are then a running
//    count plus one popcount of a bitmap word, with no search at all (the
//    paper searches per position);
//  * the windows of a run lie in one range of entries [U0, U1]; when it
//    holds at most 32, lane j keeps entry U0 + j and the warp builds a
//    range-maximum table over the keys (length << 5 | 31 - j) in five
//    shuffle levels plus the masks of equal lengths (match.any): the longest
//    length, the leftmost holder and the holders of every lane's window are
//    then two table reads and a mask, with no per-lane loop (Algorithm 2's
//    walk and Algorithm 4's ties); longer ranges take the walk itself;
//  * for the all-LR query, the CTA's 16 segments add up their numbers of LR
//    starts, one warp finds the CTA tile's place in the CSR by a decoupled
//    look-back over the tiles before it (two barriers), and every warp
//    writes its segment's offsets and, ascending, the start of every holder
//    (Algorithm 4's second walk), gathered per run in shared memory so that
//    the starts go out as contiguous runs.
//
// A lane owns one position of each run, so every per-position store of a
// warp is one contiguous 128- or 256-byte run.  A segment whose carry is
// longer than kCarry entries (windows of more than 64 compact LLR's reaching
// back across the segment start) reads LLRc in place instead of staging it.
#include <cuda_runtime.h>
#include <climits>
#include <cstdint>
#include "lr_device.cuh"
#include "lr_internal.h"

namespace lr {

namespace {

constexpr int kRuns = kSeg / kWarp;          // 8 runs of 32 positions per segment
constexpr int kSegWarps = kSegTile / kSeg;   // warps (segments) per CTA: 16
constexpr int kSegThreads = kSegWarps * kWarp;
constexpr int kCarry = 64;                   // carry entries a segment stages
constexpr int kCapW = kSeg + kCarry;         // staged entries: at most one start per position + the carry
constexpr int kEmit = 64;                    // LR starts of one run gathered in shared memory before storing
// Packed per-run word of a lane (pk): bits 0..8 the staged index v of the
// leftmost holder (all ones: none); bit 31 clear: bits 9..30 = the holders as
// a mask from v (bit 0 = v); bit 31 set: bits 9..30 = the number of holders.
constexpr int kVBitsW = 9;
constexpr uint32_t kNoneW = (1u << kVBitsW) - 1u;
constexpr uint32_t kFieldW = (1u << (31 - kVBitsW)) - 1u;
static_assert(kCapW <= (int)kNoneW, "staged indices must fit the holder-index field");
static_assert(kCapW <= (int)kFieldW, "a tie count must fit the count field");

struct __align__(16) WarpStage {
    int32_t cs[kCapW];                       // starts of the staged range LLRc[lo, c1)
    int32_t cl[kCapW];                       // lengths
    unsigned rt[6][kWarp];                   // range-max levels 0..4 and equal-length masks of one run
    uint32_t pk[kRuns][kWarp];               // the lanes' packed words of every run, kept for pass 2
    unsigned sb[kRuns];                      // bit x of word r: an entry starts at p0 + 32 r + x
    unsigned eb[kRuns];                      // bit x of word r: an entry ends at p0 + 32 r + x
    int32_t ob[kEmit];                       // one run's LR starts, gathered for coalesced stores
};

struct __align__(16) CoverWSmem {
    WarpStage w[kSegWarps];
    long long tile;
    long long tile_ex;                       // LR starts of all earlier tiles
    int32_t tot[kSegWarps];                  // the segments' numbers of LR starts
};

// Entries of the window range: staged in shared memory or read in place.
template <bool kStaged>
struct Range {
    const int32_t* cs;
    const int32_t* ce;                       // staged: lengths; in place: ends
    __device__ __forceinline__ int32_t s(int32_t v) const {
        if constexpr (kStaged) return cs[v]; else return __ldg(cs + v);
    }
    __device__ __forceinline__ int32_t len(int32_t v) const {
        if constexpr (kStaged) return ce[v]; else return __ldg(ce + v) - __ldg(cs + v) + 1;
    }
};

// Window [lw, hi] of each lane's position in run r from the bitmap words;
// us (entries started before the run) and ue (entries ended before it) move
// past the run.  The run's windows lie in [U0, U1] = [ue before, us after - 1].
__device__ __forceinline__ void run_window(const WarpStage& W, int r, int32_t& us, int32_t& ue, int32_t& lw,
                                           int32_t& hi) {
    const unsigned lane = lane_id();
    const unsigned below = (1u << lane) - 1u;
    const unsigned smap = W.sb[r], emap = W.eb[r];
    hi = us + __popc(smap & (below | (1u << lane))) - 1;
    lw = ue + __popc(emap & below);
    us += __popc(smap);
    ue += __popc(emap);
}

// Longest length b over the window [lw, hi], index vb of its leftmost
// holder and the number of holders ct, by a walk (Algorithm 2 / 4).
template <bool kStaged>
__device__ __forceinline__ void walk_best(const Range<kStaged>& R, int32_t lw, int32_t hi, int32_t& b, int32_t& vb,
                                          int32_t& ct) {
    b = 0; vb = -1; ct = 0;
    for (int32_t v = lw; v <= hi; ++v) {
        const int32_t len = R.len(v);
        const bool gt = len > b;
        ct = gt ? 1 : ct + (len == b);
        vb = gt ? v : vb;
        b = gt ? len : b;
    }
}

__device__ __forceinline__ int32_t count_of(uint32_t p) {
    // mask form: the holders' bits (none: no bits); count form: the field
    return (p >> 31) ? (int32_t)((p >> kVBitsW) & kFieldW) : __popc(p >> kVBitsW);
}

// Exclusive prefix of the lanes' tie counts within a run, and the run's
// total.  Counts below 4 (nearly all) are summed from two bit planes by
// ballots; otherwise a shuffle scan.
__device__ __forceinline__ void scan_counts(int32_t cq, int32_t& ex, int32_t& total) {
    const unsigned lane = lane_id();
    const unsigned below = (1u << lane) - 1u;
    const unsigned big = __ballot_sync(kFull, cq > 3);
    if (big == 0u) {
        const unsigned b0 = __ballot_sync(kFull, cq & 1), b1 = __ballot_sync(kFull, cq & 2);
        ex = __popc(b0 & below) + 2 * __popc(b1 & below);
        total = __popc(b0) + 2 * __popc(b1);
    } else {
        const int32_t incl = warp_incl_scan(cq);
        ex = incl - cq;
        total = __shfl_sync(kFull, incl, kWarp - 1);
    }
}

// Stages entries [lo, lo + M) when the range fits (carry C <= kCarry) and
// sets the segment's start and end bitmaps; returns whether it staged (not
// when a length reaches 2^27, which the range-max keys cannot hold).
__device__ __forceinline__ bool stage_segment(const Scratch& s, WarpStage& W, int32_t p0, int32_t lo, int32_t C,
                                              int32_t M) {
    const unsigned lane = lane_id();
    const bool fits = C <= kCarry && M <= kCapW;
    bool longlen = false;
    if (lane < kRuns) { W.sb[lane] = 0u; W.eb[lane] = 0u; }
    __syncwarp();
    for (int32_t i0 = 0; i0 < M; i0 += kWarp) {
        const int32_t i = i0 + (int32_t)lane;
        if (i < M) {
            const int32_t cs = __ldg(s.cstart + lo + i), ce = __ldg(s.cend + lo + i);
            const int32_t len = ce - cs + 1;
            if (fits) { W.cs[i] = cs; W.cl[i] = len; }
            longlen |= len >= (1 << 27);
            const unsigned xs = (unsigned)cs - (unsigned)p0, xe = (unsigned)ce - (unsigned)p0;
            if (i >= C && xs < (unsigned)kSeg) atomicOr(&W.sb[xs >> 5], 1u << (xs & 31u));
            if (xe < (unsigned)kSeg) atomicOr(&W.eb[xe >> 5], 1u << (xe & 31u));
        }
    }
    const bool staged = fits && !__any_sync(kFull, longlen);
    __syncwarp();
    return staged;
}

// Pass 1 of one segment: windows, longest lengths and leftmost starts
// (stored at once), and for the all-LR query the tie information of every
// lane in pk; returns the segment's number of LR starts.
template <bool kAll, bool kStaged>
__device__ __forceinline__ int32_t cover_pass1(int32_t n, int32_t p0, int32_t C, const Range<kStaged>& R, WarpStage& W,
                                               int32_t* __restrict__ lr_len, int32_t* __restrict__ lr_start) {
    const unsigned lane = lane_id();
    int32_t seg_total = 0;
    int32_t us = C, ue = 0;
#pragma unroll 1
    for (int r = 0; r < kRuns; ++r) {
        const int32_t k = p0 + r * kWarp + (int32_t)lane;
        const int32_t U0 = ue;
        int32_t lw, hi;
        run_window(W, r, us, ue, lw, hi);
        if (k >= n) hi = lw - 1;                            // past the string: nothing covers it
        const int32_t usz = us - U0;                        // entries of [U0, U1]
        const bool fast = kStaged && usz <= kWarp;          // staged lengths are below 2^27
        int32_t len_l = 0;
        if (fast) len_l = (int)lane < usz ? W.cl[U0 + (int)lane] : 0;
        int32_t b = 0, st = -1;
        uint32_t p = kNoneW;
        if (fast) {
            unsigned key = (int)lane < usz ? (((unsigned)len_l << 5) | (31u - lane)) : 0u;
            W.rt[0][lane] = key;
            if constexpr (kAll) W.rt[5][lane] = __match_any_sync(kFull, len_l);
#pragma unroll
            for (int l = 1; l <= 4; ++l) {
                const unsigned o = __shfl_down_sync(kFull, key, 1u << (l - 1));
                key = key > o ? key : o;
                W.rt[l][lane] = key;
            }
            __syncwarp();
            // every lane queries (an empty window reads a harmless entry and
            // is then discarded), so the warp does not diverge
            const bool valid = lw <= hi;
            const int l0 = valid ? lw - U0 : 0, h0 = valid ? hi - U0 : 0;
            int lv = 31 - __clz(h0 - l0 + 1);
            lv = lv > 4 ? 4 : lv;
            const unsigned ka = W.rt[lv][l0], kb = W.rt[lv][h0 - (1 << lv) + 1];
            const unsigned kk = ka > kb ? ka : kb;
            const int jl = 31 - (int)(kk & 31u);
            b = valid ? (int32_t)(kk >> 5) : 0;
            const int32_t sj = W.cs[valid ? U0 + jl : 0];
            st = valid ? sj : -1;
            if constexpr (kAll) {
                const unsigned range = ((2u << h0) - 1u) & ~((1u << jl) - 1u);
                const unsigned hold = (W.rt[5][jl] & range) >> jl;
                const uint32_t v = (uint32_t)(U0 + jl);
                const uint32_t pm = hold <= kFieldW ? (v | (hold << kVBitsW))
                                                    : (v | ((uint32_t)__popc(hold) << kVBitsW) | 0x80000000u);
                p = valid ? pm : kNoneW;
            }
            __syncwarp();                                   // before the next run rewrites the table
        } else {
            int32_t vb, ct;
            walk_best<kStaged>(R, lw, hi, b, vb, ct);
            st = b > 0 ? R.s(vb) : -1;
            if constexpr (kStaged) {
                if (ct == 1) p = (uint32_t)vb | (1u << kVBitsW);
                else if (ct > 1) p = (uint32_t)vb | ((uint32_t)ct << kVBitsW) | 0x80000000u;
            } else {
                p = (uint32_t)ct;                           // the count; pass 2 walks the window again
            }
        }
        if (k < n) {
            __stcs(lr_len + k, b);
            __stcs(lr_start + k, st);
        }
        if constexpr (kAll) {
            W.pk[r][lane] = p;
            seg_total += __reduce_add_sync(kFull, kStaged ? count_of(p) : (int32_t)p);
        }
    }
    return seg_total;
}

// Pass 2 of one segment (all-LR query): CSR offsets from `base` and the
// starts of every holder, ascending (Algorithm 4's second walk).  A run
// whose lanes hold at most 3 LR's each in mask form (nearly all) gathers its
// starts in shared memory without branching and stores them as one
// contiguous run; other runs walk.
template <bool kStaged>
__device__ __forceinline__ void cover_pass2(int32_t n, int32_t p0, int32_t C, int32_t M, const Range<kStaged>& R,
                                            WarpStage& W, long long base, int64_t* __restrict__ offsets,
                                            int32_t* __restrict__ starts, long long capacity) {
    const unsigned lane = lane_id();
    long long run_base = base;
    int32_t us = C, ue = 0;
#pragma unroll 1
    for (int r = 0; r < kRuns; ++r) {
        const int32_t k = p0 + r * kWarp + (int32_t)lane;
        const uint32_t p = W.pk[r][lane];
        int32_t cq, lw = 0, hi = -1, bq = 0, vb = -1;
        if constexpr (kStaged) {
            cq = count_of(p);
        } else {
            run_window(W, r, us, ue, lw, hi);
            if (k >= n) hi = lw - 1;
            walk_best<kStaged>(R, lw, hi, bq, vb, cq);
        }
        int32_t ex, T;
        scan_counts(cq, ex, T);
        long long o = run_base + ex;
        const long long rb = run_base;
        run_base += T;
        if (k < n) __stcs(reinterpret_cast<long long*>(offsets) + k, o);
        if constexpr (kStaged) {
            if (T <= kEmit && !__any_sync(kFull, (p >> 31) != 0u || cq > 3)) {
                const int32_t v0 = (int32_t)(p & kNoneW);
                const unsigned m1 = (p >> (kVBitsW + 1)) & (kFieldW >> 1);   // holders after v0, from v0 + 1
                const unsigned m2 = m1 & (m1 - 1u);
                const int32_t j2 = __ffs(m1), j3 = __ffs(m2);              // v0 + j: the 2nd and 3rd holders
                if (cq >= 1) W.ob[ex] = W.cs[v0];
                if (cq >= 2) W.ob[ex + 1] = W.cs[v0 + j2];
                if (cq >= 3) W.ob[ex + 2] = W.cs[v0 + j3];
                __syncwarp();
                if ((int32_t)lane < T && rb + lane < capacity) __stcs(starts + rb + lane, W.ob[lane]);
                if ((int32_t)lane + kWarp < T && rb + kWarp + lane < capacity)
                    __stcs(starts + rb + kWarp + lane, W.ob[kWarp + lane]);
                __syncwarp();
                continue;
            }
            if (cq == 0) continue;
            const int32_t v0 = (int32_t)(p & kNoneW);
            if (!(p >> 31)) {
                unsigned mk = (p >> kVBitsW) & kFieldW;
                while (mk) {
                    const int j = __ffs(mk) - 1;
                    mk &= mk - 1u;
                    if (o < capacity) __stcs(starts + o, W.cs[v0 + j]);
                    ++o;
                }
            } else {
                const int32_t b0 = W.cl[v0];
                for (int32_t v = v0; v < M && W.cs[v] <= k; ++v) {
                    if (W.cl[v] == b0) {
                        if (o < capacity) __stcs(starts + o, W.cs[v]);
                        ++o;
                    }
                }
            }
        } else {
            for (int32_t v = vb; v <= hi; ++v) {
                if (R.len(v) == bq) {
                    if (o < capacity) __stcs(starts + o, R.s(v));
                    ++o;
                }
            }
        }
    }
}

}  // namespace

template <bool kAll>
__global__ void __launch_bounds__(kSegThreads, 3)
k_cover_w(int32_t n, Scratch s, int32_t* __restrict__ lr_len, int32_t* __restrict__ lr_start,
          int64_t* __restrict__ offsets, int32_t* __restrict__ starts, long long capacity) {
    extern __shared__ __align__(16) unsigned char wsm_raw[];
    CoverWSmem& sm = *reinterpret_cast<CoverWSmem*>(wsm_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    WarpStage& W = sm.w[warp];
    if (tid == 0) sm.tile = atomicAdd(&s.tickets[2], 1u);
    __syncthreads();
    const long long tile = sm.tile;
    const long long g = tile * kSegWarps + warp;             // this warp's segment
    const bool live = g < s.nsegs;                           // warp-uniform
    const int32_t p0 = (int32_t)(live ? g * kSeg : 0);       // n < 2^31: positions fit 32 bits
    int32_t C = 0, M = 0, lo = 0;
    bool staged = true;
    if (live) {
        // LLRc entries [c0, c1) start inside the segment; clamped so that a
        // corrupted front end (already reported) cannot send reads out of bounds
        int32_t m = s.seg_cbase[s.nsegs];
        m = m < 0 ? 0 : (m > n ? n : m);
        int32_t c0 = s.seg_cbase[g], c1 = s.seg_cbase[g + 1];
        c0 = c0 < 0 ? 0 : (c0 > m ? m : c0);
        c1 = c1 < c0 ? c0 : (c1 > m ? m : c1);
        // the carry: the entries before c0 whose end reaches p0 (a suffix of
        // LLRc[0, c0), ends increase), 32 at a time
        lo = c0;
        while (lo > 0) {
            const int32_t idx = lo - 1 - lane;
            const bool reach = idx >= 0 && __ldg(s.cend + idx) >= p0;
            const unsigned mk = __ballot_sync(kFull, reach);
            if (mk == kFull) { lo -= kWarp; continue; }
            lo -= __ffs(~mk) - 1;
            break;
        }
        C = c0 - lo;
        M = c1 - lo;
        staged = stage_segment(s, W, p0, lo, C, M);
    }
    int32_t total = 0;
    if (live) {
        if (staged) total = cover_pass1<kAll, true>(n, p0, C, Range<true>{W.cs, W.cl}, W, lr_len, lr_start);
        else total = cover_pass1<kAll, false>(n, p0, C, Range<false>{s.cstart + lo, s.cend + lo}, W, lr_len, lr_start);
    }
    if constexpr (!kAll) return;

    // the CSR base of every segment: the CTA tile's place by a decoupled
    // look-back over the tiles (every warp reads it; warp 0 publishes), plus
    // the segments before it in the tile
    if (lane == 0) sm.tot[warp] = total;
    __syncthreads();
    int32_t tile_tot = 0, warp_ex = 0;
#pragma unroll
    for (int w = 0; w < kSegWarps; ++w) {
        const int32_t t = sm.tot[w];
        tile_tot += t;
        warp_ex += w < warp ? t : 0;
    }
    if (warp == 0) {
        const bool held = tile == s.hold_tile;
        if (lane == 0 && !held) publish(s.status_w, tile, tile == 0 ? kPrefix : kAggregate, tile_tot);
        const long long ex = (tile == 0) ? 0 : lookback(s.status_w, tile, s.err, s.qerr, s.spin_limit);
        if (lane == 0) {
            if (tile != 0 && !held) publish(s.status_w, tile, kPrefix, ex + tile_tot);
            if ((tile + 1) * kSegWarps >= s.nsegs) offsets[n] = ex + tile_tot;
            sm.tile_ex = ex;
        }
    }
    __syncthreads();
    if (!live) return;
    const long long base = sm.tile_ex + warp_ex;
    if (staged) cover_pass2<true>(n, p0, C, M, Range<true>{W.cs, W.cl}, W, base, offsets, starts, capacity);
    else cover_pass2<false>(n, p0, C, M, Range<false>{s.cstart + lo, s.cend + lo}, W, base, offsets, starts, capacity);
}

void launch_cover_w(int32_t n, const Scratch& s, int32_t* lr_len, int32_t* lr_start, int64_t* offsets,
                    int32_t* starts, long long capacity, bool all, cudaStream_t stream) {
    const unsigned grid = (unsigned)((s.nsegs + kSegWarps - 1) / kSegWarps);
    const size_t smem = sizeof(CoverWSmem);
    if (all)
        k_cover_w<true><<<grid, kSegThreads, smem, stream>>>(n, s, lr_len, lr_start, offsets, starts, capacity);
    else
        k_cover_w<false><<<grid, kSegThreads, smem, stream>>>(n, s, lr_len, lr_start, nullptr, nullptr, 0);
}

cudaError_t configure_cover_w() {
    const int smem = (int)sizeof(CoverWSmem);
    cudaError_t e = cudaFuncSetAttribute(k_cover_w<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cover_w<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

}  // namespace lr
