// Front ends of the longest-repeat query: they turn the input arrays into
// the compact LLR array LLRc (Sec. 3.2 / Sec. 4.2.1 of Tian and Xu, arXiv
// 1501.06663): every position i with L_i > 0 and L_i >= L_{i-1}, in
// ascending i, as cstart[t] = i, cend[t] = i + L_i - 1, where
// L_i = max(lcp[rank[i]], lcp[rank[i]+1]) (Lemma 1).  They also record, for
// every tile of kTile positions and every segment of kSeg positions, the
// index of its first LLRc entry (tile_cbase, seg_cbase), which the cover
// kernels start from.
//
// Two front ends compute the same LLRc:
//
//  * rank-order (the default when the suffix array is given).  Lemma 1 read
//    in rank order is L_{sa[r]} = max(lcp[r], lcp[r+1]): sa and lcp are then
//    read once, coalesced, instead of one random lcp sector per position.
//    k_part1 and k_part2 radix-partition the pairs <sa[r], L_{sa[r]}> by
//    the position, first into super-buckets of 2^20 positions, then into
//    buckets of 2^15 (packed 4-byte entries; a length of 4095 or more goes
//    to lbig).  k_bucket_llr then loads one bucket per
//    CTA, scatters its lengths into shared memory by position, and flags
//    and compacts them.
//
//  * rank gather (when only rank is given, as in the paper's data flow of
//    Sec. 4): k_gather_llr reads rank coalesced and gathers the two lcp
//    words of each position, then flags and compacts one tile.
//
// Both place their entries in LLRc with a decoupled look-back over the
// per-CTA counts (tiles handed out in order by an atomic ticket).
#include <cuda_runtime.h>
#include <cstdint>
#include "lr_device.cuh"
#include "lr_internal.h"

namespace lr {

namespace {

__device__ __forceinline__ void report(const Scratch& s, unsigned bits) {
    atomicOr(s.err, bits);
    atomicOr(s.qerr, bits);
}

// Exclusive scan of 64 ints by one warp (two per lane); returns the total.
__device__ __forceinline__ int warp_scan64(int32_t* a) {
    const int lane = lane_id();
    const int x = a[2 * lane], y = a[2 * lane + 1];
    const int incl = warp_incl_scan(x + y);
    a[2 * lane] = incl - x - y;
    a[2 * lane + 1] = incl - y;
    return __shfl_sync(kFull, incl, kWarp - 1);
}

// The strings of a batched query that overlap one CTA's flattened range
// [g0, g1), with their offsets staged in shared memory when there are at
// most kSegCap of them (else looked up in global memory).
struct SegView {
    const int64_t* off;      // global, num + 1 entries
    long long* sh;           // shared, kSegCap + 1 entries
    long long j0, j1;        // first and last string overlapping the range
    bool staged;

    // Called by the whole CTA (contains a barrier).
    __device__ void stage(const Segs& segs, const Scratch& s, long long g0, long long g1, long long* smem) {
        off = segs.off;
        sh = smem;
        // j1: the string holding the start of the tile after the range,
        // which is at or after the string holding g1 - 1
        const long long t0 = g0 / kTile, t1 = (g1 - 1) / kTile + 1;
        j0 = s.tile_seg[t0];
        j1 = (t1 < s.ntiles) ? s.tile_seg[t1] : segs.num - 1;
        if (j1 < j0) j1 = j0;                          // only after a reported bad offset table
        staged = (j1 - j0 + 2) <= kSegCap + 1;
        if (staged)
            for (long long i = threadIdx.x; i < j1 - j0 + 2; i += blockDim.x) sh[i] = __ldg(off + j0 + i);
        __syncthreads();
    }
    __device__ __forceinline__ long long at(long long j) const { return staged ? sh[j - j0] : __ldg(off + j); }
    // the string holding position g (j0 <= result <= j1); `hint` only moves forward
    __device__ __forceinline__ long long find(long long g, long long hint) const {
        if (staged) {
            long long j = hint;
            while (j < j1 && sh[j + 1 - j0] <= g) ++j;
            return j;
        }
        long long lo = hint, hi = j1;                 // last j with off[j] <= g
        while (lo < hi) {
            const long long mid = (lo + hi + 1) >> 1;
            if (__ldg(off + mid) <= g) lo = mid; else hi = mid - 1;
        }
        return lo;
    }
};

// For every tile of kTile flattened positions, the string holding its first
// position (the last j with off[j] <= tile start).
__global__ void k_seg_index(int32_t n, Scratch s, Segs segs) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= s.ntiles) return;
    const long long g = t * kTile;
    long long lo = 0, hi = segs.num - 1;
    while (lo < hi) {
        const long long mid = (lo + hi + 1) >> 1;
        if (__ldg(segs.off + mid) <= g) lo = mid; else hi = mid - 1;
    }
    s.tile_seg[t] = (int32_t)lo;
    if (t == 0 && (__ldg(segs.off) != 0 || __ldg(segs.off + segs.num) != n)) report(s, kErrInput);
    // offsets must not decrease
    for (long long j = t; j < segs.num; j += s.ntiles)
        if (__ldg(segs.off + j) > __ldg(segs.off + j + 1)) report(s, kErrInput);
}

}  // namespace

void launch_seg_index(int32_t n, const Scratch& s, const Segs& segs, cudaStream_t stream) {
    k_seg_index<<<(unsigned)((s.ntiles + 255) / 256), 256, 0, stream>>>(n, s, segs);
}

// ---------------------------------------------------------------------------
// rank gather front end
// ---------------------------------------------------------------------------

template <bool kBatch>
__global__ void __launch_bounds__(kThreads)
k_gather_llr(const int32_t* __restrict__ rank, const int32_t* __restrict__ lcp, int32_t n, Scratch s, Segs segs) {
    constexpr int kChunks = kTile / kWarp;          // 64 runs of 32 positions
    constexpr int kWarps = kThreads / kWarp;        // 8
    __shared__ int32_t Ls[kTile + 1];               // Ls[0] = L_{k0-1}, Ls[1+x] = L_{k0+x}
    __shared__ int32_t chunk[kChunks];
    __shared__ int32_t c_s[kTile];
    __shared__ int32_t c_e[kTile];
    __shared__ long long tile_s, base_s;
    __shared__ int32_t total_s;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) tile_s = atomicAdd(&s.tickets[0], 1u);
    __syncthreads();
    const long long tile = tile_s;
    const long long k0 = tile * kTile;

    // Lemma 1.  rank is streamed; the lcp pair goes through L1 (one sector
    // for 7 of 8 rank values).  Invalid input is reported and clamped so
    // every access stays in bounds.  In a batch, position k of string j has
    // its local rank at rank[k] and the string's lcp at lcp[off[j] + j ..].
    unsigned bad = 0;
    __shared__ long long seg_sh[kBatch ? kSegCap + 1 : 1];
    SegView sv{};
    if constexpr (kBatch) {
        const long long g1 = (k0 + kTile < n) ? k0 + kTile : n;
        sv.stage(segs, s, k0 > 0 ? k0 - 1 : 0, g1, seg_sh);
    }
    long long hint = kBatch ? sv.j0 : 0;
    auto llr = [&](long long k) -> int32_t {
        uint32_t r = (uint32_t)__ldcs(rank + k);
        long long base = 0, nj = n, lbase = 0;
        if constexpr (kBatch) {
            hint = sv.find(k, hint);
            base = sv.at(hint);
            nj = sv.at(hint + 1) - base;
            lbase = base + hint;
            if (base < 0 || nj < 1 || base + nj > n || k < base) { bad = 1; return 0; }   // bad offset table
        }
        if (r >= (uint32_t)nj) { bad = 1; r = 0; }
        const int32_t a = __ldg(lcp + lbase + r), b = __ldg(lcp + lbase + r + 1);
        if (kBatch && ((r == 0 && a != 0) || ((long long)r == nj - 1 && b != 0))) bad = 1;   // lcp sentinels
        int32_t L = a > b ? a : b;
        if (L < 0 || (long long)L > nj - (k - base)) { bad = 1; L = 0; }
        return L;
    };
    if (tid == 0) {
        Ls[0] = (k0 > 0) ? llr(k0 - 1) : 0;
        if (!kBatch && tile == 0 && (__ldg(lcp) != 0 || __ldg(lcp + n) != 0)) bad = 1;
    }
    hint = kBatch ? sv.j0 : 0;
    // All rank loads, then all lcp loads, then the lengths: every load of a
    // thread is in flight before the first one is used.  A batch tile that
    // lies inside one string does the same with that string's offsets and
    // checks; other batch tiles look each position's string up.
    long long sbase = 0, snj = n, slbase = 0;
    bool direct = true;
    if constexpr (kBatch) {
        const long long g1 = (k0 + kTile < n) ? k0 + kTile : n;
        const long long jk = sv.find(k0, sv.j0);
        const long long b0 = sv.at(jk), b1 = sv.at(jk + 1);
        direct = b0 >= 0 && b0 <= k0 && g1 <= b1 && b1 <= (long long)n;
        sbase = b0;
        snj = b1 - b0;
        slbase = b0 + jk;
    }
    if (direct) {
        constexpr int kPer = kTile / kThreads;
        uint32_t r[kPer];
        int32_t a[kPer], c[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const long long k = k0 + j * kThreads + tid;
            r[j] = (k < n) ? (uint32_t)__ldcs(rank + k) : 0u;
        }
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const long long k = k0 + j * kThreads + tid;
            if (k < n && (long long)r[j] >= snj) { bad = 1; r[j] = 0; }
            a[j] = (k < n) ? __ldg(lcp + slbase + r[j]) : 0;
            c[j] = (k < n) ? __ldg(lcp + slbase + r[j] + 1) : 0;
        }
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int x = j * kThreads + tid;
            const long long k = k0 + x;
            int32_t L = a[j] > c[j] ? a[j] : c[j];
            if (k < n) {
                if (kBatch && ((r[j] == 0 && a[j] != 0) || ((long long)r[j] == snj - 1 && c[j] != 0))) bad = 1;
                if (L < 0 || (long long)L > snj - (k - sbase)) { bad = 1; L = 0; }
            }
            Ls[1 + x] = (k < n) ? L : 0;
        }
    } else {
#pragma unroll
        for (int j = 0; j < kTile / kThreads; ++j) {
            const int x = j * kThreads + tid;
            Ls[1 + x] = (k0 + x < n) ? llr(k0 + x) : 0;
        }
    }
    if (bad) report(s, kErrInput);
    __syncthreads();

    // K1 flags by warp ballots over runs of 32 positions, K2 within the tile.
    unsigned masks[kChunks / kWarps];
#pragma unroll
    for (int q = 0; q < kChunks / kWarps; ++q) {
        const int c = q * kWarps + warp;
        const int x = c * kWarp + lane;
        const int32_t L = Ls[1 + x], prev = Ls[x];
        masks[q] = __ballot_sync(kFull, (k0 + x < n) && L > 0 && L >= prev);
        if (lane == 0) chunk[c] = __popc(masks[q]);
    }
    __syncthreads();
    if (warp == 0) {
        const int tot = warp_scan64(chunk);
        if (lane == 0) total_s = tot;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kChunks / kWarps; ++q) {
        const int c = q * kWarps + warp;
        const int x = c * kWarp + lane;
        if ((masks[q] >> lane) & 1u) {
            const int o = chunk[c] + __popc(masks[q] & ((1u << lane) - 1u));
            c_s[o] = (int32_t)(k0 + x);
            c_e[o] = (int32_t)(k0 + x + Ls[1 + x] - 1);
        }
    }
    // K3: the tile's place in LLRc.
    if (warp == 0) {
        const long long ex = lookback_exclusive(s.status_g, tile, total_s, s.err, s.qerr, s.spin_limit);
        if (lane == 0) {
            base_s = ex;
            s.tile_cbase[tile] = (int32_t)ex;
            if (tile == s.ntiles - 1) s.tile_cbase[s.ntiles] = (int32_t)(ex + total_s);
        }
    }
    __syncthreads();
    const long long base = base_s;
    const int total = total_s;
    // first LLRc entry of each kSeg-position segment of the tile
    if (tid < kTile / kSeg) {
        const long long sg = tile * (kTile / kSeg) + tid;
        if (sg < s.nsegs) s.seg_cbase[sg] = (int32_t)(base + chunk[tid * (kSeg / kWarp)]);
        if (sg == s.nsegs - 1) s.seg_cbase[s.nsegs] = (int32_t)(base + total);
    }
    for (int i = tid; i < total; i += kThreads) {
        s.cstart[base + i] = c_s[i];
        s.cend[base + i] = c_e[i];
    }
}

void launch_gather_front(const int32_t* rank, const int32_t* lcp, int32_t n, const Scratch& s, const Segs& segs,
                         cudaStream_t stream) {
    if (segs.num > 0)
        k_gather_llr<true><<<(unsigned)s.ntiles, kThreads, 0, stream>>>(rank, lcp, n, s, segs);
    else
        k_gather_llr<false><<<(unsigned)s.ntiles, kThreads, 0, stream>>>(rank, lcp, n, s, segs);
}

// ---------------------------------------------------------------------------
// rank-order front end
// ---------------------------------------------------------------------------

// Shared memory of a partition CTA: per-bucket counters and the round's
// entries staged in bucket order, so that each warp store writes one
// contiguous run.
struct PartSmem {
    uint32_t* hist;      // nb: entries of the round per bucket, then slot counters
    uint32_t* loff;      // nb + 1: exclusive prefix of hist (staging offsets), in
                         // place of hist (the scan reads hist before it writes)
    uint32_t* base;      // nb: the round's reserved offset in each bucket
    uint32_t* stage;     // kPartRound entries in bucket order
    uint16_t* sbk;       // kPartRound bucket ids of stage[]
};

__device__ __forceinline__ PartSmem part_smem(unsigned char* raw, int nb) {
    PartSmem p;
    p.hist = reinterpret_cast<uint32_t*>(raw);
    p.loff = p.hist;
    p.base = p.loff + nb + 1;
    p.stage = p.base + nb;
    p.sbk = reinterpret_cast<uint16_t*>(p.stage + kPartRound);
    return p;
}

// Bulk-copy staging of a level-1 round: sa[r0, r0 + kPartRound) and the
// round's lcp slice (kPartRound + 1 entries from a 16-byte-aligned start,
// rounded out to 16-byte multiples: at most kPartRound + 8 entries), at a
// 16-byte-aligned offset after the counters; it overlaps the stage area,
// which is written only after every thread has read its entries.
constexpr int kPartLcpCap = kPartRound + 8;
constexpr int kPartLoadBytes = kPartRound * 4 + kPartLcpCap * 4;
__host__ __device__ inline size_t part_load_offset(int nb) { return ((size_t)(2 * nb + 1) * 4 + 15) & ~(size_t)15; }

size_t part_smem_bytes(int nb) {
    const size_t a = (size_t)(2 * nb + 1) * 4 + (size_t)kPartRound * 6;
    const size_t b = part_load_offset(nb) + kPartLoadBytes;
    return a > b ? a : b;
}

// level 2 loads per thread: counters and stage area only
size_t part2_smem_bytes() { return (size_t)(2 * kSubPerSuper + 1) * 4 + (size_t)kPartRound * 6; }

// Exclusive scan of hist[0..nb) into loff[0..nb] by the whole CTA
// (kPartThreads threads, R consecutive buckets each, nb <= R * kPartThreads),
// and one global atomic per non-empty bucket to reserve the round's room:
// base[b] = old cursor.
template <int R>
__device__ __forceinline__ void part_reserve_r(const PartSmem& p, int nb, unsigned* cursor) {
    __shared__ uint32_t wsum[kPartThreads / kWarp];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t a[R], sum = 0;
#pragma unroll
    for (int u = 0; u < R; ++u) {
        const int b = R * tid + u;
        a[u] = (b < nb) ? p.hist[b] : 0u;
        sum += a[u];
    }
    const int incl = warp_incl_scan((int)sum);
    if (lane == kWarp - 1) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int v = (lane < kPartThreads / kWarp) ? (int)wsum[lane] : 0;
        const int wi = warp_incl_scan(v);
        if (lane < kPartThreads / kWarp) wsum[lane] = wi - v;
        if (lane == kWarp - 1) p.loff[nb] = wi;
    }
    __syncthreads();
    uint32_t ex = wsum[warp] + incl - sum;
#pragma unroll
    for (int u = 0; u < R; ++u) {
        const int b = R * tid + u;
        if (b < nb) {
            p.loff[b] = ex;
            if (a[u]) p.base[b] = atomicAdd(cursor + (size_t)b * kCursorStride, a[u]);
        }
        ex += a[u];
    }
}

// The same by warp 0 alone, for at most kWarp * R buckets (R consecutive
// buckets per lane); the other warps wait at the caller's next barrier.
// Each lane writes the staging offsets of its own buckets in place of their
// counts after reading them.
template <int R>
__device__ __forceinline__ void part_reserve_w(const PartSmem& p, int nb, unsigned* cursor) {
    if (threadIdx.x >= kWarp) return;
    const int lane = threadIdx.x;
    uint32_t a[R], sum = 0;
#pragma unroll
    for (int u = 0; u < R; ++u) {
        const int b = R * lane + u;
        a[u] = (b < nb) ? p.hist[b] : 0u;
        sum += a[u];
    }
    const int incl = warp_incl_scan((int)sum);
    uint32_t ex = (uint32_t)incl - sum;
#pragma unroll
    for (int u = 0; u < R; ++u) {
        const int b = R * lane + u;
        if (b < nb) {
            p.loff[b] = ex;
            if (a[u]) p.base[b] = atomicAdd(cursor + (size_t)b * kCursorStride, a[u]);
        }
        ex += a[u];
    }
    if (lane == kWarp - 1) p.loff[nb] = (uint32_t)incl;
}

// The exclusive scan of hist[0..nb) into loff[0..nb] alone, by warp 0, for
// at most kWarp * R buckets: k_part1 then reserves each bucket's room with
// one thread per bucket, in the same phase as its staging writes.
template <int R>
__device__ __forceinline__ void part_scan_w(const PartSmem& p, int nb) {
    if (threadIdx.x >= kWarp) return;
    const int lane = threadIdx.x;
    uint32_t a[R], sum = 0;
#pragma unroll
    for (int u = 0; u < R; ++u) {
        const int b = R * lane + u;
        a[u] = (b < nb) ? p.hist[b] : 0u;
        sum += a[u];
    }
    const int incl = warp_incl_scan((int)sum);
    uint32_t ex = (uint32_t)incl - sum;
#pragma unroll
    for (int u = 0; u < R; ++u) {
        const int b = R * lane + u;
        if (b < nb) p.loff[b] = ex;
        ex += a[u];
    }
    if (lane == kWarp - 1) p.loff[nb] = (uint32_t)incl;
}

// up to 2048 super-buckets (n <= 2^31 positions in super-buckets of 2^20)
__device__ __forceinline__ void part_reserve(const PartSmem& p, int nb, unsigned* cursor) {
    static_assert(4 * kPartThreads >= 2048, "partition CTAs too small for 2048 super-buckets");
    if (nb <= 2 * kPartThreads) part_reserve_r<2>(p, nb, cursor);
    else part_reserve_r<4>(p, nb, cursor);
}

// Slot of this lane's entry in bucket b among the entries counted so far,
// with one shared atomic per run of lanes (in lane order) that carry the
// same b: entries that arrive clustered by bucket would otherwise serialise
// on one counter.  All lanes of the warp call it; a lane with !valid gets
// no slot (and b is ignored).
__device__ __forceinline__ uint32_t run_slot(uint32_t* hist, uint32_t b, bool valid) {
    const int lane = lane_id();
    const uint32_t bk = valid ? b : 0xffffffffu;
    const uint32_t pb = __shfl_up_sync(kFull, bk, 1);
    const bool head = lane == 0 || bk != pb;
    const unsigned heads = __ballot_sync(kFull, head);
    const unsigned upto = (2u << lane) - 1u;           // lanes 0 .. lane
    const int h = 31 - __clz(heads & upto);            // head of this lane's run
    const unsigned after = heads & ~upto;
    const int next = after ? __ffs(after) - 1 : kWarp; // head of the next run
    uint32_t base = 0;
    if (head && valid) base = atomicAdd(hist + b, (uint32_t)(next - lane));
    base = __shfl_sync(kFull, base, h);
    return base + (uint32_t)(lane - h);
}

// The level-1 partition of one round's <position p[j], length L[j]> pairs
// (entry j of each thread, at round index j * kPartThreads + thread, when
// that index is below cnt), as k_part1 does it for its rank-order pairs,
// for the rank-window front end: counted per super-bucket in shared memory
// (one atomic per run of lanes with the same super-bucket, run_slot: the
// rank-window pairs come in such runs), room reserved with one global
// atomic per touched super-bucket (cursors one cache line apart), staged in
// bucket order and written out as <position mod 2^20, min(L, 4095)>.  A length of 4095 or
// more is stored in lbig (field 4095); the length of the last position of
// every bucket goes to halo (the next bucket's predecessor).  Returns 1
// after an input error (a position out of range, or more than 2^20 of them
// in a super-bucket: the positions are not a permutation).
__device__ __forceinline__ unsigned level1_scatter(const PartSmem& P, int nb, const Scratch& s, int32_t n,
                                                   const uint32_t (&p)[kPartPer], const int32_t (&L)[kPartPer],
                                                   int cnt) {
    unsigned bad = 0;
    uint32_t ent[kPartPer], key[kPartPer];          // key: bucket << 16 | slot, or ~0u
#pragma unroll
    for (int j = 0; j < kPartPer; ++j) {
        const bool in = j * kPartThreads + (int)threadIdx.x < cnt;
        const uint32_t pj = p[j];
        const bool ok = in && pj < (uint32_t)n;
        if (in && !ok) bad = 1;
        uint32_t b1 = 0;
        if (ok) {
            const int32_t Lj = L[j];
            uint32_t field = (uint32_t)Lj;
            if (field >= kEsc12) { field = kEsc12; s.lbig[pj] = Lj; }
            if ((pj & (kBucket - 1)) == kBucket - 1) s.halo[(pj >> kBucketLog) + 1] = Lj;
            b1 = pj >> kSuperLog;
            ent[j] = ((pj & (kSuper - 1)) << 12) | field;
        }
        const uint32_t slot = run_slot(P.hist, b1, ok);     // the pairs come in runs of one super-bucket
        key[j] = ok ? ((b1 << 16) | slot) : 0xffffffffu;
    }
    __syncthreads();
    const bool wscan = nb <= 8 * kWarp;
    if (wscan) part_scan_w<8>(P, nb);
    else part_reserve(P, nb, s.cursor1);
    __syncthreads();
    if (wscan) {
        for (int b = threadIdx.x; b < nb; b += kPartThreads) {
            const uint32_t c = P.loff[b + 1] - P.loff[b];
            if (c) P.base[b] = atomicAdd(s.cursor1 + (size_t)b * kCursorStride, c);
        }
    }
#pragma unroll
    for (int j = 0; j < kPartPer; ++j) {
        if (key[j] == 0xffffffffu) continue;
        const uint32_t b1 = key[j] >> 16;
        const uint32_t o = P.loff[b1] + (key[j] & 0xffffu);
        P.stage[o] = ent[j];
        P.sbk[o] = (uint16_t)b1;
    }
    __syncthreads();
    const uint32_t total = P.loff[nb];
    for (uint32_t i = threadIdx.x; i < total; i += kPartThreads) {
        const uint32_t b1 = P.sbk[i];
        const uint32_t idx = P.base[b1] + (i - P.loff[b1]);
        if (idx < (uint32_t)kSuper) s.ent1[((size_t)b1 << kSuperLog) + idx] = P.stage[i];
        else bad = 1;
    }
    return bad;
}

// Level 1: Lemma 1 in rank order.  Each CTA takes kPartRound consecutive
// ranks r, forms <sa[r], max(lcp[r], lcp[r+1])> and partitions these pairs
// into super-buckets of 2^20 positions (level1_scatter).
template <bool kBatch>
__global__ void __launch_bounds__(kPartThreads, kPartBlocks)
k_part1(const int32_t* __restrict__ sa, const int32_t* __restrict__ lcp, int32_t n, Scratch s, Segs segs, int tma) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned long long load_bar, load_bar2;
    const int nb = (int)s.nsupers;                    // <= 2048
    const PartSmem P = part_smem(smem_raw, nb);
    const long long r0 = (long long)blockIdx.x * kPartRound;
    // Full rounds (16-byte-aligned inputs) arrive by two bulk copies issued
    // before anything else: of a single string, every round but the last.
    // Of a batch, every full round's sa slice (flattened like the positions)
    // at once, on its own barrier, and then the lcp slice of a round that
    // lies inside one string, copied from the 16-byte boundary at or below
    // its first entry (shift entries earlier).  Other rounds load per thread.
    const int32_t* Ssa = reinterpret_cast<const int32_t*>(smem_raw + part_load_offset(nb));
    const int32_t* Slcp = Ssa + kPartRound;
    __shared__ int bulk_s, shift_s, sab_s;
    __shared__ long long bbase_s, bnj_s;          // batch round: its string's offset and length
    if (threadIdx.x == 0) {
        int bk = 0, shift = 0, sab = 0;
        long long lsrc = r0, cnt = kPartRound + 4;    // lcp entries copied
        if constexpr (!kBatch) {
            bk = tma && r0 + kPartRound + 4 <= (long long)n + 1;
            if (bk) {
                mbar_init(&load_bar, 1);
                mbar_fence_init();
                mbar_arrive_tx(&load_bar, (unsigned)(kPartRound * 4 + cnt * 4));
                bulk_g2s(const_cast<int32_t*>(Ssa), sa + r0, kPartRound * 4, &load_bar);
                bulk_g2s(const_cast<int32_t*>(Slcp), lcp + lsrc, (unsigned)(cnt * 4), &load_bar);
            }
        } else if (tma && r0 + kPartRound <= (long long)n) {
            sab = 1;
            mbar_init(&load_bar, 1);
            mbar_init(&load_bar2, 1);
            mbar_fence_init();
            mbar_arrive_tx(&load_bar, (unsigned)(kPartRound * 4));
            bulk_g2s(const_cast<int32_t*>(Ssa), sa + r0, kPartRound * 4, &load_bar);
            if (r0 + kPartRound < (long long)n) {
                // the round lies inside one string when the string holding
                // its first position also holds the next round's first
                // position (two independent loads; the string's offsets come
                // from warp 1)
                const long long t0 = r0 / kTile;
                const long long j = s.tile_seg[t0], jn = s.tile_seg[t0 + kPartRound / kTile];
                const long long l0 = r0 + j;          // the round's first lcp entry
                lsrc = l0 & ~3LL;
                cnt = (l0 + kPartRound + 1 - lsrc + 3) & ~3LL;
                if (j >= 0 && j < segs.num && jn == j && lsrc >= 0 && lsrc + cnt <= (long long)n + segs.num) {
                    bk = 1;
                    shift = (int)(l0 - lsrc);
                    mbar_arrive_tx(&load_bar2, (unsigned)(cnt * 4));
                    bulk_g2s(const_cast<int32_t*>(Slcp), lcp + lsrc, (unsigned)(cnt * 4), &load_bar2);
                }
            }
        }
        bulk_s = bk;
        shift_s = shift;
        sab_s = sab;
    }
    if constexpr (kBatch) {
        // the string of a round that may arrive by bulk copies: its offset
        // and length, zero when the offset table contradicts the round (every
        // entry then fails its checks below)
        if (threadIdx.x == kWarp && tma && r0 + kPartRound < (long long)n) {
            const long long j = s.tile_seg[r0 / kTile];
            long long b0 = 0, b1 = 0;
            if (j >= 0 && j < segs.num) { b0 = __ldg(segs.off + j); b1 = __ldg(segs.off + j + 1); }
            const bool ok = b0 >= 0 && b0 <= r0 && b1 > r0 + kPartRound && b1 <= (long long)n;
            bbase_s = ok ? b0 : 0;
            bnj_s = ok ? b1 - b0 : 0;
        }
    }
    for (int b = threadIdx.x; b < nb; b += kPartThreads) P.hist[b] = 0;
    // a round across strings copies no lcp slice: its string offsets use
    // the lcp part of the bulk-copy area (read only before the stage area is
    // written)
    static_assert((kSegCap + 1) * 8 <= kPartLcpCap * 4, "string offsets must fit the lcp copy area");
    long long* seg_sh = reinterpret_cast<long long*>(const_cast<int32_t*>(Slcp));
    SegView sv{};
    __syncthreads();
    const bool bulk = bulk_s != 0;
    const int shift = shift_s;
    // a round across string boundaries looks its strings up per entry
    if constexpr (kBatch) {
        if (!bulk) sv.stage(segs, s, r0, (r0 + kPartRound < n) ? r0 + kPartRound : n, seg_sh);
    }
    // bulk round of a batch: its string's offset and length (the string
    // goes on past the round, so only its first rank can lie in the round)
    uint32_t bbase = 0, bnj = 0;
    if constexpr (kBatch) {
        if (bulk) { bbase = (uint32_t)bbase_s; bnj = (uint32_t)bnj_s; }
    }
    unsigned bad = 0;
    if (!kBatch && blockIdx.x == 0 && threadIdx.x == 0 && (__ldg(lcp) != 0 || __ldg(lcp + n) != 0)) bad = 1;
    // In a batch, flattened rank index r of string j is local rank
    // r - off[j]; its suffix starts at off[j] + sa[r] and its lcp pair is at
    // lcp[off[j] + j + (r - off[j]) ..].  Positions are flattened.
    uint32_t p[kPartPer];
    int32_t L[kPartPer];
    long long hint = kBatch ? sv.j0 : 0;
    const bool sab = kBatch ? sab_s != 0 : bulk;      // sa of the round in shared memory
    bool landed = true;                               // false: the copies never landed (reported; load nothing)
    if (sab && !mbar_wait(&load_bar, 0)) landed = false;
    if (kBatch && bulk && landed && !mbar_wait(&load_bar2, 0)) landed = false;
    if (!landed && threadIdx.x == 0) report(s, kErrTimeout);
#pragma unroll
    for (int j = 0; j < kPartPer; ++j) {
        const long long r = r0 + (long long)j * kPartThreads + threadIdx.x;
        if (bulk) {
            const int x = j * kPartThreads + (int)threadIdx.x;
            if (!landed) { p[j] = 0xffffffffu; L[j] = 0; continue; }
            uint32_t pl = (uint32_t)Ssa[x];
            const int32_t a = Slcp[shift + x], c = Slcp[shift + x + 1];
            int32_t Lj = a > c ? a : c;
            if constexpr (kBatch) {
                if (x == 0 && (long long)bbase == r0 && bnj != 0 && a != 0) bad = 1;   // lcp sentinel
                if (pl >= bnj) { bad = 1; pl = 0xffffffffu; }
                else if (Lj < 0 || (uint32_t)Lj > bnj - pl) { bad = 1; Lj = 0; }
                p[j] = (pl == 0xffffffffu) ? pl : bbase + pl;
            } else {
                if (pl >= (uint32_t)n) { bad = 1; pl = 0xffffffffu; }
                else if (Lj < 0 || (long long)Lj > (long long)n - pl) { bad = 1; Lj = 0; }
                p[j] = pl;
            }
            L[j] = Lj;
        } else if (r < n) {
            if (sab && !landed) { p[j] = 0xffffffffu; L[j] = 0; continue; }
            uint32_t pl = sab ? (uint32_t)Ssa[j * kPartThreads + (int)threadIdx.x] : (uint32_t)__ldcs(sa + r);
            long long base = 0, nj = n, lidx = r;
            if constexpr (kBatch) {
                hint = sv.find(r, hint);
                base = sv.at(hint);
                nj = sv.at(hint + 1) - base;
                lidx = r + hint;
                if (base < 0 || nj < 1 || base + nj > n || r < base) {     // bad offset table
                    bad = 1; p[j] = 0xffffffffu; L[j] = 0; continue;
                }
            }
            const int32_t a = __ldcs(lcp + lidx), c = __ldg(lcp + lidx + 1);
            if (kBatch && ((r == base && a != 0) || (r == base + nj - 1 && c != 0))) bad = 1;   // lcp sentinels
            int32_t Lj = a > c ? a : c;
            if (pl >= (uint32_t)nj) { bad = 1; pl = 0xffffffffu; }
            else if (Lj < 0 || (long long)Lj > nj - pl) { bad = 1; Lj = 0; }
            p[j] = (pl == 0xffffffffu) ? pl : (uint32_t)(base + pl);
            L[j] = Lj;
        } else {
            p[j] = 0xffffffffu; L[j] = 0;
        }
    }
    // the steps of level1_scatter, with one shared atomic per entry (pairs in
    // rank order come in no runs), kept inline here (as a call they cost this
    // kernel 3 %: more register spills)
    uint32_t ent[kPartPer], key[kPartPer];          // key: bucket << 16 | slot, or ~0u
#pragma unroll
    for (int j = 0; j < kPartPer; ++j) {
        const long long r = r0 + (long long)j * kPartThreads + threadIdx.x;
        key[j] = 0xffffffffu;
        if (r >= n) continue;
        const uint32_t pj = p[j];
        if (pj >= (uint32_t)n) { bad = 1; continue; }
        const int32_t Lj = L[j];
        uint32_t field = (uint32_t)Lj;
        if (field >= kEsc12) { field = kEsc12; s.lbig[pj] = Lj; }
        if ((pj & (kBucket - 1)) == kBucket - 1) s.halo[(pj >> kBucketLog) + 1] = Lj;
        const uint32_t b1 = pj >> kSuperLog;
        ent[j] = ((pj & (kSuper - 1)) << 12) | field;
        key[j] = (b1 << 16) | atomicAdd(&P.hist[b1], 1u);
    }
    __syncthreads();
    const bool wscan = nb <= 8 * kWarp;
    if (wscan) part_scan_w<8>(P, nb);
    else part_reserve(P, nb, s.cursor1);
    __syncthreads();
    if (wscan) {
        for (int b = threadIdx.x; b < nb; b += kPartThreads) {
            const uint32_t c = P.loff[b + 1] - P.loff[b];
            if (c) P.base[b] = atomicAdd(s.cursor1 + (size_t)b * kCursorStride, c);
        }
    }
#pragma unroll
    for (int j = 0; j < kPartPer; ++j) {
        if (key[j] == 0xffffffffu) continue;
        const uint32_t b1 = key[j] >> 16;
        const uint32_t o = P.loff[b1] + (key[j] & 0xffffu);
        P.stage[o] = ent[j];
        P.sbk[o] = (uint16_t)b1;
    }
    __syncthreads();
    const uint32_t total = P.loff[nb];
    for (uint32_t i = threadIdx.x; i < total; i += kPartThreads) {
        const uint32_t b1 = P.sbk[i];
        const uint32_t idx = P.base[b1] + (i - P.loff[b1]);
        if (idx < (uint32_t)kSuper) s.ent1[((size_t)b1 << kSuperLog) + idx] = P.stage[i];
        else bad = 1;                                   // more than 2^20 positions: sa is not a permutation
    }
    if (bad) report(s, kErrInput);
}

// Rank-window front end (rank without sa, one string of 2^24 positions or
// more).  Lemma 1 in text order, max(lcp[rank[i]], lcp[rank[i] + 1]), makes
// k_gather_llr read one random lcp sector per position from HBM.  Here
// k_rank_win first partitions the pairs <rank[i], i> by rank into windows
// of 2^22 ranks (8-byte entries rank << 32 | i, in the compact LLR region,
// which is idle until k_bucket_llr).  k_part1_win then takes kPartRound
// pairs of one window per CTA, gathers their two lcp words from the
// window's 16 MB slice of lcp (CTAs run in window order, so the slice stays
// in L2 while its window is processed) and partitions <i, L_i> into the
// level-1 super-buckets like k_part1.  k_part2 and k_bucket_llr follow
// unchanged.
__host__ __device__ inline size_t win_stage_offset(int nw) { return ((size_t)(2 * nw + 1) * 4 + 15) & ~(size_t)15; }
size_t rank_win_smem_bytes(int nw) { return win_stage_offset(nw) + (size_t)kPartRound * 10; }
size_t part_scatter_smem_bytes(int nb) { return (size_t)(2 * nb + 1) * 4 + (size_t)kPartRound * 6; }

__global__ void __launch_bounds__(kPartThreads, kPartBlocks)
k_rank_win(const int32_t* __restrict__ rank, int32_t n, Scratch s, int tma) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned long long load_bar;
    const int nw = (int)s.nwins;                      // <= kMaxWins
    const PartSmem P = part_smem(smem_raw, nw);       // counters; the stage area is the 8-byte one below
    unsigned long long* stage = reinterpret_cast<unsigned long long*>(smem_raw + win_stage_offset(nw));
    uint16_t* sbk = reinterpret_cast<uint16_t*>(stage + kPartRound);
    // a full round's ranks arrive by one bulk copy into the stage area,
    // which is written only after every thread has read its ranks
    const int32_t* Srk = reinterpret_cast<const int32_t*>(stage);
    const long long i0 = (long long)blockIdx.x * kPartRound;
    const bool bulk = tma && i0 + kPartRound <= (long long)n;
    if (threadIdx.x == 0 && bulk) {
        mbar_init(&load_bar, 1);
        mbar_fence_init();
        mbar_arrive_tx(&load_bar, (unsigned)(kPartRound * 4));
        bulk_g2s(const_cast<int32_t*>(Srk), rank + i0, kPartRound * 4, &load_bar);
    }
    for (int b = threadIdx.x; b < nw; b += kPartThreads) P.hist[b] = 0;
    __syncthreads();
    unsigned bad = 0;
    bool landed = true;                               // false: the copy never landed (reported; load nothing)
    if (bulk && !mbar_wait(&load_bar, 0)) {
        landed = false;
        if (threadIdx.x == 0) report(s, kErrTimeout);
    }
    uint32_t rk[kPartPer], key[kPartPer];             // key: window << 16 | slot, or ~0u
#pragma unroll
    for (int j = 0; j < kPartPer; ++j) {
        const long long i = i0 + (long long)j * kPartThreads + threadIdx.x;
        key[j] = 0xffffffffu;
        rk[j] = 0;
        if (i >= n || !landed) continue;
        const uint32_t r = bulk ? (uint32_t)Srk[j * kPartThreads + threadIdx.x] : (uint32_t)__ldcs(rank + i);
        if (r >= (uint32_t)n) { bad = 1; continue; }
        const uint32_t w = r >> kWinLog;
        rk[j] = r;
        key[j] = (w << 16) | atomicAdd(&P.hist[w], 1u);
    }
    __syncthreads();
    if (nw <= 2 * kWarp) part_reserve_w<2>(P, nw, s.cursor_w);
    else part_reserve(P, nw, s.cursor_w);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kPartPer; ++j) {
        if (key[j] == 0xffffffffu) continue;
        const uint32_t w = key[j] >> 16;
        const uint32_t o = P.loff[w] + (key[j] & 0xffffu);
        stage[o] = ((unsigned long long)rk[j] << 32) | (uint32_t)(i0 + j * kPartThreads + threadIdx.x);
        sbk[o] = (uint16_t)w;
    }
    __syncthreads();
    const uint32_t total = P.loff[nw];
    for (uint32_t t = threadIdx.x; t < total; t += kPartThreads) {
        const uint32_t w = sbk[t];
        const uint32_t slot = P.base[w] + (t - P.loff[w]);
        const long long idx = ((long long)w << kWinLog) + slot;
        if (slot < (1u << kWinLog) && idx < n) s.went[idx] = stage[t];
        else bad = 1;                                 // a window overflows: rank is not a permutation
    }
    if (bad) report(s, kErrInput);
}

__global__ void __launch_bounds__(kPartThreads, kPartBlocks)
k_part1_win(const int32_t* __restrict__ lcp, int32_t n, Scratch s) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nb = (int)s.nsupers;
    const PartSmem P = part_smem(smem_raw, nb);
    constexpr int kRoundsPerWin = (1 << kWinLog) / kPartRound;
    const long long w = blockIdx.x / kRoundsPerWin;
    const int q = blockIdx.x % kRoundsPerWin;
    const uint32_t fill = __ldcg(s.cursor_w + (size_t)w * kCursorStride);
    const long long wsize = ((long long)n - (w << kWinLog) < (1LL << kWinLog)) ? (long long)n - (w << kWinLog)
                                                                                : (1LL << kWinLog);
    for (int b = threadIdx.x; b < nb; b += kPartThreads) P.hist[b] = 0;
    unsigned bad = 0;
    if (q == 0 && threadIdx.x == 0) {
        if ((long long)fill != wsize) bad = 1;                  // rank is not a permutation
        if (w == 0 && (__ldg(lcp) != 0 || __ldg(lcp + n) != 0)) bad = 1;   // lcp sentinels
    }
    __syncthreads();
    const long long lim = (long long)fill < wsize ? (long long)fill : wsize;
    const long long e0 = (long long)q * kPartRound;
    if (e0 >= lim) {                                  // uniform over the CTA
        if (bad) report(s, kErrInput);
        return;
    }
    const int cnt = (int)(lim - e0 < kPartRound ? lim - e0 : kPartRound);
    const unsigned long long* src = s.went + (w << kWinLog) + e0;
    uint32_t p[kPartPer];
    int32_t L[kPartPer];
#pragma unroll
    for (int j = 0; j < kPartPer; ++j) {              // all pairs in flight first: p = i, L = rank
        const int x = j * kPartThreads + (int)threadIdx.x;
        const unsigned long long e = (x < cnt) ? __ldcs(src + x) : 0xffffffffull;
        p[j] = (uint32_t)e;
        L[j] = (int32_t)(e >> 32);
    }
#pragma unroll
    for (int j = 0; j < kPartPer; ++j) {
        const int x = j * kPartThreads + (int)threadIdx.x;
        if (x >= cnt) continue;
        const uint32_t i = p[j], r = (uint32_t)L[j];
        if (i >= (uint32_t)n || r >= (uint32_t)n) { bad = 1; p[j] = 0xffffffffu; L[j] = 0; continue; }
        const int32_t a = __ldg(lcp + r), c = __ldg(lcp + r + 1);
        int32_t Lj = a > c ? a : c;
        if (Lj < 0 || (long long)Lj > (long long)n - i) { bad = 1; Lj = 0; }
        L[j] = Lj;
    }
    bad |= level1_scatter(P, nb, s, n, p, L, cnt);
    if (bad) report(s, kErrInput);
}

// Level 2: each CTA takes kPartRound entries of one super-bucket and splits
// them into its kSubPerSuper buckets, entries <position mod 2^15, field>
// (field = L, or kEsc17 when L is in lbig), the same way as level 1.
// kRuns: slots by run_slot, for level-1 entries that come clustered by
// bucket (those of the rank-window front end).
template <bool kRuns>
__global__ void __launch_bounds__(kPartThreads, kPartBlocks)
k_part2(int32_t n, Scratch s) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const PartSmem P = part_smem(smem_raw, kSubPerSuper);
    constexpr int kChunksPerSuper = kSuper / kPartRound;
    const long long b1 = blockIdx.x / kChunksPerSuper;
    const int q = blockIdx.x % kChunksPerSuper;
    const uint32_t fill = __ldcg(s.cursor1 + (size_t)b1 * kCursorStride);
    if (threadIdx.x < kSubPerSuper) P.hist[threadIdx.x] = 0;
    if (q == 0 && threadIdx.x == 0) {
        const long long want = ((long long)n - b1 * kSuper < kSuper) ? (long long)n - b1 * kSuper : kSuper;
        if ((long long)fill != want) report(s, kErrInput);
    }
    __syncthreads();
    const uint32_t i0 = (uint32_t)q * kPartRound;
    if (i0 >= fill) return;                             // uniform over the CTA
    const uint32_t* src = s.ent1 + ((size_t)b1 << kSuperLog);
    uint32_t ent[kPartPer], key[kPartPer];
#pragma unroll
    for (int j = 0; j < kPartPer; ++j) {
        const uint32_t i = i0 + j * kPartThreads + threadIdx.x;
        ent[j] = (i < fill) ? __ldcs(src + i) : 0xffffffffu;
    }
#pragma unroll
    for (int j = 0; j < kPartPer; ++j) {
        const uint32_t i = i0 + j * kPartThreads + threadIdx.x;
        if constexpr (kRuns) {
            const bool ok = i < fill;
            uint32_t b2 = 0;
            if (ok) {
                const uint32_t low20 = ent[j] >> 12, f12 = ent[j] & kEsc12;
                b2 = low20 >> kBucketLog;
                ent[j] = ((low20 & (kBucket - 1)) << 17) | (f12 == kEsc12 ? kEsc17 : f12);
            }
            const uint32_t slot = run_slot(P.hist, b2, ok);
            key[j] = ok ? ((b2 << 16) | slot) : 0xffffffffu;
        } else {
            key[j] = 0xffffffffu;
            if (i >= fill) continue;
            const uint32_t low20 = ent[j] >> 12, f12 = ent[j] & kEsc12;
            const uint32_t b2 = low20 >> kBucketLog;
            ent[j] = ((low20 & (kBucket - 1)) << 17) | (f12 == kEsc12 ? kEsc17 : f12);
            key[j] = (b2 << 16) | atomicAdd(&P.hist[b2], 1u);
        }
    }
    __syncthreads();
    const long long bb = b1 * kSubPerSuper;
    const int nsub = (int)((s.nbuckets - bb < kSubPerSuper) ? s.nbuckets - bb : kSubPerSuper);
    part_reserve_w<1>(P, nsub, s.cursor2 + (size_t)bb * kCursorStride);
    __syncthreads();
    unsigned bad = 0;
#pragma unroll
    for (int j = 0; j < kPartPer; ++j) {
        if (key[j] == 0xffffffffu) continue;
        const uint32_t b2 = key[j] >> 16;
        if ((int)b2 >= nsub) { bad = 1; continue; }
        const uint32_t o = P.loff[b2] + (key[j] & 0xffffu);
        P.stage[o] = ent[j];
        P.sbk[o] = (uint16_t)b2;
    }
    __syncthreads();
    const uint32_t total = P.loff[nsub];
    for (uint32_t i = threadIdx.x; i < total; i += kPartThreads) {
        const uint32_t b2 = P.sbk[i];
        const uint32_t idx = P.base[b2] + (i - P.loff[b2]);
        if (idx < (uint32_t)kBucket) s.ent2[((size_t)(bb + b2) << kBucketLog) + idx] = P.stage[i];
        else bad = 1;
    }
    if (bad) report(s, kErrInput);
}

// One bucket of kBucket positions per CTA: lengths scattered into shared
// memory by position, usefulness flags (K1), compaction (K2) and the
// bucket's place in LLRc by look-back (K3).  Each warp owns a contiguous
// range of 64 runs of 32 positions, so L_{k-1} comes from the lane to the
// left (or the previous run's last lane).
constexpr uint16_t kUnset = 0xfffeu;                  // no length field takes this value
constexpr uint32_t kUnset2 = 0xfffefffeu;
__global__ void __launch_bounds__(kBucketThreads)
k_bucket_llr(int32_t n, Scratch s) {
    constexpr int kChunks = kBucket / kWarp;                 // 1024 runs of 32 positions
    constexpr int kWarps = kBucketThreads / kWarp;           // 16
    constexpr int kRunsPerWarp = kChunks / kWarps;           // 64
    constexpr int kTilesPerBucket = kBucket / kTile;         // 16
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint16_t* sL = reinterpret_cast<uint16_t*>(smem_raw);                        // kBucket lengths
    unsigned* cmask = reinterpret_cast<unsigned*>(smem_raw + kBucket * 2);       // kChunks flag masks
    int32_t* ccnt = reinterpret_cast<int32_t*>(cmask + kChunks);                 // kChunks run offsets
    __shared__ int32_t wsum[kWarps];
    __shared__ long long b_s, base_s;
    __shared__ int32_t total_s;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) b_s = atomicAdd(&s.tickets[1], 1u);
    {
        // every length starts as kUnset: a position left unset after the
        // scatter means sa gave another one twice
        const uint4 u = make_uint4(kUnset2, kUnset2, kUnset2, kUnset2);
        uint4* d = reinterpret_cast<uint4*>(sL);
        for (int i = tid; i < kBucket / 8; i += kBucketThreads) d[i] = u;
    }
    __syncthreads();
    const long long b = b_s;
    const long long k0 = b * kBucket;
    const int cnt = (int)(((long long)n - k0 < kBucket) ? (long long)n - k0 : kBucket);

    // scatter the bucket's lengths into shared memory by position
    const uint32_t* ent = s.ent2 + ((size_t)b << kBucketLog);
    const uint32_t fill = __ldcg(s.cursor2 + (size_t)b * kCursorStride);
    unsigned bad = fill != (uint32_t)cnt;
    const int nent = (int)(fill < (uint32_t)cnt ? fill : (uint32_t)cnt);
    // eight loads in flight per thread before any of them is used
    constexpr int kUnroll = 8;
    for (int i0 = 0; i0 < nent; i0 += kBucketThreads * kUnroll) {
        uint32_t e[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int i = i0 + u * kBucketThreads + tid;
            e[u] = (i < nent) ? __ldcs(ent + i) : 0u;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            if (i0 + u * kBucketThreads + tid >= nent) continue;
            const uint32_t low = e[u] >> 17, f = e[u] & kEsc17;
            if (low < (uint32_t)cnt) sL[low] = (uint16_t)(f == kEsc17 ? 0xffffu : f);
            else bad = 1;
        }
    }
    __syncthreads();
    auto len_at = [&](int x) -> int32_t {                    // L of position k0 + x, 0 <= x < cnt
        const uint32_t f = sL[x];
        return f == 0xffffu ? __ldcg(s.lbig + k0 + x) : (int32_t)f;
    };

    // K1 flags, one ballot per run, runs of a warp contiguous
    int32_t left = 0;                                        // L of the position before the run
    {
        const int x0 = warp * kRunsPerWarp * kWarp;
        left = (x0 == 0) ? ((k0 > 0) ? __ldcg(s.halo + b) : 0) : (x0 - 1 < cnt ? len_at(x0 - 1) : 0);
    }
    for (int r = 0; r < kRunsPerWarp; ++r) {
        const int c = warp * kRunsPerWarp + r;
        const int x = c * kWarp + lane;
        if (x < cnt && sL[x] == kUnset) bad = 1;
        const int32_t L = (x < cnt) ? len_at(x) : 0;
        int32_t prev = __shfl_up_sync(kFull, L, 1);
        if (lane == 0) prev = left;
        left = __shfl_sync(kFull, L, kWarp - 1);
        const unsigned m = __ballot_sync(kFull, x < cnt && L > 0 && L >= prev);
        if (lane == 0) { cmask[c] = m; ccnt[c] = __popc(m); }
    }
    if (bad) report(s, kErrInput);
    __syncthreads();
    // exclusive scan of the 1024 run counts: 2 per thread
    {
        const int a0 = ccnt[2 * tid], a1 = ccnt[2 * tid + 1];
        const int incl = warp_incl_scan(a0 + a1);
        if (lane == kWarp - 1) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int v = (lane < kWarps) ? wsum[lane] : 0;
            const int wi = warp_incl_scan(v);
            if (lane < kWarps) wsum[lane] = wi - v;
            if (lane == kWarp - 1) total_s = wi;
        }
        __syncthreads();
        const int ex = wsum[warp] + incl - a0 - a1;
        ccnt[2 * tid] = ex;
        ccnt[2 * tid + 1] = ex + a0;
    }
    __syncthreads();
    if (warp == 0) {
        const long long ex = lookback_exclusive(s.status_b, b, total_s, s.err, s.qerr, s.spin_limit);
        if (lane == 0) base_s = ex;
    }
    __syncthreads();
    const long long base = base_s;
    // first LLRc entry of each tile and of each kSeg-position segment of the bucket
    if (tid < kTilesPerBucket) {
        const long long tile = b * kTilesPerBucket + tid;
        if (tile < s.ntiles) s.tile_cbase[tile] = (int32_t)(base + ccnt[tid * (kTile / kWarp)]);
        if (tile == s.ntiles - 1) s.tile_cbase[s.ntiles] = (int32_t)(base + total_s);
    }
    for (int j = tid; j < kBucket / kSeg; j += kBucketThreads) {
        const long long sg = b * (kBucket / kSeg) + j;
        if (sg < s.nsegs) s.seg_cbase[sg] = (int32_t)(base + ccnt[j * (kSeg / kWarp)]);
        if (sg == s.nsegs - 1) s.seg_cbase[s.nsegs] = (int32_t)(base + total_s);
    }
    // K3: write the kept LLR's
    for (int r = 0; r < kRunsPerWarp; ++r) {
        const int c = warp * kRunsPerWarp + r;
        const unsigned m = cmask[c];
        if ((m >> lane) & 1u) {
            const int x = c * kWarp + lane;
            const long long o = base + ccnt[c] + __popc(m & ((1u << lane) - 1u));
            s.cstart[o] = (int32_t)(k0 + x);
            s.cend[o] = (int32_t)(k0 + x + len_at(x) - 1);
        }
    }
}

size_t bucket_smem_bytes() { return (size_t)kBucket * 2 + (size_t)(kBucket / kWarp) * 8; }

void launch_partition(const int32_t* sa, const int32_t* lcp, int32_t n, const Scratch& s, const Segs& segs,
                      cudaStream_t stream) {
    const unsigned g1 = (unsigned)(((long long)n + kPartRound - 1) / kPartRound);
    // bulk copies need 16-byte-aligned sources
    const int tma = (((uintptr_t)sa | (uintptr_t)lcp) & 15u) == 0 ? 1 : 0;
    if (segs.num > 0)
        k_part1<true><<<g1, kPartThreads, part_smem_bytes((int)s.nsupers), stream>>>(sa, lcp, n, s, segs, tma);
    else
        k_part1<false><<<g1, kPartThreads, part_smem_bytes((int)s.nsupers), stream>>>(sa, lcp, n, s, segs, tma);
    const unsigned g2 = (unsigned)(s.nsupers * (kSuper / kPartRound));
    k_part2<false><<<g2, kPartThreads, part2_smem_bytes(), stream>>>(n, s);
}

void launch_rank_window_front(const int32_t* rank, const int32_t* lcp, int32_t n, const Scratch& s,
                              cudaStream_t stream) {
    const unsigned g0 = (unsigned)(((long long)n + kPartRound - 1) / kPartRound);
    const int tma = ((uintptr_t)rank & 15u) == 0 ? 1 : 0;   // bulk copies need a 16-byte-aligned source
    k_rank_win<<<g0, kPartThreads, rank_win_smem_bytes((int)s.nwins), stream>>>(rank, n, s, tma);
    const unsigned g1 = (unsigned)(s.nwins * ((1 << kWinLog) / kPartRound));
    k_part1_win<<<g1, kPartThreads, part_scatter_smem_bytes((int)s.nsupers), stream>>>(lcp, n, s);
    const unsigned g2 = (unsigned)(s.nsupers * (kSuper / kPartRound));
    k_part2<true><<<g2, kPartThreads, part2_smem_bytes(), stream>>>(n, s);
}

void launch_bucket_front(int32_t n, const Scratch& s, cudaStream_t stream) {
    k_bucket_llr<<<(unsigned)s.nbuckets, kBucketThreads, bucket_smem_bytes(), stream>>>(n, s);
}

cudaError_t configure_front() {
    cudaError_t e = cudaFuncSetAttribute(k_bucket_llr, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bucket_smem_bytes());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_part1<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)part_smem_bytes(2048));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_part1<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)part_smem_bytes(2048));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_rank_win, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rank_win_smem_bytes(kMaxWins));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_part1_win, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)part_scatter_smem_bytes(2048));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_part2<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)part2_smem_bytes());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_part2<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)part2_smem_bytes());
}

}  // namespace lr
