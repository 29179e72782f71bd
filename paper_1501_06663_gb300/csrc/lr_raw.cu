// The raw-LLR variant of the longest-repeat query and the walk statistics of
// Table 2 (Tian and Xu, arXiv 1501.06663).
//
//  * k_llr_raw: Lemma 1 in text order, the raw LLR array LLRr[i] =
//    max(lcp[rank[i]], lcp[rank[i] + 1]) (the paper's kernel K_LLRr).
//  * k_rawwalk: Algorithms 1 and 3 without compaction: every position walks
//    left over LLRr while the LLR it meets still covers it, keeping the
//    longest (the leftmost on ties) and the number of ties; for the all-LR
//    query the tie counts are scanned into CSR offsets (block scan plus a
//    decoupled look-back over tiles) and a second walk writes every start of
//    the longest length, ascending.  The 32 lanes of a warp own 32
//    consecutive positions, so every step of the walk is one coalesced load.
//    Its cost is the sum of the walk lengths, about alpha per position.
//  * k_walk_stats: per position, alpha_k (raw LLR's covering k) and beta_k
//    (compact LLR's covering k) by binary search over the monotone ends and
//    starts, with their sums, minima and maxima.
#include <cuda_runtime.h>
#include <cstdint>
#include "lr_device.cuh"
#include "lr_internal.h"

namespace lr {

namespace {

constexpr int kRawTile = 2048;
constexpr int kRawThreads = 256;
constexpr int kRawWarps = kRawThreads / kWarp;
constexpr int kRawChunks = kRawTile / kWarp;           // runs of 32 positions per tile
constexpr int kRawPerWarp = kRawChunks / kRawWarps;

__device__ __forceinline__ void report_input(const Scratch& s) {
    atomicOr(s.err, kErrInput);
    atomicOr(s.qerr, kErrInput);
}

__global__ void __launch_bounds__(256) k_llr_raw(const int32_t* __restrict__ rank, const int32_t* __restrict__ lcp,
                                                 int32_t n, Scratch s, int32_t* __restrict__ llrr) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (i == 0 && (__ldg(lcp) != 0 || __ldg(lcp + n) != 0)) bad = true;
    if (i < n) {
        uint32_t r = (uint32_t)__ldcs(rank + i);
        int32_t L = 0;
        if (r >= (uint32_t)n) {
            bad = true;
        } else {
            const int32_t a = __ldg(lcp + r), b = __ldg(lcp + r + 1);
            L = a > b ? a : b;
            if (L < 0 || (long long)L > (long long)n - i) { bad = true; L = 0; }
        }
        llrr[i] = L;
    }
    if (bad) report_input(s);
}

// Exclusive scan of the kRawChunks ints of a[] by one warp; returns the total.
__device__ __forceinline__ int scan_runs(int32_t* a) {
    constexpr int kPer = kRawChunks / kWarp;
    const int lane = lane_id();
    int c[kPer], sum = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) { c[q] = a[kPer * lane + q]; sum += c[q]; }
    const int incl = warp_incl_scan(sum);
    int run = incl - sum;
#pragma unroll
    for (int q = 0; q < kPer; ++q) { a[kPer * lane + q] = run; run += c[q]; }
    return __shfl_sync(kFull, incl, kWarp - 1);
}

template <bool kAll>
__global__ void __launch_bounds__(kRawThreads) k_rawwalk(int32_t n, const int32_t* __restrict__ llrr, Scratch s,
                                                         int32_t* __restrict__ lr_len, int32_t* __restrict__ lr_start,
                                                         int64_t* __restrict__ offsets, int32_t* __restrict__ starts,
                                                         long long capacity) {
    __shared__ int32_t run_tot[kRawChunks];
    __shared__ long long tile_s, obase_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) tile_s = atomicAdd(&s.tickets[2], 1u);
    __syncthreads();
    const long long tile = tile_s;
    const long long k0 = tile * kRawTile;
    int32_t best[kRawPerWarp], left[kRawPerWarp], cnt[kRawPerWarp], pre[kRawPerWarp];
#pragma unroll
    for (int q = 0; q < kRawPerWarp; ++q) {
        const long long k = k0 + (long long)(q * kRawWarps + warp) * kWarp + lane;
        int32_t b = 0, lm = -1, ct = 0;
        if (k < n) {
            // Algorithm 1's walk: left from k until an LLR does not cover k
            for (long long i = k; i >= 0; --i) {
                const int32_t L = __ldg(llrr + i);
                if (i + L - 1 < k) break;
                if (L > b) { b = L; lm = (int32_t)i; ct = 1; }
                else if (L == b) { lm = (int32_t)i; ++ct; }
            }
        }
        best[q] = b; left[q] = lm; cnt[q] = ct;
    }
#pragma unroll
    for (int q = 0; q < kRawPerWarp; ++q) {
        const long long k = k0 + (long long)(q * kRawWarps + warp) * kWarp + lane;
        if (k < n) { __stcs(lr_len + k, best[q]); __stcs(lr_start + k, left[q]); }
    }
    if constexpr (kAll) {
#pragma unroll
        for (int q = 0; q < kRawPerWarp; ++q) {
            const int incl = warp_incl_scan(cnt[q]);
            pre[q] = incl - cnt[q];
            if (lane == kWarp - 1) run_tot[q * kRawWarps + warp] = incl;
        }
        __syncthreads();
        if (warp == 0) {
            const int tot = scan_runs(run_tot);
            const long long ex = lookback_exclusive(s.status_o, tile, tot, s.err, s.qerr, s.spin_limit);
            if (lane == 0) {
                obase_s = ex;
                if (k0 + kRawTile >= n) offsets[n] = ex + tot;
            }
        }
        __syncthreads();
        const long long obase = obase_s;
#pragma unroll
        for (int q = 0; q < kRawPerWarp; ++q) {
            const int c = q * kRawWarps + warp;
            const long long k = k0 + (long long)c * kWarp + lane;
            if (k >= n) continue;
            const long long o = obase + run_tot[c] + pre[q];
            __stcs(reinterpret_cast<long long*>(offsets) + k, o);
            if (cnt[q] == 0) continue;
            // Algorithm 3's second walk, from k down to the leftmost holder;
            // it meets the holders right to left, so the j-th one met goes
            // to slot cnt - 1 - j to list them ascending
            int j = 0;
            for (long long i = k; i >= left[q]; --i) {
                if (__ldg(llrr + i) == best[q]) {
                    const long long slot = o + cnt[q] - 1 - j;
                    if (slot < capacity) __stcs(starts + slot, (int32_t)i);
                    ++j;
                }
            }
        }
    }
}

__device__ __forceinline__ void warp_minmax_sum(int& mn, int& mx, long long& sum) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(kFull, mn, o));
        mx = max(mx, __shfl_xor_sync(kFull, mx, o));
        sum += __shfl_xor_sync(kFull, sum, o);
    }
}

// stats[0] = alpha sum, [1] = beta sum (64-bit), then as 32-bit words at
// stats + 2: alpha min, alpha max, beta min, beta max.
__global__ void __launch_bounds__(256) k_walk_stats(int32_t n, const int32_t* __restrict__ llrr,
                                                    const int32_t* __restrict__ cstart,
                                                    const int32_t* __restrict__ cend, const int32_t* __restrict__ cbase,
                                                    long long ntiles, int32_t* __restrict__ alpha,
                                                    int32_t* __restrict__ beta, unsigned long long* __restrict__ stats) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t m = __ldg(cbase + ntiles);
    int a_min = 0x7fffffff, a_max = 0, b_min = 0x7fffffff, b_max = 0;
    long long a_sum = 0, b_sum = 0;
    if (k < n) {
        // raw: ends i + LLRr[i] - 1 never decrease (Lemma 2), so the LLR's
        // covering k are LLRr[f..k], f the first index whose end reaches k
        long long lo = 0, hi = k + 1;
        while (lo < hi) {
            const long long mid = (lo + hi) >> 1;
            if (mid + __ldg(llrr + mid) - 1 >= k) hi = mid; else lo = mid + 1;
        }
        const int32_t a = (int32_t)(k + 1 - lo);
        // compact: the window [first end >= k, last start <= k]
        int32_t l1 = 0, h1 = m;
        while (l1 < h1) {
            const int32_t mid = (l1 + h1) >> 1;
            if (__ldg(cend + mid) >= k) h1 = mid; else l1 = mid + 1;
        }
        int32_t l2 = 0, h2 = m;
        while (l2 < h2) {
            const int32_t mid = (l2 + h2) >> 1;
            if (__ldg(cstart + mid) <= k) l2 = mid + 1; else h2 = mid;
        }
        const int32_t b = (l2 - 1 >= l1) ? l2 - l1 : 0;
        if (alpha) alpha[k] = a;
        if (beta) beta[k] = b;
        a_min = a_max = a; a_sum = a;
        b_min = b_max = b; b_sum = b;
    }
    warp_minmax_sum(a_min, a_max, a_sum);
    warp_minmax_sum(b_min, b_max, b_sum);
    // block reduction, then one set of atomics per block
    __shared__ long long s_a[8], s_b[8];
    __shared__ int s_v[8][4];
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_a[warp] = a_sum; s_b[warp] = b_sum;
        s_v[warp][0] = a_min; s_v[warp][1] = a_max; s_v[warp][2] = b_min; s_v[warp][3] = b_max;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            a_sum += s_a[w]; b_sum += s_b[w];
            a_min = min(a_min, s_v[w][0]); a_max = max(a_max, s_v[w][1]);
            b_min = min(b_min, s_v[w][2]); b_max = max(b_max, s_v[w][3]);
        }
        atomicAdd(&stats[0], (unsigned long long)a_sum);
        atomicAdd(&stats[1], (unsigned long long)b_sum);
        int* w = reinterpret_cast<int*>(stats + 2);
        atomicMin(&w[0], a_min);
        atomicMax(&w[1], a_max);
        atomicMin(&w[2], b_min);
        atomicMax(&w[3], b_max);
    }
}

__global__ void k_stats_init(unsigned long long* stats) {
    stats[0] = 0;
    stats[1] = 0;
    int* w = reinterpret_cast<int*>(stats + 2);
    w[0] = 0x7fffffff; w[1] = 0; w[2] = 0x7fffffff; w[3] = 0;
}

}  // namespace

cudaError_t launch_raw_query(const int32_t* rank, const int32_t* lcp, int32_t n, const Scratch& s, int32_t* lr_len,
                             int32_t* lr_start, int64_t* offsets, int32_t* starts, long long capacity, bool all,
                             cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(s.zero_base, 0, s.zero_bytes, stream);
    if (e != cudaSuccess) return e;
    int32_t* llrr = s.lbig;
    k_llr_raw<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(rank, lcp, n, s, llrr);
    const unsigned grid = (unsigned)((n + kRawTile - 1) / kRawTile);
    if (all)
        k_rawwalk<true><<<grid, kRawThreads, 0, stream>>>(n, llrr, s, lr_len, lr_start, offsets, starts, capacity);
    else
        k_rawwalk<false><<<grid, kRawThreads, 0, stream>>>(n, llrr, s, lr_len, lr_start, nullptr, nullptr, 0);
    return cudaGetLastError();
}

cudaError_t launch_walk_stats(const int32_t* rank, const int32_t* lcp, int32_t n, const Scratch& s, int32_t* alpha,
                              int32_t* beta, unsigned long long* stats, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(s.zero_base, 0, s.zero_bytes, stream);
    if (e != cudaSuccess) return e;
    launch_gather_front(rank, lcp, n, s, Segs{nullptr, 0}, stream);       // LLRc in s.cstart / s.cend
    int32_t* llrr = s.lbig;
    k_llr_raw<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(rank, lcp, n, s, llrr);
    k_stats_init<<<1, 1, 0, stream>>>(stats);
    k_walk_stats<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(n, llrr, s.cstart, s.cend, s.tile_cbase, s.ntiles,
                                                                   alpha, beta, stats);
    return cudaGetLastError();
}

}  // namespace lr
