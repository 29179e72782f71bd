// Suffix array, rank and lcp arrays on the device: the step before the
// longest-repeat query.  The paper builds them on the host and notes that
// they can be built in parallel on a GPU by prefix doubling (Sec. 4, citing
// Osipov 2012 and Deo and Keely 2013); this is a prefix-doubling build.
//
//  * round 0: every suffix gets the key of its first 7 symbols (9 bits each,
//    symbol + 1, 0 past the end); the keys are sorted with their positions
//    (radix sort) and each position's rank becomes the sorted index of the
//    first key equal to its own (a max-scan over group heads);
//  * round r >= 1, h = 7 * 2^(r-1): key(i) = (rank(i), rank(i + h) + 1 or 0
//    past the end), sorted again; ranks are equal iff the first 7 * 2^r
//    symbols are;
//  * rounds stop when all n ranks differ: the sorted positions are the
//    suffix array and the last ranks its inverse;
//  * lcp of each pair of sa neighbours by binary lifting over the ranks of
//    every round (longest first: equal ranks at round r mean 7 * 2^r equal
//    symbols, skip them), then at most six symbol comparisons.
#include <cuda_runtime.h>
#include <cub/cub.cuh>
#include <cstdint>
#include "lr_internal.h"

namespace lr {

namespace {

constexpr int kSym0 = 7;               // symbols in the round-0 key (7 x 9 bits)

__global__ void k_keys0(const uint8_t* __restrict__ text, int32_t n, uint64_t* __restrict__ key,
                        int32_t* __restrict__ val) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t k = 0;
#pragma unroll
    for (int j = 0; j < kSym0; ++j) {
        const uint32_t c = (i + j < n) ? (uint32_t)__ldg(text + i + j) + 1u : 0u;
        k = (k << 9) | c;
    }
    key[i] = k;
    val[i] = (int32_t)i;
}

__global__ void k_keys(const int32_t* __restrict__ rank, int32_t n, long long h, uint64_t* __restrict__ key,
                       int32_t* __restrict__ val) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t second = (i + h < n) ? (uint32_t)__ldg(rank + i + h) + 1u : 0u;
    key[i] = ((uint64_t)(uint32_t)__ldg(rank + i) << 32) | second;
    val[i] = (int32_t)i;
}

// head[j] = j where sorted key j starts a group of equal keys, else 0; the
// number of groups is added to *groups.
__global__ void k_heads(const uint64_t* __restrict__ key, int32_t n, int32_t* __restrict__ head,
                        unsigned long long* __restrict__ groups) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool h = false;
    if (j < n) {
        h = (j == 0) || (key[j] != key[j - 1]);
        head[j] = h ? (int32_t)j : 0;
    }
    const unsigned b = __ballot_sync(0xffffffffu, h);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(groups, (unsigned long long)__popc(b));
}

__global__ void k_scatter_rank(const int32_t* __restrict__ sa, const int32_t* __restrict__ hp, int32_t n,
                               int32_t* __restrict__ rank) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) rank[sa[j]] = hp[j];
}

__global__ void k_lcp(const uint8_t* __restrict__ text, int32_t n, const int32_t* __restrict__ sa,
                      const int32_t* __restrict__ levels, int rounds, int32_t* __restrict__ lcp) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j > n) return;
    if (j == 0 || j == n) { lcp[j] = 0; return; }
    long long x = sa[j - 1], y = sa[j], l = 0;
    for (int r = rounds - 1; r >= 0; --r) {
        const long long len = (long long)kSym0 << r;
        const int32_t* R = levels + (size_t)r * (size_t)n;
        if (x < n && y < n && __ldg(R + x) == __ldg(R + y)) { l += len; x += len; y += len; }
    }
    for (int t = 0; t < kSym0 && x < n && y < n && __ldg(text + x) == __ldg(text + y); ++t) { ++l; ++x; ++y; }
    lcp[j] = (int32_t)l;
}

struct MaxOp {
    __device__ __forceinline__ int32_t operator()(int32_t a, int32_t b) const { return a > b ? a : b; }
};

inline unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// Builds sa, rank and lcp (n + 1 entries) of text[0..n) on `stream`; all
// device memory it needs is allocated here and freed before returning.
// Returns cudaErrorMemoryAllocation when it does not fit.
cudaError_t build_arrays(const uint8_t* text, int32_t n, int32_t* sa, int32_t* rank, int32_t* lcp,
                         cudaStream_t stream, int* rounds_out) {
    const size_t nn = (size_t)n;
    int bits = 1;
    while (bits < 31 && (1ll << bits) <= (long long)n) ++bits;
    const int max_rounds = 34;
    uint64_t *k0 = nullptr, *k1 = nullptr;
    int32_t *v0 = nullptr, *v1 = nullptr, *head = nullptr, *hp = nullptr, *levels = nullptr;
    unsigned long long* groups = nullptr;
    void* tmp = nullptr;
    size_t tmp_sort = 0, tmp_scan = 0;
    cudaError_t e = cudaSuccess;
    auto fail = [&](cudaError_t err) {
        cudaFree(k0); cudaFree(k1); cudaFree(v0); cudaFree(v1); cudaFree(head); cudaFree(hp);
        cudaFree(levels); cudaFree(groups); cudaFree(tmp);
        return err;
    };
    cub::DoubleBuffer<uint64_t> keys(nullptr, nullptr);
    cub::DoubleBuffer<int32_t> vals(nullptr, nullptr);
    e = cub::DeviceRadixSort::SortPairs(nullptr, tmp_sort, keys, vals, n, 0, 64, stream);
    if (e == cudaSuccess) e = cub::DeviceScan::InclusiveScan(nullptr, tmp_scan, head, hp, MaxOp{}, n, stream);
    if (e != cudaSuccess) return e;
    if (e == cudaSuccess) e = cudaMalloc((void**)&k0, nn * 8);
    if (e == cudaSuccess) e = cudaMalloc((void**)&k1, nn * 8);
    if (e == cudaSuccess) e = cudaMalloc((void**)&v0, nn * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&v1, nn * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&head, nn * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&hp, nn * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&groups, 8);
    if (e == cudaSuccess) e = cudaMalloc(&tmp, tmp_sort > tmp_scan ? tmp_sort : tmp_scan);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(cudaErrorMemoryAllocation); }
    // ranks of every round, for the lcp lifting; grown a round at a time
    int cap_rounds = 8;
    e = cudaMalloc((void**)&levels, (size_t)cap_rounds * nn * 4);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(cudaErrorMemoryAllocation); }
    keys = cub::DoubleBuffer<uint64_t>(k0, k1);
    vals = cub::DoubleBuffer<int32_t>(v0, v1);
    const size_t tmp_bytes = tmp_sort > tmp_scan ? tmp_sort : tmp_scan;
    int r = 0;
    for (;; ++r) {
        if (r >= max_rounds) return fail(cudaErrorUnknown);
        if (r >= cap_rounds) {                           // more rounds than room: double the level store
            int32_t* bigger = nullptr;
            if (cudaMalloc((void**)&bigger, (size_t)cap_rounds * 2 * nn * 4) != cudaSuccess) {
                cudaGetLastError();
                return fail(cudaErrorMemoryAllocation);
            }
            e = cudaMemcpyAsync(bigger, levels, (size_t)cap_rounds * nn * 4, cudaMemcpyDeviceToDevice, stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
            cudaFree(levels);
            levels = bigger;
            cap_rounds *= 2;
            if (e != cudaSuccess) return fail(e);
        }
        int end_bit;
        if (r == 0) {
            k_keys0<<<blocks(n, 256), 256, 0, stream>>>(text, n, keys.Current(), vals.Current());
            end_bit = 9 * kSym0;
        } else {
            const long long h = (long long)kSym0 << (r - 1);
            k_keys<<<blocks(n, 256), 256, 0, stream>>>(levels + (size_t)(r - 1) * nn, n, h, keys.Current(),
                                                       vals.Current());
            end_bit = 32 + bits;
        }
        size_t tb = tmp_bytes;
        e = cub::DeviceRadixSort::SortPairs(tmp, tb, keys, vals, n, 0, end_bit, stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(groups, 0, 8, stream);
        if (e != cudaSuccess) return fail(e);
        k_heads<<<blocks(n, 256), 256, 0, stream>>>(keys.Current(), n, head, groups);
        tb = tmp_bytes;
        e = cub::DeviceScan::InclusiveScan(tmp, tb, head, hp, MaxOp{}, n, stream);
        if (e != cudaSuccess) return fail(e);
        k_scatter_rank<<<blocks(n, 256), 256, 0, stream>>>(vals.Current(), hp, n, levels + (size_t)r * nn);
        unsigned long long g = 0;
        e = cudaMemcpyAsync(&g, groups, 8, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return fail(e);
        if (g == (unsigned long long)n) break;
    }
    const int rounds = r + 1;
    e = cudaMemcpyAsync(sa, vals.Current(), nn * 4, cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rank, levels + (size_t)r * nn, nn * 4, cudaMemcpyDeviceToDevice, stream);
    if (e != cudaSuccess) return fail(e);
    k_lcp<<<blocks((long long)n + 1, 256), 256, 0, stream>>>(text, n, vals.Current(), levels, rounds, lcp);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (rounds_out) *rounds_out = rounds;
    return fail(e);
}

}  // namespace lr
