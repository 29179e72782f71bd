// Suffix array, rank and lcp arrays on the device: the step before the
// longest-repeat query.  The paper builds them on the host and notes that
// they can be built in parallel on a GPU by prefix doubling (Sec. 4, citing
// Osipov 2012 and Deo and Keely 2013); this is a prefix-doubling build, for
// one string or for many strings packed back to back (string j owns
// positions [off[j], off[j+1])) in one pass.
//
//  * round 0: every suffix gets a key of its string index (most significant)
//    and its first c symbols, each in the bits its dense code needs (the
//    symbols that occur numbered 1 .. sigma, 0 past the end of its string;
//    c = 21 for DNA, 9 for 96 symbols, 7 for all 256, fewer when the string
//    index needs bits);
//    the keys are sorted with their positions (radix sort) and each
//    position's rank becomes the sorted index of the first key equal to its
//    own (a max-scan over group heads).  Strings occupy consecutive rank
//    ranges, [off[j], off[j+1]) for string j;
//  * round r >= 1, h = c * 2^(r-1): key(i) = (rank(i), rank(i + h) + 1, or 0
//    past the end of i's string), for the suffixes still in groups of two or
//    more only (the others keep their ranks), sorted again; ranks are equal
//    iff the strings and the first c * 2^r symbols are; a re-sorted suffix
//    takes the rank of its old group's start plus the offset of its new
//    group inside the old one;
//  * rounds stop when all ranks differ; the suffix array is the positions
//    sorted by rank (flattened index g holds the suffix of local rank
//    g - off[j]);
//  * lcp of each pair of sa neighbours: the round at which they parted
//    gives it within a factor of two (first c * 2^(r-1) symbols equal, fewer
//    than c * 2^r), binary lifting over the ranks of the earlier rounds
//    (equal ranks at round q mean c * 2^q equal symbols) and fewer than c
//    symbol comparisons give the rest.
#include <cuda_runtime.h>
#include <cub/cub.cuh>
#include <thrust/iterator/counting_iterator.h>
#include <cstdint>
#include "lr_internal.h"

namespace lr {

namespace {

// The string holding flattened position g: the last j with off[j] <= g.
__device__ __forceinline__ long long string_of(const int64_t* __restrict__ off, long long num, long long g) {
    long long lo = 0, hi = num - 1;
    while (lo < hi) {
        const long long mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The symbols that occur: seen[c] = 1 for every byte value c of the text.
__global__ void k_seen(const uint8_t* __restrict__ text, long long total, uint8_t* __restrict__ seen) {
    __shared__ uint8_t s[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) s[t] = 0;
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
        s[__ldg(text + i)] = 1;
    __syncthreads();
    for (int t = threadIdx.x; t < 256; t += blockDim.x)
        if (s[t]) seen[t] = 1;
}

// Dense codes 1 .. sigma of the symbols that occur (0: past the end of a
// string), bps bits each.
struct SymCodes {
    uint16_t code[256];
};

__global__ void k_keys0(const uint8_t* __restrict__ text, long long total, const int64_t* __restrict__ off,
                        long long num, int csyms, int bps, SymCodes codes, uint64_t* __restrict__ key,
                        int32_t* __restrict__ val, int32_t* __restrict__ end) {
    __shared__ uint16_t sc[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) sc[t] = codes.code[t];
    __syncthreads();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const long long j = string_of(off, num, i);
    const long long e = __ldg(off + j + 1);
    uint64_t k = (uint64_t)j;
    for (int t = 0; t < csyms; ++t) {
        const uint32_t c = (i + t < e) ? (uint32_t)sc[__ldg(text + i + t)] : 0u;
        k = (k << bps) | c;
    }
    key[i] = k;
    val[i] = (int32_t)i;
    end[i] = (int32_t)e;
}

// A rank word holds the rank in bits 0..30 and, in bit 31, whether the
// position is still in a group of two or more (then every member of its
// group is, so equal words still mean equal groups).
constexpr uint32_t kActiveBit = 0x80000000u;
constexpr uint32_t kRankMask = 0x7fffffffu;

// Round r >= 1 keys of the suffixes still in groups of two or more (act[0..A),
// ascending positions): (rank(i), rank(i + h) + 1, or 0 past the end of i's
// string).
__global__ void k_keys_act(const int32_t* __restrict__ act, long long A, const int32_t* __restrict__ rank,
                           long long h, const int32_t* __restrict__ end, uint64_t* __restrict__ key,
                           int32_t* __restrict__ val) {
    const long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A) return;
    const long long i = __ldg(act + a);
    const uint32_t second =
        (i + h < __ldg(end + i)) ? ((uint32_t)__ldg(rank + i + h) & kRankMask) + 1u : 0u;
    key[a] = ((uint64_t)((uint32_t)__ldg(rank + i) & kRankMask) << 32) | second;
    val[a] = (int32_t)i;
}

// Selects position i when its rank word carries the active bit.
struct ActiveAt {
    const int32_t* rank;
    __device__ __forceinline__ bool operator()(int32_t i) const { return ((uint32_t)__ldg(rank + i) & kActiveBit) != 0; }
};

// Round 0, over all sorted keys: head[g] = g where key g starts a group of
// equal keys, else 0; the number of groups is added to *groups; sep[g] = 0
// where g starts a group; flags[g] = 1 where g is in a group of two or
// more.  A block takes kHeadsPer x 256 consecutive keys and adds its count
// with one atomic: adds on the one counter serialise (one per 256 keys cost
// ~5 ms at n = 256 Mi).
constexpr int kHeadsThreads = 256;
constexpr int kHeadsPer = 16;
__global__ void __launch_bounds__(kHeadsThreads)
k_heads(const uint64_t* __restrict__ key, long long total, int32_t* __restrict__ head,
        unsigned long long* __restrict__ groups, uint8_t* __restrict__ sep, uint8_t* __restrict__ flags) {
    __shared__ int wsum[kHeadsThreads / 32];
    const long long g0 = (long long)blockIdx.x * (kHeadsThreads * kHeadsPer) + threadIdx.x;
    int cnt = 0;
#pragma unroll 4
    for (int u = 0; u < kHeadsPer; ++u) {
        const long long g = g0 + (long long)u * kHeadsThreads;
        if (g < total) {
            const uint64_t k = __ldg(key + g);
            const bool h = (g == 0) || (k != __ldg(key + g - 1));
            head[g] = h ? (int32_t)g : 0;
            cnt += h;
            if (h) sep[g] = 0;
            flags[g] = !h || (g + 1 < total && __ldg(key + g + 1) == k);
        }
    }
    cnt = __reduce_add_sync(0xffffffffu, (unsigned)cnt);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kHeadsThreads / 32; ++w) t += (unsigned long long)wsum[w];
        if (t) atomicAdd(groups, t);
    }
}

__global__ void k_scatter_rank(const int32_t* __restrict__ sorted, const int32_t* __restrict__ hp, long long total,
                               int32_t* __restrict__ rank) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < total) rank[sorted[g]] = hp[g];
}

// Round r >= 1, over the re-sorted keys key[0..A): mh[a] = a where key a
// starts a new group, mo[a] = a where it starts a group of the previous
// round (its first half, the old rank, changes); else 0.
__global__ void k_marks(const uint64_t* __restrict__ key, long long A, int32_t* __restrict__ mh,
                        int32_t* __restrict__ mo) {
    const long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A) return;
    const uint64_t k = __ldg(key + a);
    bool nh = true, oh = true;
    if (a > 0) {
        const uint64_t p = __ldg(key + a - 1);
        nh = k != p;
        oh = (k >> 32) != (p >> 32);
    }
    mh[a] = nh ? (int32_t)a : 0;
    mo[a] = oh ? (int32_t)a : 0;
}

// Round r >= 1: an old group (rank g0 = its first sorted index) holds its
// re-sorted members at a0 .. a0 + size - 1, so member a sits at sorted index
// g0 + a - a0 and its new rank is the index of its new group's first member,
// g0 + ah - a0 (ah, a0: max-scans of the marks), with the active bit when
// the new group has two or more members.  New group starts inside an old
// group take sep = r.
__global__ void k_update(const uint64_t* __restrict__ key, const int32_t* __restrict__ val,
                         const int32_t* __restrict__ ah, const int32_t* __restrict__ a0, long long A,
                         int32_t* __restrict__ rank, uint8_t* __restrict__ sep, int round) {
    const long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A) return;
    const uint64_t k = __ldg(key + a);
    const long long g0 = (long long)(k >> 32), s0 = __ldg(a0 + a), hh = __ldg(ah + a);
    const bool act = (a > 0 && __ldg(key + a - 1) == k) || (a + 1 < A && __ldg(key + a + 1) == k);
    rank[__ldg(val + a)] = (int32_t)((uint32_t)(g0 + (hh - s0)) | (act ? kActiveBit : 0u));
    if (hh == a && s0 != a) sep[g0 + (a - s0)] = (uint8_t)round;
}

// Round 0: the active bit on the ranks (in sorted order) of keys in groups
// of two or more.
__global__ void k_mark_active(int32_t* __restrict__ hp, const uint8_t* __restrict__ flags, long long total) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < total && flags[g]) hp[g] = (int32_t)((uint32_t)hp[g] | kActiveBit);
}

__global__ void k_iota(int32_t* __restrict__ v, long long total) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) v[i] = (int32_t)i;
}

// lcp of sorted neighbours g - 1, g of one string, written in the layout the
// queries take (string j's n_j + 1 entries at off[j] + j), and the string-
// local sa and rank (index g read as a rank for sa, as a position for rank:
// both lie in string j's range [off[j], off[j+1])).  The two suffixes parted
// at round r = sep[g]: their first csyms * 2^(r-1) symbols are equal (none
// for r = 0) and fewer than csyms * 2^r are; the rest is found by binary
// lifting over the ranks of rounds r - 2 .. 0 (equal ranks at round q mean
// csyms * 2^q more equal symbols, longest first), then fewer than csyms
// symbol comparisons.
__global__ void k_lcp(const uint8_t* __restrict__ text, long long total, const int64_t* __restrict__ off,
                      long long num, const int32_t* __restrict__ sorted, const int32_t* __restrict__ levels,
                      int rounds, int csyms, const uint8_t* __restrict__ sep, const int32_t* __restrict__ frank,
                      int32_t* __restrict__ sa, int32_t* __restrict__ rank, int32_t* __restrict__ lcp) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const long long j = string_of(off, num, g);
    const long long a = __ldg(off + j), e = __ldg(off + j + 1);
    sa[g] = (int32_t)(sorted[g] - a);
    rank[g] = (int32_t)(frank[g] - a);
    int32_t out = 0;
    if (g > a) {
        long long x = sorted[g - 1], y = sorted[g], l = 0;
        int r = sep[g];
        r = r < rounds ? r : rounds - 1;               // every index parts by the last round
        if (r > 0) {
            l = (long long)csyms << (r - 1);
            x += l;
            y += l;
        }
        for (int q = r - 2; q >= 0; --q) {
            const long long len = (long long)csyms << q;
            const int32_t* R = levels + (size_t)q * (size_t)total;
            if (x < e && y < e && __ldg(R + x) == __ldg(R + y)) { l += len; x += len; y += len; }
        }
        for (int t = 0; t < csyms && x < e && y < e && __ldg(text + x) == __ldg(text + y); ++t) { ++l; ++x; ++y; }
        out = (int32_t)l;
    }
    lcp[g + j] = out;                                  // lcp[0] of string j is 0 (g == a)
}

// The closing sentinel lcp[n_j] = 0 of every string (and the only entry of
// an empty one).
__global__ void k_lcp_tails(const int64_t* __restrict__ off, long long num, int32_t* __restrict__ lcp) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < num) lcp[__ldg(off + j + 1) + j] = 0;
}

// Sets *bad unless off[0] = 0, off[num] = total and off never decreases.
__global__ void k_check_off(const int64_t* __restrict__ off, long long num, long long total,
                            unsigned long long* __restrict__ bad) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j > num) return;
    const long long v = __ldg(off + j);
    bool b = v < 0 || v > total || (j == 0 && v != 0) || (j == num && v != total);
    if (j < num && __ldg(off + j + 1) < v) b = true;
    if (b) atomicOr(bad, 1ull);
}

struct MaxOp {
    __device__ __forceinline__ int32_t operator()(int32_t a, int32_t b) const { return a > b ? a : b; }
};

inline unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

size_t sort_temp_bytes(long long n) {
    size_t a = 0, b = 0, c = 0;
    cub::DoubleBuffer<uint64_t> keys(nullptr, nullptr);
    cub::DoubleBuffer<int32_t> vals(nullptr, nullptr), pos(nullptr, nullptr);
    cub::DeviceRadixSort::SortPairs(nullptr, a, keys, vals, (int)n, 0, 64, (cudaStream_t)0);
    cub::DeviceScan::InclusiveScan(nullptr, b, (int32_t*)nullptr, (int32_t*)nullptr, MaxOp{}, (int)n, (cudaStream_t)0);
    cub::DeviceRadixSort::SortPairs(nullptr, c, pos, vals, (int)n, 0, 32, (cudaStream_t)0);
    size_t d = 0;
    cub::DeviceSelect::If(nullptr, d, thrust::counting_iterator<int32_t>(0), (int32_t*)nullptr,
                          (unsigned long long*)nullptr, (int)n, ActiveAt{nullptr}, (cudaStream_t)0);
    if (b > a) a = b;
    if (d > a) a = d;
    return (c > a ? c : a) + 256;
}

inline size_t al(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

// Layout of the work memory for n positions and `rounds` rank levels.
size_t index_work_bytes(long long n, int rounds) {
    const size_t nn = (size_t)n;
    return al(nn * 8) * 2 + al(nn * 4) * 5 + al(nn) + al((size_t)rounds * nn * 4) + al(64) + al(sort_temp_bytes(n));
}

cudaError_t IndexWork::alloc(long long n, int rounds) {
    release();
    const size_t nn = (size_t)n;
    bytes = index_work_bytes(n, rounds);
    cudaError_t e = cudaMalloc((void**)&base, bytes);
    if (e != cudaSuccess) { cudaGetLastError(); base = nullptr; bytes = 0; return cudaErrorMemoryAllocation; }
    unsigned char* p = base;
    k0 = (uint64_t*)p; p += al(nn * 8);
    k1 = (uint64_t*)p; p += al(nn * 8);
    v0 = (int32_t*)p; p += al(nn * 4);
    v1 = (int32_t*)p; p += al(nn * 4);
    head = (int32_t*)p; p += al(nn * 4);
    hp = (int32_t*)p; p += al(nn * 4);
    end = (int32_t*)p; p += al(nn * 4);
    sep = (uint8_t*)p; p += al(nn);
    levels = (int32_t*)p; p += al((size_t)rounds * nn * 4);
    misc = (unsigned long long*)p; p += al(64);
    tmp = p;
    tmp_bytes = sort_temp_bytes(n);
    cap_n = n;
    cap_rounds = rounds;
    return cudaSuccess;
}

void IndexWork::release() {
    if (base) cudaFree(base);
    base = nullptr;
    bytes = 0;
    cap_n = 0;
    cap_rounds = 0;
}

// Builds sa, rank (string-local, at the strings' offsets) and lcp (n_j + 1
// entries per string at off[j] + j) of text[0..total) split by the device
// offset table off[0..num]; `w` must hold `total` positions.  When more
// rounds are needed than w holds and `grow` is set, w is reallocated (which
// waits for the device); otherwise cudaErrorMemoryAllocation.
cudaError_t build_arrays_batch(const uint8_t* text, long long total, const int64_t* off, long long num, int32_t* sa,
                               int32_t* rank, int32_t* lcp, IndexWork& w, bool grow, cudaStream_t stream,
                               int* rounds_out) {
    if (total > w.cap_n) return cudaErrorMemoryAllocation;
    // every kernel below trusts the offset table: check it first
    cudaError_t e = cudaMemsetAsync(w.misc, 0, 16, stream);
    if (e != cudaSuccess) return e;
    k_check_off<<<blocks(num + 1, 256), 256, 0, stream>>>(off, num, total, w.misc + 1);
    e = cudaMemcpyAsync(&w.groups_host, w.misc + 1, 8, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return e;
    if (w.groups_host != 0) return cudaErrorInvalidValue;
    k_lcp_tails<<<blocks(num, 256), 256, 0, stream>>>(off, num, lcp);
    if (total == 0) {
        if (rounds_out) *rounds_out = 0;
        return cudaGetLastError();
    }
    const size_t nn = (size_t)total;
    // the alphabet that occurs, coded densely: more symbols per round-0 key
    // for a small alphabet (21 for DNA, 9 for 96 symbols, 7 for all 256)
    uint8_t* seen = reinterpret_cast<uint8_t*>(w.head);
    e = cudaMemsetAsync(seen, 0, 256, stream);
    if (e != cudaSuccess) return e;
    k_seen<<<(unsigned)(total < (1 << 22) ? blocks(total, 256) : 1216), 256, 0, stream>>>(text, total, seen);
    uint8_t seen_h[256];
    e = cudaMemcpyAsync(seen_h, seen, 256, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return e;
    SymCodes codes;
    int sigma = 0;
    for (int c = 0; c < 256; ++c) codes.code[c] = seen_h[c] ? (uint16_t)++sigma : (uint16_t)0;
    int bps = 1;
    while ((1 << bps) <= sigma) ++bps;                     // codes 0 .. sigma
    int jobbits = 0;
    while (jobbits < 40 && (1ll << jobbits) < num) ++jobbits;
    const int csyms = (63 - jobbits) / bps;
    int bits = 1;
    while (bits < 31 && (1ll << bits) <= total) ++bits;
    cub::DoubleBuffer<uint64_t> keys(w.k0, w.k1);
    cub::DoubleBuffer<int32_t> vals(w.v0, w.v1);
    e = cudaMemsetAsync(w.sep, 0xff, nn, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.misc, 0, 24, stream);
    if (e != cudaSuccess) return e;
    // round 0: every suffix by its string and first csyms symbols
    k_keys0<<<blocks(total, 256), 256, 0, stream>>>(text, total, off, num, csyms, bps, codes, keys.Current(),
                                                    vals.Current(), w.end);
    size_t tb = w.tmp_bytes;
    e = cub::DeviceRadixSort::SortPairs(w.tmp, tb, keys, vals, (int)total, 0, jobbits + bps * csyms, stream);
    if (e != cudaSuccess) return e;
    uint8_t* flags = reinterpret_cast<uint8_t*>(keys.Alternate());
    k_heads<<<blocks(total, kHeadsThreads * kHeadsPer), kHeadsThreads, 0, stream>>>(keys.Current(), total, w.head,
                                                                                  w.misc, w.sep, flags);
    tb = w.tmp_bytes;
    e = cub::DeviceScan::InclusiveScan(w.tmp, tb, w.head, w.hp, MaxOp{}, (int)total, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&w.groups_host, w.misc, 8, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return e;
    int rounds = 1;
    const int32_t* sorted = nullptr;                       // the suffix array (flattened) at the end
    if (w.groups_host == (unsigned long long)total) {
        // all first keys differ: the sorted positions are the suffix array
        k_scatter_rank<<<blocks(total, 256), 256, 0, stream>>>(vals.Current(), w.hp, total, w.levels);
        sorted = vals.Current();
    } else {
        // the suffixes in groups of two or more (act, in w.head) are the only
        // ones sorted again; then the ranks go back to position order by a
        // radix sort keyed by position (streaming passes instead of one random
        // 4-byte store per position)
        long long A = 0;
        k_mark_active<<<blocks(total, 256), 256, 0, stream>>>(w.hp, flags, total);
        {
            cub::DoubleBuffer<int32_t> pos(vals.Current(), vals.Alternate());
            cub::DoubleBuffer<int32_t> rnk(w.hp, w.levels);
            tb = w.tmp_bytes;
            e = cub::DeviceRadixSort::SortPairs(w.tmp, tb, pos, rnk, (int)total, 0, bits, stream);
            if (e == cudaSuccess && rnk.Current() != w.levels)
                e = cudaMemcpyAsync(w.levels, rnk.Current(), nn * 4, cudaMemcpyDeviceToDevice, stream);
            if (e != cudaSuccess) return e;
        }
        // the active positions, ascending (their rank words are then read in order)
        tb = w.tmp_bytes;
        e = cub::DeviceSelect::If(w.tmp, tb, thrust::counting_iterator<int32_t>(0), w.head, w.misc + 2, (int)total,
                                  ActiveAt{w.levels}, stream);
        if (e != cudaSuccess) return e;
        for (int r = 1;; ++r) {
            e = cudaMemcpyAsync(&w.groups_host, w.misc + 2, 8, cudaMemcpyDeviceToHost, stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
            if (e != cudaSuccess) return e;
            A = (long long)w.groups_host;
            if (A == 0) { rounds = r; break; }
            if (r >= 40 || A > total) return cudaErrorUnknown;
            if (r >= w.cap_rounds) {                          // more rounds than the level store holds
                if (!grow) return cudaErrorMemoryAllocation;
                IndexWork bigger;
                e = bigger.alloc(w.cap_n, w.cap_rounds * 2);
                if (e != cudaSuccess) return e;
                e = cudaMemcpyAsync(bigger.levels, w.levels, (size_t)w.cap_rounds * nn * 4, cudaMemcpyDeviceToDevice,
                                    stream);
                if (e == cudaSuccess) e = cudaMemcpyAsync(bigger.end, w.end, nn * 4, cudaMemcpyDeviceToDevice, stream);
                if (e == cudaSuccess) e = cudaMemcpyAsync(bigger.sep, w.sep, nn, cudaMemcpyDeviceToDevice, stream);
                if (e == cudaSuccess) e = cudaMemcpyAsync(bigger.head, w.head, (size_t)A * 4, cudaMemcpyDeviceToDevice,
                                                          stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
                if (e != cudaSuccess) { bigger.release(); return e; }
                w.release();
                w = bigger;
                bigger.base = nullptr;                        // owned by w now
                keys = cub::DoubleBuffer<uint64_t>(w.k0, w.k1);
                vals = cub::DoubleBuffer<int32_t>(w.v0, w.v1);
            }
            const int32_t* prev = w.levels + (size_t)(r - 1) * nn;
            int32_t* level = w.levels + (size_t)r * nn;
            e = cudaMemcpyAsync(level, prev, nn * 4, cudaMemcpyDeviceToDevice, stream);   // settled ranks stay
            if (e != cudaSuccess) return e;
            const long long h = (long long)csyms << (r - 1);
            k_keys_act<<<blocks(A, 256), 256, 0, stream>>>(w.head, A, prev, h, w.end, keys.Current(), vals.Current());
            tb = w.tmp_bytes;
            e = cub::DeviceRadixSort::SortPairs(w.tmp, tb, keys, vals, (int)A, 0, 32 + bits, stream);
            if (e != cudaSuccess) return e;
            int32_t* mh = reinterpret_cast<int32_t*>(keys.Alternate());
            int32_t* mo = mh + nn;
            int32_t* a0 = vals.Alternate();
            k_marks<<<blocks(A, 256), 256, 0, stream>>>(keys.Current(), A, mh, mo);
            tb = w.tmp_bytes;
            e = cub::DeviceScan::InclusiveScan(w.tmp, tb, mh, w.hp, MaxOp{}, (int)A, stream);
            tb = w.tmp_bytes;
            if (e == cudaSuccess) e = cub::DeviceScan::InclusiveScan(w.tmp, tb, mo, a0, MaxOp{}, (int)A, stream);
            if (e != cudaSuccess) return e;
            k_update<<<blocks(A, 256), 256, 0, stream>>>(keys.Current(), vals.Current(), w.hp, a0, A, level, w.sep, r);
            tb = w.tmp_bytes;
            e = cub::DeviceSelect::If(w.tmp, tb, thrust::counting_iterator<int32_t>(0), w.head, w.misc + 2,
                                      (int)total, ActiveAt{level}, stream);
            if (e != cudaSuccess) return e;
        }
        // the suffix array: positions sorted by their final (distinct) ranks
        int32_t* kk = reinterpret_cast<int32_t*>(w.k0);
        e = cudaMemcpyAsync(kk, w.levels + (size_t)(rounds - 1) * nn, nn * 4, cudaMemcpyDeviceToDevice, stream);
        if (e != cudaSuccess) return e;
        k_iota<<<blocks(total, 256), 256, 0, stream>>>(w.v0, total);
        cub::DoubleBuffer<int32_t> fk(kk, kk + nn);
        cub::DoubleBuffer<int32_t> fv(w.v0, w.v1);
        tb = w.tmp_bytes;
        e = cub::DeviceRadixSort::SortPairs(w.tmp, tb, fk, fv, (int)total, 0, bits, stream);
        if (e != cudaSuccess) return e;
        sorted = fv.Current();
    }
    k_lcp<<<blocks(total, 256), 256, 0, stream>>>(text, total, off, num, sorted, w.levels, rounds, csyms, w.sep,
                                                  w.levels + (size_t)(rounds - 1) * nn, sa, rank, lcp);
    if (rounds_out) *rounds_out = rounds;
    return cudaGetLastError();
}

// One string: the work memory is allocated here and freed before returning.
cudaError_t build_arrays(const uint8_t* text, int32_t n, int32_t* sa, int32_t* rank, int32_t* lcp,
                         cudaStream_t stream, int* rounds_out) {
    IndexWork w;
    cudaError_t e = w.alloc(n, 8);
    if (e != cudaSuccess) return e;
    int64_t* off = nullptr;                                         // {0, n}
    if (cudaMalloc((void**)&off, 16) != cudaSuccess) { cudaGetLastError(); w.release(); return cudaErrorMemoryAllocation; }
    const int64_t h_off[2] = {0, (int64_t)n};
    e = cudaMemcpyAsync(off, h_off, sizeof(h_off), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = build_arrays_batch(text, n, off, 1, sa, rank, lcp, w, true, stream, rounds_out);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cudaFree(off);
    w.release();
    return e;
}

}  // namespace lr
