// Device helpers shared by the longest-repeat kernels: accesses of tile
// status words and the warp-cooperative decoupled look-back
// of a single-pass prefix scan (Merrill and Garland, "Single-pass Parallel
// Prefix Scan with Decoupled Look-back", NVIDIA TR 2016), written for this
// library.
#pragma once
#include <cstdint>
#include "lr_internal.h"

namespace lr {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;

// Error bits the kernels OR into the context's device error word.
constexpr unsigned kErrInput = 1u;     // rank out of [0, n), lcp[0] / lcp[n] not 0, or an lcp too long
constexpr unsigned kErrTimeout = 2u;   // a bounded wait on another tile gave up

// A status word holds a 2-bit flag and a 62-bit value.
constexpr unsigned long long kFlagShift = 62;
constexpr unsigned long long kValMask = (1ull << kFlagShift) - 1;
constexpr unsigned long long kAggregate = 1ull;   // value = this tile's own total
constexpr unsigned long long kPrefix = 2ull;      // value = total of tiles 0..this one

// A status word carries its own value and guards no other data (readers
// use only the flag and the count in it), so relaxed gpu-scope accesses
// suffice: no fence makes a publishing thread wait for its earlier stores.
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & (kWarp - 1); }

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ int warp_incl_scan(int v) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
        int y = __shfl_up_sync(kFull, v, o);
        if (lane >= (unsigned)o) v += y;
    }
    return v;
}

__device__ __forceinline__ void publish(unsigned long long* status, long long tile, unsigned long long flag,
                                        long long value) {
    st_relaxed(&status[tile], (flag << kFlagShift) | (unsigned long long)value);
}

// Called by one whole warp after the tile published its aggregate.  Sums the
// totals of all earlier tiles by looking back over their status words and
// returns that exclusive prefix (the same value in every lane); it does not
// publish the inclusive prefix.  Lane j reads tile base - j; only the tiles
// after the nearest one holding an inclusive prefix (and that one) are
// needed, so only their lanes wait for a word still unset.  Waits only on
// earlier tiles, which were scheduled before this one; after `limit` polls
// (kSpinLimit unless a test shortens it) a missing word counts as a prefix
// of 0 and a timeout is recorded in both error words.
__device__ __forceinline__ long long lookback(const unsigned long long* status, long long tile, unsigned* err,
                                              unsigned* qerr, int limit) {
    const unsigned lane = lane_id();
    long long exclusive = 0;
    long long base = tile - 1;
    int polls = 0;
    while (base >= 0) {
        const long long t = base - (long long)lane;
        unsigned long long w = (t >= 0) ? ld_relaxed(&status[t]) : (kPrefix << kFlagShift);
        unsigned pmask;
        int stop;
        for (;;) {
            pmask = __ballot_sync(kFull, (w >> kFlagShift) == kPrefix);
            stop = pmask ? __ffs(pmask) - 1 : kWarp - 1;
            const bool missing = (int)lane <= stop && (w >> kFlagShift) == 0;
            if (!__any_sync(kFull, missing)) break;
            if (++polls >= limit) {
                if (lane == 0) {
                    atomicOr(err, kErrTimeout);
                    atomicOr(qerr, kErrTimeout);
                }
                if (missing) w = kPrefix << kFlagShift;
                continue;
            }
            __nanosleep(64);
            if (missing) w = ld_relaxed(&status[t]);
        }
        const long long contrib = ((int)lane <= stop) ? (long long)(w & kValMask) : 0;
        exclusive += warp_sum_ll(contrib);
        if (pmask) break;
        base -= kWarp;
    }
    return exclusive;
}

// Publish-aggregate, look back, publish-prefix in one call (one whole warp).
__device__ __forceinline__ long long lookback_exclusive(unsigned long long* status, long long tile,
                                                       long long aggregate, unsigned* err, unsigned* qerr,
                                                       int limit) {
    const unsigned lane = lane_id();
    if (lane == 0) publish(status, tile, tile == 0 ? kPrefix : kAggregate, aggregate);
    if (tile == 0) return 0;
    const long long ex = lookback(status, tile, err, qerr, limit);
    if (lane == 0) publish(status, tile, kPrefix, ex + aggregate);
    return ex;
}

}  // namespace lr

// ---------------------------------------------------------------------------
// mbarriers and bulk (TMA) copies global -> shared, for producer / consumer
// pipelines inside one CTA.  Every wait is bounded (kMbarSpinLimit polls).

namespace lr {

constexpr int kMbarSpinLimit = 1 << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes initialised mbarriers visible to the async (bulk copy) proxy.
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar)) : "memory");
}

// Arrives and adds `bytes` to the transaction count the phase waits for.
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity to complete; false after the
// poll limit (the caller reports a timeout).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    for (int i = 0; i < kMbarSpinLimit; ++i) {
        if (mbar_test(bar, parity)) return true;
        if (i > 8) __nanosleep(64);
    }
    return false;
}

// Orders this thread's earlier generic-proxy accesses to shared memory
// before later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

}  // namespace lr
