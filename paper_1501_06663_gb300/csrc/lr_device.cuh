// Device helpers shared by the longest-repeat kernels: acquire/release
// accesses of tile status words and the warp-cooperative decoupled look-back
// of a single-pass prefix scan (Merrill and Garland, "Single-pass Parallel
// Prefix Scan with Decoupled Look-back", NVIDIA TR 2016), written for this
// library.
#pragma once
#include <cstdint>

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

// Upper bound on polls of one status word before a wait is declared lost
// (about a second at the back-off below).
constexpr int kSpinLimit = 1 << 23;

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
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

// Polls `w` until its flag is set; after kSpinLimit polls records a timeout
// in both error words and returns a prefix of 0 so the caller can finish.
__device__ __forceinline__ unsigned long long wait_flag(const unsigned long long* w, unsigned* err, unsigned* qerr) {
    unsigned long long v = ld_acquire(w);
    int polls = 0;
    while ((v >> kFlagShift) == 0) {
        if (++polls >= kSpinLimit) {
            atomicOr(err, kErrTimeout);
            atomicOr(qerr, kErrTimeout);
            return kPrefix << kFlagShift;
        }
        __nanosleep(32);
        v = ld_acquire(w);
    }
    return v;
}

__device__ __forceinline__ void publish(unsigned long long* status, long long tile, unsigned long long flag,
                                        long long value) {
    st_release(&status[tile], (flag << kFlagShift) | (unsigned long long)value);
}

// Called by one whole warp after the tile published its aggregate.  Sums the
// totals of all earlier tiles by looking back over their status words and
// returns that exclusive prefix (the same value in every lane); it does not
// publish the inclusive prefix.  Waits only on earlier tiles, which were
// scheduled before this one.
__device__ __forceinline__ long long lookback(const unsigned long long* status, long long tile, unsigned* err,
                                              unsigned* qerr) {
    const unsigned lane = lane_id();
    long long exclusive = 0;
    long long base = tile - 1;
    while (base >= 0) {
        const long long t = base - (long long)lane;
        const unsigned long long w = (t >= 0) ? wait_flag(&status[t], err, qerr) : (kPrefix << kFlagShift);
        const unsigned pmask = __ballot_sync(kFull, (w >> kFlagShift) == kPrefix);
        const int stop = pmask ? __ffs(pmask) - 1 : kWarp - 1;
        const long long contrib = ((int)lane <= stop) ? (long long)(w & kValMask) : 0;
        exclusive += warp_sum_ll(contrib);
        if (pmask) break;
        base -= kWarp;
    }
    return exclusive;
}

// Publish-aggregate, look back, publish-prefix in one call (one whole warp).
__device__ __forceinline__ long long lookback_exclusive(unsigned long long* status, long long tile,
                                                       long long aggregate, unsigned* err, unsigned* qerr) {
    const unsigned lane = lane_id();
    if (lane == 0) publish(status, tile, tile == 0 ? kPrefix : kAggregate, aggregate);
    if (tile == 0) return 0;
    const long long ex = lookback(status, tile, err, qerr);
    if (lane == 0) publish(status, tile, kPrefix, ex + aggregate);
    return ex;
}

}  // namespace lr
