// lr_query_all_static: the all-LR query for callers that must not allocate
// device memory.  It runs the existing rank-gather front end and cover
// kernel unchanged; only their scratch comes from a fixed array in the
// library's device image instead of a context.
#include <cuda_runtime.h>
#include <cstdint>
#include <mutex>
#include "lr.h"
#include "lr_internal.h"
#include "lr_device.cuh"

namespace {

constexpr long long kStaticMaxN = 1LL << 20;              // LR_STATIC_MAX_N in lr.h
constexpr size_t kAlignS = 256;
constexpr size_t align_s(size_t v) { return (v + kAlignS - 1) / kAlignS * kAlignS; }

// Scratch layout for n <= kStaticMaxN (rank-gather front end + cover kernel).
constexpr long long kTilesMax = (kStaticMaxN + lr::kTile - 1) / lr::kTile;
constexpr long long kSegsMax = (kStaticMaxN + lr::kSeg - 1) / lr::kSeg;
constexpr size_t kOffStatusG = kAlignS;                   // [0, 256): tickets, per-query and sticky error bits
constexpr size_t kOffStatusO = align_s(kOffStatusG + (size_t)kTilesMax * 8);
constexpr size_t kOffStatusW = align_s(kOffStatusO + (size_t)kTilesMax * 8);
constexpr size_t kZeroEnd = kOffStatusW + (size_t)((kStaticMaxN + lr::kSegTile - 1) / lr::kSegTile) * 8;
constexpr size_t kOffCbase = align_s(kZeroEnd);
constexpr size_t kOffSegCbase = align_s(kOffCbase + (size_t)(kTilesMax + 1) * 4);
constexpr size_t kOffCstart = align_s(kOffSegCbase + (size_t)(kSegsMax + 1) * 4);
constexpr size_t kOffCend = align_s(kOffCstart + (size_t)kStaticMaxN * 4);
constexpr size_t kStaticBytes = align_s(kOffCend + (size_t)kStaticMaxN * 4);   // about 8.1 MB

// The array itself.  Host code must not use its name as an address: it is a
// host-side stand-in.  The device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_lr_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};                  // device address per device, set up once

lr_status static_scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return LR_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_lr_static_scratch);   // the device is current here
        if (e != cudaSuccess || !p) { cudaGetLastError(); return LR_ERR_CUDA; }
        if (lr::configure_kernels() != cudaSuccess) { cudaGetLastError(); return LR_ERR_CUDA; }
        g_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[dev];
    return LR_OK;
}

}  // namespace

extern "C" lr_status lr_query_all_static(lr_stream_t stream, const int32_t* d_rank, const int32_t* d_lcp,
                                         int32_t n, int32_t* d_lr_len, int32_t* d_lr_start,
                                         int64_t* d_offsets, int32_t* d_starts, int64_t starts_capacity,
                                         int64_t* h_total) {
    if (!d_rank || !d_lcp || !d_lr_len || !d_lr_start || !d_offsets) return LR_ERR_ARG;
    if (starts_capacity < 0 || (starts_capacity > 0 && !d_starts)) return LR_ERR_ARG;
    if (n < 1 || (long long)n > kStaticMaxN) return LR_ERR_ARG;    // larger inputs need lr_query_all
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return LR_ERR_CUDA; }
    unsigned char* b = nullptr;
    lr_status st = static_scratch_address(dev, &b);
    if (st != LR_OK) return st;

    lr::Scratch s = {};
    s.tickets = reinterpret_cast<unsigned*>(b);
    s.qerr = reinterpret_cast<unsigned*>(b + 16);
    s.err = reinterpret_cast<unsigned*>(b + 32);
    s.status_g = reinterpret_cast<unsigned long long*>(b + kOffStatusG);
    s.status_o = reinterpret_cast<unsigned long long*>(b + kOffStatusO);
    s.status_w = reinterpret_cast<unsigned long long*>(b + kOffStatusW);
    s.tile_cbase = reinterpret_cast<int32_t*>(b + kOffCbase);
    s.seg_cbase = reinterpret_cast<int32_t*>(b + kOffSegCbase);
    s.cstart = reinterpret_cast<int32_t*>(b + kOffCstart);
    s.cend = reinterpret_cast<int32_t*>(b + kOffCend);
    s.ntiles = lr::num_tiles(n);
    s.nsegs = lr::num_segs(n);
    // what every query must find at zero: tickets, both error words, the
    // look-back words of both kernels (one memset, no allocation)
    s.zero_base = b;
    s.zero_bytes = kZeroEnd;
    cudaStream_t strm = (cudaStream_t)stream;
    cudaError_t e = lr::launch_query(nullptr, d_rank, d_lcp, n, s, d_lr_len, d_lr_start, d_offsets, d_starts,
                                     starts_capacity, true, strm, nullptr, nullptr);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LR_ERR_NOMEM : LR_ERR_CUDA;
    if (!h_total) return LR_OK;
    unsigned bits = 0;
    int64_t total = 0;
    e = cudaMemcpyAsync(&total, d_offsets + n, sizeof(total), cudaMemcpyDeviceToHost, strm);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, s.err, sizeof(bits), cudaMemcpyDeviceToHost, strm);
    if (e == cudaSuccess) e = cudaStreamSynchronize(strm);
    if (e != cudaSuccess) return LR_ERR_CUDA;
    *h_total = total;
    if (bits & lr::kErrTimeout) return LR_ERR_TIMEOUT;
    if (bits & lr::kErrInput) return LR_ERR_SENTINEL;
    return total > starts_capacity ? LR_ERR_CAPACITY : LR_OK;
}
