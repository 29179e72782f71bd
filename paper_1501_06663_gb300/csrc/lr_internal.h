// Internal declarations shared by the kernels and the C ABI layer of liblr.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace lr {

constexpr int kTile = 2048;        // positions per tile (one CTA)
constexpr int kThreads = 256;      // threads per CTA
constexpr int kCoverCap = 4096;    // compact LLR's a tile stages in shared memory

// Device scratch of one query, carved out of one allocation by the context.
struct TileScratch {
    unsigned* tickets;             // [0] ticket of k_llr_compact, [1] of k_cover
    unsigned* qerr;                // error bits of this query (cleared with the tickets)
    unsigned* err;                 // sticky device error bits (kErr*), read by the host
    unsigned long long* status_c;  // per-tile look-back words, LLRc counts
    unsigned long long* status_o;  // per-tile look-back words, LR counts
    int32_t* cbase;                // ntiles + 1: compact LLR's starting before tile j
    int32_t* cstart;               // n: compact LLR starts (ascending)
    int32_t* cend;                 // n: compact LLR ends   (ascending)
    long long ntiles;
    void* zero_base;               // tickets + status words, cleared before every query
    size_t zero_bytes;
};

inline long long num_tiles(long long n) { return (n + kTile - 1) / kTile; }

cudaError_t configure_kernels();
size_t cover_smem_bytes();
constexpr int kMaxPhases = 8;

// Optional per-kernel events: ev[i] is recorded before kernel i and
// ev[count] after the last one.
struct PhaseEvents {
    cudaEvent_t ev[kMaxPhases + 1];
    bool enabled = false;
};

cudaError_t launch_query(const int32_t* rank, const int32_t* lcp, int32_t n, const TileScratch& s,
                         int32_t* lr_len, int32_t* lr_start, int64_t* offsets, int32_t* starts,
                         long long capacity, bool all, cudaStream_t stream, int* launches,
                         PhaseEvents* events);

}  // namespace lr
