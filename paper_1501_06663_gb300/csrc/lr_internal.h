// Internal declarations shared by the kernels and the C ABI layer of liblr.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include "lr.h"

namespace lr {

// Tiles of the gather front end (and the granularity of tile_cbase).
constexpr int kTile = 2048;          // positions per tile (one CTA)
constexpr int kThreads = 256;        // threads per tile CTA
// Tiles of the tile cover kernel: kTile x (1, 2 or 4) positions, kThreads x the same threads.
// Segments of the warp-segment cover kernel (one warp each), and the
// granularity of seg_cbase.
constexpr int kSegLog = 8;
constexpr int kSeg = 1 << kSegLog;   // positions per warp segment
constexpr int kSegTile = 4096;       // positions per CTA of the warp-segment cover (its look-back unit)

// Rank-order front end: a two-level radix partition of <position, L> by the
// position, into super-buckets of 2^20 and then buckets of 2^15 positions.
constexpr int kSuperLog = 20;
constexpr int kSuper = 1 << kSuperLog;         // positions per super-bucket
constexpr int kBucketLog = 15;
constexpr int kBucket = 1 << kBucketLog;       // positions per bucket (one bucket CTA)
constexpr int kSubPerSuper = kSuper / kBucket; // 32
constexpr int kBucketThreads = 512;            // threads of the bucket CTA
constexpr int kPartThreads = 512;              // threads of a partition CTA
constexpr int kPartBlocks = 4;                 // partition CTAs per SM (registers: 32 per thread)
constexpr int kPartPer = 8;                    // entries per thread per partition CTA
constexpr int kPartRound = kPartThreads * kPartPer;   // 4096 entries per partition CTA
constexpr uint32_t kEsc12 = 0xfffu;            // 12-bit length field of level 1: value in lbig
constexpr uint32_t kEsc17 = 0x1ffffu;          // 17-bit length field of level 2: value in lbig
constexpr int kCursorStride = 32;              // one 128-byte line per partition cursor
// Rank-window front end (rank without sa, one string): the pairs
// <rank[i], i> partitioned by rank into windows of 2^22 ranks, so that the
// lcp words of a window (16 MB) are gathered from L2.  Used from n = 2^24 on
// (below that, all of lcp fits in L2 and the plain gather is as good).
constexpr int kWinLog = 22;
constexpr int kMaxWins = 512;                  // n < 2^31
constexpr long long kRankWinMinN = 1LL << 24;

// Polls of a look-back status word before the wait is declared lost (a
// few seconds at most; the kernel then reports kErrTimeout and finishes).
constexpr int kSpinLimit = 1 << 23;

// Device scratch of one query, carved out of one allocation by the context.
struct Scratch {
    unsigned* tickets;             // [0] gather tiles, [1] buckets, [2] cover tiles
    unsigned* qerr;                // error bits of this query (cleared with the tickets)
    unsigned* err;                 // sticky device error bits (kErr*), read by the host
    unsigned long long* status_g;  // look-back words of the gather front end (per tile)
    unsigned long long* status_b;  // look-back words of the rank-order front end (per bucket)
    unsigned long long* status_o;  // look-back words of the cover kernel (per cover tile)
    int32_t* tile_cbase;           // ntiles + 1: compact LLR's starting before tile j
    int32_t* cstart;               // n: compact LLR starts (ascending)
    int32_t* cend;                 // n: compact LLR ends   (ascending)
    uint32_t* ent1;                // nsupers x 2^20: level-1 entries <pos mod 2^20, min(L, 4095)>
    uint32_t* ent2;                // nbuckets x 2^15: level-2 entries <pos mod 2^15, min(L, 2^17-1)>
    unsigned* cursor1;             // fill counts of ent1, one per kCursorStride words (cleared per query)
    unsigned* cursor2;             // fill counts of ent2, one per kCursorStride words (cleared per query)
    int32_t* lbig;                 // n: L of positions whose length field escaped
    int32_t* halo;                 // nbuckets + 1: L of the position before each bucket
    int32_t* tile_seg;             // ntiles: first string overlapping each tile (batched queries)
    int32_t* seg_cbase;            // nsegs + 1: compact LLR's starting before segment j (kSeg positions)
    unsigned long long* status_w;  // look-back words of the warp-segment cover kernel (per kSegTile tile)
    long long ntiles;
    long long nsegs;
    long long nbuckets;
    long long nsupers;
    void* zero_base;               // tickets, status words and cursors, cleared before every query
    size_t zero_bytes;
    unsigned* cursor_w = nullptr;  // fill counts of the rank windows, one per kCursorStride words (cleared
                                   // per query); null where the scratch has no room for the rank-window front
    unsigned long long* went = nullptr;   // n: rank-window entries rank << 32 | i (in the cstart / cend region)
    long long nwins = 0;
    int spin_limit = kSpinLimit;   // polls of one look-back wait before it gives up
    long long hold_tile = -1;      // test hook: this cover tile never publishes its look-back word
};

__host__ __device__ inline long long num_tiles(long long n) { return (n + kTile - 1) / kTile; }
__host__ __device__ inline long long num_cover_tiles(long long n, int tiles_per) {
    return (n + (long long)kTile * tiles_per - 1) / ((long long)kTile * tiles_per);
}
__host__ __device__ inline long long num_segs(long long n) { return (n + kSeg - 1) / kSeg; }
__host__ __device__ inline long long num_seg_tiles(long long n) { return (n + kSegTile - 1) / kSegTile; }
inline long long num_buckets(long long n) { return (n + kBucket - 1) / kBucket; }
inline long long num_supers(long long n) { return (n + kSuper - 1) / kSuper; }
inline long long num_wins(long long n) { return (n + (1LL << kWinLog) - 1) >> kWinLog; }

constexpr int kMaxPhases = 8;

// Optional per-kernel events: ev[i] is recorded before kernel i and
// ev[count] after the last one.
struct PhaseEvents {
    cudaEvent_t ev[kMaxPhases + 1];
    bool enabled = false;
    int count = 0;                 // phases recorded by the last query
};

// Strings of a batched query: string j occupies the flattened positions
// [off[j], off[j+1]); its local sa / rank live at the same offsets, its lcp
// (n_j + 1 entries) at off[j] + j.  num == 0 means one string, no table.
struct Segs {
    const int64_t* off;            // device, num + 1 entries
    long long num;
};
constexpr int kSegCap = 1024;      // strings per CTA a front end keeps in shared memory

// Kernel shape choices a query can take (picked by lr_autotune_*).
struct Shape {
    bool tile_cover = true;        // the tile cover kernel (else the warp-segment one)
    int cover_tiles_per = 2;       // its tile = kTile x this (1, 2 or 4)
};

// Launches the whole query on `stream`: the front end (rank-order when sa is
// non-null, else the rank gather) and the cover kernel.
cudaError_t launch_query(const int32_t* sa, const int32_t* rank, const int32_t* lcp, int32_t n, const Scratch& s,
                         int32_t* lr_len, int32_t* lr_start, int64_t* offsets, int32_t* starts,
                         long long capacity, bool all, cudaStream_t stream, int* launches,
                         PhaseEvents* events, const Segs& segs = Segs{nullptr, 0}, const Shape& shape = Shape{});

// Front ends (lr_front.cu) and the cover kernel (lr_cover.cu).
void launch_seg_index(int32_t n, const Scratch& s, const Segs& segs, cudaStream_t stream);
void launch_gather_front(const int32_t* rank, const int32_t* lcp, int32_t n, const Scratch& s, const Segs& segs,
                         cudaStream_t stream);
void launch_partition(const int32_t* sa, const int32_t* lcp, int32_t n, const Scratch& s, const Segs& segs,
                      cudaStream_t stream);
void launch_bucket_front(int32_t n, const Scratch& s, cudaStream_t stream);
// k_rank_win, k_part1_win and k_part2 (the rank-window front end up to the bucket kernel)
void launch_rank_window_front(const int32_t* rank, const int32_t* lcp, int32_t n, const Scratch& s,
                              cudaStream_t stream);
void launch_cover(int32_t n, const Scratch& s, int32_t* lr_len, int32_t* lr_start, int64_t* offsets,
                  int32_t* starts, long long capacity, bool all, int tiles_per, cudaStream_t stream);
void launch_cover_w(int32_t n, const Scratch& s, int32_t* lr_len, int32_t* lr_start, int64_t* offsets,
                    int32_t* starts, long long capacity, bool all, cudaStream_t stream);

cudaError_t configure_kernels();

// The raw-LLR variant (Algorithms 1 and 3 on the GPU, no compaction) and the
// walk statistics of Table 2 (lr_raw.cu).  Both keep LLRr in s.lbig.
cudaError_t launch_raw_query(const int32_t* rank, const int32_t* lcp, int32_t n, const Scratch& s, int32_t* lr_len,
                             int32_t* lr_start, int64_t* offsets, int32_t* starts, long long capacity, bool all,
                             cudaStream_t stream);
cudaError_t launch_walk_stats(const int32_t* rank, const int32_t* lcp, int32_t n, const Scratch& s, int32_t* alpha,
                              int32_t* beta, unsigned long long* stats, cudaStream_t stream);

// Suffix array, rank and lcp of device texts by prefix doubling
// (lr_index.cu).  IndexWork is the work memory for up to cap_n positions
// and cap_rounds doubling rounds (released explicitly).
struct IndexWork {
    unsigned char* base = nullptr;
    size_t bytes = 0;
    uint64_t *k0 = nullptr, *k1 = nullptr;
    int32_t *v0 = nullptr, *v1 = nullptr, *head = nullptr, *hp = nullptr, *end = nullptr, *levels = nullptr;
    uint8_t* sep = nullptr;        // per sorted index: the round at which it started a group
    unsigned long long* misc = nullptr;
    void* tmp = nullptr;
    size_t tmp_bytes = 0;
    long long cap_n = 0;
    int cap_rounds = 0;
    unsigned long long groups_host = 0;
    cudaError_t alloc(long long n, int rounds);
    void release();
};
size_t index_work_bytes(long long n, int rounds);
// Many strings (string j = text[off[j], off[j+1]), off on the device): sa and
// rank string-local at the strings' offsets, lcp (n_j + 1 entries) at
// off[j] + j.  Waits for `stream` once per round.
cudaError_t build_arrays_batch(const uint8_t* text, long long total, const int64_t* off, long long num, int32_t* sa,
                               int32_t* rank, int32_t* lcp, IndexWork& w, bool grow, cudaStream_t stream,
                               int* rounds_out);
// One string; allocates and frees its own work memory.
cudaError_t build_arrays(const uint8_t* text, int32_t n, int32_t* sa, int32_t* rank, int32_t* lcp,
                         cudaStream_t stream, int* rounds_out);

// Scratch management (lr_api.cu): bytes of a scratch block for n positions,
// and the carving of such a block (laid out for cap_n >= n) into `s`.
size_t scratch_size(long long n);
void carve_scratch(unsigned char* base, long long cap_n, long long n, unsigned* d_err, Scratch* s);
// The lr_status for the device error bits of a query.
lr_status status_of_bits(unsigned bits);

}  // namespace lr
