// Launch sequence of one longest-repeat query on a stream: clear the
// per-query status words, run a front end (lr_front.cu) that builds the
// compact LLR array (rank order from sa; rank windows from rank alone for
// one long string; else the rank gather), then a cover kernel (the tile
// cover of lr_cover.cu by default, or the warp-segment cover of
// lr_cover_w.cu when the shape asks for it).
#include <cuda_runtime.h>
#include <cstdint>
#include "lr_internal.h"

namespace lr {

cudaError_t configure_front();
cudaError_t configure_cover();
cudaError_t configure_cover_w();

cudaError_t configure_kernels() {
    cudaError_t e = configure_front();
    if (e == cudaSuccess) e = configure_cover();
    return e == cudaSuccess ? configure_cover_w() : e;
}

cudaError_t launch_query(const int32_t* sa, const int32_t* rank, const int32_t* lcp, int32_t n, const Scratch& s,
                         int32_t* lr_len, int32_t* lr_start, int64_t* offsets, int32_t* starts,
                         long long capacity, bool all, cudaStream_t stream, int* launches,
                         PhaseEvents* events, const Segs& segs, const Shape& shape) {
    cudaError_t e = cudaMemsetAsync(s.zero_base, 0, s.zero_bytes, stream);
    if (e != cudaSuccess) return e;
    const bool timed = events && events->enabled;
    int k = 0;
    auto mark = [&]() { if (timed) cudaEventRecord(events->ev[k], stream); ++k; };
    if (segs.num > 0) launch_seg_index(n, s, segs, stream);                     // k_seg_index
    const bool rankwin = !sa && segs.num == 0 && s.cursor_w && (long long)n >= kRankWinMinN;
    if (sa) {
        mark();
        launch_partition(sa, lcp, n, s, segs, stream);      // k_part1, k_part2
        mark();
        launch_bucket_front(n, s, stream);                  // k_bucket_llr
    } else if (rankwin) {
        mark();
        launch_rank_window_front(rank, lcp, n, s, stream);  // k_rank_win, k_part1_win, k_part2
        mark();
        launch_bucket_front(n, s, stream);                  // k_bucket_llr
    } else {
        mark();
        launch_gather_front(rank, lcp, n, s, segs, stream); // k_gather_llr
    }
    mark();
    if (shape.tile_cover)
        launch_cover(n, s, lr_len, lr_start, offsets, starts, capacity, all, shape.cover_tiles_per, stream);
    else
        launch_cover_w(n, s, lr_len, lr_start, offsets, starts, capacity, all, stream);
    if (timed) cudaEventRecord(events->ev[k], stream);
    if (launches) *launches = (sa ? 4 : (rankwin ? 5 : 2)) + (segs.num > 0 ? 1 : 0);
    if (events) events->count = k;
    return cudaGetLastError();
}

}  // namespace lr
