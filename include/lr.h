/*
 * lr.h -- C ABI of the GB300 longest-repeat query library (liblr.so).
 *
 * The library answers the longest repeat (LR) query of Tian and Xu, "On
 * Longest Repeat Queries Using GPU" (arXiv 1501.06663), Sec. 2: for every
 * position k of a string S[0..n), the longest substrings that cover k and
 * occur at least twice in S (overlapping occurrences count), or the fact
 * that none exists (S[k] is a singleton).  Several LR's may tie; the
 * "all" calls list every one of them.
 *
 * Inputs are the arrays the paper builds on the host before the query and
 * copies to the GPU (Sec. 4), here 0-based:
 *   sa[r]   = start of the r-th smallest suffix                  (int32, n entries)
 *   rank[i] = r  iff  sa[r] = i                                   (int32, n entries)
 *   lcp[0] = lcp[n] = 0, lcp[r] = |lcp(S[sa[r-1]..], S[sa[r]..])| for 0<r<n
 *                                                                  (int32, n+1 entries)
 * The string itself is not needed.  Lemma 1 gives the length of the
 * left-bounded longest repeat at i as L_i = max(lcp[rank[i]], lcp[rank[i]+1]),
 * which read in rank order is L_{sa[r]} = max(lcp[r], lcp[r+1]).  A query
 * takes sa or rank (at least one; when both are given, sa is used unless
 * lr_autotune chose the rank front end for queries of that size):
 *   - with sa, the lengths are computed in rank order (sa and lcp read
 *     once, coalesced) and radix-partitioned back to text order;
 *   - with rank only, each position gathers its two lcp words, the paper's
 *     own data flow (Sec. 4): one random 32-byte sector per position.  For
 *     one string of 2^24 positions or more (not a batch, not the static
 *     call), the pairs <rank[i], i> are first partitioned into windows of
 *     2^22 ranks, so that each window's gathers hit L2, and then join the
 *     sa path's partition.
 * All give identical results.  sa must be a permutation of [0, n) and rank
 * its inverse; a violation that the kernels detect is reported as
 * LR_ERR_SENTINEL, and no input ever makes a kernel access memory out of
 * bounds.
 *
 * Outputs, per position k (0-based):
 *   lr_len[k]    length of LR_k, 0 if none                          (int32)
 *   lr_start[k]  start of the leftmost LR_k, -1 if none             (int32)
 * and, for the "all" calls, a CSR list of every LR_k:
 *   offsets[k] .. offsets[k+1]  the range of starts[] for position k (int64, n+1)
 *   starts[j]    start positions, ascending within each k             (int32)
 * so lr_start[k] == starts[offsets[k]] whenever lr_len[k] > 0.
 *
 * Conventions for every call:
 *  - d_* pointers are device memory owned by the caller; h_* pointers are
 *    host memory.  No pointer is retained after the call returns.
 *  - Calls are asynchronous on `stream` (NULL = the legacy default stream)
 *    unless they take an h_* output, which makes them wait for the stream.
 *  - The library owns only its scratch (tile status words, the compact LLR
 *    array, the partition buffers: about 20 bytes per position; the device
 *    copies of lr_query_all_host; the work memory of the GPU array builds),
 *    cached in the context and grown on demand; a context must not be used
 *    from two host threads at once.
 *  - No C++ exception crosses this interface.  Errors are returned as
 *    lr_status.  Malformed device inputs (a rank outside [0, n), lcp[0] or
 *    lcp[n] not 0) are detected by the kernels, never read out of bounds,
 *    and reported through lr_device_status() (or by the synchronising calls).
 */
#ifndef LR_H_
#define LR_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LR_OK = 0,
    LR_ERR_ARG = 1,        /* null pointer, n out of [1, 2^31 - 2], bad option  */
    LR_ERR_SENTINEL = 2,   /* lcp[0] or lcp[n] is not 0, or a rank is out of range */
    LR_ERR_CAPACITY = 3,   /* starts_capacity < total; *h_total holds the total   */
    LR_ERR_NOMEM = 4,      /* a scratch allocation failed                          */
    LR_ERR_CUDA = 5,       /* a CUDA runtime call failed; see lr_last_cuda_error   */
    LR_ERR_TIMEOUT = 6,    /* a device-side wait gave up (results are invalid)    */
    LR_ERR_BUSY = 7        /* the serving engine has no room for the job           */
} lr_status;

typedef struct lr_ctx lr_ctx;
typedef struct CUstream_st* lr_stream_t;   /* same type as cudaStream_t */

/* Create a context bound to CUDA device `device`.  *ctx is NULL on failure. */
lr_status lr_create(lr_ctx** ctx, int device);
/* Free the context and its scratch.  Waits for work the context queued. */
lr_status lr_destroy(lr_ctx* ctx);
/* Human-readable name of a status code (static string). */
const char* lr_status_str(lr_status s);
/* The last cudaError_t value seen by the context (0 if none). */
lr_status lr_last_cuda_error(lr_ctx* ctx, int* code);

/*
 * Wait for `stream` and return the status the kernels of the context's
 * previous asynchronous calls recorded (LR_OK, LR_ERR_SENTINEL or
 * LR_ERR_TIMEOUT), then clear it.
 */
lr_status lr_device_status(lr_ctx* ctx, lr_stream_t stream);

/*
 * Leftmost LR of every position (Algorithm 2: compaction of the LLR array,
 * Sec. 3.2, then for each k the longest compact LLR covering k, the leftmost
 * on ties).  d_sa, d_rank: n int32 (one may be NULL); d_lcp: n+1 int32;
 * d_lr_start, d_lr_len: n int32 outputs.  Asynchronous.
 */
lr_status lr_query_leftmost(lr_ctx* ctx, lr_stream_t stream,
                            const int32_t* d_sa, const int32_t* d_rank, const int32_t* d_lcp, int32_t n,
                            int32_t* d_lr_start, int32_t* d_lr_len);

/*
 * All LR's of every position (Algorithm 4 / Corollary 2: compaction, then
 * the longest length per position and every compact LLR of that length that
 * covers it), as the CSR described above.
 *   d_offsets       n+1 int64 output; d_offsets[n] is the total
 *   d_starts        output of starts_capacity int32 entries; entries past
 *                   the capacity are not written
 *   h_total         optional host output.  If non-NULL the call waits for
 *                   `stream`, stores the total and returns LR_ERR_CAPACITY
 *                   when it exceeds starts_capacity (lr_len, lr_start and
 *                   offsets are still complete), or a device status.  If
 *                   NULL the call is asynchronous; read d_offsets[n] and
 *                   lr_device_status() later.
 */
lr_status lr_query_all(lr_ctx* ctx, lr_stream_t stream,
                       const int32_t* d_sa, const int32_t* d_rank, const int32_t* d_lcp, int32_t n,
                       int32_t* d_lr_len, int32_t* d_lr_start,
                       int64_t* d_offsets, int32_t* d_starts, int64_t starts_capacity,
                       int64_t* h_total);

/*
 * lr_query_all on host buffers: copies sa (or rank) and lcp to device memory owned
 * by the context, runs the query on `stream`, copies the results back and
 * waits.  h_starts holds starts_capacity entries; *h_total receives the
 * total, and LR_ERR_CAPACITY is returned if it does not fit (the other
 * outputs are complete).  Host buffers may be pageable; pinned buffers copy
 * faster.
 */
lr_status lr_query_all_host(lr_ctx* ctx, lr_stream_t stream,
                            const int32_t* h_sa, const int32_t* h_rank, const int32_t* h_lcp, int32_t n,
                            int32_t* h_lr_len, int32_t* h_lr_start,
                            int64_t* h_offsets, int32_t* h_starts, int64_t starts_capacity,
                            int64_t* h_total);

/*
 * The step before the query: sa, rank and lcp of device text, built on the
 * GPU.  The paper builds these arrays on the host and notes they could be
 * built in parallel on the GPU by prefix doubling (Sec. 4); these calls do
 * that: radix sorts of (string index, first symbols) keys, then of
 * (rank(i), rank(i + h)) pairs of the suffixes not yet told apart, for
 * doubling h until all ranks differ, and
 * the lcp of sa neighbours from the round at which they parted plus binary
 * lifting over the ranks of the earlier rounds.
 *
 * lr_build_arrays: one string, d_text n bytes (any values); outputs in the
 * layout the queries take: d_sa and d_rank n entries, d_lcp n + 1
 * (lcp[0] = lcp[n] = 0).
 * lr_batch_build_arrays: many strings packed back to back, in the layout of
 * lr_batch_desc: string j = d_text[d_off[j], d_off[j+1]) (empty strings
 * allowed); its local sa and rank at the same offsets of d_sa / d_rank, its
 * lcp (n_j + 1 entries) at d_lcp + d_off[j] + j (total + num entries).
 *
 * Work memory, about (37 + 4 R) bytes per position for R doubling rounds
 * (R is about log2 of the longest repeat / c, plus 2, c = 7 .. 63 symbols
 * per round-0 key by the alphabet size), is kept in the
 * context and grown on demand (LR_ERR_NOMEM when it does not fit).  A batch
 * of more than 2^29 positions is built in chunks of whole strings of at
 * most 2^29 positions (one string longer than that is a chunk of its own),
 * so its work memory follows the chunk; its offset table is then also
 * checked on the host.  Both calls wait for `stream` (once per round);
 * *rounds (may be NULL) receives R (the largest over the chunks).
 * An offset table that does not start at 0, end at total or never
 * decrease is reported as LR_ERR_SENTINEL before any symbol is read.
 */
typedef struct {
    int64_t num;                /* number of strings (>= 1) */
    int64_t total;              /* d_off[num]: total symbols, 0 <= total <= 2^31 - 2 */
    const int64_t* d_off;       /* num + 1 device offsets, d_off[0] = 0, non-decreasing */
    const uint8_t* d_text;      /* total bytes */
} lr_text_batch;

lr_status lr_build_arrays(lr_ctx* ctx, lr_stream_t stream, const uint8_t* d_text, int32_t n,
                          int32_t* d_sa, int32_t* d_rank, int32_t* d_lcp, int32_t* rounds);
lr_status lr_batch_build_arrays(lr_ctx* ctx, lr_stream_t stream, const lr_text_batch* batch,
                                int32_t* d_sa, int32_t* d_rank, int32_t* d_lcp, int32_t* rounds);

/*
 * The raw-LLR variant (Sec. 3.1, Algorithms 1 and 3; the paper's GPU
 * kernels K_LLRr and K_rawwalk of Sec. 4.1): no compaction; every position
 * walks left over the raw LLR array LLRr while the LLR's it meets cover it.
 * The results are exactly those of lr_query_all / lr_query_leftmost; the
 * cost is the sum of the walk lengths, about alpha per position (Table 2),
 * which the paper compares against the compact array.  Takes rank (text
 * order) and lcp only; arguments, outputs and errors as lr_query_all /
 * lr_query_leftmost.
 */
lr_status lr_query_all_raw(lr_ctx* ctx, lr_stream_t stream, const int32_t* d_rank, const int32_t* d_lcp,
                           int32_t n, int32_t* d_lr_len, int32_t* d_lr_start,
                           int64_t* d_offsets, int32_t* d_starts, int64_t starts_capacity, int64_t* h_total);
lr_status lr_query_leftmost_raw(lr_ctx* ctx, lr_stream_t stream, const int32_t* d_rank, const int32_t* d_lcp,
                                int32_t n, int32_t* d_lr_start, int32_t* d_lr_len);

/*
 * Walk statistics of Table 2 on the device: alpha_k, the number of raw LLR's
 * covering position k (the steps of Algorithm 1's walk that meet a covering
 * LLR), and beta_k, the number of compact (useful, Sec. 3.2) LLR's covering
 * k.  d_alpha / d_beta (n entries each) receive the per-position values when
 * non-NULL; *h_summary receives n, m = |LLRc|, the sums, minima and maxima
 * (the call waits for `stream`).  Errors as lr_query_all.
 */
typedef struct {
    int64_t n, m;
    int64_t alpha_sum, beta_sum;
    int32_t alpha_min, alpha_max, beta_min, beta_max;
} lr_walk_summary;

lr_status lr_walk_stats(lr_ctx* ctx, lr_stream_t stream, const int32_t* d_rank, const int32_t* d_lcp, int32_t n,
                        int32_t* d_alpha, int32_t* d_beta, lr_walk_summary* h_summary);

/*
 * Batched query: many strings of uneven length in one set of launches over
 * a flattened position space (the strings back to back).  String j owns the
 * flattened positions [d_off[j], d_off[j+1]); its own (local, 0-based) sa or
 * rank array sits at the same offsets of d_sa / d_rank, and its lcp array
 * (n_j + 1 entries, lcp[0] = lcp[n_j] = 0) at d_lcp + d_off[j] + j.  Empty
 * strings are allowed.  The outputs cover the flattened positions; lr_start
 * and starts hold flattened positions (subtract d_off[j] for string-local
 * ones).  The per-string results are exactly those of lr_query_all run on
 * each string alone.  LLR's never run past their string (an lcp value is at
 * most the suffix length), so compact LLR's of consecutive strings keep
 * strictly increasing starts and ends and the flattened cover step needs
 * no string boundaries; only Lemma 1 reads the string table.
 */
typedef struct {
    int64_t num;                /* number of strings (>= 1) */
    int64_t total;              /* d_off[num]: flattened positions, 1 <= total <= 2^31 - 2 */
    const int64_t* d_off;       /* num + 1 device offsets, d_off[0] = 0, non-decreasing */
    const int32_t* d_sa;        /* flattened local suffix arrays, or NULL */
    const int32_t* d_rank;      /* flattened local rank arrays, or NULL (sa wins when both are given) */
    const int32_t* d_lcp;       /* flattened local lcp arrays, total + num entries */
} lr_batch_desc;

lr_status lr_batch_query_all(lr_ctx* ctx, lr_stream_t stream, const lr_batch_desc* batch,
                             int32_t* d_lr_len, int32_t* d_lr_start,
                             int64_t* d_offsets, int32_t* d_starts, int64_t starts_capacity,
                             int64_t* h_total);

/*
 * Autotuning.  Kernel shape choices (the cover kernel: warp segments of 256
 * positions, or CTA tiles of 2048, 4096 or 8192 positions; the front end,
 * when both sa and rank are given) are timed on the given batch (a single
 * string is a batch with num = 1) and the fastest is remembered in the
 * context for batches of the same shape class (total size and mean string
 * length, both rounded to powers of two).  Later queries of that class use
 * it; the default is the tile cover with 4096-position tiles and the
 * rank-order front end (code 9).  *choice receives the chosen shape code: bit 3 clear: the
 * warp-segment cover (bits 0 and 2 clear); bit 3 set: the tile cover, with
 * bit 0: 4096-position tiles, bit 2: 8192-position tiles, neither: 2048;
 * bit 1: the rank front end (timed as the rank gather; a single query of
 * 2^24 positions or more with this code takes the rank windows).  The outputs are overwritten.
 * lr_autotune_save / _load write and read the remembered choices as a small
 * text file (one "class code" pair per line; invalid codes are skipped).
 */
lr_status lr_autotune(lr_ctx* ctx, lr_stream_t stream, const lr_batch_desc* batch,
                      int32_t* d_lr_len, int32_t* d_lr_start, int64_t* d_offsets, int32_t* d_starts,
                      int64_t starts_capacity, int32_t* choice);
lr_status lr_autotune_save(lr_ctx* ctx, const char* path);
lr_status lr_autotune_load(lr_ctx* ctx, const char* path);

/*
 * Captured plans: the launch sequence of one batched query with fixed
 * inputs, outputs and sizes, captured once into a CUDA graph (with its own
 * scratch, owned by the plan) and replayed by lr_plan_launch.  For batch
 * shapes that repeat, it removes the per-launch host overhead.  The plan
 * keeps the device pointers it was created with: refill those buffers in
 * place between launches.  The shape is the context's tuned choice at
 * creation time.  Launches of one plan must not overlap (they share its
 * scratch): issue them on one stream.  lr_plan_launch only enqueues;
 * lr_plan_result waits for the stream, stores the number of LR starts of
 * the last launch in *h_total (when non-NULL) and reports its input errors
 * (LR_ERR_SENTINEL), timeouts and LR_ERR_CAPACITY.  lr_plan_destroy waits
 * for the device and frees everything the plan owns.
 */
typedef struct lr_plan lr_plan;
lr_status lr_plan_create(lr_ctx* ctx, const lr_batch_desc* batch,
                         int32_t* d_lr_len, int32_t* d_lr_start, int64_t* d_offsets, int32_t* d_starts,
                         int64_t starts_capacity, lr_plan** plan);
lr_status lr_plan_launch(lr_plan* plan, lr_stream_t stream);
lr_status lr_plan_result(lr_plan* plan, lr_stream_t stream, int64_t* h_total);
lr_status lr_plan_destroy(lr_plan* plan);

/*
 * Serving: a request loop with continuous batching (no paper counterpart;
 * it drives the batched query of lr_batch_query_all).
 *
 * The server owns `slots` batch slots in device memory, each holding the
 * inputs, outputs and scratch of one batch of up to max_batch_positions
 * positions and max_batch_jobs jobs.  At start it sizes them from the free
 * HBM (hbm_fraction of what cudaMemGetInfo reports) and fails with
 * LR_ERR_NOMEM if not even one slot fits.  A submitted job waits in a queue
 * until the slot being filled has room for it (HBM-based admission); its
 * sa (or rank) and lcp are then copied to the device and stay resident in
 * the slot until its results are back in host memory.  The slot being
 * filled is closed and launched (one batched query, then a kernel that
 * makes every job's results string-local) when it is full, when fewer than
 * max_inflight slots are on the GPU, or when its oldest job has waited
 * batch_window_us.  Jobs that arrive while other slots run are admitted into
 * the next slot, and the copies of one slot overlap the kernels of another
 * (one CUDA stream per slot).  A batch whose device checks report an input
 * error is re-run one job at a time so that only the offending job fails.
 * Each job's results equal those of lr_query_all on that job alone.
 *
 * A worker thread inside the library runs the loop; all functions here are
 * thread-safe.  Host buffers of a job must stay valid until the job is done
 * or cancelled; page-locked (pinned) buffers let the copies run
 * asynchronously.
 */
typedef struct lr_server lr_server;

typedef struct {
    int32_t device;
    int32_t slots;                 /* batch slots; 0 = 4 */
    int32_t max_inflight;          /* slots on the GPU at once; 0 = 2 */
    int64_t max_batch_positions;   /* positions per slot; 0 = 2^26 */
    int32_t max_batch_jobs;        /* jobs per slot; 0 = 4096 */
    int32_t max_queue;             /* queued jobs before lr_server_submit answers LR_ERR_BUSY; 0 = 65536 */
    int32_t batch_window_us;       /* longest wait of an admitted job while other slots run; 0 = 2000 */
    double hbm_fraction;           /* share of the free device memory the slots may take; 0 = 0.5 */
    double starts_factor;          /* initial starts buffer of a slot, in entries per position; 0 = 2
                                      (it grows, within the budget, when a batch needs more) */
    int32_t text_jobs;             /* nonzero: slots also take text jobs (sa / rank / lcp built on
                                      the GPU; about 90 more bytes of device memory per position) */
} lr_server_config;

typedef struct {
    const int32_t* h_sa;           /* host, n entries, or NULL */
    const int32_t* h_rank;         /* host, n entries, or NULL (sa wins when both are given) */
    const int32_t* h_lcp;          /* host, n + 1 entries; NULL for a text job */
    int32_t n;                     /* 1 <= n <= max_batch_positions */
    int32_t* h_lr_len;             /* host outputs, as lr_query_all: n */
    int32_t* h_lr_start;           /* n, string-local positions */
    int64_t* h_offsets;            /* n + 1 */
    int32_t* h_starts;             /* starts_capacity entries (NULL when 0) */
    int64_t starts_capacity;
    const uint8_t* h_text;         /* text job: the string itself (n bytes) and no sa, rank or lcp; its
                                      arrays are built on the GPU with the rest of its batch
                                      (lr_batch_build_arrays); needs a server started with text_jobs */
} lr_job;

enum { LR_JOB_QUEUED = 0, LR_JOB_ADMITTED = 1, LR_JOB_RUNNING = 2, LR_JOB_DONE = 3, LR_JOB_CANCELLED = 4 };

typedef struct {
    int64_t submitted, completed, cancelled, failed;   /* jobs */
    int64_t batches, positions;                        /* batches launched, positions completed */
    double p50_us, p99_us, mean_us, max_us;            /* submit-to-done latency of completed jobs */
    int32_t slots;
    int64_t slot_positions;
    int64_t device_bytes;                              /* device memory the server holds */
} lr_server_stats;

/* Starts the worker thread.  cfg may be NULL (all defaults, device 0). */
lr_status lr_server_start(const lr_server_config* cfg, lr_server** server);
/* Queues a job; *job_id identifies it.  LR_ERR_BUSY: the queue is full;
 * LR_ERR_NOMEM: the job can never fit a slot; LR_ERR_ARG: bad job. */
lr_status lr_server_submit(lr_server* server, const lr_job* job, int64_t* job_id);
/* Non-blocking: *state = LR_JOB_*.  For a done job *result is its status
 * (LR_OK; LR_ERR_CAPACITY with *total the needed size, lr_len, lr_start and
 * offsets still written; LR_ERR_SENTINEL for bad input ...) and *total its
 * number of LR starts.  A job's record is dropped once poll or wait has
 * reported it done or cancelled (later calls on its id: LR_ERR_ARG).
 * result and total may be NULL. */
lr_status lr_server_poll(lr_server* server, int64_t job_id, int32_t* state, lr_status* result, int64_t* total);
/* Waits up to timeout_ms (< 0: no limit) until the job is done or
 * cancelled; LR_ERR_TIMEOUT if it is not.  Outputs as for poll (state may
 * be NULL). */
lr_status lr_server_wait(lr_server* server, int64_t job_id, int32_t timeout_ms, int32_t* state,
                         lr_status* result, int64_t* total);
/* Cancels a job still in the queue; LR_ERR_BUSY once it has been admitted. */
lr_status lr_server_cancel(lr_server* server, int64_t job_id);
/* Counters and latency percentiles; reset != 0 clears them afterwards. */
lr_status lr_server_stats_get(lr_server* server, int32_t reset, lr_server_stats* stats);
/* Cancels queued jobs, finishes admitted ones, stops the thread and frees
 * everything the server holds. */
lr_status lr_server_stop(lr_server* server);

/*
 * lr_query_all_static -- lr_query_all for callers that cannot allocate.
 *
 * The paper has no counterpart of this entry point; it exists for library
 * users who are not allowed to allocate device memory at query time: code
 * that runs inside another framework's per-request callback (where a device
 * allocation would synchronise the whole device and stall unrelated work),
 * or services that fix their memory budget once at start-up.  It needs no
 * context and allocates nothing: its working memory is one array of about
 * 8 MB compiled into this library's device image, which every GPU that
 * loads the library keeps until the process exits.
 *
 * Same inputs and outputs as lr_query_all with rank (the rank-gather front
 * end), for 1 <= n <= LR_STATIC_MAX_N; larger n is rejected with
 * LR_ERR_ARG (use lr_query_all).  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current);
 * make that first call before any stream capture.  All calls on a device
 * share the one array and leave their contents in it (the parts that must
 * start at zero are cleared by every call), so calls on the same device
 * must not overlap on the GPU: two streams running it at the same time
 * race.  Errors of the kernels (bad input, a lost wait) are only reported
 * when h_total is given, which makes the call wait for `stream`.
 */
#define LR_STATIC_MAX_N 1048576
lr_status lr_query_all_static(lr_stream_t stream,
                              const int32_t* d_rank, const int32_t* d_lcp, int32_t n,
                              int32_t* d_lr_len, int32_t* d_lr_start,
                              int64_t* d_offsets, int32_t* d_starts, int64_t starts_capacity,
                              int64_t* h_total);

/*
 * Test hook for the bounded device-side waits (off by default; changes no
 * result while off).  Every kernel that waits for another CTA's look-back
 * status word gives up after a bounded number of polls, records a timeout
 * and finishes, so a lost wait never hangs the GPU; this hook makes such a
 * wait run out on purpose without any fault.  While it is on, the cover
 * kernel's look-back unit number `tile` (a tile of 4096 positions with the
 * default warp-segment cover or with the tile cover's default shape) never
 * publishes its status word, and every look-back wait of the context's
 * queries gives up after `spin_limit` polls (1 .. 2^23; the default is
 * 2^23).  A query whose cover has more than tile + 1 units then waits for a
 * word that nothing sets, gives up, and reports LR_ERR_TIMEOUT
 * (through h_total or lr_device_status); its outputs are invalid.  tile < 0
 * switches the hook off and restores the default limit; the context stays
 * usable throughout.  LR_ERR_ARG for a spin_limit out of range.
 */
lr_status lr_test_hold_lookback(lr_ctx* ctx, int64_t tile, int32_t spin_limit);

/*
 * Kernels launched by the most recent query of this context (for the
 * benchmark's launch accounting): 4 with sa, 2 with rank only, one more for
 * a batch; 2 for the raw-LLR variant, 4 for lr_walk_stats.
 */
int32_t lr_last_launch_count(lr_ctx* ctx);

/*
 * Per-kernel timing (instrumentation, off by default).  While enabled, each
 * query records a CUDA event on its stream before and after every kernel it
 * launches.  lr_phase_times() waits for the last query's events and writes
 * the duration in milliseconds of each of its phases, in launch order, into
 * ms[0 .. cap); it returns the number of phases of that query, or -1 if
 * timing was off or an event failed.  The phases are: with sa, the
 * partition (two kernels), the bucket front end and the cover kernel;
 * with rank only, the gather front end and the cover kernel.
 */
lr_status lr_set_phase_timing(lr_ctx* ctx, int32_t enable);
int32_t lr_phase_times(lr_ctx* ctx, float* ms, int32_t cap);

/*
 * Size of the compact LLR array of the context's last query (the number of
 * useful LLR's, Sec. 3.2), read back after waiting for `stream`.
 */
lr_status lr_last_compact_size(lr_ctx* ctx, lr_stream_t stream, int64_t* m);

#ifdef __cplusplus
}
#endif

#endif /* LR_H_ */
