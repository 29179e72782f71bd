// Serving loop of liblr (declared in include/lr.h): continuous batching of
// query jobs over slots of device memory.  A worker thread admits queued
// jobs into the slot being filled (host-to-device copies on that slot's
// stream), closes and launches slots (one batched query plus a kernel that
// makes the results string-local), and copies each job's results back.
// Stream callbacks only wake the worker; every CUDA call is made with the
// server lock released.
#include <cuda_runtime.h>
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>
#include "lr.h"
#include "lr_internal.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr size_t kAlignS = 256;
constexpr int kTextRounds = 12;                      // doubling rounds a text slot holds (grown on demand)
inline size_t align_s(size_t v) { return (v + kAlignS - 1) / kAlignS * kAlignS; }

// Turns the flattened results of a batched query into per-job ones: every
// lr_start and start loses its string's offset, and job j's CSR offsets are
// rebased to 0 and written to loc_off[off[j] + j ..] (n_j + 1 entries, the
// lcp layout).  job_total[j] = number of LR starts of job j.  Strings are
// non-empty.  One thread per flattened position.
__global__ void k_localize(int32_t total, int32_t num, const int64_t* __restrict__ off,
                           const int64_t* __restrict__ offsets, int32_t* __restrict__ lr_start,
                           int32_t* __restrict__ starts, long long capacity, int64_t* __restrict__ loc_off,
                           int64_t* __restrict__ job_total) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    int lo = 0, hi = num - 1;                       // the last j with off[j] <= g
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= g) lo = mid; else hi = mid - 1;
    }
    const long long a = __ldg(off + lo);
    const long long oa = __ldg(offsets + a);
    const long long o0 = __ldg(offsets + g), o1 = __ldg(offsets + g + 1);
    const int32_t st = lr_start[g];
    if (st >= 0) lr_start[g] = (int32_t)(st - a);
    loc_off[g + lo] = o0 - oa;
    const long long t1 = o1 < capacity ? o1 : capacity;
    for (long long t = o0; t < t1; ++t) starts[t] -= (int32_t)a;
    if (g + 1 == __ldg(off + lo + 1)) {
        loc_off[g + 1 + lo] = o1 - oa;
        job_total[lo] = o1 - oa;
    }
}

enum JobKind { kSaJob, kRankJob, kTextJob };

struct Job {
    int64_t id = 0;
    lr_job spec{};
    JobKind kind = kSaJob;
    int32_t state = LR_JOB_QUEUED;
    lr_status result = LR_OK;
    int64_t total = 0;
    Clock::time_point t_submit;
    int64_t off = 0;                                 // flattened offset inside its slot
    int idx = 0;                                     // index inside its slot's batch
};

enum SlotState { kFree, kFilling, kReady, kRunning };

struct Slot {
    lr_server* srv = nullptr;
    SlotState state = kFree;
    int phase = 0;                                   // 1: query in flight, 2: result copies in flight
    bool signaled = false;                           // set by the stream callback
    bool blocked = false;                            // the queue head did not fit
    bool copy_failed = false;                        // a host-to-device copy of an admitted job failed
    cudaStream_t stream = nullptr;
    unsigned char* mem = nullptr;
    int32_t *d_in = nullptr, *d_lcp = nullptr, *d_len = nullptr, *d_start = nullptr, *d_starts = nullptr;
    int64_t *d_off = nullptr, *d_offsets = nullptr, *d_locoff = nullptr, *d_jobtot = nullptr;
    unsigned* d_err = nullptr;
    unsigned char* scratch = nullptr;
    int64_t cap = 0;                                 // entries of d_starts
    int64_t* h_off = nullptr;                        // pinned: offsets table, then job totals, then error bits
    int64_t* h_jobtot = nullptr;
    unsigned* h_err = nullptr;
    std::vector<Job*> jobs;
    int64_t used = 0;
    JobKind kind = kSaJob;
    uint8_t* d_text = nullptr;                       // text jobs: the strings, and the build's work memory
    lr::IndexWork index_work;
    Clock::time_point t_first;
};

}  // namespace

struct lr_server {
    int device = 0;
    lr_server_config cfg{};
    int64_t P = 0;                                   // positions per slot
    int32_t J = 0;                                   // jobs per slot
    int nslots = 0;
    std::unique_ptr<Slot[]> slots;
    size_t budget = 0;
    std::atomic<int64_t> device_bytes{0};

    std::mutex mu;
    std::condition_variable cv;                      // wakes the worker
    std::condition_variable cv_done;                 // wakes waiters
    std::deque<Job*> queue;
    int64_t queued = 0;                              // QUEUED jobs (the deque may hold cancelled ones)
    std::unordered_map<int64_t, Job*> jobs;
    int64_t next_id = 1;
    bool stopping = false;
    int filling = -1;
    std::deque<int> ready;
    int running = 0;
    std::thread worker;
    // text slots are launched by builder threads: their array build waits on
    // the stream once per doubling round, which would stall the worker
    std::vector<std::thread> builders;
    std::deque<int> to_build;
    std::condition_variable cv_build;
    bool builders_stop = false;

    int64_t submitted = 0, completed = 0, cancelled = 0, failed = 0, batches = 0, positions = 0;
    std::vector<double> lat_us;
};

namespace {

void CUDART_CB on_stream_done(void* p) {
    Slot* s = static_cast<Slot*>(p);
    std::lock_guard<std::mutex> lk(s->srv->mu);
    s->signaled = true;
    s->srv->cv.notify_one();
}

// Device bytes of one slot (without d_starts) for P positions and J jobs.
struct SlotLayout {
    size_t in, lcp, off, len, start, offsets, locoff, jobtot, err, scratch, text, total;
};

SlotLayout slot_layout(int64_t P, int32_t J, bool text) {
    SlotLayout L;
    size_t o = 0;
    L.in = o;       o = align_s(o + (size_t)P * 4);
    L.lcp = o;      o = align_s(o + (size_t)(P + J) * 4);
    L.off = o;      o = align_s(o + (size_t)(J + 1) * 8);
    L.len = o;      o = align_s(o + (size_t)P * 4);
    L.start = o;    o = align_s(o + (size_t)P * 4);
    L.offsets = o;  o = align_s(o + (size_t)(P + 1) * 8);
    L.locoff = o;   o = align_s(o + (size_t)(P + J) * 8);
    L.jobtot = o;   o = align_s(o + (size_t)J * 8);
    L.err = o;      o = align_s(o + 256);
    L.scratch = o;  o = align_s(o + lr::scratch_size(P));
    L.text = o;     o = align_s(o + (text ? (size_t)P : 0));
    L.total = o;
    return L;
}

void free_slot(Slot& s) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    if (s.mem) cudaFree(s.mem);
    if (s.d_starts) cudaFree(s.d_starts);
    if (s.h_off) cudaFreeHost(s.h_off);
    s.index_work.release();
    if (s.stream) cudaStreamDestroy(s.stream);
    s.mem = nullptr; s.d_starts = nullptr; s.h_off = nullptr; s.stream = nullptr;
}

cudaError_t alloc_slot(lr_server* S, Slot& s, const SlotLayout& L, int64_t cap) {
    s.srv = S;
    cudaError_t e = cudaMalloc((void**)&s.mem, L.total);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s.d_starts, (size_t)cap * 4);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&s.h_off, (size_t)(2 * S->J + 2) * 8 + 64);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { cudaGetLastError(); return e; }
    s.cap = cap;
    unsigned char* b = s.mem;
    s.d_in = (int32_t*)(b + L.in);
    s.d_lcp = (int32_t*)(b + L.lcp);
    s.d_off = (int64_t*)(b + L.off);
    s.d_len = (int32_t*)(b + L.len);
    s.d_start = (int32_t*)(b + L.start);
    s.d_offsets = (int64_t*)(b + L.offsets);
    s.d_locoff = (int64_t*)(b + L.locoff);
    s.d_jobtot = (int64_t*)(b + L.jobtot);
    s.d_err = (unsigned*)(b + L.err);
    s.scratch = b + L.scratch;
    s.d_text = S->cfg.text_jobs ? b + L.text : nullptr;
    if (S->cfg.text_jobs) {
        e = s.index_work.alloc(S->P, kTextRounds);
        if (e != cudaSuccess) return e;
        S->device_bytes += (int64_t)s.index_work.bytes;
    }
    s.h_jobtot = s.h_off + (S->J + 1);
    s.h_err = (unsigned*)(s.h_jobtot + S->J);
    S->device_bytes += (int64_t)L.total + cap * 4;
    return cudaSuccess;
}

// Grows d_starts to hold `need` entries if the budget allows.  The slot's
// stream is idle.
bool grow_starts(lr_server* S, Slot& s, int64_t need) {
    int64_t want = std::max(need, s.cap * 2);
    const int64_t have = S->device_bytes.load();
    if (have + (want - s.cap) * 4 > (int64_t)S->budget) want = need;
    if (have + (want - s.cap) * 4 > (int64_t)S->budget) return false;
    int32_t* p = nullptr;
    if (cudaMalloc((void**)&p, (size_t)want * 4) != cudaSuccess) { cudaGetLastError(); return false; }
    cudaFree(s.d_starts);
    S->device_bytes += (want - s.cap) * 4;
    s.d_starts = p;
    s.cap = want;
    return true;
}

cudaError_t launch_batch(lr_server* S, Slot& s) {
    const int num = (int)s.jobs.size();
    s.h_off[0] = 0;
    for (int j = 0; j < num; ++j) s.h_off[j + 1] = s.h_off[j] + s.jobs[j]->spec.n;
    const int32_t total = (int32_t)s.used;
    cudaError_t e = cudaMemcpyAsync(s.d_off, s.h_off, (size_t)(num + 1) * 8, cudaMemcpyHostToDevice, s.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.d_err, 0, 4, s.stream);
    if (e != cudaSuccess) return e;
    if (s.kind == kTextJob) {
        // sa (into d_in), rank (into d_len, overwritten by the query) and
        // lcp of every string of the batch, built on the GPU; this waits for
        // the slot's stream once per doubling round
        const int64_t before = (int64_t)s.index_work.bytes;
        e = lr::build_arrays_batch(s.d_text, total, s.d_off, num, s.d_in, s.d_len, s.d_lcp, s.index_work, true,
                                   s.stream, nullptr);
        S->device_bytes += (int64_t)s.index_work.bytes - before;
        if (e != cudaSuccess) return e;
    }
    const bool use_sa = s.kind != kRankJob;
    lr::Scratch sc;
    lr::carve_scratch(s.scratch, S->P, total, s.d_err, &sc);
    e = lr::launch_query(use_sa ? s.d_in : nullptr, use_sa ? nullptr : s.d_in, s.d_lcp, total, sc, s.d_len,
                         s.d_start, s.d_offsets, s.d_starts, s.cap, true, s.stream, nullptr, nullptr,
                         lr::Segs{s.d_off, num}, lr::Shape{});
    if (e != cudaSuccess) return e;
    k_localize<<<(unsigned)((total + 255) / 256), 256, 0, s.stream>>>(total, num, s.d_off, s.d_offsets, s.d_start,
                                                                       s.d_starts, s.cap, s.d_locoff, s.d_jobtot);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s.h_jobtot, s.d_jobtot, (size_t)num * 8, cudaMemcpyDeviceToHost, s.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.h_err, s.d_err, 4, cudaMemcpyDeviceToHost, s.stream);
    s.phase = 1;
    if (e == cudaSuccess) e = cudaLaunchHostFunc(s.stream, on_stream_done, &s);
    return e;
}

// Copies job j's results (string-local, in the slot) to its host buffers.
cudaError_t copy_out(Slot& s, int j, int64_t base) {
    Job* job = s.jobs[j];
    const lr_job& q = job->spec;
    cudaError_t e = cudaMemcpyAsync(q.h_lr_len, s.d_len + job->off, (size_t)q.n * 4, cudaMemcpyDeviceToHost, s.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(q.h_lr_start, s.d_start + job->off, (size_t)q.n * 4, cudaMemcpyDeviceToHost, s.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(q.h_offsets, s.d_locoff + job->off + j, (size_t)(q.n + 1) * 8, cudaMemcpyDeviceToHost,
                            s.stream);
    if (e == cudaSuccess && job->result == LR_OK && job->total > 0)
        e = cudaMemcpyAsync(q.h_starts, s.d_starts + base, (size_t)job->total * 4, cudaMemcpyDeviceToHost, s.stream);
    return e;
}

// Runs the slot's jobs one at a time (after a batch reported an input error
// or outgrew its starts buffer), waiting for each.
void run_solo(lr_server* S, Slot& s) {
    for (int j = 0; j < (int)s.jobs.size(); ++j) {
        Job* job = s.jobs[j];
        const int32_t n = job->spec.n;
        int64_t* d_loc = s.d_locoff + job->off + j;
        for (int attempt = 0; attempt < 2; ++attempt) {
            lr::Scratch sc;
            lr::carve_scratch(s.scratch, S->P, n, s.d_err, &sc);
            cudaError_t e = cudaMemsetAsync(s.d_err, 0, 4, s.stream);
            if (e == cudaSuccess)
                e = lr::launch_query(s.kind != kRankJob ? s.d_in + job->off : nullptr,
                                     s.kind != kRankJob ? nullptr : s.d_in + job->off,
                                     s.d_lcp + job->off + j, n, sc, s.d_len + job->off, s.d_start + job->off, d_loc,
                                     s.d_starts, s.cap, true, s.stream, nullptr, nullptr);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(s.h_jobtot, d_loc + n, 8, cudaMemcpyDeviceToHost, s.stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(s.h_err, s.d_err, 4, cudaMemcpyDeviceToHost, s.stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s.stream);
            if (e != cudaSuccess) { cudaGetLastError(); job->result = LR_ERR_CUDA; break; }
            job->total = s.h_jobtot[0];
            job->result = lr::status_of_bits(*s.h_err);
            if (job->result != LR_OK) break;
            if (job->total > s.cap && job->total <= job->spec.starts_capacity) {
                if (attempt == 0 && grow_starts(S, s, job->total)) continue;   // again, with room for its starts
                job->result = LR_ERR_NOMEM;
                break;
            }
            if (job->total > job->spec.starts_capacity) job->result = LR_ERR_CAPACITY;
            e = copy_out(s, j, 0);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s.stream);
            if (e != cudaSuccess) { cudaGetLastError(); job->result = LR_ERR_CUDA; }
            break;
        }
    }
}

// Marks the slot's jobs done and frees the slot.
void finish(lr_server* S, Slot& s) {
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    for (Job* job : s.jobs) {
        job->state = LR_JOB_DONE;
        S->lat_us.push_back(std::chrono::duration<double, std::micro>(now - job->t_submit).count());
        if (job->result == LR_OK || job->result == LR_ERR_CAPACITY) {
            ++S->completed;
            S->positions += job->spec.n;
        } else {
            ++S->failed;
        }
    }
    s.jobs.clear();
    s.used = 0;
    s.phase = 0;
    s.state = kFree;
    --S->running;
    S->cv_done.notify_all();
}

void fail_all(Slot& s, lr_status st) {
    for (Job* job : s.jobs) job->result = st;
}

// Next step of a running slot after its stream callback fired.
void advance(lr_server* S, Slot& s) {
    if (s.phase == 1) {
        if (s.copy_failed) {
            fail_all(s, LR_ERR_CUDA);
            finish(S, s);
            return;
        }
        const int num = (int)s.jobs.size();
        int64_t sum = 0;
        for (int j = 0; j < num; ++j) sum += s.h_jobtot[j];
        if (*s.h_err != 0 || sum > s.cap) {
            if (*s.h_err == 0 && grow_starts(S, s, sum)) {
                if (launch_batch(S, s) == cudaSuccess) return;
                cudaGetLastError();
                fail_all(s, LR_ERR_CUDA);
                cudaStreamSynchronize(s.stream);
                finish(S, s);
                return;
            }
            run_solo(S, s);
            finish(S, s);
            return;
        }
        int64_t base = 0;
        cudaError_t e = cudaSuccess;
        for (int j = 0; j < num && e == cudaSuccess; ++j) {
            Job* job = s.jobs[j];
            job->total = s.h_jobtot[j];
            job->result = job->total > job->spec.starts_capacity ? LR_ERR_CAPACITY : LR_OK;
            e = copy_out(s, j, base);
            base += job->total;
        }
        s.phase = 2;
        if (e == cudaSuccess) e = cudaLaunchHostFunc(s.stream, on_stream_done, &s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail_all(s, LR_ERR_CUDA);
            cudaStreamSynchronize(s.stream);
            finish(S, s);
        }
        return;
    }
    finish(S, s);                                    // phase 2: the copies are done
}

// Moves queued jobs into the slot being filled.  Called with the lock held;
// returns the admitted jobs (their copies are issued after unlocking).
int admit_locked(lr_server* S, std::vector<Job*>& admitted) {
    admitted.clear();
    while (!S->queue.empty()) {
        Job* job = S->queue.front();
        if (job->state == LR_JOB_CANCELLED) { S->queue.pop_front(); continue; }
        if (S->filling < 0) {
            for (int i = 0; i < S->nslots; ++i)
                if (S->slots[i].state == kFree) { S->filling = i; break; }
            if (S->filling < 0) break;
            Slot& f = S->slots[S->filling];
            f.state = kFilling;
            f.used = 0;
            f.blocked = false;
            f.copy_failed = false;
            f.kind = job->kind;
            f.jobs.clear();
        }
        Slot& f = S->slots[S->filling];
        if (f.used + job->spec.n > S->P || (int)f.jobs.size() >= S->J || f.kind != job->kind) {
            f.blocked = true;
            break;
        }
        S->queue.pop_front();
        --S->queued;
        if (f.jobs.empty()) f.t_first = Clock::now();
        job->off = f.used;
        job->idx = (int)f.jobs.size();
        job->state = LR_JOB_ADMITTED;
        f.used += job->spec.n;
        f.jobs.push_back(job);
        admitted.push_back(job);
    }
    return S->filling;
}

// Host-to-device copies of newly admitted jobs, on their slot's stream.
cudaError_t copy_in(Slot& s, const std::vector<Job*>& admitted) {
    cudaError_t e = cudaSuccess;
    for (Job* job : admitted) {
        const int j = job->idx;
        const lr_job& q = job->spec;
        if (job->kind == kTextJob) {
            e = cudaMemcpyAsync(s.d_text + job->off, q.h_text, (size_t)q.n, cudaMemcpyHostToDevice, s.stream);
        } else {
            const int32_t* src = job->kind == kSaJob ? q.h_sa : q.h_rank;
            e = cudaMemcpyAsync(s.d_in + job->off, src, (size_t)q.n * 4, cudaMemcpyHostToDevice, s.stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(s.d_lcp + job->off + j, q.h_lcp, (size_t)(q.n + 1) * 4, cudaMemcpyHostToDevice,
                                    s.stream);
        }
        if (e != cudaSuccess) break;
    }
    return e;
}

void builder_main(lr_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_build.wait(lk, [&]() { return S->builders_stop || !S->to_build.empty(); });
        if (S->to_build.empty()) return;                 // stopping, nothing left
        Slot& s = S->slots[S->to_build.front()];
        S->to_build.pop_front();
        lk.unlock();
        cudaError_t e = launch_batch(S, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail_all(s, LR_ERR_CUDA);
            cudaStreamSynchronize(s.stream);
            finish(S, s);
        }
        lk.lock();
    }
}

void worker_main(lr_server* S) {
    cudaSetDevice(S->device);
    std::vector<Job*> admitted;
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool did = false;
        for (int i = 0; i < S->nslots; ++i) {
            Slot& s = S->slots[i];
            if (!s.signaled) continue;
            s.signaled = false;
            lk.unlock();
            advance(S, s);
            lk.lock();
            did = true;
        }
        const int f = admit_locked(S, admitted);
        if (!admitted.empty()) {
            lk.unlock();
            cudaError_t e = copy_in(S->slots[f], admitted);
            lk.lock();
            if (e != cudaSuccess) {
                cudaGetLastError();
                S->slots[f].copy_failed = true;
            }
            did = true;
        }
        // Close the slot being filled when it is due.
        if (S->filling >= 0) {
            Slot& s = S->slots[S->filling];
            const bool due = !s.jobs.empty() &&
                             (s.blocked || s.used >= S->P || (int)s.jobs.size() >= S->J || S->stopping ||
                              S->running + (int)S->ready.size() < S->cfg.max_inflight ||
                              Clock::now() - s.t_first >= std::chrono::microseconds(S->cfg.batch_window_us));
            if (due) {
                s.state = kReady;
                S->ready.push_back(S->filling);
                S->filling = -1;
                did = true;
            }
        }
        while (S->running < S->cfg.max_inflight && !S->ready.empty()) {
            Slot& s = S->slots[S->ready.front()];
            S->ready.pop_front();
            s.state = kRunning;
            ++S->running;
            ++S->batches;
            for (Job* job : s.jobs) job->state = LR_JOB_RUNNING;
            if (s.kind == kTextJob && !S->builders.empty()) {
                S->to_build.push_back((int)(&s - S->slots.get()));
                S->cv_build.notify_one();
                did = true;
                continue;
            }
            lk.unlock();
            cudaError_t e = launch_batch(S, s);
            if (e != cudaSuccess) {
                cudaGetLastError();
                fail_all(s, LR_ERR_CUDA);
                cudaStreamSynchronize(s.stream);
                finish(S, s);
            }
            lk.lock();
            did = true;
        }
        bool idle = S->queued == 0 && S->filling < 0 && S->ready.empty() && S->running == 0;
        if (S->stopping && idle) break;
        if (did) continue;
        if (S->filling >= 0 && !S->slots[S->filling].jobs.empty())
            S->cv.wait_until(lk, S->slots[S->filling].t_first + std::chrono::microseconds(S->cfg.batch_window_us));
        else
            S->cv.wait_for(lk, std::chrono::milliseconds(50));
    }
}

bool job_finished(const Job* j) { return j->state == LR_JOB_DONE || j->state == LR_JOB_CANCELLED; }

// Reports a finished job and drops its record (lock held).
void report_locked(lr_server* S, Job* job, lr_status* result, int64_t* total) {
    if (result) *result = job->result;
    if (total) *total = job->total;
    S->jobs.erase(job->id);
    delete job;
}

}  // namespace

extern "C" {

lr_status lr_server_start(const lr_server_config* cfg_in, lr_server** out) {
    if (!out) return LR_ERR_ARG;
    *out = nullptr;
    lr_server_config cfg{};
    if (cfg_in) cfg = *cfg_in;
    if (cfg.device < 0 || cfg.slots < 0 || cfg.max_inflight < 0 || cfg.max_batch_positions < 0 ||
        cfg.max_batch_jobs < 0 || cfg.max_queue < 0 || cfg.batch_window_us < 0 || cfg.hbm_fraction < 0 ||
        cfg.hbm_fraction > 1 || cfg.starts_factor < 0 || cfg.starts_factor > 64)
        return LR_ERR_ARG;
    if (cfg.slots == 0) cfg.slots = 4;
    if (cfg.max_inflight == 0) cfg.max_inflight = 2;
    if (cfg.max_batch_positions == 0) cfg.max_batch_positions = 1LL << 26;
    if (cfg.max_batch_jobs == 0) cfg.max_batch_jobs = 4096;
    if (cfg.max_queue == 0) cfg.max_queue = 65536;
    if (cfg.batch_window_us == 0) cfg.batch_window_us = 2000;
    if (cfg.hbm_fraction == 0) cfg.hbm_fraction = 0.5;
    if (cfg.starts_factor == 0) cfg.starts_factor = 2.0;
    if (cfg.max_batch_positions > 2147483646LL - cfg.max_batch_jobs) return LR_ERR_ARG;

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) { cudaGetLastError(); return LR_ERR_CUDA; }
    if (cudaSetDevice(cfg.device) != cudaSuccess) { cudaGetLastError(); return LR_ERR_CUDA; }
    struct Restore { int d; ~Restore() { if (d >= 0) cudaSetDevice(d); } } restore{prev};
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { cudaGetLastError(); return LR_ERR_CUDA; }
    if (lr::configure_kernels() != cudaSuccess) { cudaGetLastError(); return LR_ERR_CUDA; }

    lr_server* S = new (std::nothrow) lr_server();
    if (!S) return LR_ERR_NOMEM;
    S->device = cfg.device;
    S->cfg = cfg;
    S->P = cfg.max_batch_positions;
    S->J = cfg.max_batch_jobs;
    S->budget = (size_t)((double)free_b * cfg.hbm_fraction);
    const SlotLayout L = slot_layout(S->P, S->J, cfg.text_jobs != 0);
    const int64_t cap0 = (int64_t)(cfg.starts_factor * (double)S->P) + 1024;
    const size_t per_slot = L.total + (size_t)cap0 * 4 + (cfg.text_jobs ? lr::index_work_bytes(S->P, kTextRounds) : 0);
    const int fit = (int)std::min<size_t>((size_t)cfg.slots, S->budget / per_slot);
    if (fit < 1) { delete S; return LR_ERR_NOMEM; }
    S->nslots = fit;
    S->slots.reset(new (std::nothrow) Slot[fit]);
    if (!S->slots) { delete S; return LR_ERR_NOMEM; }
    for (int i = 0; i < fit; ++i) {
        if (alloc_slot(S, S->slots[i], L, cap0) != cudaSuccess) {
            for (int k = 0; k <= i; ++k) free_slot(S->slots[k]);
            delete S;
            return LR_ERR_NOMEM;
        }
    }
    try {
        if (cfg.text_jobs)
            for (int i = 0; i < cfg.max_inflight; ++i) S->builders.emplace_back(builder_main, S);
        S->worker = std::thread(worker_main, S);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->builders_stop = true;
        }
        S->cv_build.notify_all();
        for (auto& t : S->builders) if (t.joinable()) t.join();
        for (int k = 0; k < fit; ++k) free_slot(S->slots[k]);
        delete S;
        return LR_ERR_NOMEM;
    }
    *out = S;
    return LR_OK;
}

lr_status lr_server_submit(lr_server* S, const lr_job* q, int64_t* job_id) {
    if (!S || !q || !job_id) return LR_ERR_ARG;
    const bool text = q->h_text != nullptr && !q->h_sa && !q->h_rank && !q->h_lcp;
    if (q->n < 1 || !q->h_lr_len || !q->h_lr_start || !q->h_offsets) return LR_ERR_ARG;
    if (!text && (!q->h_lcp || (!q->h_sa && !q->h_rank))) return LR_ERR_ARG;
    if (text && !S->cfg.text_jobs) return LR_ERR_ARG;
    if (q->starts_capacity < 0 || (q->starts_capacity > 0 && !q->h_starts)) return LR_ERR_ARG;
    if (q->n > S->P) return LR_ERR_NOMEM;
    Job* job = new (std::nothrow) Job();
    if (!job) return LR_ERR_NOMEM;
    job->spec = *q;
    job->kind = text ? kTextJob : (q->h_sa ? kSaJob : kRankJob);
    job->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping || S->queued >= S->cfg.max_queue) { delete job; return LR_ERR_BUSY; }
    job->id = S->next_id++;
    S->jobs[job->id] = job;
    S->queue.push_back(job);
    ++S->queued;
    ++S->submitted;
    *job_id = job->id;
    S->cv.notify_one();
    return LR_OK;
}

lr_status lr_server_poll(lr_server* S, int64_t id, int32_t* state, lr_status* result, int64_t* total) {
    if (!S || !state) return LR_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) return LR_ERR_ARG;
    Job* job = it->second;
    *state = job->state;
    if (job_finished(job)) report_locked(S, job, result, total);
    return LR_OK;
}

lr_status lr_server_wait(lr_server* S, int64_t id, int32_t timeout_ms, int32_t* state, lr_status* result,
                         int64_t* total) {
    if (!S) return LR_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto done = [&]() {
        auto it = S->jobs.find(id);
        return it == S->jobs.end() || job_finished(it->second);
    };
    if (timeout_ms < 0) S->cv_done.wait(lk, done);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) return LR_ERR_TIMEOUT;
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) return LR_ERR_ARG;
    if (state) *state = it->second->state;
    report_locked(S, it->second, result, total);
    return LR_OK;
}

lr_status lr_server_cancel(lr_server* S, int64_t id) {
    if (!S) return LR_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) return LR_ERR_ARG;
    Job* job = it->second;
    if (job->state == LR_JOB_CANCELLED) return LR_OK;
    if (job->state != LR_JOB_QUEUED) return LR_ERR_BUSY;
    job->state = LR_JOB_CANCELLED;
    --S->queued;
    ++S->cancelled;
    S->cv_done.notify_all();
    return LR_OK;
}

lr_status lr_server_stats_get(lr_server* S, int32_t reset, lr_server_stats* st) {
    if (!S || !st) return LR_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    *st = lr_server_stats{};
    st->submitted = S->submitted;
    st->completed = S->completed;
    st->cancelled = S->cancelled;
    st->failed = S->failed;
    st->batches = S->batches;
    st->positions = S->positions;
    st->slots = S->nslots;
    st->slot_positions = S->P;
    st->device_bytes = S->device_bytes.load();
    std::vector<double> v = S->lat_us;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            size_t k = (size_t)(p * (double)(v.size() - 1) + 0.5);
            return v[std::min(k, v.size() - 1)];
        };
        st->p50_us = pct(0.50);
        st->p99_us = pct(0.99);
        double sum = 0;
        for (double x : v) sum += x;
        st->mean_us = sum / (double)v.size();
        st->max_us = v.back();
    }
    if (reset) {
        S->lat_us.clear();
        S->submitted = S->completed = S->cancelled = S->failed = S->batches = S->positions = 0;
    }
    return LR_OK;
}

lr_status lr_server_stop(lr_server* S) {
    if (!S) return LR_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        for (Job* job : S->queue)
            if (job->state == LR_JOB_QUEUED) {
                job->state = LR_JOB_CANCELLED;
                --S->queued;
                ++S->cancelled;
            }
        S->cv.notify_all();
        S->cv_done.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->builders_stop = true;
    }
    S->cv_build.notify_all();
    for (auto& t : S->builders) if (t.joinable()) t.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    for (int i = 0; i < S->nslots; ++i) free_slot(S->slots[i]);
    if (prev >= 0) cudaSetDevice(prev);
    for (auto& kv : S->jobs) delete kv.second;
    delete S;
    return LR_OK;
}

}  // extern "C"
