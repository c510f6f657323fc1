// mtb_server.cu -- serving: continuous admission of alignment jobs under a
// device-memory budget.  Host code around the library's own alignment path.
//
// A job is one exposure stack in host memory.  The server owns one device arena
// of `budget_bytes`, `slots` compute streams and `copy_streams` copy streams.
// A worker thread admits waiting jobs in arrival order whenever a slot is free
// and the arena has room for the job's images, workspace and shifts -- also
// while other jobs are on the GPU.  For an admitted job it enqueues
//   - the copy of its exposures to the device (Sec. III-B copies each exposure
//     to the GPU once), split over the copy streams, which serve jobs in
//     admission order so that the first admitted job's copy finishes first.
//     Page-locked host memory is read by a copy kernel straight over the host
//     link: a copy engine that has been idle for some milliseconds takes up to
//     ~15x longer for its next 504 MB copy (2.4 ms back to back; p99 19 ms
//     with 20 ms between copies, p90 34 ms with 100 ms), while SM loads of the
//     same memory keep their pace (p99 2.4 and 4.7 ms).  Pageable memory goes
//     through cudaMemcpyAsync;
//   - on the job's compute stream, after those copies: the whole alignment
//     (pyramids, bitmaps and search stay in the arena for the job's life), the
//     copy of its shifts and search status word to a pinned slot buffer, and a
//     host function that completes the job.
// The host function (a CUDA callback thread) copies the shifts to the caller's
// buffer, stamps the completion time, returns the job's memory to the arena and
// wakes the worker, which may then admit the next job.  The worker never holds
// the server lock across a CUDA call, so the callback never waits behind one.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mtb_arena.h"
#include "mtb_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

using mtb::kArenaAlign;
using mtb::round_up;

using Arena = mtb::Arena<MTB_SERVER_MAX_SLOTS>;  // at most `slots` jobs hold memory

constexpr int kRunning = 1;  // job status while queued or on the GPU


struct Job {
    uint64_t id = 0;
    mtb_job_t desc = {};
    mtb_layout_t layout = {};
    size_t bytes = 0, off = 0;
    int slot = -1;
    int status = kRunning;
    Clock::time_point t_submit, t_admit, t_enqueued, t_callback, t_done;
};

struct SlotCtx {
    mtb_server *server = nullptr;
    int slot = 0;
};

// Pinned per-slot result area: the search status word, then the shifts.
struct SlotResult {
    int32_t status;
    int32_t pad[3];
    int32_t shifts[2 * MTB_MAX_EXPOSURES];
};

}  // namespace

struct mtb_server {
    mtb_server_config_t cfg = {};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> pending;
    std::vector<std::shared_ptr<Job>> running;  // per slot
    std::unordered_map<uint64_t, std::shared_ptr<Job>> jobs;
    uint64_t next_id = 1;
    std::unique_ptr<Arena> arena;
    uint8_t *arena_base = nullptr;
    SlotResult *results = nullptr;  // pinned, one per slot
    SlotResult *results_dev = nullptr;  // the same area as the device addresses it (null: copy engines)
    std::vector<SlotCtx> ctx;
    std::vector<cudaStream_t> compute, copy;
    std::vector<cudaEvent_t> copied;  // [slot][copy stream]
    std::thread worker;
    bool paused = false, stop = false;
    int n_running = 0;
    // statistics
    uint64_t admitted = 0, completed = 0, refused = 0, failed = 0;
    size_t peak_bytes = 0;
    int peak_running = 0;
};

namespace {

size_t job_bytes(const mtb_job_t &j, mtb_layout_t *L) {
    if (mtb::check_stack_args(j.n_exposures, j.w, j.h, j.levels, j.noise_tol, j.ref_idx) != MTB_OK) return 0;
    if (mtb::compute_layout(j.n_exposures, j.w, j.h, j.levels, L) != MTB_OK) return 0;
    return mtb_host_workspace_bytes(j.n_exposures, j.w, j.h, j.levels);
}

// Completes the job in `slot` (lock held).
void finish_locked(mtb_server *s, int slot, int status) {
    std::shared_ptr<Job> job = s->running[slot];
    s->running[slot].reset();
    --s->n_running;
    job->status = status;
    job->t_done = Clock::now();
    s->arena->release(job->off, job->bytes);
    ++s->completed;
    if (status != MTB_OK) ++s->failed;
    s->cv_done.notify_all();
    s->cv_work.notify_one();
}

// Host function at the end of a job's compute stream.  Makes no CUDA call.
void CUDART_CB job_done(void *p) {
    const Clock::time_point t_cb = Clock::now();
    SlotCtx *c = static_cast<SlotCtx *>(p);
    mtb_server *s = c->server;
    std::lock_guard<std::mutex> lock(s->mu);
    Job &job = *s->running[c->slot];
    job.t_callback = t_cb;
    const SlotResult &r = s->results[c->slot];
    std::memcpy(job.desc.host_shifts_out, r.shifts, (size_t)job.desc.n_exposures * 2 * sizeof(int32_t));
    finish_locked(s, c->slot, r.status == 0 ? MTB_OK : r.status);
}

// Enqueues an admitted job (lock NOT held).
int enqueue_job(mtb_server *s, const Job &job) {
    const int slot = job.slot;
    const int C = s->cfg.copy_streams;
    cudaStream_t st = s->compute[slot];
    uint8_t *base = s->arena_base + job.off;
    const size_t img_bytes = (size_t)job.desc.n_exposures * job.desc.w * job.desc.h * 3;
    uint8_t *d_img = base;
    uint8_t *ws = base + round_up(img_bytes, kArenaAlign);
    int32_t *d_shifts = reinterpret_cast<int32_t *>(ws + job.layout.total_bytes);
    // the copy in, in C parts of whole 256-byte units
    const size_t part = round_up((img_bytes + C - 1) / C, kArenaAlign);
    const uint8_t *view = mtb::host_device_view(job.desc.host_images);
    for (int c = 0; c < C; ++c) {
        const size_t lo = std::min(img_bytes, part * c), hi = std::min(img_bytes, part * (c + 1));
        if (hi > lo) {
            if (view) {
                if (mtb::launch_copy_in(view + lo, d_img + lo, hi - lo, s->copy[c]) != cudaSuccess) return MTB_ERR_CUDA;
            } else if (cudaMemcpyAsync(d_img + lo, job.desc.host_images + lo, hi - lo, cudaMemcpyHostToDevice,
                                       s->copy[c]) != cudaSuccess) {
                return MTB_ERR_CUDA;
            }
        }
        cudaEvent_t ev = s->copied[slot * C + c];
        if (cudaEventRecord(ev, s->copy[c]) != cudaSuccess || cudaStreamWaitEvent(st, ev, 0) != cudaSuccess)
            return MTB_ERR_CUDA;
    }
    const int rc = mtb_align_stack_ex(d_img, job.desc.n_exposures, job.desc.w, job.desc.h, job.desc.levels,
                                      job.desc.noise_tol, job.desc.ref_idx, d_shifts, nullptr, nullptr, ws,
                                      job.layout.total_bytes, st);
    if (rc != MTB_OK) return rc;
    SlotResult *r = &s->results[slot];
    SlotResult *rd = s->results_dev ? s->results_dev + slot : nullptr;
    if (rd) {
        if (mtb::launch_copy_out(reinterpret_cast<const int32_t *>(ws + job.layout.status_offset), &rd->status, 1,
                                 d_shifts, rd->shifts, job.desc.n_exposures * 2, st) != cudaSuccess)
            return MTB_ERR_CUDA;
    } else if (cudaMemcpyAsync(&r->status, ws + job.layout.status_offset, sizeof(int32_t), cudaMemcpyDeviceToHost,
                               st) != cudaSuccess ||
               cudaMemcpyAsync(r->shifts, d_shifts, (size_t)job.desc.n_exposures * 2 * sizeof(int32_t),
                               cudaMemcpyDeviceToHost, st) != cudaSuccess) {
        return MTB_ERR_CUDA;
    }
    if (cudaLaunchHostFunc(st, job_done, &s->ctx[slot]) != cudaSuccess) return MTB_ERR_CUDA;
    return MTB_OK;
}

bool admissible_locked(const mtb_server *s) {
    return !s->paused && !s->pending.empty() && s->n_running < s->cfg.slots;
}

void worker_loop(mtb_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        s->cv_work.wait(lock, [s] { return s->stop || admissible_locked(s); });
        if (s->stop) return;
        // only the first waiting job may be admitted: arrival order is kept, so a
        // large job is never overtaken indefinitely by smaller ones
        std::shared_ptr<Job> job = s->pending.front();
        size_t off = 0;
        if (!s->arena->alloc(job->bytes, &off)) {
            s->cv_work.wait(lock);  // until a completion frees memory (or stop)
            continue;
        }
        s->pending.pop_front();
        int slot = 0;
        while (s->running[slot]) ++slot;
        job->off = off;
        job->slot = slot;
        job->t_admit = Clock::now();
        s->running[slot] = job;
        ++s->n_running;
        ++s->admitted;
        s->peak_bytes = std::max(s->peak_bytes, s->arena->in_use());
        s->peak_running = std::max(s->peak_running, s->n_running);
        lock.unlock();
        const int rc = enqueue_job(s, *job);
        const Clock::time_point t_enq = Clock::now();
        if (rc != MTB_OK) {
            // nothing of this job may still run when its memory is given back
            cudaStreamSynchronize(s->compute[slot]);
            for (cudaStream_t c : s->copy) cudaStreamSynchronize(c);
            cudaGetLastError();
        }
        lock.lock();
        job->t_enqueued = t_enq;
        if (job->t_callback < t_enq) job->t_callback = t_enq;  // (the callback may already have run)
        if (rc != MTB_OK) finish_locked(s, slot, rc);
    }
}

int check_config(const mtb_server_config_t *c) {
    if (!c || c->budget_bytes < (1u << 20) || c->slots < 1 || c->slots > MTB_SERVER_MAX_SLOTS ||
        c->copy_streams < 1 || c->copy_streams > MTB_SERVER_MAX_COPY_STREAMS || c->max_pending < 0)
        return MTB_ERR_INVALID_ARG;
    return MTB_OK;
}

void release_resources(mtb_server *s) {
    for (cudaStream_t st : s->compute) cudaStreamDestroy(st);
    for (cudaStream_t st : s->copy) cudaStreamDestroy(st);
    for (cudaEvent_t ev : s->copied) cudaEventDestroy(ev);
    if (s->results) cudaFreeHost(s->results);
    if (s->arena_base) cudaFree(s->arena_base);
}

}  // namespace

extern "C" {

size_t mtb_job_bytes(const mtb_job_t *job) {
    if (!job) return 0;
    mtb_layout_t L;
    return job_bytes(*job, &L);
}

int mtb_server_create(const mtb_server_config_t *config, mtb_server_t **out) {
    if (!out) return MTB_ERR_INVALID_ARG;
    *out = nullptr;
    int rc = check_config(config);
    if (rc != MTB_OK) return rc;
    mtb_server *s = new (std::nothrow) mtb_server();
    if (!s) return MTB_ERR_OOM;
    s->cfg = *config;
    s->cfg.budget_bytes = config->budget_bytes / kArenaAlign * kArenaAlign;
    const int S = s->cfg.slots, C = s->cfg.copy_streams;
    try {  // host allocations first: after this point nothing throws
        s->running.resize(S);
        s->ctx.resize(S);
        s->compute.reserve(S);
        s->copy.reserve(C);
        s->copied.reserve((size_t)S * C);
        s->arena.reset(new Arena(s->cfg.budget_bytes));
    } catch (...) {
        delete s;
        return MTB_ERR_OOM;
    }
    if (cudaGetDevice(&s->device) != cudaSuccess) rc = MTB_ERR_CUDA;
    void *p = nullptr;
    if (rc == MTB_OK && cudaMalloc(&p, s->cfg.budget_bytes) != cudaSuccess) rc = MTB_ERR_OOM;
    s->arena_base = static_cast<uint8_t *>(p);
    p = nullptr;
    if (rc == MTB_OK && cudaHostAlloc(&p, sizeof(SlotResult) * S, cudaHostAllocMapped) != cudaSuccess)
        rc = MTB_ERR_OOM;
    s->results = static_cast<SlotResult *>(p);
    if (rc == MTB_OK) {
        void *d = nullptr;
        if (cudaHostGetDevicePointer(&d, p, 0) == cudaSuccess) s->results_dev = static_cast<SlotResult *>(d);
        else cudaGetLastError();
    }
    for (int k = 0; rc == MTB_OK && k < S; ++k) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) rc = MTB_ERR_CUDA;
        else s->compute.push_back(st);
        s->ctx[k] = SlotCtx{s, k};
    }
    for (int k = 0; rc == MTB_OK && k < C; ++k) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) rc = MTB_ERR_CUDA;
        else s->copy.push_back(st);
    }
    for (int k = 0; rc == MTB_OK && k < S * C; ++k) {
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) rc = MTB_ERR_CUDA;
        else s->copied.push_back(ev);
    }
    if (rc != MTB_OK) {
        cudaGetLastError();
        release_resources(s);
        delete s;
        return rc;
    }
    try {
        s->worker = std::thread(worker_loop, s);
    } catch (...) {
        release_resources(s);
        delete s;
        return MTB_ERR_OOM;
    }
    *out = s;
    return MTB_OK;
}

int mtb_server_submit(mtb_server_t *s, const mtb_job_t *job, uint64_t *job_id) {
    if (!s || !job || !job_id || !job->host_images || !job->host_shifts_out) return MTB_ERR_INVALID_ARG;
    std::shared_ptr<Job> j;
    try {
        j = std::make_shared<Job>();
    } catch (...) {
        return MTB_ERR_OOM;
    }
    j->desc = *job;
    j->bytes = job_bytes(*job, &j->layout);
    if (j->bytes == 0) return MTB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    if (j->bytes > s->cfg.budget_bytes ||
        (s->cfg.max_pending > 0 && (int)s->pending.size() >= s->cfg.max_pending)) {
        ++s->refused;
        return MTB_ERR_BUSY;
    }
    j->id = s->next_id;
    j->t_submit = Clock::now();
    try {
        s->jobs.emplace(j->id, j);
        s->pending.push_back(j);
    } catch (...) {
        s->jobs.erase(j->id);
        return MTB_ERR_OOM;
    }
    ++s->next_id;
    s->cv_work.notify_one();
    *job_id = j->id;
    return MTB_OK;
}

int mtb_server_poll(mtb_server_t *s, uint64_t job_id) {
    if (!s) return MTB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    return it == s->jobs.end() ? MTB_ERR_INVALID_ARG : it->second->status;
}

namespace {

int wait_job(mtb_server_t *s, uint64_t job_id, double *times_ms, int n_times) {
    if (!s) return MTB_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return MTB_ERR_INVALID_ARG;
    std::shared_ptr<Job> j = it->second;
    s->cv_done.wait(lock, [&j] { return j->status != kRunning; });
    if (times_ms) {
        using ms = std::chrono::duration<double, std::milli>;
        const bool ran = j->t_enqueued != Clock::time_point{};  // admitted and enqueued
        const double t[5] = {ms(j->t_done - j->t_submit).count(), ms(j->t_admit - j->t_submit).count(),
                             ran ? ms(j->t_enqueued - j->t_admit).count() : 0.0,
                             ran ? ms(j->t_callback - j->t_enqueued).count() : 0.0,
                             ran ? ms(j->t_done - j->t_callback).count() : 0.0};
        for (int k = 0; k < n_times && k < 5; ++k) times_ms[k] = t[k];
    }
    s->jobs.erase(job_id);
    return j->status;
}

}  // namespace

int mtb_server_wait(mtb_server_t *s, uint64_t job_id, double *times_ms) { return wait_job(s, job_id, times_ms, 2); }

int mtb_server_wait_phases(mtb_server_t *s, uint64_t job_id, double *times_ms) {
    return wait_job(s, job_id, times_ms, 5);
}

int mtb_server_pause(mtb_server_t *s, int paused) {
    if (!s) return MTB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    s->paused = paused != 0;
    s->cv_work.notify_one();
    return MTB_OK;
}

int mtb_server_stats(mtb_server_t *s, uint64_t *values, int n_values) {
    if (!s || !values || n_values < MTB_SERVER_STATS) return MTB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    values[0] = s->admitted;
    values[1] = s->completed;
    values[2] = s->refused;
    values[3] = s->failed;
    values[4] = s->pending.size();
    values[5] = (uint64_t)s->n_running;
    values[6] = s->arena->in_use();
    values[7] = s->peak_bytes;
    values[8] = (uint64_t)s->peak_running;
    return MTB_OK;
}

void mtb_server_destroy(mtb_server_t *s) {
    if (!s) return;
    {
        std::unique_lock<std::mutex> lock(s->mu);
        s->paused = false;
        s->cv_work.notify_one();
        s->cv_done.wait(lock, [s] { return s->pending.empty() && s->n_running == 0; });
        s->stop = true;
        s->cv_work.notify_one();
    }
    s->worker.join();
    release_resources(s);
    delete s;
}

}  // extern "C"
