// Continuous-batching server for HyperANF jobs.
//
// Jobs (a CSR graph, m, runs, seed) arrive at any time through
// hanf_server_submit.  A fixed set of worker threads, each with its own CUDA
// stream, admits queued jobs in arrival order as soon as a worker is free and
// the job's workspace fits in the device arena the caller reserved (first-fit
// allocation, coalescing free list): the admitted job's context is created in
// its slice of the arena and the whole of Algorithm 2 runs as one CUDA graph
// on the worker's stream, so jobs of different workers overlap on the GPU.
// Streams carry priorities in arrival order: a job admitted while others run
// ranks below them, so the oldest job runs nearly as if alone and newer jobs
// use the SMs it leaves free.
// Each job has its own context, so its result does not depend on what else is
// running.  hanf_server_wait returns a job's N(t), T and timings.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hanf.h"
#include "hanf_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Job {
    uint64_t id = 0;
    hanf_job spec{};
    size_t bytes = 0;
    int32_t status = 1;            // 1 queued, 2 running, 0 or <0 finished
    bool cancelled = false;
    std::string error;
    std::vector<double> N;         // runs x (T+1)
    std::vector<int32_t> T;
    int32_t T_max = 0;
    Clock::time_point t_submit, t_start, t_end;
};

// First-fit allocator over [0, size) with coalescing, 256-byte granules.
class Arena {
public:
    void reset(size_t size) { free_.clear(); if (size) free_[0] = size; }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = (bytes + 255) & ~size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = (bytes + 255) & ~size_t(255);
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t largest() const
    {
        size_t m = 0;
        for (auto &kv : free_) m = std::max(m, kv.second);
        return m;
    }

private:
    std::map<size_t, size_t> free_;
};

}  // namespace

struct hanf_server {
    uint8_t *arena = nullptr;
    size_t arena_bytes = 0;
    Arena alloc;
    hanf_opts base{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Job>> jobs;
    std::vector<std::thread> workers;
    // streams[w][k]: worker w's stream at priority level k (0 = highest)
    std::vector<std::vector<cudaStream_t>> streams;
    int prio_greatest = 0, levels = 1;
    int next_level = 0;            // level of the next admitted job (arrival order)
    uint64_t next_id = 1;
    bool stopping = false;
    int running = 0;
    uint64_t completed = 0, failed = 0;
};

namespace {

int server_fail(int code, const std::string &msg)
{
    hanf::record_error(msg);
    return code;
}

hanf_opts job_opts(const hanf_server *s, const hanf_job &j, cudaStream_t st)
{
    hanf_opts o = s->base;
    o.runs = j.runs;
    o.use_graph = 1;
    o.profile = 0;
    o.seeds = nullptr;
    o.stream = st;
    o.l2_hot_bytes = -1;   // jobs share the GPU: no context-wide L2 set-aside
    return o;
}

// Run one admitted job in its arena slice; fills the job's results.
void run_job(hanf_server *s, Job &job, uint8_t *ws, cudaStream_t st)
{
    const hanf_job &j = job.spec;
    hanf_opts o = job_opts(s, j, st);
    hanf_ctx *ctx = nullptr;
    int rc = hanf_create(&ctx, j.n, j.arcs, j.offsets, j.targets, j.graph_on_device, j.log2m,
                         j.seed, &o, ws, job.bytes);
    if (rc == HANF_OK) {
        const int32_t cap = j.max_iter > 0 ? j.max_iter + 1 : 4097;
        std::vector<double> N((size_t)j.runs * cap);
        std::vector<int32_t> T(j.runs);
        rc = hanf_run(ctx, cap - 1, N.data(), cap, T.data());
        if (rc == HANF_OK) {
            int32_t Tm = 0;
            for (int r = 0; r < j.runs; ++r) Tm = std::max(Tm, T[r]);
            job.N.assign((size_t)j.runs * (Tm + 1), 0.0);
            for (int r = 0; r < j.runs; ++r)
                std::copy(N.begin() + (size_t)r * cap, N.begin() + (size_t)r * cap + Tm + 1,
                          job.N.begin() + (size_t)r * (Tm + 1));
            job.T = T;
            job.T_max = Tm;
        }
        if (rc != HANF_OK) job.error = hanf_last_error();
        hanf_destroy(ctx);
    } else {
        job.error = hanf_last_error();
    }
    job.status = rc;
}

void worker_main(hanf_server *s, int w)
{
    cudaSetDevice(s->device);
    for (;;) {
        std::shared_ptr<Job> job;
        size_t off = 0;
        cudaStream_t st = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            for (;;) {
                if (s->stopping) return;
                // arrival order: only the oldest queued job may be admitted
                while (!s->queue.empty() && s->queue.front()->cancelled) s->queue.pop_front();
                if (!s->queue.empty() && s->alloc.alloc(s->queue.front()->bytes, &off)) {
                    job = s->queue.front();
                    s->queue.pop_front();
                    break;
                }
                s->cv_work.wait(lk);
            }
            job->status = 2;
            job->t_start = Clock::now();
            // jobs admitted while others run get lower priorities, in arrival
            // order: the oldest job's blocks are scheduled first, the newer
            // ones fill the SMs it leaves free; an idle GPU starts over
            if (s->running == 0) s->next_level = 0;
            st = s->streams[w][std::min(s->next_level, s->levels - 1)];
            ++s->next_level;
            ++s->running;
        }
        run_job(s, *job, s->arena + off, st);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            job->t_end = Clock::now();
            s->alloc.release(off, job->bytes);
            --s->running;
            if (job->status == HANF_OK) ++s->completed;
            else ++s->failed;
        }
        s->cv_work.notify_all();   // memory freed: the queue head may fit now
        s->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

int hanf_server_create(hanf_server **out, void *arena, size_t arena_bytes, int32_t workers,
                       const hanf_opts *base)
{
    if (!out || !arena || arena_bytes == 0) return server_fail(HANF_EINVAL, "NULL argument");
    if (reinterpret_cast<uintptr_t>(arena) & 255)
        return server_fail(HANF_EINVAL, "arena is not 256-byte aligned");
    if (workers < 1 || workers > 64) return server_fail(HANF_EINVAL, "workers outside 1..64");
    hanf_server *s = new (std::nothrow) hanf_server();
    if (!s) return server_fail(HANF_ENOMEM, "host allocation failed");
    s->arena = static_cast<uint8_t *>(arena);
    s->arena_bytes = arena_bytes;
    s->alloc.reset(arena_bytes);
    if (base) s->base = *base;
    else hanf_default_opts(&s->base);
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return server_fail(HANF_ECUDA, "no CUDA device");
    }
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) least = greatest = 0;
    s->prio_greatest = greatest;
    s->levels = least - greatest + 1;
    s->streams.assign(workers, std::vector<cudaStream_t>(s->levels, nullptr));
    for (int w = 0; w < workers; ++w)
        for (int k = 0; k < s->levels; ++k)
            if (cudaStreamCreateWithPriority(&s->streams[w][k], cudaStreamNonBlocking,
                                             greatest + k) != cudaSuccess) {
                for (auto &row : s->streams)
                    for (cudaStream_t x : row)
                        if (x) cudaStreamDestroy(x);
                delete s;
                return server_fail(HANF_ECUDA, "stream creation failed");
            }
    for (int w = 0; w < workers; ++w) s->workers.emplace_back(worker_main, s, w);
    *out = s;
    return HANF_OK;
}

int hanf_server_submit(hanf_server *s, const hanf_job *job, uint64_t *id_out)
{
    if (!s || !job || !id_out) return server_fail(HANF_EINVAL, "NULL argument");
    if (job->runs < 1 || job->max_iter < 0) return server_fail(HANF_EINVAL, "bad job options");
    hanf_opts o = job_opts(s, *job, nullptr);
    size_t bytes = 0;
    int rc = hanf_workspace_size(job->n, job->arcs, job->log2m, &o, job->graph_on_device ? 0 : 1,
                                 &bytes);
    if (rc) return rc;
    auto j = std::make_shared<Job>();
    j->spec = *job;
    j->bytes = bytes;
    j->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) return server_fail(HANF_ESTATE, "server is shutting down");
        if (((bytes + 255) & ~size_t(255)) > s->arena_bytes)
            return server_fail(HANF_ENOMEM, "job needs " + std::to_string(bytes) +
                                                " bytes, more than the whole arena");
        j->id = s->next_id++;
        s->jobs[j->id] = j;
        s->queue.push_back(j);
    }
    s->cv_work.notify_all();
    *id_out = j->id;
    return HANF_OK;
}

int hanf_server_wait(hanf_server *s, uint64_t id, int32_t timeout_ms, double *N_out, int32_t cap,
                     int32_t *T_out, double *info_out)
{
    if (!s) return server_fail(HANF_EINVAL, "NULL server");
    std::shared_ptr<Job> job;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->jobs.find(id);
        if (it == s->jobs.end()) return server_fail(HANF_EINVAL, "unknown job id");
        job = it->second;
        auto finished = [&] { return job->status <= 0 || job->cancelled; };
        if (timeout_ms < 0) {
            s->cv_done.wait(lk, finished);
        } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished)) {
            return server_fail(HANF_ETIMEOUT, "job not finished within the timeout");
        }
        s->jobs.erase(it);
    }
    if (job->cancelled) return server_fail(HANF_ECANCELLED, "job was cancelled");
    if (info_out) {
        info_out[0] = ms_between(job->t_submit, job->t_end);    // latency
        info_out[1] = ms_between(job->t_submit, job->t_start);  // queued
        info_out[2] = ms_between(job->t_start, job->t_end);     // on a worker
        info_out[3] = (double)job->T_max;
        info_out[4] = (double)job->bytes;
    }
    if (job->status != HANF_OK) return server_fail(job->status, job->error);
    const int32_t R = job->spec.runs, Tm = job->T_max;
    if (T_out)
        for (int r = 0; r < R; ++r) T_out[r] = job->T[r];
    if (N_out) {
        for (int r = 0; r < R; ++r)
            for (int t = 0; t < cap; ++t)
                N_out[(size_t)r * cap + t] = t <= Tm ? job->N[(size_t)r * (Tm + 1) + t] : 0.0;
        if (Tm + 1 > cap) return server_fail(HANF_ERANGE, "cap smaller than T+1");
    }
    return HANF_OK;
}

int hanf_server_cancel(hanf_server *s, uint64_t id)
{
    if (!s) return server_fail(HANF_EINVAL, "NULL server");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->jobs.find(id);
        if (it == s->jobs.end()) return server_fail(HANF_EINVAL, "unknown job id");
        if (it->second->status != 1) return server_fail(HANF_ESTATE, "job already started");
        it->second->cancelled = true;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
    return HANF_OK;
}

int hanf_server_stats(hanf_server *s, double *out, int32_t nout)
{
    if (!s || !out) return server_fail(HANF_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    const double v[6] = {(double)s->queue.size(), (double)s->running, (double)s->completed,
                         (double)s->failed, (double)s->alloc.largest(), (double)s->arena_bytes};
    for (int i = 0; i < nout && i < 6; ++i) out[i] = v[i];
    return HANF_OK;
}

void hanf_server_destroy(hanf_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
        for (auto &j : s->queue) j->cancelled = true;
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    for (auto &t : s->workers) t.join();
    for (auto &row : s->streams)
        for (cudaStream_t st : row) cudaStreamDestroy(st);
    delete s;
}

}  // extern "C"
