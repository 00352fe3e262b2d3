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
// Small jobs (at most kBatchMaxNodes nodes, default pass limit) that are
// queued together share a context: the worker that admits the oldest queued
// job also takes the later queued small jobs with the same m, runs and graph
// placement (up to kMaxBatch jobs and kBatchTotalNodes stored nodes), lays
// their graphs out as one padded disjoint union (num_graphs = K) and runs
// Algorithm 2 once for all of them, so they share launches, not just the GPU.
// Every job's result is the same as alone (the batch keeps a separate N(t),
// T and seeds per graph; N(t) is an exact sum either way).  A batch whose
// context cannot be created or run puts its jobs back at the head of the
// queue, to be run alone with their own status.
// hanf_server_wait returns a job's N(t), T and timings.
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

constexpr int kMaxBatch = 64;               // jobs in one shared context
constexpr int64_t kBatchMaxNodes = 65536;    // jobs up to this size are batched
constexpr int64_t kBatchTotalNodes = 1 << 21;  // stored nodes of one batch
constexpr int kBatchScan = 256;              // queued jobs looked at for a batch

struct Job {
    uint64_t id = 0;
    hanf_job spec{};
    size_t bytes = 0;
    int32_t status = 1;            // 1 queued, 2 running, 0 or <0 finished
    bool cancelled = false;
    bool alone = false;            // run in a context of its own (a batch failed)
    int32_t outcome = 0;           // the run's status, published as `status` under the lock
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
    uint64_t contexts = 0;         // contexts created (a batch counts once)
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

bool batchable(const Job &j)
{
    return !j.alone && !j.cancelled && j.spec.n <= kBatchMaxNodes && j.spec.max_iter == 0;
}

bool same_class(const Job &a, const Job &b)
{
    return a.spec.log2m == b.spec.log2m && a.spec.runs == b.spec.runs &&
           (a.spec.graph_on_device != 0) == (b.spec.graph_on_device != 0);
}

// Layout of a batch: graph g owns stored nodes [base[g], base[g+1]) (64-aligned)
// and arcs [abase[g], abase[g+1]).
struct BatchPlan {
    std::vector<int64_t> base, nodes, abase;
    std::vector<uint64_t> seeds;
    int64_t n = 0, arcs = 0;
    size_t csr_bytes = 0;          // device batches: the union CSR, before the workspace
    size_t ws_bytes = 0;
    size_t total() const { return csr_bytes + ws_bytes; }
};

hanf_opts batch_opts(const hanf_server *s, const BatchPlan &b, int32_t runs, cudaStream_t st)
{
    hanf_opts o = s->base;
    o.runs = runs;
    o.use_graph = 1;
    o.profile = 0;
    o.seeds = nullptr;
    o.stream = st;
    o.l2_hot_bytes = -1;
    o.num_graphs = (int32_t)b.nodes.size();
    o.graph_base = b.base.data();
    o.graph_nodes = b.nodes.data();
    o.graph_seeds = b.seeds.data();
    return o;
}

int plan_batch(const hanf_server *s, const std::vector<std::shared_ptr<Job>> &jobs, BatchPlan *b)
{
    b->base.assign(1, 0);
    b->abase.assign(1, 0);
    b->nodes.clear();
    b->seeds.clear();
    for (auto &j : jobs) {
        b->nodes.push_back(j->spec.n);
        b->seeds.push_back(j->spec.seed);
        b->base.push_back(b->base.back() + (j->spec.n + 63) / 64 * 64);
        b->abase.push_back(b->abase.back() + j->spec.arcs);
    }
    b->n = b->base.back();
    b->arcs = b->abase.back();
    const bool dev = jobs[0]->spec.graph_on_device != 0;
    b->csr_bytes = dev ? ((size_t)8 * (b->n + 1) + 255) / 256 * 256 +
                             ((size_t)4 * std::max<int64_t>(b->arcs, 1) + 255) / 256 * 256
                       : 0;
    hanf_opts o = batch_opts(s, *b, jobs[0]->spec.runs, nullptr);
    return hanf_workspace_size(b->n, b->arcs, jobs[0]->spec.log2m, &o, dev ? 0 : 1, &b->ws_bytes);
}

// The graphs of a device batch, as one union CSR: graph g's offsets shifted by
// its first arc, padding nodes without arcs, its targets shifted by its first
// node.  One grid row per graph.
struct BatchTables {
    const int64_t *off[kMaxBatch];
    const int32_t *tgt[kMaxBatch];
    int64_t base[kMaxBatch + 1], abase[kMaxBatch + 1], nodes[kMaxBatch];
    int32_t K;
};

__global__ void k_batch_csr(BatchTables b, int64_t *off_out, int32_t *tgt_out)
{
    const int g = blockIdx.y;
    const int64_t span = b.base[g + 1] - b.base[g], n_g = b.nodes[g];
    const int64_t a_g = b.abase[g + 1] - b.abase[g];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t i = i0; i < span; i += stride)
        off_out[b.base[g] + i] = b.abase[g] + b.off[g][i < n_g ? i : n_g] - b.off[g][0];
    for (int64_t e = i0; e < a_g; e += stride)
        tgt_out[b.abase[g] + e] = b.tgt[g][e] + (int32_t)b.base[g];
    if (g == b.K - 1 && i0 == 0) off_out[b.base[b.K]] = b.abase[b.K];
}

// Run an admitted batch in its arena slice.  Returns false if the batch as a
// whole failed (its jobs then go back to the queue to run alone).
bool run_batch(hanf_server *s, std::vector<std::shared_ptr<Job>> &jobs, const BatchPlan &b,
               uint8_t *ws, cudaStream_t st)
{
    const int K = (int)jobs.size();
    const int32_t R = jobs[0]->spec.runs;
    const bool dev = jobs[0]->spec.graph_on_device != 0;
    std::vector<int64_t> h_off;
    std::vector<int32_t> h_tgt;
    const int64_t *off = nullptr;
    const int32_t *tgt = nullptr;
    uint8_t *wsp = ws + b.csr_bytes;
    if (dev) {
        int64_t *d_off = reinterpret_cast<int64_t *>(ws);
        int32_t *d_tgt =
            reinterpret_cast<int32_t *>(ws + ((size_t)8 * (b.n + 1) + 255) / 256 * 256);
        BatchTables t;
        std::memset(&t, 0, sizeof t);
        t.K = K;
        for (int g = 0; g < K; ++g) {
            t.off[g] = jobs[g]->spec.offsets;
            t.tgt[g] = jobs[g]->spec.targets;
            t.nodes[g] = b.nodes[g];
        }
        for (int g = 0; g <= K; ++g) {
            t.base[g] = b.base[g];
            t.abase[g] = b.abase[g];
        }
        k_batch_csr<<<dim3(64, K), 256, 0, st>>>(t, d_off, d_tgt);
        if (cudaGetLastError() != cudaSuccess) return false;
        off = d_off;
        tgt = d_tgt;
    } else {
        h_off.assign(b.n + 1, 0);
        h_tgt.resize(std::max<int64_t>(b.arcs, 1));
        for (int g = 0; g < K; ++g) {
            const hanf_job &j = jobs[g]->spec;
            for (int64_t i = 0; i < b.base[g + 1] - b.base[g]; ++i)
                h_off[b.base[g] + i] = b.abase[g] + j.offsets[i < j.n ? i : j.n] - j.offsets[0];
            for (int64_t e = 0; e < j.arcs; ++e)
                h_tgt[b.abase[g] + e] = j.targets[e] + (int32_t)b.base[g];
        }
        h_off[b.n] = b.arcs;
        off = h_off.data();
        tgt = h_tgt.data();
    }
    hanf_opts o = batch_opts(s, b, R, st);
    hanf_ctx *ctx = nullptr;
    int rc = hanf_create(&ctx, b.n, b.arcs, off, tgt, dev ? 1 : 0, jobs[0]->spec.log2m, 0, &o, wsp,
                         b.ws_bytes);
    if (rc != HANF_OK) return false;
    const int32_t cap = 4097, S = K * R;
    std::vector<double> N((size_t)S * cap);
    std::vector<int32_t> T(S);
    rc = hanf_run(ctx, cap - 1, N.data(), cap, T.data());
    hanf_destroy(ctx);
    if (rc != HANF_OK) return false;
    for (int g = 0; g < K; ++g) {
        Job &job = *jobs[g];
        int32_t Tm = 0;
        job.T.assign(T.begin() + (size_t)g * R, T.begin() + (size_t)(g + 1) * R);
        for (int r = 0; r < R; ++r) Tm = std::max(Tm, job.T[r]);
        job.N.assign((size_t)R * (Tm + 1), 0.0);
        for (int r = 0; r < R; ++r) {
            const double *row = N.data() + (size_t)(g * R + r) * cap;
            std::copy(row, row + Tm + 1, job.N.begin() + (size_t)r * (Tm + 1));
        }
        job.T_max = Tm;
        job.outcome = HANF_OK;
    }
    return true;
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
    job.outcome = rc;
}

// The oldest queued job, and (if it is small) the later queued small jobs of
// its class, as many as the batch limits and the free arena allow.  Called
// with the lock held; removes the admitted jobs from the queue and allocates
// their slice.  Returns false if nothing can be admitted now.
bool admit(hanf_server *s, std::vector<std::shared_ptr<Job>> *jobs, BatchPlan *b, size_t *off,
           size_t *bytes)
{
    while (!s->queue.empty() && s->queue.front()->cancelled) s->queue.pop_front();
    if (s->queue.empty()) return false;
    std::shared_ptr<Job> head = s->queue.front();
    jobs->assign(1, head);
    if (batchable(*head)) {
        int64_t stored = (head->spec.n + 63) / 64 * 64;
        const int scan = std::min<int>((int)s->queue.size(), kBatchScan);
        for (int i = 1; i < scan && (int)jobs->size() < kMaxBatch; ++i) {
            const std::shared_ptr<Job> &j = s->queue[i];
            if (!batchable(*j) || !same_class(*head, *j)) continue;
            const int64_t span = (j->spec.n + 63) / 64 * 64;
            if (stored + span > kBatchTotalNodes) break;
            stored += span;
            jobs->push_back(j);
        }
        // a batch that does not fit the free arena shrinks, down to the head
        while (jobs->size() > 1) {
            if (plan_batch(s, *jobs, b) == HANF_OK && s->alloc.alloc(b->total(), off)) {
                *bytes = b->total();
                break;
            }
            jobs->pop_back();
        }
    }
    if (jobs->size() == 1) {
        if (!s->alloc.alloc(head->bytes, off)) return false;
        *bytes = head->bytes;
    }
    for (auto &j : *jobs)
        s->queue.erase(std::find(s->queue.begin(), s->queue.end(), j));
    return true;
}

void worker_main(hanf_server *s, int w)
{
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<std::shared_ptr<Job>> jobs;
        BatchPlan plan;
        size_t off = 0, bytes = 0;
        cudaStream_t st = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            for (;;) {
                if (s->stopping) return;
                // arrival order: the oldest queued job is admitted first
                if (admit(s, &jobs, &plan, &off, &bytes)) break;
                s->cv_work.wait(lk);
            }
            const Clock::time_point now = Clock::now();
            for (auto &j : jobs) {
                j->status = 2;
                j->t_start = now;
            }
            // jobs admitted while others run get lower priorities, in arrival
            // order: the oldest job's blocks are scheduled first, the newer
            // ones fill the SMs it leaves free; an idle GPU starts over
            if (s->running == 0) s->next_level = 0;
            st = s->streams[w][std::min(s->next_level, s->levels - 1)];
            ++s->next_level;
            ++s->running;
            ++s->contexts;
        }
        bool requeue = false;
        if (jobs.size() == 1) run_job(s, *jobs[0], s->arena + off, st);
        else requeue = !run_batch(s, jobs, plan, s->arena + off, st);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            const Clock::time_point now = Clock::now();
            s->alloc.release(off, bytes);
            --s->running;
            if (requeue) {
                // put the batch back, oldest first, to run one by one
                for (auto it = jobs.rbegin(); it != jobs.rend(); ++it) {
                    (*it)->alone = true;
                    (*it)->status = 1;
                    s->queue.push_front(*it);
                }
            } else {
                for (auto &j : jobs) {
                    j->t_end = now;
                    j->status = j->outcome;   // a waiter sees the result and its times together
                    if (j->status == HANF_OK) ++s->completed;
                    else ++s->failed;
                }
            }
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
    const double v[7] = {(double)s->queue.size(), (double)s->running, (double)s->completed,
                         (double)s->failed, (double)s->alloc.largest(), (double)s->arena_bytes,
                         (double)s->contexts};
    for (int i = 0; i < nout && i < 7; ++i) out[i] = v[i];
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
