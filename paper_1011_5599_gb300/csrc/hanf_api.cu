// C ABI of the GB300 HyperANF library: argument checking, workspace layout,
// graph preprocessing (validation, degree classes, hub segments, transpose),
// and the iteration drivers (host loop, or one CUDA graph whose while node
// repeats the pass until the device-side control block says stop).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "hanf.h"
#include "hanf_internal.cuh"

using hanf::DevCtl;
using hanf::Plan;

namespace {
thread_local std::string g_err;
}

void hanf::record_error(const char *msg) { g_err = msg; }

namespace {

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(HANF_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

constexpr int32_t kDefaultSmall = 256;    // hanf_autotune's choice on R-MAT scale 27 and 24
constexpr int32_t kDefaultSmallWide = 32; // its choice for rows of 512 bytes and more (web-like, R = 8)
constexpr int32_t kDefaultHub = 16384;
constexpr int32_t kDefaultHistory = 4096;
constexpr int64_t kStageRows = 65536;   // rows per chunk of a relabelled register read

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Host-side splitmix64 output step, for the run seeds.
uint64_t host_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// alpha_m of the HyperLogLog estimator (published constants).
double hll_alpha(int m)
{
    switch (m) {
    case 16: return 0.673;
    case 32: return 0.697;
    case 64: return 0.709;
    default: return 0.7213 / (1.0 + 1.079 / (double)m);
    }
}

struct Sizes {
    int64_t n, arcs;
    int32_t log2m, m, R, W, layout, K, S;
    int32_t d_small, d_hub, history;
    bool copy_graph, transpose, relabel, node_stats, est_fused;
    int64_t nwords, ntiles, max_hub, max_seg, scan_elems;
};

struct Layout {
    size_t off, tgt, in_off, in_src, regs0, regs1, F0, F1, cand, cand0, cand1, nodes;
    size_t seg_node, seg_beg, seg_end, hub_first, hub_part, hub_any;
    size_t blk_q, est_acc, ecache, hist, lc, seeds, ctl, scan_tmp, blk_counts, blk_offs;
    size_t seg_counts, seg_offs, totals, perm, inv, off2, tgt2, rcounts, roffs, stage;
    size_t ns_prev, ns_dist, ns_reach, ns_ecc, ns_rad;
    size_t slot_T, slot_changed, blk_graph, g_base, g_nodes, hr;
    size_t total;
};

int make_sizes(int64_t n, int64_t arcs, int32_t log2m, const hanf_opts &o, int32_t copy_graph,
               Sizes *s)
{
    if (log2m < 4 || log2m > 8) return fail(HANF_EINVAL, "log2m=%d outside 4..8", log2m);
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(HANF_EINVAL, "n=%lld out of range", (long long)n);
    if (arcs < 0) return fail(HANF_EINVAL, "arcs=%lld negative", (long long)arcs);
    if (o.runs < 1 || o.runs > hanf::kMaxRuns)
        return fail(HANF_EINVAL, "runs=%d outside 1..%d", o.runs, hanf::kMaxRuns);
    if (o.frontier < HANF_FRONTIER_OFF || o.frontier > HANF_FRONTIER_AUTO)
        return fail(HANF_EINVAL, "frontier=%d invalid", o.frontier);
    if (o.push_den < 1) return fail(HANF_EINVAL, "push_den=%d < 1", o.push_den);
    if (o.dense_den < 0) return fail(HANF_EINVAL, "dense_den=%d < 0", o.dense_den);
    if (o.gather_variant < 0 || o.gather_variant > 4)
        return fail(HANF_EINVAL, "gather_variant=%d invalid", o.gather_variant);
    if (o.small_max_deg < 0 || o.hub_min_deg < 0 || o.history_cap < 0)
        return fail(HANF_EINVAL, "negative tuning option");
    s->n = n;
    s->arcs = arcs;
    s->log2m = log2m;
    s->m = 1 << log2m;
    s->R = o.runs;
    s->layout = o.layout;
    if (o.layout < 0 || o.layout > 1) return fail(HANF_EINVAL, "layout=%d invalid", o.layout);
    if (o.layout == 1 && (o.runs != 1 || log2m < 5))
        return fail(HANF_EINVAL, "the bit-sliced layout needs runs = 1 and log2m >= 5");
    s->W = s->m * s->R;
    if (o.layout == 0 && s->W != 16 && s->W != 32 && s->W != 64 && s->W != 128 && s->W != 256 && s->W != 512 &&
        s->W != 1024 && s->W != 2048)
        return fail(HANF_EINVAL, "runs * m = %d must be a power of two (runs 1, 2, 4 or 8)", s->W);
    if (o.layout == 1) s->W = 5 * s->m / 8;
    s->d_small = o.small_max_deg ? o.small_max_deg
                                 : (o.layout == 0 && s->W >= 512 ? kDefaultSmallWide : kDefaultSmall);
    s->d_hub = o.hub_min_deg ? o.hub_min_deg : kDefaultHub;
    if (s->d_hub < 2) return fail(HANF_EINVAL, "hub_min_deg=%d < 2", s->d_hub);
    if (s->d_small > s->d_hub) s->d_small = s->d_hub;
    s->history = o.history_cap ? o.history_cap : kDefaultHistory;
    s->copy_graph = copy_graph != 0;
    s->transpose = o.frontier == HANF_FRONTIER_AUTO;
    s->K = o.num_graphs ? o.num_graphs : 1;
    if (s->K < 1) return fail(HANF_EINVAL, "num_graphs=%d < 1", o.num_graphs);
    if (s->K > 1) {
        if (!o.graph_base || !o.graph_nodes) return fail(HANF_EINVAL, "batch tables are NULL");
        if (o.graph_base[0] != 0 || o.graph_base[s->K] != n)
            return fail(HANF_EINVAL, "graph_base must start at 0 and end at n");
        for (int g = 0; g < s->K; ++g) {
            if ((o.graph_base[g] & 63) != 0 || o.graph_base[g + 1] < o.graph_base[g])
                return fail(HANF_EINVAL, "graph %d does not start at a multiple of 64", g);
            if (o.graph_nodes[g] < 0 || o.graph_nodes[g] > o.graph_base[g + 1] - o.graph_base[g])
                return fail(HANF_EINVAL, "graph %d has more nodes than its range", g);
        }
    }
    s->S = s->K * s->R;
    s->relabel = o.relabel != 0 && n > 0 && s->K == 1;
    s->node_stats = o.node_stats != 0;
    // only the changed counters' size() is evaluated after a pass (one graph,
    // byte registers, no per-node statistics, which keep the block sums)
    s->est_fused = s->layout == 0 && s->K == 1 && !s->node_stats;
    s->nwords = std::max<int64_t>(1, (n + 63) / 64);
    s->ntiles = hanf::classify_blocks(n);
    s->max_hub = arcs / (s->d_hub + 1) + 1;
    s->max_seg = 2 * (arcs / s->d_hub) + 2;
    if (s->max_seg >= (int64_t(1) << 31))   // hub segments are numbered with int32
        return fail(HANF_EINVAL, "hub_min_deg=%d is too small for %lld arcs", s->d_hub,
                    (long long)arcs);
    int64_t biggest = std::max<int64_t>({n + 1, 3 * s->ntiles + 1, s->max_hub + 1,
                                         hanf::relabel_count_elems(n)});
    s->scan_elems = hanf::scan_tmp_elems(biggest) * 2 + 64;
    return HANF_OK;
}

Layout make_layout(const Sizes &s)
{
    Layout L{};
    size_t at = 0;
    auto take = [&](size_t bytes) {
        size_t here = at;
        at += align256(std::max<size_t>(bytes, 16));
        return here;
    };
    const size_t rows = (size_t)std::max<int64_t>(s.n, 1);
    L.off = s.copy_graph ? take(sizeof(int64_t) * (s.n + 1)) : 0;
    L.tgt = s.copy_graph ? take(sizeof(int32_t) * std::max<int64_t>(s.arcs, 1)) : 0;
    L.in_off = s.transpose ? take(sizeof(int64_t) * (s.n + 1)) : 0;
    L.in_src = s.transpose ? take(sizeof(int32_t) * std::max<int64_t>(s.arcs, 1)) : 0;
    L.regs0 = take(rows * s.W);
    L.regs1 = take(std::max(rows * s.W, sizeof(int64_t) * (s.n + 1)));
    L.F0 = take(8 * s.nwords);
    L.F1 = take(8 * s.nwords);
    L.cand = take(8 * s.nwords);
    L.cand0 = s.transpose ? take(4 * rows) : 0;
    L.cand1 = s.transpose ? take(4 * rows) : 0;
    L.nodes = take(4 * rows);
    L.seg_node = take(4 * s.max_seg);
    L.seg_beg = take(8 * s.max_seg);
    L.seg_end = take(8 * s.max_seg);
    L.hub_first = take(4 * (s.max_hub + 1));
    L.hub_part = take((size_t)s.max_seg * s.W);
    L.hub_any = take(s.max_seg);
    L.blk_q = take(16 * s.nwords * s.R);
    L.est_acc = take(16 * (size_t)s.S);
    L.ecache = s.est_fused ? take(8 * rows * (size_t)s.R) : 0;
    L.hr = s.layout == 0 ? take(2 * rows * (size_t)s.R) : 0;
    L.hist = take(8 * (size_t)s.history * s.S);
    L.lc = take(8 * (s.m + 1));
    L.seeds = take(8 * (size_t)s.S);
    L.slot_T = take(4 * (size_t)s.S);
    L.slot_changed = take(8 * (size_t)s.S);
    if (s.K > 1) {
        L.blk_graph = take(4 * (size_t)s.nwords);
        L.g_base = take(8 * (size_t)(s.K + 1));
        L.g_nodes = take(8 * (size_t)s.K);
    }
    L.ctl = take(sizeof(DevCtl));
    L.scan_tmp = take(8 * s.scan_elems);
    L.blk_counts = take(8 * (3 * s.ntiles + 1));
    L.blk_offs = take(8 * (3 * s.ntiles + 1));
    L.seg_counts = take(8 * (s.max_hub + 1));
    L.seg_offs = take(8 * (s.max_hub + 1));
    L.totals = take(8 * 4);
    if (s.relabel) {
        L.perm = take(4 * rows);
        L.inv = take(4 * rows);
        L.off2 = take(8 * (s.n + 1));
        L.tgt2 = take(4 * std::max<int64_t>(s.arcs, 1));
        L.rcounts = take(8 * hanf::relabel_count_elems(s.n));
        L.roffs = take(8 * hanf::relabel_count_elems(s.n));
    }
    if (s.node_stats) {
        const size_t cells = rows * (size_t)s.R;
        L.ns_prev = take(8 * cells);
        L.ns_dist = take(8 * cells);
        L.ns_reach = take(8 * cells);
        L.ns_ecc = take(4 * cells);
        L.ns_rad = take(4 * cells);
    }
    if (s.relabel || s.layout || s.node_stats)
        L.stage = take((size_t)std::min<int64_t>(std::max<int64_t>(s.n, 1), kStageRows) *
                       std::max(std::max(s.W, s.m), 8));
    L.total = at;
    return L;
}

hanf_opts opts_or_default(const hanf_opts *o)
{
    hanf_opts d;
    hanf_default_opts(&d);
    return o ? *o : d;
}

}  // namespace

struct hanf_ctx {
    Plan plan;
    Sizes sz;
    hanf_opts opts;
    cudaStream_t stream;
    DevCtl host_ctl;
    uint64_t seed;
    int nsm;
    cudaEvent_t ev[4];
    double union_ms, est_ms;
    int64_t launches;
    cudaGraphExec_t gexec;
    cudaStream_t capture_stream;
    hanf::PassFork fork;         // side stream + events of the union launch
    std::vector<uint64_t> seeds;
    std::vector<double> trace;   // 8 values per pass (hanf_trace)
    const int32_t *perm;         // input id -> stored row (relabelled), or null
    uint8_t *stage;              // staging rows for relabelled register reads
    size_t l2_window;            // bytes of hot rows kept persisting in L2 (0 = off)
    int graph_passes;            // passes in one iteration of the graph's loop body
    bool in_pass;                // between hanf_pass_begin and hanf_pass_end
    size_t l2_limit_before;      // the context's persisting-L2 limit before create
};

namespace {

int read_ctl(hanf_ctx *c)
{
    CU(cudaMemcpyAsync(&c->host_ctl, c->plan.ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return HANF_OK;
}

// Back to t = 0: control block, counters initialised (each node adds itself)
// and N(0).
int reset(hanf_ctx *c, int32_t max_t)
{
    DevCtl h;
    std::memset(&h, 0, sizeof h);
    h.max_t = max_t;
    CU(cudaMemcpyAsync(c->plan.ctl, &h, sizeof h, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemsetAsync(c->plan.slot_T, 0xff, sizeof(int32_t) * c->plan.S, c->stream));   // -1
    CU(cudaMemsetAsync(c->plan.est_acc, 0, 16 * (size_t)c->plan.S, c->stream));
    CU(hanf::launch_init(c->plan, c->stream));
    int nl = 1;
    CU(hanf::launch_estimate(c->plan, c->stream, &nl));
    c->launches = nl;
    c->union_ms = 0;
    c->est_ms = 0;
    c->trace.clear();
    CU(cudaStreamSynchronize(c->stream));   // h lives on this stack frame
    c->host_ctl = h;
    return HANF_OK;
}

// Access-policy window over the hottest rows of the buffer the coming pass
// reads (stored first), or none (bytes = 0).
int set_l2_window(hanf_ctx *c, cudaStream_t stream, const void *base, size_t bytes)
{
    cudaStreamAttrValue v;
    std::memset(&v, 0, sizeof v);
    v.accessPolicyWindow.base_ptr = const_cast<void *>(base);
    v.accessPolicyWindow.num_bytes = bytes;
    v.accessPolicyWindow.hitRatio = bytes ? 1.0f : 0.0f;
    v.accessPolicyWindow.hitProp = bytes ? cudaAccessPropertyPersisting : cudaAccessPropertyNormal;
    v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    CU(cudaStreamSetAttribute(stream, cudaStreamAttributeAccessPolicyWindow, &v));
    if (c->fork.side)
        CU(cudaStreamSetAttribute(c->fork.side, cudaStreamAttributeAccessPolicyWindow, &v));
    return HANF_OK;
}

int one_pass(hanf_ctx *c)
{
    const bool prof = c->opts.profile != 0;
    const DevCtl before = c->host_ctl;
    int nl = 0;
    if (c->l2_window) {
        const int rc = set_l2_window(c, c->stream, c->plan.regs[c->host_ctl.parity], c->l2_window);
        if (rc) return rc;
    }
    const cudaError_t le = hanf::launch_pass(c->plan, c->stream, 0, 0, prof ? c->ev[0] : nullptr,
                                             prof ? c->ev[1] : nullptr, &nl, &c->fork);
    if (c->l2_window) {
        const int rc = set_l2_window(c, c->stream, nullptr, 0);
        if (rc) return rc;
    }
    CU(le);
    c->launches += nl;
    int rc = read_ctl(c);
    if (rc) return rc;
    if (prof) {
        float ms = 0;
        CU(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
        c->union_ms += ms;
        const DevCtl &a = c->host_ctl;
        const double row[8] = {(double)before.t,
                               (double)a.mode,
                               (double)a.last_changed,
                               (double)ms,
                               (double)(a.arcs_scanned - before.arcs_scanned),
                               (double)(a.arcs_gathered - before.arcs_gathered),
                               (double)(a.own_reads - before.own_reads),
                               (double)(a.writes - before.writes)};
        c->trace.insert(c->trace.end(), row, row + 8);
    }
    return HANF_OK;
}

int build_graph(hanf_ctx *c)
{
    if (c->gexec) return HANF_OK;
    cudaGraph_t g = nullptr;
    CU(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    CU(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CU(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    if (!c->capture_stream) CU(cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
    CU(cudaStreamBeginCaptureToGraph(c->capture_stream, body, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    int nl = 0;
    cudaError_t le = cudaSuccess;
    if (c->l2_window) {
        // two passes a loop iteration, each with the window over the hot rows
        // of the buffer it reads (a run starts at t = 0, reading regs[0])
        for (int q = 0; q < 2 && le == cudaSuccess; ++q) {
            if (set_l2_window(c, c->capture_stream, c->plan.regs[q], c->l2_window) != HANF_OK)
                le = cudaErrorUnknown;
            else
                le = hanf::launch_pass(c->plan, c->capture_stream, h, 1, nullptr, nullptr, &nl,
                                       &c->fork);
        }
        if (le == cudaSuccess && set_l2_window(c, c->capture_stream, nullptr, 0) != HANF_OK)
            le = cudaErrorUnknown;
        c->graph_passes = 2;
    } else {
        le = hanf::launch_pass(c->plan, c->capture_stream, h, 1, nullptr, nullptr, &nl, &c->fork);
        c->graph_passes = 1;
    }
    cudaGraph_t captured = nullptr;
    cudaError_t ee = cudaStreamEndCapture(c->capture_stream, &captured);
    if (le != cudaSuccess || ee != cudaSuccess) {
        cudaGraphDestroy(g);
        return fail(HANF_ECUDA, "graph capture failed: %s / %s", cudaGetErrorString(le),
                    cudaGetErrorString(ee));
    }
    cudaError_t ie = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        c->gexec = nullptr;
        return fail(HANF_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(ie));
    }
    return HANF_OK;
}

// Status of a loop stopped by the device: ERANGE (history or pass limit) or
// ESTATE (a scatter pass found a register outside 0..31).
int ctl_fail(int32_t err)
{
    if (err == HANF_ESTATE)
        return fail(HANF_ESTATE, "a scatter pass exceeded its compare-and-swap bound "
                                 "(registers outside 0..31)");
    return fail(err, "history capacity exhausted");
}

int pass_launch_count(const hanf_ctx *c)
{
    const Plan &p = c->plan;
    const bool scatter = !p.layout && p.in_off && p.scatter_den > 0;
    return 5 + (p.in_off ? 1 : 0) + (p.n_hub ? 1 : 0) + (p.S > 8 ? 1 : 0) +
           (!p.layout && p.W <= 128 ? 1 : 0) + (scatter ? 2 : 0) + (p.est_fused ? 3 : 2) +
           (!p.layout && p.first_warps > 0 ? 2 : 0);   // the pass-0 kernels
}

}  // namespace

extern "C" {

void hanf_default_opts(hanf_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->runs = 1;
    o->frontier = HANF_FRONTIER_AUTO;
    o->push_den = 4;
    o->small_max_deg = 0;
    o->hub_min_deg = 0;
    o->history_cap = 0;
    o->use_graph = 0;
    o->profile = 0;
    o->dense_den = 0;
    o->scatter_den = 0;
    o->relabel = 1;
    o->gather_variant = 0;
    o->layout = 0;
    o->node_stats = 0;
    o->num_graphs = 1;
    o->graph_base = nullptr;
    o->graph_nodes = nullptr;
    o->graph_seeds = nullptr;
    o->seeds = nullptr;
    o->stream = nullptr;
}

int hanf_workspace_size(int64_t n, int64_t arcs, int32_t log2m, const hanf_opts *opts,
                        int32_t copy_graph, size_t *bytes_out)
{
    if (!bytes_out) return fail(HANF_EINVAL, "bytes_out is NULL");
    Sizes s;
    int rc = make_sizes(n, arcs, log2m, opts_or_default(opts), copy_graph, &s);
    if (rc) return rc;
    *bytes_out = make_layout(s).total;
    return HANF_OK;
}

int hanf_create(hanf_ctx **out, int64_t n, int64_t arcs, const int64_t *offsets,
                const int32_t *targets, int32_t graph_on_device, int32_t log2m, uint64_t seed,
                const hanf_opts *opts, void *workspace, size_t workspace_bytes)
{
    if (!out) return fail(HANF_EINVAL, "out is NULL");
    const hanf_opts o = opts_or_default(opts);
    Sizes s;
    int rc = make_sizes(n, arcs, log2m, o, graph_on_device ? 0 : 1, &s);
    if (rc) return rc;
    if (!offsets || (arcs > 0 && !targets)) return fail(HANF_EINVAL, "CSR pointer is NULL");
    const Layout L = make_layout(s);
    if (!workspace) return fail(HANF_EINVAL, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(workspace) & 255)
        return fail(HANF_EINVAL, "workspace is not 256-byte aligned");
    if (workspace_bytes < L.total)
        return fail(HANF_ENOMEM, "workspace of %zu bytes, %zu needed", workspace_bytes, L.total);

    hanf_ctx *c = new (std::nothrow) hanf_ctx();
    if (!c) return fail(HANF_ENOMEM, "host allocation failed");
    auto bail = [&](int code) {
        if (c->ev[0]) for (auto &e : c->ev) if (e) cudaEventDestroy(e);
        if (c->fork.side) cudaStreamDestroy(c->fork.side);
        if (c->fork.fork) cudaEventDestroy(c->fork.fork);
        if (c->fork.join) cudaEventDestroy(c->fork.join);
        delete c;
        return code;
    };
    c->sz = s;
    c->opts = o;
    c->seed = seed;
    c->stream = static_cast<cudaStream_t>(o.stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bail(fail(HANF_ECUDA, "no CUDA device"));
    for (auto &e : c->ev)
        if (cudaEventCreate(&e) != cudaSuccess) return bail(fail(HANF_ECUDA, "event create failed"));
    int prio = 0;   // the side stream runs at the priority of the context's stream
    if (cudaStreamGetPriority(c->stream, &prio) != cudaSuccess) prio = 0;
    if (cudaStreamCreateWithPriority(&c->fork.side, cudaStreamNonBlocking, prio) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork.join, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(HANF_ECUDA, "side stream create failed"));

    uint8_t *ws = static_cast<uint8_t *>(workspace);
    Plan &p = c->plan;
    std::memset(&p, 0, sizeof p);
    p.n = n;
    p.arcs = arcs;
    p.b = log2m;
    p.m = s.m;
    p.R = s.R;
    p.W = s.W;
    p.layout = s.layout;
    p.nwords = s.nwords;
    p.frontier = o.frontier;
    p.push_den = o.push_den;
    // dense pulls while changed in-arcs >= arcs * dense_num / dense_den.  The
    // per-arc bitmap test pays off sooner with wide rows: with 512-byte rows
    // (web-like graph, 8 runs) a tested pass beat a dense one below about 92%
    // of the successors changed, while with 64- and 128-byte rows it was
    // slower even at 82% (R-MAT 27 pass 4: 34 against 23 ms)
    p.dense_num = o.dense_den ? 1 : (p.W >= 512 ? 15 : 1);
    p.dense_den = o.dense_den ? o.dense_den : (p.W >= 512 ? 16 : 2);
    // scatter passes by default for rows of at most 128 bytes: with wider rows a
    // pushed pair costs a whole row of compare-and-swaps and the systolic pull
    // measured faster (web-like graph, 512-byte rows)
    p.scatter_den = o.scatter_den == 0 ? (p.W <= 128 && !p.layout ? 8 : 0)
                                       : std::max(o.scatter_den, 0);
    p.scatter_seg = 2048;     // in-arcs per segment of a long in-list
    p.scatter_inline = 256;   // in-lists up to this length are pushed whole
    p.history_cap = s.history;
    cudaStream_t st = c->stream;
    if (s.copy_graph) {
        int64_t *doff = reinterpret_cast<int64_t *>(ws + L.off);
        int32_t *dtgt = reinterpret_cast<int32_t *>(ws + L.tgt);
        if (cudaMemcpyAsync(doff, offsets, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            (arcs > 0 && cudaMemcpyAsync(dtgt, targets, sizeof(int32_t) * arcs,
                                         cudaMemcpyHostToDevice, st) != cudaSuccess))
            return bail(fail(HANF_ECUDA, "graph upload failed: %s",
                             cudaGetErrorString(cudaGetLastError())));
        p.off = doff;
        p.tgt = dtgt;
    } else {
        p.off = offsets;
        p.tgt = targets;
    }
    p.regs[0] = ws + L.regs0;
    p.regs[1] = ws + L.regs1;
    p.F[0] = reinterpret_cast<unsigned long long *>(ws + L.F0);
    p.F[1] = reinterpret_cast<unsigned long long *>(ws + L.F1);
    p.cand = reinterpret_cast<unsigned long long *>(ws + L.cand);
    if (s.transpose) {
        p.cand_list[0] = reinterpret_cast<int32_t *>(ws + L.cand0);
        p.cand_list[1] = reinterpret_cast<int32_t *>(ws + L.cand1);
    }
    p.d_small = s.d_small;
    p.d_hub = s.d_hub;
    int32_t *nodes = reinterpret_cast<int32_t *>(ws + L.nodes);
    p.nodes = nodes;
    p.hub_part = ws + L.hub_part;
    p.hub_any = ws + L.hub_any;
    p.blk_q = reinterpret_cast<unsigned long long *>(ws + L.blk_q);
    p.est_acc = reinterpret_cast<unsigned long long *>(ws + L.est_acc);
    p.est_fused = s.est_fused ? 1 : 0;
    p.ecache = s.est_fused ? reinterpret_cast<double *>(ws + L.ecache) : nullptr;
    p.hr = s.layout == 0 ? reinterpret_cast<uint16_t *>(ws + L.hr) : nullptr;
    p.hist = reinterpret_cast<double *>(ws + L.hist);
    p.lc = reinterpret_cast<const double *>(ws + L.lc);
    p.seeds = reinterpret_cast<const uint64_t *>(ws + L.seeds);
    p.ctl = reinterpret_cast<DevCtl *>(ws + L.ctl);
    p.amm = hll_alpha(s.m) * (double)s.m * (double)s.m;
    int64_t *scan_tmp = reinterpret_cast<int64_t *>(ws + L.scan_tmp);
    int64_t *totals = reinterpret_cast<int64_t *>(ws + L.totals);

    p.K = s.K;
    p.S = s.S;
    p.slot_T = reinterpret_cast<int32_t *>(ws + L.slot_T);
    p.slot_changed = reinterpret_cast<unsigned long long *>(ws + L.slot_changed);
    if (s.K > 1) {
        // batch tables: the graph of every 64-node block, bases, node counts
        std::vector<int32_t> bg(s.nwords, 0);
        for (int g = 0; g < s.K; ++g)
            for (int64_t b = o.graph_base[g] >> 6; b < ((o.graph_base[g + 1] + 63) >> 6) && b < s.nwords; ++b)
                bg[b] = g;
        int32_t *d_bg = reinterpret_cast<int32_t *>(ws + L.blk_graph);
        int64_t *d_base = reinterpret_cast<int64_t *>(ws + L.g_base);
        int64_t *d_nodes = reinterpret_cast<int64_t *>(ws + L.g_nodes);
        if (cudaMemcpyAsync(d_bg, bg.data(), 4 * s.nwords, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(d_base, o.graph_base, 8 * (s.K + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(d_nodes, o.graph_nodes, 8 * s.K, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return bail(fail(HANF_ECUDA, "batch table upload failed"));
        p.blk_graph = d_bg;
        p.g_base = d_base;
        p.g_nodes = d_nodes;
    }

    // 1. validate the CSR on the device
    if (cudaMemsetAsync(p.ctl, 0, sizeof(DevCtl), st) != cudaSuccess ||
        hanf::launch_validate(p, st) != cudaSuccess || read_ctl(c) != HANF_OK)
        return bail(fail(HANF_ECUDA, "validation failed: %s", g_err.c_str()));
    if (c->host_ctl.bad_graph)
        return bail(fail(HANF_EINVAL, "invalid CSR: offsets must start at 0, end at arcs and "
                                      "not decrease; targets must lie in [0, n)"));

    // 1b. store nodes by decreasing in-degree class: the relabelled CSR
    //     replaces the input one for everything below
    if (s.relabel) {
        int32_t *perm = reinterpret_cast<int32_t *>(ws + L.perm);
        int32_t *inv = reinterpret_cast<int32_t *>(ws + L.inv);
        int64_t *off2 = reinterpret_cast<int64_t *>(ws + L.off2);
        int32_t *tgt2 = reinterpret_cast<int32_t *>(ws + L.tgt2);
        if (hanf::launch_relabel(p.off, p.tgt, n, arcs,
                                 reinterpret_cast<unsigned long long *>(p.regs[1]),
                                 reinterpret_cast<int64_t *>(ws + L.rcounts),
                                 reinterpret_cast<int64_t *>(ws + L.roffs), scan_tmp, s.scan_elems,
                                 perm, inv, reinterpret_cast<int64_t *>(p.regs[0]), off2,
                                 tgt2, st) != cudaSuccess)
            return bail(fail(HANF_ECUDA, "relabelling failed: %s",
                             cudaGetErrorString(cudaGetLastError())));
        p.off = off2;
        p.tgt = tgt2;
        p.orig_id = inv;
        c->perm = perm;
    }
    if (s.relabel || s.layout || s.node_stats) c->stage = ws + L.stage;
    if (s.node_stats) {
        p.node_stats = 1;
        p.ns_prev = reinterpret_cast<double *>(ws + L.ns_prev);
        p.ns_dist = reinterpret_cast<double *>(ws + L.ns_dist);
        p.ns_reach = reinterpret_cast<double *>(ws + L.ns_reach);
        p.ns_ecc = reinterpret_cast<int32_t *>(ws + L.ns_ecc);
        p.ns_rad = reinterpret_cast<int32_t *>(ws + L.ns_rad);
    }

    // 2. degree classes -> [small | medium | hub] node lists
    int64_t tot[4] = {0, 0, 0, 0};
    if (cudaMemsetAsync(totals, 0, 4 * sizeof(int64_t), st) != cudaSuccess ||
        hanf::launch_classify(p, s.d_small, s.d_hub, reinterpret_cast<int64_t *>(ws + L.blk_counts),
                              reinterpret_cast<int64_t *>(ws + L.blk_offs), scan_tmp, s.scan_elems,
                              nodes, totals, st) != cudaSuccess ||
        cudaMemcpyAsync(tot, totals, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return bail(fail(HANF_ECUDA, "degree classification failed: %s",
                         cudaGetErrorString(cudaGetLastError())));
    p.n_small = tot[0];
    p.n_med = tot[1] - tot[0];
    p.n_hub = tot[2] - tot[1];

    // 3. hub segments
    p.seg_node = reinterpret_cast<int32_t *>(ws + L.seg_node);
    p.seg_beg = reinterpret_cast<int64_t *>(ws + L.seg_beg);
    p.seg_end = reinterpret_cast<int64_t *>(ws + L.seg_end);
    p.hub_seg_first = reinterpret_cast<int32_t *>(ws + L.hub_first);
    if (p.n_hub > 0) {
        int64_t nseg = 0;
        if (hanf::launch_hub_segments(p, s.d_hub, reinterpret_cast<int64_t *>(ws + L.seg_counts),
                                      reinterpret_cast<int64_t *>(ws + L.seg_offs), scan_tmp,
                                      s.scan_elems, const_cast<int32_t *>(p.seg_node),
                                      const_cast<int64_t *>(p.seg_beg),
                                      const_cast<int64_t *>(p.seg_end),
                                      const_cast<int32_t *>(p.hub_seg_first), totals + 3,
                                      st) != cudaSuccess ||
            cudaMemcpyAsync(&nseg, totals + 3, sizeof(int64_t), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return bail(fail(HANF_ECUDA, "hub segmentation failed: %s",
                             cudaGetErrorString(cudaGetLastError())));
        p.n_seg = nseg;
    }

    // 4. transpose for systolic signalling (regs[1] is free scratch until init)
    if (s.transpose) {
        int64_t *in_off = reinterpret_cast<int64_t *>(ws + L.in_off);
        int32_t *in_src = reinterpret_cast<int32_t *>(ws + L.in_src);
        // after relabelling, regs[1] still holds the input in-degrees and
        // regs[0] is free scratch for the permuted counts
        if (hanf::launch_transpose(p, in_off, in_src, reinterpret_cast<int64_t *>(p.regs[1]),
                                   scan_tmp, s.scan_elems,
                                   s.relabel ? reinterpret_cast<const unsigned long long *>(p.regs[1])
                                             : nullptr,
                                   s.relabel ? p.orig_id : nullptr,
                                   reinterpret_cast<int64_t *>(p.regs[0]), st) != cudaSuccess)
            return bail(fail(HANF_ECUDA, "transpose failed: %s",
                             cudaGetErrorString(cudaGetLastError())));
        p.in_off = in_off;
        p.in_src = in_src;
    }

    // 5. run seeds and the linear-counting table m ln(m/V), V = 1..m
    c->seeds.resize(s.S);
    for (int g = 0; g < s.K; ++g)
        for (int r = 0; r < s.R; ++r) {
            const uint64_t base_seed = (s.K > 1 && o.graph_seeds) ? o.graph_seeds[g] : seed;
            c->seeds[(size_t)g * s.R + r] =
                (s.K == 1 && o.seeds) ? o.seeds[r] : host_splitmix64(base_seed + (uint64_t)r);
        }
    std::vector<double> lc(s.m + 1, 0.0);
    for (int V = 1; V <= s.m; ++V) lc[V] = (double)s.m * std::log((double)s.m / (double)V);
    if (cudaMemcpyAsync(const_cast<uint64_t *>(p.seeds), c->seeds.data(), 8 * (size_t)s.S,
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(const_cast<double *>(p.lc), lc.data(), 8 * (s.m + 1),
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
        return bail(fail(HANF_ECUDA, "constant upload failed"));
    p.union_warps = s.layout ? hanf::packed_occupancy_warps(s.m, c->nsm)
                             : hanf::union_occupancy_warps(s.W, c->nsm);
    p.scatter_warps = s.layout ? 0 : hanf::scatter_occupancy_warps(s.W, c->nsm);
    p.union_async_warps = s.layout ? 0 : hanf::union_async_warps(s.W, c->nsm);
    p.warp_variant = ((o.gather_variant == 2 || o.gather_variant == 4) && p.union_async_warps > 0) ? 2 : 1;
    // asynchronous copies in the small-degree kernel by default (rows of at
    // most 128 bytes; measured 26.4 -> 25.1 ms a dense R-MAT 27 pass)
    // pass 0 from the two-byte c_0 records (byte layout, rows up to 1 KB)
    p.first_warps = p.hr ? hanf::first_pass_warps(s.W, c->nsm) : 0;
    p.small_variant = ((o.gather_variant == 0 || o.gather_variant >= 3) && !s.layout &&
                       s.W <= 128 && hanf::small_async_blocks(s.W) > 0)
                          ? 3
                          : 0;

    // persisting-L2 window: explicit size, or by default 64 MiB for counter
    // arrays of 1 GiB and more (measured best on R-MAT 27, m = 64)
    const int64_t l2_want = o.l2_hot_bytes != 0
                                ? o.l2_hot_bytes
                                : ((int64_t)std::max<int64_t>(n, 1) * s.W >= (int64_t(1) << 30)
                                       ? int64_t(64) << 20
                                       : 0);
    if (l2_want > 0 && s.layout == 0) {
        // persisting L2 lines for the hottest counter rows (host-loop driver)
        int max_persist = 0, max_window = 0;
        size_t before = 0;
        if (cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev) !=
                cudaSuccess ||
            cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, dev) !=
                cudaSuccess ||
            cudaDeviceGetLimit(&before, cudaLimitPersistingL2CacheSize) != cudaSuccess)
            return bail(fail(HANF_ECUDA, "L2 persistence queries failed"));
        const size_t want = std::min<size_t>({(size_t)l2_want, (size_t)max_persist,
                                              (size_t)max_window, (size_t)std::max<int64_t>(n, 1) * s.W});
        if (want > 0) {
            if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, std::max(want, before)) != cudaSuccess)
                return bail(fail(HANF_ECUDA, "cannot set the persisting L2 limit"));
            c->l2_window = want;
            c->l2_limit_before = before;
        }
    }

    rc = reset(c, s.history);
    if (rc) return bail(rc);
    *out = c;
    return HANF_OK;
}

int hanf_estimate(hanf_ctx *c, double *N_out)
{
    if (!c || !N_out) return fail(HANF_EINVAL, "NULL argument");
    int rc = read_ctl(c);
    if (rc) return rc;
    CU(cudaMemcpyAsync(N_out, c->plan.hist + (int64_t)c->host_ctl.t * c->plan.S,
                       sizeof(double) * c->plan.S, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return HANF_OK;
}

int hanf_iterate(hanf_ctx *c, int64_t *changed_out)
{
    if (!c) return fail(HANF_EINVAL, "NULL context");
    if (c->in_pass) return fail(HANF_ESTATE, "a stepped pass is open");
    int rc = read_ctl(c);
    if (rc) return rc;
    if (c->host_ctl.done) {
        if (changed_out) *changed_out = 0;
        return c->host_ctl.err ? ctl_fail(c->host_ctl.err) : HANF_OK;
    }
    rc = one_pass(c);
    if (rc) return rc;
    if (changed_out) *changed_out = (int64_t)c->host_ctl.last_changed;
    if (c->host_ctl.err) return ctl_fail(c->host_ctl.err);
    return HANF_OK;
}

namespace {

// Run passes from the current state until stabilisation (or ctl.max_t), then
// copy N(0..T) and the T_r out.
int drive(hanf_ctx *c, double *N_out, int32_t cap, int32_t *T_out, int32_t max_iter);

}  // namespace

int hanf_run(hanf_ctx *c, int32_t max_iter, double *N_out, int32_t cap, int32_t *T_out)
{
    if (!c || !N_out || !T_out) return fail(HANF_EINVAL, "NULL argument");
    if (cap < 1 || max_iter < 1) return fail(HANF_EINVAL, "cap and max_iter must be >= 1");
    if (c->in_pass) return fail(HANF_ESTATE, "a stepped pass is open");
    const int32_t max_t = std::min<int32_t>(std::min(max_iter, cap), c->sz.history);
    int rc = reset(c, max_t);
    if (rc) return rc;
    return drive(c, N_out, cap, T_out, max_iter);
}

int hanf_continue(hanf_ctx *c, int32_t max_iter, double *N_out, int32_t cap, int32_t *T_out)
{
    if (!c || !N_out || !T_out) return fail(HANF_EINVAL, "NULL argument");
    if (cap < 1 || max_iter < 1) return fail(HANF_EINVAL, "cap and max_iter must be >= 1");
    if (c->in_pass) return fail(HANF_ESTATE, "a stepped pass is open");
    int rc = read_ctl(c);
    if (rc) return rc;
    DevCtl h = c->host_ctl;
    h.max_t = std::min<int32_t>(std::min<int64_t>((int64_t)h.t + max_iter, cap), c->sz.history);
    const bool limited = h.err == HANF_ERANGE && h.t < h.max_t;
    if (limited) {   // resume after a run that hit its pass limit
        h.err = HANF_OK;
        h.done = 0;
    }
    CU(cudaMemcpyAsync(c->plan.ctl, &h, sizeof h, cudaMemcpyHostToDevice, c->stream));
    if (limited) {
        // that run stopped before estimating N(t) at its last t
        int nl = 0;
        CU(hanf::launch_estimate(c->plan, c->stream, &nl));
        c->launches += nl;
    }
    CU(cudaStreamSynchronize(c->stream));
    c->host_ctl = h;
    return drive(c, N_out, cap, T_out, max_iter);
}

}  // extern "C"

namespace {

int drive(hanf_ctx *c, double *N_out, int32_t cap, int32_t *T_out, int32_t max_iter)
{
    int rc = HANF_OK;
    if (c->host_ctl.done) {
        // already stable (or stopped): nothing to run
    } else if (c->opts.use_graph) {
        rc = build_graph(c);
        if (rc) return rc;
        CU(cudaGraphLaunch(c->gexec, c->stream));
        rc = read_ctl(c);
        if (rc) return rc;
        const int64_t gp = std::max(c->graph_passes, 1);
        c->launches += (((int64_t)c->host_ctl.passes + gp - 1) / gp) * gp * pass_launch_count(c);
    } else {
        for (;;) {
            rc = one_pass(c);
            if (rc) return rc;
            if (c->host_ctl.done) break;
        }
    }
    const DevCtl &h = c->host_ctl;
    const int32_t S = c->plan.S;
    const int32_t T = h.t;   // N(0..T) valid (T = t at stop)
    const int32_t have = h.err ? T : T + 1;
    std::vector<double> hist((size_t)std::max(have, 1) * S);
    std::vector<int32_t> slotT(S);
    CU(cudaMemcpyAsync(hist.data(), c->plan.hist, sizeof(double) * have * S,
                       cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(slotT.data(), c->plan.slot_T, sizeof(int32_t) * S, cudaMemcpyDeviceToHost,
                       c->stream));
    CU(cudaStreamSynchronize(c->stream));
    for (int r = 0; r < S; ++r) {
        for (int t = 0; t < cap; ++t)
            N_out[(int64_t)r * cap + t] = t < have ? hist[(size_t)t * S + r] : 0.0;
        T_out[r] = slotT[r] >= 0 ? slotT[r] : T;
    }
    if (h.err == HANF_ESTATE) return ctl_fail(h.err);
    if (h.err) return fail(HANF_ERANGE, "no stabilisation within %d passes / %d values", max_iter, cap);
    return HANF_OK;
}

}  // namespace

extern "C" {

int hanf_registers(hanf_ctx *c, int32_t run, int64_t first, int64_t count, uint8_t *out)
{
    if (!c || (!out && count > 0)) return fail(HANF_EINVAL, "NULL argument");
    if (run < 0 || run >= c->plan.R) return fail(HANF_EINVAL, "run %d out of range", run);
    if (first < 0 || count < 0 || first + count > c->plan.n)
        return fail(HANF_EINVAL, "node range out of bounds");
    if (count == 0) return HANF_OK;
    int rc = read_ctl(c);
    if (rc) return rc;
    const uint8_t *regs = c->plan.regs[c->host_ctl.parity];
    const int W = c->plan.W, m = c->plan.m;
    if (c->plan.layout) {
        // bit-sliced storage: unpack one byte per register, chunk by chunk
        for (int64_t i = 0; i < count; i += kStageRows) {
            const int64_t k = std::min<int64_t>(kStageRows, count - i);
            CU(hanf::launch_unpack_rows(regs, c->perm, first + i, k, m, c->stage, c->stream));
            CU(cudaMemcpyAsync(out + i * m, c->stage, (size_t)k * m, cudaMemcpyDeviceToHost,
                               c->stream));
            CU(cudaStreamSynchronize(c->stream));
        }
        return HANF_OK;
    }
    if (!c->perm) {
        const uint8_t *src = regs + first * W + (int64_t)run * m;
        CU(cudaMemcpy2DAsync(out, m, src, W, m, count, cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
        return HANF_OK;
    }
    // relabelled storage: gather the rows into input order, chunk by chunk
    for (int64_t i = 0; i < count; i += kStageRows) {
        const int64_t k = std::min<int64_t>(kStageRows, count - i);
        CU(hanf::launch_gather_rows(regs, c->perm, first + i, k, W, c->stage, c->stream));
        CU(cudaMemcpy2DAsync(out + i * m, m, c->stage + (int64_t)run * m, W, m, k,
                             cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
    }
    return HANF_OK;
}

int hanf_digest(hanf_ctx *c, int32_t run, int64_t first, int64_t count, uint64_t *digest_out)
{
    if (!c || !digest_out) return fail(HANF_EINVAL, "NULL argument");
    if (run < 0 || run >= c->plan.R) return fail(HANF_EINVAL, "run %d out of range", run);
    if (first < 0 || count < 0 || first + count > c->plan.n)
        return fail(HANF_EINVAL, "node range out of bounds");
    unsigned long long *d = &c->plan.ctl->digest;
    CU(cudaMemsetAsync(d, 0, sizeof *d, c->stream));
    CU(hanf::launch_digest(c->plan, run, first, count, c->perm, d, c->stream));
    unsigned long long h = 0;
    CU(cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    *digest_out = h;
    return HANF_OK;
}

// ---- one pass in steps, for node-sharded runs ----

int hanf_pass_begin(hanf_ctx *c, int32_t *started_out)
{
    if (!c || !started_out) return fail(HANF_EINVAL, "NULL argument");
    if (c->in_pass) return fail(HANF_ESTATE, "a pass is already open");
    if (c->plan.layout != 0 || c->plan.K != 1)
        return fail(HANF_ESTATE, "stepped passes need the byte layout and one graph");
    int rc = read_ctl(c);
    if (rc) return rc;
    *started_out = 0;
    if (c->host_ctl.done) return c->host_ctl.err ? ctl_fail(c->host_ctl.err) : HANF_OK;
    if (c->l2_window) {
        rc = set_l2_window(c, c->stream, c->plan.regs[c->host_ctl.parity], c->l2_window);
        if (rc) return rc;
    }
    int nl = 0;
    const cudaError_t le = hanf::launch_pass_union(c->plan, c->stream, nullptr, nullptr, &nl, &c->fork);
    if (c->l2_window) {
        rc = set_l2_window(c, c->stream, nullptr, 0);
        if (rc) return rc;
    }
    CU(le);
    c->launches += nl;
    c->in_pass = true;
    *started_out = 1;
    return HANF_OK;
}

int hanf_pass_collect(hanf_ctx *c, int64_t first, int64_t count, int32_t *ids, uint8_t *rows,
                      int64_t cap, int64_t *n_out)
{
    if (!c || !n_out || (cap > 0 && (!ids || !rows))) return fail(HANF_EINVAL, "NULL argument");
    if (!c->in_pass) return fail(HANF_ESTATE, "no pass is open");
    if (first < 0 || count < 0 || first + count > c->plan.n || cap < 0)
        return fail(HANF_EINVAL, "node range out of bounds");
    if ((reinterpret_cast<uintptr_t>(rows) & 15) != 0)
        return fail(HANF_EINVAL, "rows must be 16-byte aligned");
    unsigned long long *d = &c->plan.ctl->shard_count;
    CU(cudaMemsetAsync(d, 0, sizeof *d, c->stream));
    CU(hanf::launch_shard_collect(c->plan, first, count, ids, rows, cap, c->stream));
    unsigned long long found = 0;
    CU(cudaMemcpyAsync(&found, d, sizeof found, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    c->launches += 1;
    *n_out = (int64_t)found;
    if ((int64_t)found > cap)
        return fail(HANF_ERANGE, "%lld changed nodes, room for %lld", (long long)found,
                    (long long)cap);
    return HANF_OK;
}

int hanf_pass_apply(hanf_ctx *c, const int32_t *ids, const uint8_t *rows, int64_t k)
{
    if (!c || (k > 0 && (!ids || !rows)) || k < 0) return fail(HANF_EINVAL, "bad argument");
    if (!c->in_pass) return fail(HANF_ESTATE, "no pass is open");
    if ((reinterpret_cast<uintptr_t>(rows) & 15) != 0)
        return fail(HANF_EINVAL, "rows must be 16-byte aligned");
    CU(hanf::launch_shard_apply(c->plan, c->perm, ids, rows, k, c->stream));
    if (k > 0) c->launches += 1;
    return HANF_OK;
}

int hanf_pass_end(hanf_ctx *c, int64_t *changed_out)
{
    if (!c) return fail(HANF_EINVAL, "NULL context");
    if (!c->in_pass) return fail(HANF_ESTATE, "no pass is open");
    c->in_pass = false;
    int nl = 0;
    CU(hanf::launch_pass_end(c->plan, c->stream, 0, 0, &nl));
    c->launches += nl;
    const int rc = read_ctl(c);
    if (rc) return rc;
    if (changed_out) *changed_out = (int64_t)c->host_ctl.last_changed;
    if (c->host_ctl.err) return ctl_fail(c->host_ctl.err);
    return HANF_OK;
}

int hanf_current_t(hanf_ctx *c, int32_t *t_out)
{
    if (!c || !t_out) return fail(HANF_EINVAL, "NULL argument");
    int rc = read_ctl(c);
    if (rc) return rc;
    *t_out = c->host_ctl.t;
    return HANF_OK;
}

int hanf_counters(hanf_ctx *c, double *out, int32_t nout)
{
    if (!c || !out) return fail(HANF_EINVAL, "NULL argument");
    int rc = read_ctl(c);
    if (rc) return rc;
    const DevCtl &h = c->host_ctl;
    const double v[10] = {(double)h.passes,        (double)h.arcs_scanned, (double)h.arcs_gathered,
                          (double)h.own_reads,     (double)h.writes,       (double)h.passes,
                          c->union_ms,             (double)c->launches,    c->est_ms,
                          (double)h.push_passes};
    for (int i = 0; i < nout && i < 10; ++i) out[i] = v[i];
    return HANF_OK;
}

int hanf_trace(hanf_ctx *c, double *out, int32_t max_rows, int32_t *rows_out)
{
    if (!c || !rows_out || (max_rows > 0 && !out)) return fail(HANF_EINVAL, "NULL argument");
    const int32_t rows = (int32_t)(c->trace.size() / 8);
    const int32_t k = std::min(rows, std::max(max_rows, 0));
    std::copy(c->trace.begin(), c->trace.begin() + 8 * (size_t)k, out);
    *rows_out = k;
    return HANF_OK;
}

int hanf_stats(const double *N, int32_t T, double alpha, int32_t exclude_zero, double *out5)
{
    if (!N || !out5 || T < 0) return fail(HANF_EINVAL, "bad argument");
    const double base = exclude_zero ? N[0] : 0.0;
    double M = N[0];
    for (int t = 1; t <= T; ++t) M = std::max(M, N[t]);
    double prev = 0.0, mean = 0.0, second = 0.0;
    out5[0] = out5[1] = NAN;
    bool found = false;
    for (int t = 0; t <= T; ++t) {
        const double H = (N[t] - base) / (M - base);
        const double h = H - prev;
        mean += t * h;
        second += (double)t * t * h;
        if (!found && H >= alpha) {
            found = true;
            out5[0] = t;
            out5[1] = t == 0 ? 0.0 : (t - 1) + (alpha - prev) / (H - prev);
        }
        prev = H;
    }
    out5[2] = mean;
    out5[3] = second - mean * mean;
    out5[4] = out5[3] / mean;
    return HANF_OK;
}

}  // extern "C"

namespace {

struct CkpHeader {
    char magic[8];
    int64_t n, arcs, nwords;
    int32_t log2m, R, layout, relabel, W, history, K, pad;
    uint64_t seed_hash;
};

struct CkpParts {
    size_t header, ctl, regs, bits, hist, blk, acc, cache, slots, total;
};

CkpParts ckp_parts(const hanf_ctx *c)
{
    const Plan &p = c->plan;
    CkpParts q;
    q.header = sizeof(CkpHeader);
    q.ctl = sizeof(DevCtl);
    q.regs = (size_t)std::max<int64_t>(p.n, 1) * p.W;
    q.bits = (size_t)p.nwords * 8;
    q.hist = (size_t)p.history_cap * p.S * 8;
    q.blk = (size_t)p.nwords * p.R * 16;
    q.acc = (size_t)p.S * 16;
    q.cache = p.est_fused ? (size_t)std::max<int64_t>(p.n, 1) * p.R * 8 : 0;
    q.slots = (size_t)p.S * 4;
    q.total = q.header + q.ctl + 2 * q.regs + 2 * q.bits + q.hist + q.blk + q.acc + q.cache +
              q.slots;
    return q;
}

CkpHeader ckp_header(const hanf_ctx *c)
{
    CkpHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, "HANFCKP2", 8);
    h.n = c->plan.n;
    h.arcs = c->plan.arcs;
    h.nwords = c->plan.nwords;
    h.log2m = c->plan.b;
    h.R = c->plan.R;
    h.layout = c->plan.layout;
    h.relabel = c->perm != nullptr;
    h.W = c->plan.W;
    h.history = c->plan.history_cap;
    h.K = c->plan.K;
    uint64_t x = 0x9E3779B97F4A7C15ull;
    for (uint64_t sd : c->seeds) x = host_splitmix64(x ^ sd);
    h.seed_hash = x;
    return h;
}

}  // namespace

extern "C" {

int hanf_checkpoint_size(hanf_ctx *c, size_t *bytes_out)
{
    if (!c || !bytes_out) return fail(HANF_EINVAL, "NULL argument");
    *bytes_out = ckp_parts(c).total;
    return HANF_OK;
}

int hanf_checkpoint_save(hanf_ctx *c, void *buf, size_t bytes)
{
    if (!c || !buf) return fail(HANF_EINVAL, "NULL argument");
    const CkpParts q = ckp_parts(c);
    if (bytes < q.total) return fail(HANF_ENOMEM, "checkpoint needs %zu bytes", q.total);
    int rc = read_ctl(c);
    if (rc) return rc;
    uint8_t *o = static_cast<uint8_t *>(buf);
    const CkpHeader h = ckp_header(c);
    std::memcpy(o, &h, sizeof h);
    std::memcpy(o + q.header, &c->host_ctl, sizeof(DevCtl));
    uint8_t *d = o + q.header + q.ctl;
    const Plan &p = c->plan;
    CU(cudaMemcpyAsync(d, p.regs[0], q.regs, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(d + q.regs, p.regs[1], q.regs, cudaMemcpyDeviceToHost, c->stream));
    d += 2 * q.regs;
    CU(cudaMemcpyAsync(d, p.F[0], q.bits, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(d + q.bits, p.F[1], q.bits, cudaMemcpyDeviceToHost, c->stream));
    d += 2 * q.bits;
    CU(cudaMemcpyAsync(d, p.hist, q.hist, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(d + q.hist, p.blk_q, q.blk, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(d + q.hist + q.blk, p.est_acc, q.acc, cudaMemcpyDeviceToHost, c->stream));
    if (q.cache)
        CU(cudaMemcpyAsync(d + q.hist + q.blk + q.acc, p.ecache, q.cache, cudaMemcpyDeviceToHost,
                           c->stream));
    CU(cudaMemcpyAsync(d + q.hist + q.blk + q.acc + q.cache, p.slot_T, q.slots,
                       cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return HANF_OK;
}

int hanf_checkpoint_load(hanf_ctx *c, const void *buf, size_t bytes)
{
    if (!c || !buf) return fail(HANF_EINVAL, "NULL argument");
    const CkpParts q = ckp_parts(c);
    if (bytes < q.total) return fail(HANF_EINVAL, "checkpoint of %zu bytes, %zu expected", bytes, q.total);
    const uint8_t *in = static_cast<const uint8_t *>(buf);
    CkpHeader h;
    std::memcpy(&h, in, sizeof h);
    const CkpHeader mine = ckp_header(c);
    if (std::memcmp(&h, &mine, sizeof h) != 0)
        return fail(HANF_EINVAL, "checkpoint belongs to another graph, layout or seed set");
    DevCtl ctl;
    std::memcpy(&ctl, in + q.header, sizeof ctl);
    const uint8_t *d = in + q.header + q.ctl;
    const Plan &p = c->plan;
    CU(cudaMemcpyAsync(p.ctl, &ctl, sizeof ctl, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(p.regs[0], d, q.regs, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(p.regs[1], d + q.regs, q.regs, cudaMemcpyHostToDevice, c->stream));
    d += 2 * q.regs;
    CU(cudaMemcpyAsync(p.F[0], d, q.bits, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(p.F[1], d + q.bits, q.bits, cudaMemcpyHostToDevice, c->stream));
    d += 2 * q.bits;
    CU(cudaMemcpyAsync(p.hist, d, q.hist, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(p.blk_q, d + q.hist, q.blk, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(p.est_acc, d + q.hist + q.blk, q.acc, cudaMemcpyHostToDevice, c->stream));
    if (q.cache)
        CU(cudaMemcpyAsync(p.ecache, d + q.hist + q.blk + q.acc, q.cache, cudaMemcpyHostToDevice,
                           c->stream));
    CU(cudaMemcpyAsync(p.slot_T, d + q.hist + q.blk + q.acc + q.cache, q.slots,
                       cudaMemcpyHostToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    c->host_ctl = ctl;
    return HANF_OK;
}

}  // extern "C"

namespace {

// Copy per-node values of run r, input ids first.., to the host in chunks.
int copy_node_values(hanf_ctx *c, const void *src_all, int elem, int32_t run, int64_t first,
                     int64_t count, void *out)
{
    const uint8_t *src = static_cast<const uint8_t *>(src_all) + (size_t)run * c->plan.n * elem;
    for (int64_t i = 0; i < count; i += kStageRows) {
        const int64_t k = std::min<int64_t>(kStageRows, count - i);
        CU(hanf::launch_gather_node_values(src, c->perm, first + i, k, elem, c->stage, c->stream));
        CU(cudaMemcpyAsync(static_cast<uint8_t *>(out) + (size_t)i * elem, c->stage, (size_t)k * elem,
                           cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
    }
    return HANF_OK;
}

int check_node_range(hanf_ctx *c, int32_t run, int64_t first, int64_t count)
{
    if (!c) return fail(HANF_EINVAL, "NULL context");
    if (!c->plan.node_stats) return fail(HANF_ESTATE, "context created without node_stats");
    if (run < 0 || run >= c->plan.R) return fail(HANF_EINVAL, "run %d out of range", run);
    if (first < 0 || count < 0 || first + count > c->plan.n)
        return fail(HANF_EINVAL, "node range out of bounds");
    return HANF_OK;
}

}  // namespace

extern "C" {

int hanf_node_stats(hanf_ctx *c, int32_t run, int64_t first, int64_t count, double *reach,
                    double *dist, int32_t *ecc)
{
    int rc = check_node_range(c, run, first, count);
    if (rc) return rc;
    if (reach && (rc = copy_node_values(c, c->plan.ns_prev, 8, run, first, count, reach))) return rc;
    if (dist && (rc = copy_node_values(c, c->plan.ns_dist, 8, run, first, count, dist))) return rc;
    if (ecc && (rc = copy_node_values(c, c->plan.ns_ecc, 4, run, first, count, ecc))) return rc;
    return HANF_OK;
}

int hanf_node_radius(hanf_ctx *c, double alpha, int32_t run, int64_t first, int64_t count,
                     int32_t *radius)
{
    int rc = check_node_range(c, run, first, count);
    if (rc) return rc;
    rc = read_ctl(c);
    if (rc) return rc;
    if (!c->host_ctl.done || c->host_ctl.err) return fail(HANF_ESTATE, "no completed run to replay");
    Plan &p = c->plan;
    const size_t cells = (size_t)std::max<int64_t>(p.n, 1) * p.R;
    CU(cudaMemcpyAsync(p.ns_reach, p.ns_prev, 8 * cells, cudaMemcpyDeviceToDevice, c->stream));
    const int32_t T = c->host_ctl.t;
    p.ns_radius_mode = 1;
    p.ns_alpha = alpha;
    rc = reset(c, std::max<int32_t>(T + 1, 1));
    while (rc == HANF_OK && !c->host_ctl.done) rc = one_pass(c);
    p.ns_radius_mode = 0;
    if (rc) return rc;
    if (radius) return copy_node_values(c, p.ns_rad, 4, run, first, count, radius);
    return HANF_OK;
}

int hanf_ed_interval(const double *N, int32_t T, double alpha, double eps, int32_t *lo,
                     int32_t *hi)
{
    if (!N || !lo || !hi || T < 0 || eps < 0) return fail(HANF_EINVAL, "bad argument");
    double M = N[0];
    for (int t = 1; t <= T; ++t) M = std::max(M, N[t]);
    *lo = -1;
    *hi = -1;
    for (int t = 0; t <= T; ++t) {
        const double H = N[t] / M;
        if (H <= alpha * (1.0 - 2.0 * eps)) *lo = t;
        if (*hi < 0 && H >= alpha * (1.0 + 2.0 * eps)) *hi = t;
    }
    return HANF_OK;
}

int hanf_stats_runs(const double *N, int32_t R, int32_t cap, const int32_t *T, double alpha,
                    int32_t exclude_zero, double *out10)
{
    if (!N || !T || !out10 || R < 1 || cap < 1) return fail(HANF_EINVAL, "bad argument");
    double sum[5] = {0, 0, 0, 0, 0}, sq[5] = {0, 0, 0, 0, 0};
    for (int r = 0; r < R; ++r) {
        if (T[r] < 0 || T[r] >= cap) return fail(HANF_EINVAL, "T[%d] outside 0..cap-1", r);
        double s5[5];
        const int rc = hanf_stats(N + (size_t)r * cap, T[r], alpha, exclude_zero, s5);
        if (rc) return rc;
        for (int k = 0; k < 5; ++k) {
            sum[k] += s5[k];
            sq[k] += s5[k] * s5[k];
        }
    }
    for (int k = 0; k < 5; ++k) {
        const double mean = sum[k] / R;
        out10[k] = mean;
        out10[5 + k] = R > 1 ? std::sqrt(std::max(0.0, (sq[k] - R * mean * mean) / (R - 1))) : 0.0;
    }
    return HANF_OK;
}

void hanf_destroy(hanf_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    if (c->fork.side) {
        cudaStreamSynchronize(c->fork.side);
        cudaStreamDestroy(c->fork.side);
    }
    if (c->fork.fork) cudaEventDestroy(c->fork.fork);
    if (c->fork.join) cudaEventDestroy(c->fork.join);
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->l2_window) {
        cudaCtxResetPersistingL2Cache();
        cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, c->l2_limit_before);
    }
    delete c;
}

const char *hanf_last_error(void) { return g_err.c_str(); }

}  // extern "C"
