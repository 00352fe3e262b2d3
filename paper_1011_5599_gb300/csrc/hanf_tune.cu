// Autotuner: picks the launch parameters of the union pass for one graph by
// timing them.  The tuned knobs are the degree split (small_max_deg: nodes
// per lane group vs per warp; hub_min_deg: segment length of hub nodes), the
// gather variant (register batches, or asynchronous copies for the warp or
// the small-degree kernel) and, as a second stage on the best of those,
// whether late passes push (scatter) or pull (systolic).  Each candidate gets
// its own context in the caller's workspace, one untimed warm-up run and one
// timed run of the whole of Algorithm 2; the fastest wins.  Results are remembered in a text
// cache (one "key value..." line per tuned shape) so that later calls with the
// same GPU, row width and graph size skip the timing.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "hanf.h"
#include "hanf_internal.cuh"

namespace {

int tune_fail(int code, const std::string &msg)
{
    hanf::record_error(msg);
    return code;
}

std::string shape_key(int64_t n, int64_t arcs, int32_t log2m, const hanf_opts &o)
{
    cudaDeviceProp prop;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    std::string gpu = prop.name;
    for (char &ch : gpu)
        if (ch == ' ') ch = '_';
    const int W = (1 << log2m) * o.runs;
    const int ln = n > 0 ? (int)std::lround(std::log2((double)n)) : 0;
    const int la = arcs > 0 ? (int)std::lround(std::log2((double)arcs)) : 0;
    char buf[256];
    snprintf(buf, sizeof buf, "%s|W%d|L%d|n2^%d|a2^%d|f%d|r%d", gpu.c_str(), W, o.layout, ln, la,
             o.frontier, o.relabel);
    return buf;
}

bool cache_lookup(const char *path, const std::string &key, int32_t *small, int32_t *hub,
                  int32_t *variant, int32_t *scatter, double *ms)
{
    if (!path) return false;
    std::ifstream in(path);
    std::string line;
    bool found = false;
    while (std::getline(in, line)) {   // the last entry for a key wins
        std::istringstream ss(line);
        std::string k;
        int32_t a, b, c, d;
        double t;
        if ((ss >> k >> a >> b >> c >> d >> t) && k == key) {
            *small = a;
            *hub = b;
            *variant = c;
            *scatter = d;
            *ms = t;
            found = true;
        }
    }
    return found;
}

}  // namespace

extern "C" int hanf_autotune(int64_t n, int64_t arcs, const int64_t *offsets,
                             const int32_t *targets, int32_t graph_on_device, int32_t log2m,
                             uint64_t seed, const hanf_opts *base, void *workspace,
                             size_t workspace_bytes, const char *cache_path, hanf_opts *best_out,
                             double *best_ms_out)
{
    if (!best_out) return tune_fail(HANF_EINVAL, "best_out is NULL");
    hanf_opts o;
    if (base) o = *base;
    else hanf_default_opts(&o);
    o.use_graph = 1;
    o.profile = 0;
    const std::string key = shape_key(n, arcs, log2m, o);
    int32_t cs, ch, cv, cd;
    double cms;
    if (cache_lookup(cache_path, key, &cs, &ch, &cv, &cd, &cms)) {
        *best_out = o;
        best_out->small_max_deg = cs;
        best_out->hub_min_deg = ch;
        best_out->gather_variant = cv;
        best_out->scatter_den = cd;
        if (best_ms_out) *best_ms_out = cms;
        return HANF_OK;
    }
    double best_ms = INFINITY;
    hanf_opts best = o;
    std::vector<double> N(4096 * (size_t)std::max(o.runs, 1));
    std::vector<int32_t> T(std::max(o.runs, 1));
    cudaStream_t st = static_cast<cudaStream_t>(o.stream);
    // one candidate: a context, an untimed warm-up run, a timed run; returns
    // a status (a candidate that does not fit the workspace is skipped)
    auto trial = [&](const hanf_opts &c) -> int {
        size_t need = 0;
        int rc = hanf_workspace_size(n, arcs, log2m, &c, graph_on_device ? 0 : 1, &need);
        if (rc) return rc;
        if (need > workspace_bytes) return HANF_OK;
        hanf_ctx *ctx = nullptr;
        rc = hanf_create(&ctx, n, arcs, offsets, targets, graph_on_device, log2m, seed, &c,
                         workspace, workspace_bytes);
        if (rc) return rc;
        rc = hanf_run(ctx, 4096, N.data(), 4096, T.data());
        if (rc == HANF_OK) {
            if (st) cudaStreamSynchronize(st);
            else cudaDeviceSynchronize();
            const auto t0 = std::chrono::steady_clock::now();
            rc = hanf_run(ctx, 4096, N.data(), 4096, T.data());
            const double ms =
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                    .count();
            if (rc == HANF_OK && ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        hanf_destroy(ctx);
        return rc;
    };
    const int32_t smalls[] = {32, 128, 256, 1024, 4096};
    const int32_t hubs[] = {4096, 16384, 65536};
    const int32_t variants[] = {1, 2, 3};
    for (int32_t vsm : smalls)
        for (int32_t vh : hubs)
            for (int32_t gv : variants) {
                if (gv >= 2 && ((1 << log2m) * o.runs > 128 || o.layout)) continue;   // not applicable
                hanf_opts c = o;
                c.small_max_deg = vsm;
                c.hub_min_deg = vh;
                c.gather_variant = gv;
                const int rc = trial(c);
                if (rc) return rc;
            }
    // stage 2 on the best split: the pass flavour the row width does not
    // default to (pushes for rows up to 128 bytes, pulls for wider ones)
    if (std::isfinite(best_ms) && o.frontier == HANF_FRONTIER_AUTO && !o.layout &&
        o.scatter_den == 0) {
        hanf_opts c = best;
        c.scatter_den = (1 << log2m) * o.runs <= 128 ? -1 : 8;
        const int rc = trial(c);
        if (rc) return rc;
    }
    if (!std::isfinite(best_ms))
        return tune_fail(HANF_ENOMEM, "no candidate fits in the workspace");
    if (cache_path) {
        std::ofstream out(cache_path, std::ios::app);
        out << key << ' ' << best.small_max_deg << ' ' << best.hub_min_deg << ' '
            << best.gather_variant << ' ' << best.scatter_den << ' ' << best_ms << '\n';
    }
    *best_out = best;
    if (best_ms_out) *best_ms_out = best_ms;
    return HANF_OK;
}
