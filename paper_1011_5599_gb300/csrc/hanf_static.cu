// Allocation-free estimator: hanf_estimate_static.
//
// Some callers cannot allocate device memory while they run: a serving loop
// whose device memory was all reserved at start-up, or a process that embeds
// this library next to an allocator that owns the whole GPU, where a
// cudaMalloc would fail or would synchronise the device at a bad moment.  For
// them this entry point computes N = sum_v size(c[v]) of a register array the
// caller already holds, with its only scratch (the per-block partial sums) in
// a fixed array that lives inside the library.  It allocates nothing.
//
// The scratch is one file-scope device array of kStaticScratchDoubles
// doubles (8 MiB).  Every GPU that loads the library keeps its own copy until
// the process exits.  Host code may not use the array's name as a device
// address (on the host it is only a stand-in), so the first call in each CUDA
// context (normally: on each device) looks the address up with
// cudaGetSymbolAddress while that context is current and remembers it under
// the context's process-unique id; make that first call before any stream
// capture.  Keying by context id keeps the address right for a context
// created after cudaDeviceReset and for driver-API contexts other than the
// primary one.  All calls in a context share the array and it keeps the
// previous call's contents: each call writes every partial before reading
// it, so nothing has to be cleared, but calls that overlap on the GPU (on
// different streams, or from different host threads) race on it and must be
// serialised by the caller.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "hanf.h"
#include "hanf_internal.cuh"

namespace {

constexpr int64_t kStaticScratchDoubles = int64_t(1) << 20;   // 8 MiB
constexpr int kThreads = 256;
constexpr int kChunk = 4096;      // block partials summed by one first-level CTA
constexpr int kMaxContexts = 64;

static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

struct LcTable {
    double v[257];   // m ln(m / V) for V = 0..m (entry 0 unused)
};

// The scratch's device address per CUDA context, keyed by the context's id
// (unique for the life of the process).  Driver entry points are looked up
// through the runtime, so the library does not link the driver library.
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);
std::mutex g_setup_mutex;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
unsigned long long g_ctx_ids[kMaxContexts];
double *g_scratch_ptr[kMaxContexts];
int g_contexts = 0;

// the message is read back with hanf_last_error()
int static_fail(int code, const std::string &msg)
{
    hanf::record_error(msg);
    return code;
}

// size() of run r of node v: alpha_m m^2 / sum_j 2^-M[j] with the sum taken
// exactly as an integer of 2^(31-M[j]) terms, and linear counting m ln(m/V)
// when that estimate is at most 5m/2 and V registers are empty.
// A register above 31 is outside the layout: the node's size is NaN, which
// makes the run's N NaN.
__device__ double static_node_size(const uint8_t *regs, int64_t v, int r, int m, int64_t W,
                                   double amm, const LcTable &lc)
{
    const uint4 *q = reinterpret_cast<const uint4 *>(regs + v * W + (int64_t)r * m);
    unsigned long long S = 0;
    int V = 0;
    bool bad = false;
    for (int k = 0; k < (m >> 4); ++k) {
        const uint4 x = q[k];
        const uint32_t w4[4] = {x.x, x.y, x.z, x.w};
        for (int j = 0; j < 4; ++j) {
            for (int s = 0; s < 32; s += 8) {
                const uint32_t M = (w4[j] >> s) & 0xffu;
                bad |= M > 31u;
                S += M <= 31u ? 1ull << (31 - M) : 0ull;
                V += M == 0;
            }
        }
    }
    if (bad) return __longlong_as_double(0x7ff8000000000000ll);   // quiet NaN
    const double Z = 1.0 / ((double)S * 0x1p-31);
    double E = amm * Z;
    if (E <= 2.5 * (double)m && V > 0) E = lc.v[V];
    return E;
}

// Partial sum of size() over each block of 64 nodes and each run; a warp per
// (run, block), fixed butterfly order.
__global__ void k_static_blocks(const uint8_t *regs, int64_t n, int m, int R, double amm,
                                LcTable lc, double *part, int64_t nblk)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t W = (int64_t)R * m;
    for (int64_t it = warp; it < nblk * R; it += nwarps) {
        const int r = (int)(it / nblk);
        const int64_t blk = it - (int64_t)r * nblk;
        const int64_t v0 = blk * 64 + lane, v1 = v0 + 32;
        double s = (v0 < n ? static_node_size(regs, v0, r, m, W, amm, lc) : 0.0) +
                   (v1 < n ? static_node_size(regs, v1, r, m, W, amm, lc) : 0.0);
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) part[it] = s;
    }
}

// Fixed-shape sum of `count` values per run (run-major rows of length
// `count`): grid (ceil(count / kChunk), R), one partial per CTA.
__global__ void k_static_reduce(const double *in, int64_t count, double *out, int64_t out_stride)
{
    __shared__ double sh[kThreads];
    const int r = blockIdx.y;
    const int64_t i0 = (int64_t)blockIdx.x * kChunk;
    double s = 0.0;
    for (int j = threadIdx.x; j < kChunk; j += kThreads) {
        const int64_t i = i0 + j;
        if (i < count) s += in[(int64_t)r * count + i];
    }
    sh[threadIdx.x] = s;
    for (int w = kThreads / 2; w; w >>= 1) {
        __syncthreads();
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    }
    if (threadIdx.x == 0) out[(int64_t)r * out_stride + blockIdx.x] = sh[0];
}

double static_alpha(int m)
{
    switch (m) {
    case 16: return 0.673;
    case 32: return 0.697;
    case 64: return 0.709;
    default: return 0.7213 / (1.0 + 1.079 / (double)m);
    }
}

}  // namespace

extern "C" int hanf_estimate_static(const uint8_t *regs, int64_t n, int32_t log2m, int32_t runs,
                                    double *N_out, void *stream)
{
    if (log2m < 4 || log2m > 8) return static_fail(HANF_EINVAL, "log2m outside 4..8");
    if (runs < 1 || runs > 8) return static_fail(HANF_EINVAL, "runs outside 1..8");
    if (n < 0 || n >= (int64_t(1) << 31)) return static_fail(HANF_EINVAL, "n out of range");
    if (!N_out || (n > 0 && !regs)) return static_fail(HANF_EINVAL, "NULL pointer");
    if (reinterpret_cast<uintptr_t>(regs) & 15)
        return static_fail(HANF_EINVAL, "hanf_estimate_static: regs must be 16-byte aligned "
                                        "(rows are read as 16-byte vectors)");
    if (reinterpret_cast<uintptr_t>(N_out) & 7)
        return static_fail(HANF_EINVAL, "hanf_estimate_static: N_out must be 8-byte aligned");
    const int m = 1 << log2m;
    const int64_t nblk = std::max<int64_t>(1, (n + 63) / 64);
    const int64_t nred = (nblk + kChunk - 1) / kChunk;
    const int64_t need = (int64_t)runs * (nblk + nred);
    if (need > kStaticScratchDoubles) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "hanf_estimate_static: %d runs x %lld nodes need %lld scratch doubles, more "
                 "than the fixed %lld (8 MiB); use hanf_estimate with a workspace instead",
                 runs, (long long)n, (long long)need, (long long)kStaticScratchDoubles);
        return static_fail(HANF_EINVAL, buf);
    }
    cudaError_t e;
    double *scratch = nullptr;
    {
        // once per context, with that context current: the scratch's address
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_ctx_get_current || !g_ctx_get_id) {
            cudaDriverEntryPointQueryResult q1, q2;
            void *f1 = nullptr, *f2 = nullptr;
            if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault,
                                                 &q1) != cudaSuccess ||
                cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault,
                                                 &q2) != cudaSuccess ||
                q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
                return static_fail(HANF_ECUDA, "hanf_estimate_static: the driver's context "
                                               "queries are unavailable");
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
            g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
        }
        void *ptr = nullptr;
        void *ctx = nullptr;
        if (g_ctx_get_current(&ctx) != 0 || !ctx) {
            // no context current on this thread yet: the symbol lookup makes
            // the runtime's primary context current
            e = cudaGetSymbolAddress(&ptr, g_static_scratch);
            if (e != cudaSuccess)
                return static_fail(HANF_ECUDA, std::string("cudaGetSymbolAddress failed: ") +
                                                   cudaGetErrorString(e));
            if (g_ctx_get_current(&ctx) != 0 || !ctx)
                return static_fail(HANF_ECUDA, "hanf_estimate_static: no current CUDA context");
        }
        unsigned long long id = 0;
        if (g_ctx_get_id(ctx, &id) != 0)
            return static_fail(HANF_ECUDA, "hanf_estimate_static: cuCtxGetId failed");
        for (int i = 0; i < g_contexts; ++i)
            if (g_ctx_ids[i] == id) scratch = g_scratch_ptr[i];
        if (!scratch) {
            if (!ptr) {
                e = cudaGetSymbolAddress(&ptr, g_static_scratch);
                if (e != cudaSuccess)
                    return static_fail(HANF_ECUDA, std::string("cudaGetSymbolAddress failed: ") +
                                                       cudaGetErrorString(e));
            }
            scratch = static_cast<double *>(ptr);
            // a full table forgets its oldest entry
            const int slot = g_contexts < kMaxContexts ? g_contexts++ : (int)(id % kMaxContexts);
            g_ctx_ids[slot] = id;
            g_scratch_ptr[slot] = scratch;
        }
    }
    LcTable lc;
    for (int V = 0; V <= 256; ++V)
        lc.v[V] = (V >= 1 && V <= m) ? (double)m * std::log((double)m / (double)V) : 0.0;
    const double amm = static_alpha(m) * (double)m * (double)m;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *part = scratch;                              // runs x nblk
    double *red = scratch + (int64_t)runs * nblk;        // runs x nred
    const int64_t warps = std::min<int64_t>(nblk * runs, 152 * 64);
    k_static_blocks<<<(unsigned)((warps * 32 + kThreads - 1) / kThreads), kThreads, 0, s>>>(
        regs, n, m, runs, amm, lc, part, nblk);
    k_static_reduce<<<dim3((unsigned)nred, (unsigned)runs), kThreads, 0, s>>>(part, nblk, red, nred);
    k_static_reduce<<<dim3(1, (unsigned)runs), kThreads, 0, s>>>(red, nred, N_out, 1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return static_fail(HANF_ECUDA, cudaGetErrorString(e));
    return HANF_OK;
}
