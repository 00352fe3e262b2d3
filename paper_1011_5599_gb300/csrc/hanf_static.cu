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
// address (on the host it is only a stand-in), so the first call on each
// device looks the address up with cudaGetSymbolAddress while that device is
// current and remembers it; make that first call before any stream capture.
// All calls on a device share the array and it keeps the previous call's
// contents: each call writes every partial before reading it, so nothing has
// to be cleared, but calls that overlap on the GPU (on different streams, or
// from different host threads) race on it and must be serialised by the
// caller.
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
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

struct LcTable {
    double v[257];   // m ln(m / V) for V = 0..m (entry 0 unused)
};

std::mutex g_setup_mutex;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

// the message is read back with hanf_last_error()
int static_fail(int code, const std::string &msg)
{
    hanf::record_error(msg);
    return code;
}

// size() of run r of node v: alpha_m m^2 / sum_j 2^-M[j] with the sum taken
// exactly as an integer of 2^(31-M[j]) terms, and linear counting m ln(m/V)
// when that estimate is at most 5m/2 and V registers are empty.
__device__ double static_node_size(const uint8_t *regs, int64_t v, int r, int m, int64_t W,
                                   double amm, const LcTable &lc)
{
    const uint4 *q = reinterpret_cast<const uint4 *>(regs + v * W + (int64_t)r * m);
    unsigned long long S = 0;
    int V = 0;
    for (int k = 0; k < (m >> 4); ++k) {
        const uint4 x = q[k];
        const uint32_t w4[4] = {x.x, x.y, x.z, x.w};
        for (int j = 0; j < 4; ++j) {
            for (int s = 0; s < 32; s += 8) {
                const uint32_t M = (w4[j] >> s) & 0xffu;
                S += 1ull << (31 - M);
                V += M == 0;
            }
        }
    }
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
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(HANF_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return static_fail(HANF_ECUDA, "device index too large");
    double *scratch;
    {
        // once per device, with that device current: the scratch's address
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_ptr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_static_scratch);
            if (e != cudaSuccess)
                return static_fail(HANF_ECUDA, std::string("cudaGetSymbolAddress failed: ") +
                                                   cudaGetErrorString(e));
            g_scratch_ptr[dev] = static_cast<double *>(ptr);
        }
        scratch = g_scratch_ptr[dev];
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
