// CUDA kernels of the GB300 HyperANF library (sm_103a).
//
// Counter layout: node v owns one row of W = R*m bytes at regs[p] + v*W; run
// r's m registers are bytes [r*m, (r+1)*m) of the row, one register per byte
// (values 0..31).  A row is moved as W/16 uint4 vectors by a "lane group" of
// LANES = min(32, W/16) threads, VPL = W/(16*LANES) vectors per lane, so every
// gather of a successor counter is a run of fully used 16-byte loads.
//
// The union (Algorithm 2's inner loop, Section 3.2) is Jacobi: pass t reads
// regs[p] (= c_t) and writes regs[p^1].  regs[p^1] holds c_{t-1} on entry, so
// a node needs a store only if its counter changes now or changed in the
// previous pass; every other row already equals c_{t+1}.  Successors that did
// not change in the previous pass are skipped (Section 3.3, tracking modified
// counters): the changed set is a bitmap F[p] of n bits.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "hanf_internal.cuh"

namespace hanf {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------- hashing

// splitmix64 output step (Steele, Lea, Flood): golden-ratio increment, then
// two xor-shift-multiply rounds and a final xor-shift.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ---------------------------------------------------------------- rows

// Resident blocks per SM the union kernels are compiled for: three (at most
// 80 registers a thread) while a lane holds one 16-byte vector of a row,
// two where it holds several, so that the rows in flight stay in registers.
__host__ __device__ constexpr int min_blocks(int vectors_per_lane)
{
    return vectors_per_lane >= 2 ? 2 : 3;
}

template <int LANES, int VPL>
struct Row {
    uint4 v[VPL];
};

// Register-wise max of four byte registers (Section 3.3, union via broadword
// programming).  Registers never exceed 31, so bit 7 of every byte is free and
// serves as the guard bit of the paper's parallel compare: setting it is the
// same as adding 0x80 to every byte, and in d = a + 0x80..80 - b every byte
// stays within 97..159, so no byte carries into or borrows from its
// neighbour (one three-input add), and bit 7 of byte i of d is set iff
// a_i >= b_i.  A byte permute that replicates each byte's top bit turns d
// into the selection mask (0xff where a_i >= b_i), and the result is
// (a & mask) | (b & ~mask), one three-input logic operation.
__device__ __forceinline__ uint32_t bmax(uint32_t a, uint32_t b)
{
    const uint32_t d = a + 0x80808080u - b;
    uint32_t mask;
    // prmt with selector nibbles 8..11: byte i of the result replicates the
    // sign bit of byte i of d (the __byte_perm intrinsic ignores that bit)
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(mask) : "r"(d), "r"(0u), "r"(0xBA98u));
    return (a & mask) | (b & ~mask);
}

__device__ __forceinline__ uint4 vmax4(uint4 a, uint4 b)
{
    return make_uint4(bmax(a.x, b.x), bmax(a.y, b.y), bmax(a.z, b.z), bmax(a.w, b.w));
}

__device__ __forceinline__ bool veq(uint4 a, uint4 b)
{
    return ((a.x ^ b.x) | (a.y ^ b.y) | (a.z ^ b.z) | (a.w ^ b.w)) == 0u;
}

template <int LANES, int VPL>
__device__ __forceinline__ void row_zero(Row<LANES, VPL> &r)
{
#pragma unroll
    for (int k = 0; k < VPL; ++k) r.v[k] = make_uint4(0u, 0u, 0u, 0u);
}

template <int LANES, int VPL>
__device__ __forceinline__ void row_load(Row<LANES, VPL> &r, const uint8_t *base, int64_t row,
                                         int gl)
{
    const uint4 *q = reinterpret_cast<const uint4 *>(base) + row * (LANES * VPL) + gl;
#pragma unroll
    for (int k = 0; k < VPL; ++k) r.v[k] = __ldg(q + k * LANES);
}

template <int LANES, int VPL>
__device__ __forceinline__ void row_store(uint8_t *base, int64_t row, const Row<LANES, VPL> &r,
                                          int gl)
{
    uint4 *q = reinterpret_cast<uint4 *>(base) + row * (LANES * VPL) + gl;
#pragma unroll
    for (int k = 0; k < VPL; ++k) q[k * LANES] = r.v[k];
}

template <int LANES, int VPL>
__device__ __forceinline__ void row_max(Row<LANES, VPL> &a, const Row<LANES, VPL> &b)
{
#pragma unroll
    for (int k = 0; k < VPL; ++k) a.v[k] = vmax4(a.v[k], b.v[k]);
}

// Register-wise max across the lane groups of a warp (all lanes take part).
template <int LANES, int VPL>
__device__ __forceinline__ void row_warp_max(Row<LANES, VPL> &r)
{
#pragma unroll
    for (int s = LANES; s < 32; s <<= 1) {
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            r.v[k].x = bmax(r.v[k].x, __shfl_xor_sync(kFull, r.v[k].x, s));
            r.v[k].y = bmax(r.v[k].y, __shfl_xor_sync(kFull, r.v[k].y, s));
            r.v[k].z = bmax(r.v[k].z, __shfl_xor_sync(kFull, r.v[k].z, s));
            r.v[k].w = bmax(r.v[k].w, __shfl_xor_sync(kFull, r.v[k].w, s));
        }
    }
}

template <int LANES>
__device__ __forceinline__ uint32_t group_or(uint32_t x)
{
#pragma unroll
    for (int s = 1; s < LANES; s <<= 1) x |= __shfl_xor_sync(kFull, x, s);
    return x;
}

__device__ __forceinline__ bool test_bit(const unsigned long long *bits, int32_t v)
{
    return (__ldg(bits + (v >> 6)) >> (v & 63)) & 1ull;
}

// ---------------------------------------------------------------- size() and exact N(t)

// size() of a counter (Algorithm 1 with linear counting) from the exact
// integer S = sum_j 2^(31 - M[j]) over its M registers and the number V of
// empty registers.  sum = S * 2^-31 is exact (M <= S < 2^40); it is built
// from the bits of S, and E <= 5m/2 is decided on the bit patterns of the two
// positive doubles, so that only the division and the product use the
// (narrow, on this GPU) double-precision pipe; each is rounded once, as IEEE
// double arithmetic does it.
__device__ __forceinline__ double size_from_sums(const Plan &p, unsigned long long S, int V, int M)
{
    const int L = 64 - __clzll((long long)S);   // S in [2^(L-1), 2^L)
    const unsigned long long sum_bits = ((unsigned long long)(1023 + L - 1 - 31) << 52) |
                                        ((S << (53 - L)) & ((1ull << 52) - 1ull));
    const double Z = 1.0 / __longlong_as_double((long long)sum_bits);
    double E = p.amm * Z;
    if (__double_as_longlong(E) <= __double_as_longlong(2.5 * (double)M) && V > 0) E = p.lc[V];
    return E;
}

// Adds 2^(31 - M) for each of the four byte registers M of w to S, and the
// number of empty ones to V.  Registers are below 32, so a funnel shift in
// wrap mode takes its amount (modulo 32) straight from the low bits of the
// word, byte i after w >> 8i, and mad.wide adds the 32-bit term to the 64-bit
// sum in one instruction; w + 0x7f..7f sets bit 7 exactly in the non-zero
// bytes (no byte carries into the next).
__device__ __forceinline__ void word_sums(uint32_t w, unsigned long long &S, int &V)
{
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        uint32_t term;
        asm("shf.r.wrap.b32 %0, %1, %2, %3;" : "=r"(term) : "r"(0x80000000u), "r"(0u), "r"(w >> (8 * i)));
        asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(S) : "r"(term), "r"(1u));
    }
    V += __popc(~(w + 0x7f7f7f7fu) & 0x80808080u);
}

__device__ __forceinline__ void vec_sums(uint4 x, unsigned long long &S, int &V)
{
    word_sums(x.x, S, V);
    word_sums(x.y, S, V);
    word_sums(x.z, S, V);
    word_sums(x.w, S, V);
}

// N(t) = sum_v size(c_t[v]) is kept exactly, as a signed 128-bit integer of
// units 2^-52 ("Q52").  Every size() value is 0 or lies in (1, 2^40): linear
// counting gives m ln(m/V) > 1 for V < m registers empty (0 for V = m), and
// the raw estimate is taken only above 5m/2 or with no empty register, where
// it exceeds 2 alpha_m m > 20.  So E * 2^52 is an integer below 2^92 and a
// sum over fewer than 2^31 nodes fits.  Integer addition is exact and
// commutative: the sum does not depend on the order of the additions (atomics
// included) and is rounded to double once.
struct Q128 {
    unsigned long long lo, hi;
};

__device__ __forceinline__ void q_add(Q128 &a, const Q128 &b)
{
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(a.lo), "+l"(a.hi) : "l"(b.lo), "l"(b.hi));
}

__device__ __forceinline__ void q_sub(Q128 &a, const Q128 &b)
{
    asm("sub.cc.u64 %0, %0, %2;\n\tsubc.u64 %1, %1, %3;" : "+l"(a.lo), "+l"(a.hi) : "l"(b.lo), "l"(b.hi));
}

// E (0, or in (1, 2^40)) in Q52: mantissa << (exponent - 1023).
__device__ __forceinline__ Q128 q_from(double E)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(E);
    const int ex = (int)(bits >> 52);
    Q128 q{0ull, 0ull};
    if (ex == 0) return q;
    const unsigned long long mant = (bits & ((1ull << 52) - 1ull)) | (1ull << 52);
    const int sh = ex - 1023;
    if (sh <= 0) {
        q.lo = mant >> (-sh);   // 0 < E < 2 (E < 1 does not occur, see above)
    } else {
        q.lo = mant << sh;
        q.hi = mant >> (64 - sh);
    }
    return q;
}

__device__ __forceinline__ Q128 q_shfl_xor(const Q128 &a, int o, unsigned mask = kFull)
{
    return Q128{__shfl_xor_sync(mask, a.lo, o), __shfl_xor_sync(mask, a.hi, o)};
}

// *q += a for a 128-bit value in memory (q[0] low word, q[1] high word).  The
// carry out of each low-word addition is exactly what that addition adds to
// the high word, whatever the order the atomics take, so the sum is exact.
__device__ __forceinline__ void q_atomic_add(unsigned long long *q, const Q128 &a)
{
    if ((a.lo | a.hi) == 0ull) return;
    unsigned long long hi = a.hi;
    if (a.lo) {
        const unsigned long long old = atomicAdd(q, a.lo);
        if (old + a.lo < old) hi += 1ull;
    }
    if (hi) atomicAdd(q + 1, hi);
}

// Round a Q52 value to the nearest double (ties to even): the value itself
// when it has at most 53 significant bits, else its top 53 bits rounded by
// the next bit and the bits below it.
__device__ __forceinline__ double q_to_double(Q128 a)
{
    const bool neg = (long long)a.hi < 0;
    if (neg) {
        const Q128 z{0ull, 0ull};
        Q128 t = z;
        q_sub(t, a);
        a = t;
    }
    double r;
    if (a.hi == 0ull && a.lo < (1ull << 53)) {
        r = (double)a.lo * 0x1p-52;
    } else {
        const int nb = a.hi ? 128 - __clzll((long long)a.hi) : 64 - __clzll((long long)a.lo);
        int sh = nb - 53;   // 1 .. 75
        unsigned long long top = sh >= 64 ? a.hi >> (sh - 64) : (a.lo >> sh) | (a.hi << (64 - sh));
        const int hb = sh - 1;   // the rounding bit; the sticky bits lie below it
        const bool half = hb >= 64 ? (a.hi >> (hb - 64)) & 1ull : (a.lo >> hb) & 1ull;
        bool sticky;
        if (hb >= 64)
            sticky = a.lo != 0ull || (hb > 64 && (a.hi & ((1ull << (hb - 64)) - 1ull)) != 0ull);
        else
            sticky = hb > 0 && (a.lo & ((1ull << hb) - 1ull)) != 0ull;
        if (half && (sticky || (top & 1ull))) top += 1ull;
        if (top == (1ull << 53)) {
            top >>= 1;
            sh += 1;
        }
        r = (double)top * __longlong_as_double((long long)(1023 + sh - 52) << 52);
    }
    return neg ? -r : r;
}

// ---------------------------------------------------------------- union

// Pass flavours (DevCtl::mode, chosen by k_prep before every pass):
//   kModeTest   pull: every node scans its arcs, gathering only successors
//               that changed in the previous pass (bitmap F_t);
//   kModePush   systolic: only candidate nodes (changed nodes and their
//               predecessors) scan their arcs, gathering changed successors;
//   kModeDense  pull without the per-arc test, used at t = 0, with the
//               frontier off, and while most counters still change: merging an
//               unchanged successor is harmless, max being idempotent.
//   kModeScatter pure push: each node changed by the last pass raises the new
//               counters of its predecessors (k_scatter), used once the changed
//               nodes have few in-arcs; the pull kernels sit the pass out.
constexpr int kModeTest = 0;
constexpr int kModePush = 1;
constexpr int kModeDense = 2;
constexpr int kModeScatter = 3;

// Gather the counters of arcs [beg, end) of one node, one lane group per
// node (all lanes of the group share beg/end).  Each lane loads U/LANES
// targets of a batch of U (one batch ahead), tests its own targets against
// the changed bitmap, and the group then issues the U row gathers together.
template <int LANES, int VPL, int U>
__device__ __forceinline__ void group_gather(const int32_t *__restrict__ tgt, const uint8_t *rc,
                                             const unsigned long long *Fc, bool test,
                                             int64_t beg, int64_t end, int gl, unsigned gmask,
                                             int gbase, Row<LANES, VPL> &acc, bool &any,
                                             uint32_t &gathered)
{
    constexpr int TPL = (U + LANES - 1) / LANES;
    int32_t nxt[TPL];
#pragma unroll
    for (int k = 0; k < TPL; ++k) {
        const int j = gl + k * LANES;
        nxt[k] = (j < U && beg + j < end) ? __ldg(tgt + beg + j) : -1;
    }
    for (int64_t e = beg; e < end; e += U) {
        int32_t cur[TPL];
#pragma unroll
        for (int k = 0; k < TPL; ++k) {
            cur[k] = nxt[k];
            const int j = gl + k * LANES;
            nxt[k] = (j < U && e + U + j < end) ? __ldg(tgt + e + U + j) : -1;
        }
#pragma unroll
        for (int k = 0; k < TPL; ++k)
            if (cur[k] >= 0 && test && !test_bit(Fc, cur[k])) cur[k] = -1;
        int32_t w[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            w[u] = LANES == 1 ? cur[u] : __shfl_sync(gmask, cur[u / LANES], gbase + (u % LANES));
        Row<LANES, VPL> x[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (w[u] >= 0) row_load(x[u], rc, w[u], gl);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (w[u] >= 0) {
                row_max(acc, x[u]);
                any = true;
                ++gathered;
            }
    }
}

// Sparse variant for passes that test the changed bitmap: most successors
// fail the test, so a lane group scans UT arcs per batch (UT/LANES targets
// and bitmap words per lane, all in flight together, the next batch's
// targets loaded ahead), then gathers only the rows that passed, packed into
// rounds of at most SUBR rows.
template <int LANES, int VPL, int UT>
__device__ __forceinline__ void group_gather_sparse(const int32_t *__restrict__ tgt,
                                                    const uint8_t *rc,
                                                    const unsigned long long *Fc, int64_t beg,
                                                    int64_t end, int gl, unsigned gmask, int gbase,
                                                    Row<LANES, VPL> &acc, bool &any,
                                                    uint32_t &gathered)
{
    constexpr int TPL = UT / LANES;   // targets per lane and batch
    constexpr int SUBR = LANES < 4 ? LANES : 4;
    int32_t nxt[TPL];
#pragma unroll
    for (int k = 0; k < TPL; ++k) {
        const int64_t j = beg + (int64_t)k * LANES + gl;
        nxt[k] = j < end ? __ldg(tgt + j) : -1;
    }
    for (int64_t e = beg; e < end; e += UT) {
        int32_t cur[TPL];
#pragma unroll
        for (int k = 0; k < TPL; ++k) {
            cur[k] = nxt[k];
            const int64_t j = e + UT + (int64_t)k * LANES + gl;
            nxt[k] = j < end ? __ldg(tgt + j) : -1;
        }
#pragma unroll
        for (int k = 0; k < TPL; ++k)
            if (cur[k] >= 0 && !test_bit(Fc, cur[k])) cur[k] = -1;
#pragma unroll
        for (int k = 0; k < TPL; ++k) {
            // lanes of this group holding a target that passed (absolute
            // lane bits; the same value on every lane of the group)
            unsigned live = __ballot_sync(gmask, cur[k] >= 0) & gmask;
            while (live) {
                int32_t w[SUBR];
#pragma unroll
                for (int u = 0; u < SUBR; ++u) {
                    const int src = live ? __ffs(live) - 1 : gbase;
                    w[u] = __shfl_sync(gmask, cur[k], src);
                    if (!live) w[u] = -1;
                    live &= live - 1u;
                }
                Row<LANES, VPL> x[SUBR];
#pragma unroll
                for (int u = 0; u < SUBR; ++u)
                    if (w[u] >= 0) row_load(x[u], rc, w[u], gl);
#pragma unroll
                for (int u = 0; u < SUBR; ++u)
                    if (w[u] >= 0) {
                        row_max(acc, x[u]);
                        any = true;
                        ++gathered;
                    }
            }
        }
    }
}

// Gather the counters of arcs [beg, end) with the whole warp (beg/end warp-
// uniform).  Lane i loads target e+i of each batch of 32 (one batch ahead,
// coalesced) and tests it; lane group g then merges the targets of lanes
// g, g+GPW, ..., SUB rows in flight at a time.
template <int LANES, int VPL>
__device__ __forceinline__ void warp_gather(const int32_t *__restrict__ tgt, const uint8_t *rc,
                                            const unsigned long long *Fc, bool test, int64_t beg,
                                            int64_t end, int g, int gl, Row<LANES, VPL> &acc,
                                            bool &any, uint32_t &gathered)
{
    constexpr int GPW = 32 / LANES;
    constexpr int SUB = (8 / VPL) < LANES ? (8 / VPL) : LANES;
    const int lane = threadIdx.x & 31;
    int32_t nxt = beg + lane < end ? __ldg(tgt + beg + lane) : -1;
    for (int64_t e = beg; e < end; e += 32) {
        int32_t cur = nxt;
        nxt = e + 32 + lane < end ? __ldg(tgt + e + 32 + lane) : -1;
        if (cur >= 0 && test && !test_bit(Fc, cur)) cur = -1;
        const unsigned live = __ballot_sync(kFull, cur >= 0);
        if (live == 0) continue;
        any = true;
        gathered += __popc(live);
#pragma unroll
        for (int s = 0; s < LANES; s += SUB) {
            int32_t w[SUB];
#pragma unroll
            for (int u = 0; u < SUB; ++u) w[u] = __shfl_sync(kFull, cur, (s + u) * GPW + g);
            Row<LANES, VPL> x[SUB];
#pragma unroll
            for (int u = 0; u < SUB; ++u)
                if (w[u] >= 0) row_load(x[u], rc, w[u], gl);
#pragma unroll
            for (int u = 0; u < SUB; ++u)
                if (w[u] >= 0) row_max(acc, x[u]);
        }
    }
}

// New counter of v = max(acc, c_t[v]); store it if it changed or if `stale`
// (v changed in the previous pass, or t = 0, when the target buffer holds
// only the rows of nodes without arcs).  Returns
// the mask of runs whose counter changed (same value on all lanes of the
// group).  Every lane of the warp must call it.
template <int LANES, int VPL>
__device__ __forceinline__ uint32_t node_finish(const Plan &p, int cur, const Row<LANES, VPL> &acc,
                                                bool need, bool stale, int32_t v, int gl,
                                                uint32_t &c_own, uint32_t &c_write,
                                                const Row<LANES, VPL> *pre = nullptr)
{
    Row<LANES, VPL> own, nw;
    uint32_t mask = 0;
    if (need) {
        if (pre) own = *pre;
        else row_load(own, p.regs[cur], v, gl);
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            nw.v[k] = vmax4(acc.v[k], own.v[k]);
            const int run = ((k * LANES + gl) << 4) >> p.b;
            if (!veq(nw.v[k], own.v[k])) mask |= 1u << run;
        }
    }
    mask = group_or<LANES>(mask);
    if (need && (mask || stale)) {
        row_store(p.regs[cur ^ 1], v, nw, gl);
        if (gl == 0) ++c_write;
    }
    if (need && gl == 0) ++c_own;
    return mask;
}

// Changed-node tallies of one thread, kept in registers for the whole kernel
// and flushed once at its end: a reduction per node on the few shared
// counters would queue every warp of the GPU on one L2 slice.
struct MarkTally {
    uint32_t nodes = 0;   // lane 0: changed nodes seen by the warp
    uint32_t fresh = 0;   // any lane: nodes it marked first (scatter passes)
    uint32_t runs = 0;    // lane r < R: nodes whose run-r counter changed (one graph;
                          // in scatter passes raises, which may repeat a node)
};

// Per-run change tallies of the nodes marked by one warp call (`ch` marks the
// lanes holding a changed node, `bal` is their ballot).
__device__ __forceinline__ void tally_runs(const Plan &p, bool ch, unsigned bal, int32_t v,
                                           uint32_t mask, MarkTally &mt)
{
    const int lane = threadIdx.x & 31;
    if (p.K == 1) {
        // lane r counts run r: read the changed leaders' masks, or ballot
        // run by run, whichever takes fewer warp operations
        if (__popc(bal) < p.R) {
            for (unsigned b = bal; b; b &= b - 1u) {
                const uint32_t mg = __shfl_sync(kFull, mask, __ffs(b) - 1);
                mt.runs += (mg >> lane) & 1u;
            }
        } else {
            for (int r = 0; r < p.R; ++r) {
                const unsigned br = __ballot_sync(kFull, ch && ((mask >> r) & 1u));
                if (lane == r) mt.runs += __popc(br);
            }
        }
    } else {
        // a batch: lanes may hold nodes of different graphs; one reduction
        // per graph present and run
        const int g = ch ? __ldg(p.blk_graph + (v >> 6)) : -1;
        const unsigned peers = __match_any_sync(kFull, g);
        const bool head = ch && __ffs(peers) - 1 == lane;
        for (int r = 0; r < p.R; ++r) {
            const unsigned br = __ballot_sync(kFull, ch && ((mask >> r) & 1u)) & peers;
            if (head && br) atomicAdd(&p.slot_changed[g * p.R + r], (unsigned long long)__popc(br));
        }
    }
}

// Record the nodes whose counters changed: the bitmap bit at once (a
// fire-and-forget reduction), the counts in the tally.  Called by all lanes;
// `leader` marks one lane per node, `mask` is its mask of changed runs.
__device__ __forceinline__ void warp_mark(const Plan &p, int cur, bool leader, int32_t v,
                                          uint32_t mask, MarkTally &mt)
{
    const bool ch = leader && mask != 0;
    const unsigned bal = __ballot_sync(kFull, ch);
    if (bal == 0) return;
    const int lane = threadIdx.x & 31;
    if (lane == 0) mt.nodes += __popc(bal);
    if (ch) atomicOr(&p.F[cur ^ 1][v >> 6], 1ull << (v & 63));
    tally_runs(p, ch, bal, v, mask, mt);
}

__device__ __forceinline__ unsigned warp_sum_u32(unsigned x)
{
#pragma unroll
    for (int s = 16; s; s >>= 1) x += __shfl_xor_sync(kFull, x, s);
    return x;
}

__device__ __forceinline__ void flush_counters(const Plan &p, int cur, const MarkTally &mt,
                                               uint32_t scan, uint32_t gather, uint32_t own,
                                               uint32_t write)
{
    const unsigned s0 = warp_sum_u32(scan), s1 = warp_sum_u32(gather);
    const unsigned s2 = warp_sum_u32(own), s3 = warp_sum_u32(write);
    const unsigned nodes = mt.nodes + warp_sum_u32(mt.fresh);   // lane 0
    const int lane = threadIdx.x & 31;
    DevCtl *c = p.ctl;
    if (lane == 0) {
        if (s0) atomicAdd(&c->arcs_scanned, (unsigned long long)s0);
        if (s1) atomicAdd(&c->arcs_gathered, (unsigned long long)s1);
        if (s2) atomicAdd(&c->own_reads, (unsigned long long)s2);
        if (s3) atomicAdd(&c->writes, (unsigned long long)s3);
        if (nodes) atomicAdd(&c->changed_count[cur ^ 1], (unsigned long long)nodes);
    }
    if (p.K == 1 && lane < p.R && mt.runs)
        atomicAdd(&p.slot_changed[lane], (unsigned long long)mt.runs);
}

// Union pass over small nodes (degree <= small_max_deg): a lane group per
// node, GPW nodes per warp, warps striding over the small-node list.
// Rows of at most 128 bytes get a separate instantiation for passes that test
// the changed bitmap (SPARSE): each instantiation returns at once when the
// pass is not its kind, which keeps both register footprints small.
template <int LANES, int VPL>
constexpr bool has_sparse_path() { return VPL == 1 && LANES <= 8; }

template <int LANES, int VPL, bool SPARSE>
__global__ void __launch_bounds__(kBlock, min_blocks(VPL)) k_union_small(Plan p)
{
    constexpr int GPW = 32 / LANES;
    constexpr int U = 4 / VPL > 0 ? 4 / VPL : 1;
    const DevCtl *ctl = p.ctl;
    if (ctl->done || ctl->mode == kModeScatter || (ctl->t == 0 && p.first_warps)) return;
    if constexpr (has_sparse_path<LANES, VPL>()) {
        if (SPARSE != (ctl->mode != kModeDense)) return;
    }
    const int cur = ctl->parity;
    const bool first = ctl->t == 0;
    const bool test = ctl->mode != kModeDense;
    const bool push = ctl->mode == kModePush;
    const uint8_t *rc = p.regs[cur];
    const unsigned long long *Fc = p.F[cur];
    const int lane = threadIdx.x & 31, g = lane / LANES, gl = lane % LANES;
    const int gbase = g * LANES;
    const unsigned gmask = LANES == 32 ? kFull : (((1u << LANES) - 1u) << gbase);
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t c_scan = 0, c_gather = 0, c_own = 0, c_write = 0;
    MarkTally mt;
    // systolic passes visit the small-degree candidates only
    const int32_t *list = push ? p.cand_list[0] : p.nodes;
    const int64_t count = push ? (int64_t)ctl->cand_count[0] : p.n_small;
    // dense and systolic passes need almost every visited node's own counter:
    // load it next to the gathers instead of after them
    const bool own_early = !test || push;
    const int64_t stride = nwarps * GPW;
    // node ids two iterations ahead, arc ranges one iteration ahead
    int64_t idx_ahead = warp * GPW + g;
    int32_t v_next = idx_ahead < count ? __ldg(list + idx_ahead) : -1;
    int64_t beg_next = v_next >= 0 ? __ldg(p.off + v_next) : 0;
    int64_t end_next = v_next >= 0 ? __ldg(p.off + v_next + 1) : 0;
    idx_ahead += stride;
    int32_t v_after = idx_ahead < count ? __ldg(list + idx_ahead) : -1;
    for (int64_t base = warp * GPW; base < count; base += stride) {
        const int32_t v = v_next;
        const int64_t beg = beg_next, end = end_next;
        const bool valid = v >= 0;
        v_next = v_after;
        beg_next = v_next >= 0 ? __ldg(p.off + v_next) : 0;
        end_next = v_next >= 0 ? __ldg(p.off + v_next + 1) : 0;
        idx_ahead += stride;
        v_after = idx_ahead < count ? __ldg(list + idx_ahead) : -1;
        Row<LANES, VPL> own;
        if (valid && own_early) row_load(own, rc, v, gl);
        Row<LANES, VPL> acc;
        row_zero(acc);
        bool any = false;
        if (valid) {
            if constexpr (SPARSE)
                group_gather_sparse<LANES, VPL, 4 * LANES>(p.tgt, rc, Fc, beg, end, gl, gmask,
                                                           gbase, acc, any, c_gather);
            else
                group_gather<LANES, VPL, U>(p.tgt, rc, Fc, test, beg, end, gl, gmask, gbase, acc,
                                            any, c_gather);
            if (gl == 0) c_scan += (uint32_t)(end - beg);
        }
        const bool inR = valid && !first && test_bit(Fc, v);
        const bool need = valid && (any || inR);
        const uint32_t mask = node_finish(p, cur, acc, need, inR || first, v, gl, c_own, c_write,
                                          own_early ? &own : nullptr);
        warp_mark(p, cur, gl == 0 && valid, v, mask, mt);
    }
    flush_counters(p, cur, mt, c_scan, gl == 0 ? c_gather : 0u, c_own, c_write);
}

// Union pass over medium nodes (a warp per node) and hub segments (a warp
// merges up to hub_min_deg arcs of a hub into a partial row, combined later
// by k_hub_finish).  Hub segments come first so the longest items start
// early.
template <int LANES, int VPL>
__global__ void __launch_bounds__(kBlock, min_blocks(VPL)) k_union_warp(Plan p)
{
    const DevCtl *ctl = p.ctl;
    if (ctl->done || ctl->mode == kModeScatter || (ctl->t == 0 && p.first_warps)) return;
    const int cur = ctl->parity;
    const bool first = ctl->t == 0;
    const bool test = ctl->mode != kModeDense;
    const bool push = ctl->mode == kModePush;
    // systolic passes visit the medium-degree candidates only
    const int32_t *med = push ? p.cand_list[1] : p.nodes + p.n_small;
    const int64_t total = p.n_seg + (push ? (int64_t)ctl->cand_count[1] : p.n_med);
    const uint8_t *rc = p.regs[cur];
    const unsigned long long *Fc = p.F[cur];
    const int lane = threadIdx.x & 31, g = lane / LANES, gl = lane % LANES;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t c_scan = 0, c_gather = 0, c_own = 0, c_write = 0;
    MarkTally mt;
    for (int64_t it = warp; it < total; it += nwarps) {
        const bool seg = it < p.n_seg;
        const int32_t v = seg ? __ldg(p.seg_node + it) : __ldg(med + (it - p.n_seg));
        const bool take = !seg || !push || test_bit(p.cand, v);
        Row<LANES, VPL> acc;
        row_zero(acc);
        bool any = false;
        if (take) {
            const int64_t beg = seg ? __ldg(p.seg_beg + it) : __ldg(p.off + v);
            const int64_t end = seg ? __ldg(p.seg_end + it) : __ldg(p.off + v + 1);
            warp_gather<LANES, VPL>(p.tgt, rc, Fc, test, beg, end, g, gl, acc, any, c_gather);
            if (lane == 0) c_scan += (uint32_t)(end - beg);
        }
        row_warp_max(acc);
        any = __any_sync(kFull, any);
        if (seg) {
            if (g == 0) row_store(p.hub_part, it, acc, gl);
            if (lane == 0) p.hub_any[it] = any ? 1 : 0;
        } else {
            const bool inR = take && !first && test_bit(Fc, v);
            const bool need = take && (any || inR) && g == 0;
            const uint32_t mask = node_finish(p, cur, acc, need, inR || first, v, gl, c_own, c_write);
            warp_mark(p, cur, lane == 0, v, mask, mt);
        }
    }
    flush_counters(p, cur, mt, c_scan, lane == 0 ? c_gather : 0u, c_own, c_write);
}

// ---------------------------------------------------------------- asynchronous gathers

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc, bool valid)
{
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
    const int n = valid ? 16 : 0;   // 0: nothing is read, the 16 bytes are zero-filled
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(gsrc), "r"(n)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Pipeline depth (stages of 32 arcs in the shared-memory ring of a warp).
template <int LANES>
struct AsyncCfg {
    static constexpr int W = 16 * LANES;
    static constexpr int D = W <= 64 ? 4 : 2;
    static constexpr size_t smem_per_warp = (size_t)D * 32 * W;
    static constexpr size_t smem_per_block = smem_per_warp * (kBlock / 32);
};

// Per-stage bookkeeping kept in shared memory next to the ring.
struct StageMeta {
    int64_t item;   // work item the stage belongs to, -1 if empty
    int32_t valid;  // rows actually gathered
    int32_t last;   // 1 if it is the item's last stage
};

// Union pass over medium nodes and hub segments with the row gathers in
// flight as asynchronous copies: every warp streams its work items as stages
// of up to 32 arcs; the targets of a stage are loaded one stage ahead, the
// rows of D-1 stages are in flight while the oldest is merged from shared
// memory.  Rows of skipped successors are zero-filled, the identity of max.
// For rows of at most 128 bytes (LANES <= 8, one vector per lane).
template <int LANES>
__global__ void __launch_bounds__(kBlock, 2) k_union_warp_async(Plan p)
{
    using Cfg = AsyncCfg<LANES>;
    constexpr int GPW = 32 / LANES;
    constexpr int D = Cfg::D;
    static_assert(GPW * LANES == 32, "lane groups tile the warp");
    extern __shared__ uint4 smem_raw[];
    const DevCtl *ctl = p.ctl;
    if (ctl->done || ctl->mode == kModeScatter || (ctl->t == 0 && p.first_warps)) return;
    const int cur = ctl->parity;
    const bool first = ctl->t == 0;
    const bool test = ctl->mode != kModeDense;
    const bool push = ctl->mode == kModePush;
    const uint8_t *rc = p.regs[cur];
    const unsigned long long *Fc = p.F[cur];
    const int32_t *med = push ? p.cand_list[1] : p.nodes + p.n_small;
    const int64_t total = p.n_seg + (push ? (int64_t)ctl->cand_count[1] : p.n_med);
    const int lane = threadIdx.x & 31, g = lane / LANES, gl = lane % LANES;
    const int wib = threadIdx.x >> 5;
    uint4 *ring = smem_raw + (size_t)wib * (Cfg::smem_per_warp / 16);
    StageMeta *meta = reinterpret_cast<StageMeta *>(smem_raw + (Cfg::smem_per_block / 16)) + wib * D;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t c_scan = 0, c_gather = 0, c_own = 0, c_write = 0;
    MarkTally mt;

    // ---- producer state (warp-uniform) ----
    int64_t p_it = warp - nwarps, p_e = 0, p_end = 0;
    auto next_item = [&]() {
        // advance to the next item that has arcs to merge; untaken hub
        // segments (systolic pass, hub not a candidate) just publish "nothing"
        for (;;) {
            p_it += nwarps;
            if (p_it >= total) return;
            if (p_it < p.n_seg) {
                const int32_t v = __ldg(p.seg_node + p_it);
                if (push && !test_bit(p.cand, v)) {
                    if (lane == 0) p.hub_any[p_it] = 0;
                    continue;
                }
                p_e = __ldg(p.seg_beg + p_it);
                p_end = __ldg(p.seg_end + p_it);
            } else {
                const int32_t v = __ldg(med + (p_it - p.n_seg));
                p_e = __ldg(p.off + v);
                p_end = __ldg(p.off + v + 1);
            }
            if (lane == 0) c_scan += (uint32_t)(p_end - p_e);
            return;
        }
    };
    next_item();
    // targets of the next stage to issue, loaded one stage ahead
    int32_t t_next = (p_it < total && p_e + lane < p_end) ? __ldg(p.tgt + p_e + lane) : -1;

    auto produce = [&](int slot) {
        uint4 *buf = ring + (size_t)slot * 32 * LANES;
        if (p_it >= total) {
            if (lane == 0) meta[slot].item = -1;
            cp_async_commit();
            return;
        }
        int32_t w = t_next;
        const int64_t it = p_it;
        const bool last = p_e + 32 >= p_end;
        // advance the producer and prefetch the following stage's targets
        p_e += 32;
        if (last) next_item();
        t_next = (p_it < total && p_e + lane < p_end) ? __ldg(p.tgt + p_e + lane) : -1;
        if (w >= 0 && test && !test_bit(Fc, w)) w = -1;
        const unsigned live = __ballot_sync(kFull, w >= 0);
        // lane (g, gl) copies the gl-th 16 bytes of rows g, g+GPW, ...
#pragma unroll
        for (int k = 0; k < LANES; ++k) {
            const int r = g + GPW * k;
            const int32_t wr = __shfl_sync(kFull, w, r);
            const uint8_t *src = wr >= 0 ? rc + (int64_t)wr * Cfg::W + gl * 16 : rc;
            cp_async16(buf + r * LANES + gl, src, wr >= 0);
        }
        cp_async_commit();
        if (lane == 0) {
            meta[slot].item = it;
            meta[slot].valid = __popc(live);
            meta[slot].last = last ? 1 : 0;
        }
    };

    Row<LANES, 1> acc;
    row_zero(acc);
    bool any = false;
    auto consume = [&](int slot) -> bool {
        cp_async_wait<D - 1>();
        __syncwarp();
        const StageMeta m = meta[slot];
        if (m.item < 0) {
            __syncwarp();
            return false;
        }
        const uint4 *buf = ring + (size_t)slot * 32 * LANES;
#pragma unroll
        for (int k = 0; k < LANES; ++k) acc.v[0] = vmax4(acc.v[0], buf[(g + GPW * k) * LANES + gl]);
        if (m.valid) any = true;
        c_gather += m.valid;
        __syncwarp();
        if (m.last) {
            row_warp_max(acc);
            const bool anyw = any;   // warp-uniform: every lane saw the same stages
            if (m.item < p.n_seg) {
                if (g == 0) row_store(p.hub_part, m.item, acc, gl);
                if (lane == 0) p.hub_any[m.item] = anyw ? 1 : 0;
            } else {
                const int32_t v = __ldg(med + (m.item - p.n_seg));
                const bool inR = !first && test_bit(Fc, v);
                const bool need = (anyw || inR) && g == 0;
                const uint32_t mask = node_finish(p, cur, acc, need, inR || first, v, gl, c_own, c_write);
                warp_mark(p, cur, lane == 0, v, mask, mt);
            }
            row_zero(acc);
            any = false;
        }
        return true;
    };

#pragma unroll
    for (int s = 0; s < D - 1; ++s) produce(s);
    for (int k = 0;; ++k) {
        produce((k + D - 1) % D);
        if (!consume(k % D) && p_it >= total) break;
    }
    cp_async_wait<0>();
    flush_counters(p, cur, mt, c_scan, lane == 0 ? c_gather : 0u, c_own, c_write);
}

// Small-degree union with asynchronous row copies (gather_variant 3; rows of
// at most 128 bytes, dense passes): each lane copies its 16-byte share of a
// batch of UA rows into its own shared-memory slots with cp.async and merges
// the previous batch meanwhile, so a lane group keeps up to 2 x UA rows in
// flight without holding them in registers.  A lane only ever reads the
// slots it filled itself, so cp.async.wait_group is the only wait (no
// cross-lane barrier); rows a batch does not use are zero-filled, which
// leaves the max unchanged.
template <int LANES>
struct SmallAsyncCfg {
    static constexpr int UA = 8;                                        // rows per batch
    static constexpr size_t smem_per_warp = 2 * (size_t)UA * 32 * sizeof(uint4);
    static constexpr size_t smem_per_block = smem_per_warp * (kBlock / 32);
};

template <int LANES>
__global__ void __launch_bounds__(kBlock, 3) k_union_small_async(Plan p)
{
    constexpr int GPW = 32 / LANES;
    constexpr int UA = SmallAsyncCfg<LANES>::UA;
    constexpr int TPL = (UA + LANES - 1) / LANES;
    extern __shared__ uint4 async_rows[];
    const DevCtl *ctl = p.ctl;
    if (ctl->done || ctl->mode != kModeDense || (ctl->t == 0 && p.first_warps)) return;
    const int cur = ctl->parity;
    const bool first = ctl->t == 0;
    const uint8_t *rc = p.regs[cur];
    const unsigned long long *Fc = p.F[cur];
    const int lane = threadIdx.x & 31, g = lane / LANES, gl = lane % LANES;
    const int gbase = g * LANES;
    const unsigned gmask = ((1u << LANES) - 1u) << gbase;
    uint4 *ring = async_rows + (size_t)(threadIdx.x >> 5) * (2 * UA * 32);
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t c_scan = 0, c_gather = 0, c_own = 0, c_write = 0;
    MarkTally mt;
    const int32_t *list = p.nodes;
    const int64_t count = p.n_small;
    const int64_t stride = nwarps * GPW;
    int64_t idx_ahead = warp * GPW + g;
    int32_t v_next = idx_ahead < count ? __ldg(list + idx_ahead) : -1;
    int64_t beg_next = v_next >= 0 ? __ldg(p.off + v_next) : 0;
    int64_t end_next = v_next >= 0 ? __ldg(p.off + v_next + 1) : 0;
    idx_ahead += stride;
    int32_t v_after = idx_ahead < count ? __ldg(list + idx_ahead) : -1;
    // targets of a batch at e: each lane its TPL share
    auto load_targets = [&](int32_t (&t)[TPL], int64_t e, int64_t end) {
#pragma unroll
        for (int k = 0; k < TPL; ++k) {
            const int j = gl + k * LANES;
            t[k] = (j < UA && e + j < end) ? __ldg(p.tgt + e + j) : -1;
        }
    };
    // copy the batch's rows into stage `st`: lane gl copies bytes
    // [16 gl, 16 gl + 16) of each row; every lane of the warp takes part
    auto issue = [&](const int32_t (&t)[TPL], int st) {
#pragma unroll
        for (int u = 0; u < UA; ++u) {
            const int32_t w = __shfl_sync(kFull, t[u / LANES], gbase + (u % LANES));
            const uint8_t *src = w >= 0 ? rc + (int64_t)w * (16 * LANES) + gl * 16 : rc;
            cp_async16(ring + (st * UA + u) * 32 + lane, src, w >= 0);
        }
        cp_async_commit();
    };
    for (int64_t base = warp * GPW; base < count; base += stride) {
        const int32_t v = v_next;
        const int64_t beg = beg_next, end = end_next;
        const bool valid = v >= 0;
        v_next = v_after;
        beg_next = v_next >= 0 ? __ldg(p.off + v_next) : 0;
        end_next = v_next >= 0 ? __ldg(p.off + v_next + 1) : 0;
        idx_ahead += stride;
        v_after = idx_ahead < count ? __ldg(list + idx_ahead) : -1;
        Row<LANES, 1> own;
        if (valid) row_load(own, rc, v, gl);
        Row<LANES, 1> acc;
        row_zero(acc);
        // the lane groups of a warp walk their nodes' batches in lockstep:
        // the warp loops over the longest arc range among its groups
        const int64_t len = valid ? end - beg : 0;
        int64_t len_max = len;
#pragma unroll
        for (int o = LANES; o < 32; o <<= 1)
            len_max = max(len_max, (int64_t)__shfl_xor_sync(kFull, (long long)len_max, o));
        if (len_max > 0) {
            int32_t t[TPL];
            load_targets(t, beg, valid ? end : beg);
            issue(t, 0);
            load_targets(t, beg + UA, valid ? end : beg);
            int st = 0;
            for (int64_t k = 0; k < len_max; k += UA) {
                if (k + UA < len_max) {
                    issue(t, st ^ 1);
                    load_targets(t, beg + k + 2 * UA, valid ? end : beg);
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
#pragma unroll
                for (int u = 0; u < UA; ++u)
                    acc.v[0] = vmax4(acc.v[0], ring[(st * UA + u) * 32 + lane]);
                st ^= 1;
            }
        }
        (void)gmask;
        if (valid && gl == 0) {
            c_scan += (uint32_t)len;
            c_gather += (uint32_t)len;
        }
        const bool any = len > 0;
        const bool inR = valid && !first && test_bit(Fc, v);
        const bool need = valid && (any || inR);
        const uint32_t mask = node_finish(p, cur, acc, need, inR || first, v, gl, c_own, c_write, &own);
        warp_mark(p, cur, gl == 0 && valid, v, mask, mt);
    }
    cp_async_wait<0>();
    flush_counters(p, cur, mt, c_scan, gl == 0 ? c_gather : 0u, c_own, c_write);
}

// Hub nodes: combine the segment partials written by k_union_warp, then
// finish like any other node.  A lane group per hub.
template <int LANES, int VPL>
__global__ void __launch_bounds__(kBlock) k_hub_finish(Plan p)
{
    constexpr int GPW = 32 / LANES;
    const DevCtl *ctl = p.ctl;
    if (ctl->done || p.n_hub == 0 || ctl->mode == kModeScatter) return;
    const int cur = ctl->parity;
    const bool first = ctl->t == 0;
    const bool push = ctl->mode == kModePush;
    const unsigned long long *Fc = p.F[cur];
    const int lane = threadIdx.x & 31, g = lane / LANES, gl = lane % LANES;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t c_own = 0, c_write = 0;
    MarkTally mt;
    for (int64_t base = warp * GPW; base < p.n_hub; base += nwarps * GPW) {
        const int64_t h = base + g;
        const bool valid = h < p.n_hub;
        const int32_t v = valid ? p.nodes[p.n_small + p.n_med + h] : 0;
        const bool take = valid && (!push || test_bit(p.cand, v));
        Row<LANES, VPL> acc;
        row_zero(acc);
        bool any = false;
        if (take) {
            for (int32_t s = p.hub_seg_first[h]; s < p.hub_seg_first[h + 1]; ++s) {
                if (p.hub_any[s]) {
                    Row<LANES, VPL> x;
                    row_load(x, p.hub_part, s, gl);
                    row_max(acc, x);
                    any = true;
                }
            }
        }
        const bool inR = take && !first && test_bit(Fc, v);
        const bool need = take && (any || inR);
        const uint32_t mask = node_finish(p, cur, acc, need, inR || first, v, gl, c_own, c_write);
        warp_mark(p, cur, gl == 0 && valid, v, mask, mt);
    }
    flush_counters(p, cur, mt, 0u, 0u, c_own, c_write);
}

// ---------------------------------------------------------------- pass 0 from the c_0 records

// At t = 0 every counter holds its own node only: run r's register idx_r(u)
// = rho_r(u), every other register 0 (Algorithm 2's initialisation).  So
// pass 0, c_1[v] = max(c_0[v], max_{v->w} c_0[w]), needs one two-byte record
// (idx << 8 | rho) a successor and run, written by k_init, instead of the
// successor's W-byte row: one sector request instead of W/32.  The successors'
// registers are merged into a row of one 32-bit word a register in shared
// memory (atomicMax), which is then packed into bytes and finished as in the
// other passes.  The result is the same row, so the pass is the same; the
// pull kernels sit it out (they return at t = 0 when first_warps is set).

// Lane gl's 16-byte chunk of a shared-memory row of word registers, cleared
// behind it for the next node.
__device__ __forceinline__ uint4 pack_chunk(uint32_t *row_words, int byte0)
{
    uint4 *q = reinterpret_cast<uint4 *>(row_words + byte0);
    uint32_t out[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint4 a = q[i];
        out[i] = a.x | (a.y << 8) | (a.z << 16) | (a.w << 24);
        q[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    return make_uint4(out[0], out[1], out[2], out[3]);
}

// Merge the records of arcs [e0, end) taken `stride` apart, KB at a time, into
// the word row: every run's register of every successor.
template <int KB>
__device__ __forceinline__ void merge_records(const Plan &p, uint32_t *row_words, int64_t e0,
                                              int64_t end, int stride)
{
    for (; e0 < end; e0 += (int64_t)KB * stride) {
        int32_t w[KB];
#pragma unroll
        for (int k = 0; k < KB; ++k) {
            const int64_t e = e0 + (int64_t)k * stride;
            w[k] = e < end ? __ldg(p.tgt + e) : -1;
        }
        if (p.R == 8) {
            // eight runs: a successor's records are one aligned 16-byte vector
            // (four successors at a time)
#pragma unroll
            for (int k0 = 0; k0 < KB; k0 += 4) {
                uint4 rec[4];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    rec[k] = (k0 + k < KB && w[k0 + k] >= 0)
                                 ? __ldg(reinterpret_cast<const uint4 *>(p.hr) + w[k0 + k])
                                 : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (k0 + k < KB && w[k0 + k] >= 0) {
                        const uint32_t q[4] = {rec[k].x, rec[k].y, rec[k].z, rec[k].w};
#pragma unroll
                        for (int r = 0; r < 8; ++r) {
                            const uint32_t e = (q[r >> 1] >> (16 * (r & 1))) & 0xffffu;
                            atomicMax(row_words + r * p.m + (e >> 8), e & 0xffu);
                        }
                    }
            }
            continue;
        }
        for (int r = 0; r < p.R; ++r) {
            uint32_t rec[KB];
#pragma unroll
            for (int k = 0; k < KB; ++k)
                rec[k] = w[k] >= 0 ? (uint32_t)__ldg(p.hr + (int64_t)w[k] * p.R + r) : 0u;
#pragma unroll
            for (int k = 0; k < KB; ++k)
                if (w[k] >= 0) atomicMax(row_words + r * p.m + (rec[k] >> 8), rec[k] & 0xffu);
        }
    }
}

// The node's own counter c_0[v], lane gl's chunks.
template <int LANES, int VPL>
__device__ __forceinline__ void own_singleton(Row<LANES, VPL> &own, const Plan &p, int32_t v, int gl)
{
#pragma unroll
    for (int k = 0; k < VPL; ++k) {
        const int byte0 = (k * LANES + gl) << 4;
        const uint32_t e = __ldg(p.hr + (int64_t)v * p.R + (byte0 >> p.b));
        const int rel = (int)(e >> 8) - (byte0 & (p.m - 1));
        const uint32_t val = (rel >= 0 && rel < 16) ? (e & 0xffu) << ((rel & 3) * 8) : 0u;
        const int q = rel >> 2;
        own.v[k] = make_uint4(q == 0 ? val : 0u, q == 1 ? val : 0u, q == 2 ? val : 0u,
                              q == 3 ? val : 0u);
    }
}

constexpr int kFirstBlocks = 4;   // resident blocks an SM the pass-0 kernels are built for

// Pass 0 over small nodes: a lane group per node, as k_union_small.
template <int LANES, int VPL>
__global__ void __launch_bounds__(kBlock, kFirstBlocks) k_first_small(Plan p)
{
    constexpr int GPW = 32 / LANES;
    constexpr int WB = 16 * LANES * VPL;   // registers a row (all runs)
    __shared__ __align__(16) uint32_t words[kBlock / 32][GPW * WB];
    const DevCtl *ctl = p.ctl;
    if (ctl->done || ctl->t != 0 || p.first_warps == 0) return;
    const int cur = ctl->parity;
    const int lane = threadIdx.x & 31, g = lane / LANES, gl = lane % LANES;
    uint32_t *row_words = words[threadIdx.x >> 5] + g * WB;
    for (int i = gl; i < WB; i += LANES) row_words[i] = 0u;
    __syncwarp();
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t c_scan = 0, c_own = 0, c_write = 0;
    MarkTally mt;
    const int64_t count = p.n_small;
    const int64_t stride = nwarps * GPW;
    int64_t idx = warp * GPW + g;
    int32_t v_next = idx < count ? __ldg(p.nodes + idx) : -1;
    for (int64_t base = warp * GPW; base < count; base += stride) {
        const int32_t v = v_next;
        idx += stride;
        v_next = idx < count ? __ldg(p.nodes + idx) : -1;
        const bool valid = v >= 0;
        const int64_t beg = valid ? __ldg(p.off + v) : 0, end = valid ? __ldg(p.off + v + 1) : 0;
        merge_records<8>(p, row_words, beg + gl, end, LANES);
        __syncwarp();
        Row<LANES, VPL> acc, own;
#pragma unroll
        for (int k = 0; k < VPL; ++k) acc.v[k] = pack_chunk(row_words, (k * LANES + gl) << 4);
        if (valid) own_singleton(own, p, v, gl);
        __syncwarp();
        if (valid && gl == 0) c_scan += (uint32_t)(end - beg);
        // every listed node has arcs; pass 0 stores every row it visits
        const uint32_t mask = node_finish(p, cur, acc, valid, true, v, gl, c_own, c_write, &own);
        warp_mark(p, cur, gl == 0 && valid, v, mask, mt);
    }
    flush_counters(p, cur, mt, c_scan, gl == 0 ? c_scan : 0u, c_own, c_write);
}

// Pass 0 over hub segments and medium nodes: a warp per item, as k_union_warp.
template <int LANES, int VPL>
__global__ void __launch_bounds__(kBlock, kFirstBlocks) k_first_warp(Plan p)
{
    constexpr int WB = 16 * LANES * VPL;
    __shared__ __align__(16) uint32_t words[kBlock / 32][WB];
    const DevCtl *ctl = p.ctl;
    if (ctl->done || ctl->t != 0 || p.first_warps == 0) return;
    const int cur = ctl->parity;
    const int lane = threadIdx.x & 31, g = lane / LANES, gl = lane % LANES;
    uint32_t *row_words = words[threadIdx.x >> 5];
    for (int i = lane; i < WB; i += 32) row_words[i] = 0u;
    __syncwarp();
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t c_scan = 0, c_own = 0, c_write = 0;
    MarkTally mt;
    const int64_t total = p.n_seg + p.n_med;
    for (int64_t it = warp; it < total; it += nwarps) {
        const bool seg = it < p.n_seg;
        const int32_t v = seg ? __ldg(p.seg_node + it) : __ldg(p.nodes + p.n_small + (it - p.n_seg));
        const int64_t beg = seg ? __ldg(p.seg_beg + it) : __ldg(p.off + v);
        const int64_t end = seg ? __ldg(p.seg_end + it) : __ldg(p.off + v + 1);
        merge_records<4>(p, row_words, beg + lane, end, 32);
        __syncwarp();
        Row<LANES, VPL> acc, own;
        if (g == 0) {
#pragma unroll
            for (int k = 0; k < VPL; ++k) acc.v[k] = pack_chunk(row_words, (k * LANES + gl) << 4);
        }
        __syncwarp();
        if (lane == 0) c_scan += (uint32_t)(end - beg);
        if (seg) {
            if (g == 0) row_store(p.hub_part, it, acc, gl);
            if (lane == 0) p.hub_any[it] = end > beg ? 1 : 0;
        } else {
            if (g == 0) own_singleton(own, p, v, gl);
            const uint32_t mask = node_finish(p, cur, acc, g == 0, true, v, gl, c_own, c_write, &own);
            warp_mark(p, cur, lane == 0, v, mask, mt);
        }
    }
    flush_counters(p, cur, mt, c_scan, lane == 0 ? c_scan : 0u, c_own, c_write);
}

// ---------------------------------------------------------------- pass control

// Choose pull or systolic push for the coming pass and reset its counters.
// Section 3.3: systolic computation once fewer than n/push_den counters
// changed.
__global__ void k_prep(Plan p)
{
    DevCtl *c = p.ctl;
    if (c->done) return;
    const long long changed = (long long)c->last_changed;
    int mode = kModeTest;
    const long long in_arcs = (long long)c->changed_in_arcs;
    if (c->t == 0 || p.frontier == HANF_FRONTIER_OFF)
        mode = kModeDense;
    else if (p.frontier == HANF_FRONTIER_AUTO && p.in_off != nullptr && p.layout == 0 &&
             p.scatter_den > 0 && in_arcs * p.scatter_den < p.arcs &&
             in_arcs / p.scatter_seg + in_arcs / p.scatter_inline + 1 <= p.n)
        mode = kModeScatter;   // the segment list fits the candidate lists
    else if (p.frontier == HANF_FRONTIER_AUTO && p.in_off != nullptr && changed * p.push_den < p.n)
        mode = kModePush;
    else if (p.in_off != nullptr
                 ? (long long)c->changed_in_arcs * p.dense_den >= p.arcs * p.dense_num
                 : changed * p.dense_den >= p.n * p.dense_num)
        mode = kModeDense;   // most successors changed: skip the per-arc test
    c->mode = mode;
    c->changed_count[c->parity ^ 1] = 0;
    c->cand_count[0] = 0;
    c->cand_count[1] = 0;
    c->changed_in_arcs = 0;     // the estimator sums it again after this pass
}

__global__ void k_clear(Plan p)
{
    const DevCtl *c = p.ctl;
    if (c->done) return;
    unsigned long long *fn = p.F[c->parity ^ 1];
    const bool push = c->mode == kModePush;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.nwords || i < p.S;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < p.nwords) {
            fn[i] = 0ull;
            if (push) p.cand[i] = 0ull;
        }
        if (i < p.S) p.slot_changed[i] = 0ull;
    }
}

// Systolic signalling: every node changed by the previous pass marks itself
// and its predecessors (through the transposed graph) as candidates.  The
// first marking of a node appends it to the candidate list of its degree
// class (warp-aggregated), so the union kernels visit candidates only; hubs
// are found through their segments.
__device__ __forceinline__ void cand_append(const Plan &p, bool fresh, int32_t u)
{
    int cls = -1;
    if (fresh) {
        const int64_t deg = __ldg(p.off + u + 1) - __ldg(p.off + u);
        cls = deg <= p.d_small ? 0 : (deg <= p.d_hub ? 1 : -1);
    }
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const unsigned bal = __ballot_sync(kFull, cls == k);
        if (bal == 0) continue;
        const int first = __ffs(bal) - 1;
        unsigned long long base = 0;
        if (lane == first) base = atomicAdd(&p.ctl->cand_count[k], (unsigned long long)__popc(bal));
        base = __shfl_sync(kFull, base, first);
        if (cls == k) p.cand_list[k][base + __popc(bal & ((1u << lane) - 1u))] = u;
    }
}

__global__ void k_mark(Plan p)
{
    const DevCtl *c = p.ctl;
    if (c->done || c->mode != kModePush) return;
    const unsigned long long *Fc = p.F[c->parity];
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // 32 bitmap words per warp iteration (lane l: word i0 + l * nwarps), the
    // non-zero ones in order
    for (int64_t i0 = warp; i0 < p.nwords; i0 += nwarps * 32) {
        const int64_t iw = i0 + (int64_t)lane * nwarps;
        const unsigned long long mine = iw < p.nwords ? Fc[iw] : 0ull;
        for (unsigned nz = __ballot_sync(kFull, mine != 0ull); nz; nz &= nz - 1u) {
            const int src_lane = __ffs(nz) - 1;
            const int64_t i = i0 + (int64_t)src_lane * nwarps;
            unsigned long long bits = __shfl_sync(kFull, mine, src_lane);
            while (bits) {
                const int32_t w = (int32_t)(i * 64 + (__ffsll((long long)bits) - 1));
                bits &= bits - 1;
                const int64_t beg = p.in_off[w], deg = p.in_off[w + 1] - beg;
                // item 0 is w itself, item j >= 1 its (j-1)-th predecessor
                for (int64_t j0 = 0; j0 <= deg; j0 += 32) {
                    const int64_t j = j0 + lane;
                    const int32_t u = j == 0 ? w : (j <= deg ? __ldg(p.in_src + beg + j - 1) : -1);
                    bool fresh = false;
                    if (u >= 0) {
                        const unsigned long long bit = 1ull << (u & 63);
                        fresh = (atomicOr(&p.cand[u >> 6], bit) & bit) == 0ull;
                    }
                    cand_append(p, fresh, u);
                }
            }
        }
    }
}

// Slots (graph, run) that a pass left unchanged end at that pass (batches
// with more than 8 slots; smaller ones are handled by k_post).
// ---------------------------------------------------------------- scatter (pure push)

// Scatter pass: Section 3.3's systolic computation carried to its end.  Once
// the nodes changed by the last pass (F_t) have few in-arcs, every w in F_t
// pushes c_t[w] into the new counter of each predecessor v, and nothing else
// is visited.  Jacobi is kept: pushes read c_t (regs[p], untouched by the
// pass) and raise c_{t+1} (regs[p^1]) with a compare-and-swap byte max, which
// commutes, so the result does not depend on the order of the pushes.
// regs[p^1] holds c_{t-1} on entry, which equals c_t except on F_t: those
// rows are copied first (k_scatter_seed), before any push lands.
__device__ __forceinline__ unsigned long long pack64(uint32_t lo, uint32_t hi)
{
    return (unsigned long long)lo | ((unsigned long long)hi << 32);
}

__device__ __forceinline__ unsigned long long bmax64(unsigned long long a, unsigned long long b)
{
    return pack64(bmax((uint32_t)a, (uint32_t)b), bmax((uint32_t)(a >> 32), (uint32_t)(b >> 32)));
}

// Raise the eight registers at q to at least those of `mine`.  `now` is a
// value read from q earlier (possibly stale: registers only grow during the
// pass, so a stale value is never above the current one).  Returns whether
// this call raised q.  Every failed compare-and-swap means another thread
// raised a register of q, which can happen at most 8 x 31 times, so the loop
// always ends within its bound; `bad` records the impossible case.
__device__ __forceinline__ bool raise64(unsigned long long *q, unsigned long long now,
                                        unsigned long long mine, bool &bad)
{
    for (int it = 0; it <= 8 * 31; ++it) {
        const unsigned long long want = bmax64(now, mine);
        if (want == now) return false;
        const unsigned long long seen = atomicCAS(q, now, want);
        if (seen == now) return true;
        now = seen;
    }
    bad = true;
    return false;
}

// (node, predecessor) pairs a lane group of a scatter pass keeps in flight:
// two rows of one vector a lane, one for wider lane rows.  (Four rows need
// more than 80 registers; two resident blocks of 128 registers measured
// slower than three of 80.)
template <int LANES, int VPL>
constexpr int kScatterRows = (LANES < 2 ? LANES : 2) / VPL > 0 ? (LANES < 2 ? LANES : 2) / VPL : 1;

// Copy the rows of F_t into regs[p^1] (they hold c_{t-1} there) and cut the
// in-arc lists longer than p.scatter_inline into segments, listed in
// cand_list[0] (node) / cand_list[1] (segment index), counted in
// cand_count[0].  A lane per changed node, a warp per non-zero bitmap word.
__global__ void __launch_bounds__(kBlock) k_scatter_seed(Plan p)
{
    const DevCtl *ctl = p.ctl;
    if (ctl->done || ctl->mode != kModeScatter) return;
    const int cur = ctl->parity;
    const unsigned long long *Fc = p.F[cur];
    const uint4 *src = reinterpret_cast<const uint4 *>(p.regs[cur]);
    uint4 *dst = reinterpret_cast<uint4 *>(p.regs[cur ^ 1]);
    const int vec = p.W >> 4;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t c_write = 0;
    bool bad = false;
    // a warp reads 32 bitmap words at once (lane l: word i0 + l * nwarps, so
    // that small bitmaps still spread over all warps), then handles the
    // non-zero ones in order
    for (int64_t i0 = warp; i0 < p.nwords; i0 += nwarps * 32) {
        const int64_t iw = i0 + (int64_t)lane * nwarps;
        const unsigned long long mine = iw < p.nwords ? Fc[iw] : 0ull;
        for (unsigned nz = __ballot_sync(kFull, mine != 0ull); nz; nz &= nz - 1u) {
            const int src_lane = __ffs(nz) - 1;
            const int64_t i = i0 + (int64_t)src_lane * nwarps;
            const unsigned long long bits = __shfl_sync(kFull, mine, src_lane);
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                const int bit = lane + 32 * h;
                const int32_t w = (int32_t)(i * 64 + bit);
                int32_t nseg = 0;
                if ((bits >> bit) & 1ull) {
#pragma unroll 4
                    for (int k = 0; k < vec; ++k) dst[(int64_t)w * vec + k] = src[(int64_t)w * vec + k];
                    ++c_write;
                    const int64_t d = p.in_off[w + 1] - p.in_off[w];
                    if (d > p.scatter_inline) nseg = (int32_t)((d + p.scatter_seg - 1) / p.scatter_seg);
                }
                int32_t incl = nseg;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t t = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += t;
                }
                const int32_t total = __shfl_sync(kFull, incl, 31);
                if (total == 0) continue;
                unsigned long long base = 0;
                if (lane == 31) base = atomicAdd(&p.ctl->cand_count[0], (unsigned long long)total);
                base = __shfl_sync(kFull, base, 31);
                const unsigned long long first = base + (unsigned long long)(incl - nseg);
                for (int32_t j = 0; j < nseg; ++j) {
                    if (first + j >= (unsigned long long)p.n) {   // k_prep's bound broken
                        bad = true;
                        break;
                    }
                    p.cand_list[0][first + j] = w;
                    p.cand_list[1][first + j] = j;
                }
            }
        }
    }
    flush_counters(p, cur, MarkTally(), 0u, 0u, 0u, c_write);
    if (bad) p.ctl->err = HANF_ESTATE;
}

// Push the (changed node w, predecessor v) pairs of up to 32 entries, one per
// lane (entry: node w_l, its in-arcs [beg_l, beg_l + cnt_l)).  The entries'
// pairs are numbered consecutively and taken 32 at a time, a pair per lane
// (its entry found by binary search over the entries' prefix sums), so short
// in-arc lists fill whole warps; lane group g then merges the pairs of lanes
// g*LANES .. g*LANES+LANES-1, SUB rows in flight.  Warp-uniform control flow.
template <int LANES, int VPL>
__device__ __forceinline__ void scatter_entries(const Plan &p, int cur, int32_t w_l, int64_t beg_l,
                                                int32_t cnt_l, MarkTally &mt, uint32_t &pairs,
                                                uint32_t &raised, bool &bad)
{
    constexpr int SUB = kScatterRows<LANES, VPL>;
    const int lane = threadIdx.x & 31, gl = lane % LANES, gbase = lane - gl;
    const uint8_t *rc = p.regs[cur];
    uint8_t *rn = p.regs[cur ^ 1];
    int32_t incl = cnt_l;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    const int32_t total = __shfl_sync(kFull, incl, 31);
    const int32_t excl = incl - cnt_l;
    for (int32_t base = 0; base < total; base += 32) {
        const int32_t q = base + lane;
        // entry of pair q: the last lane whose prefix sum is <= q
        int lo = 0;
#pragma unroll
        for (int st = 16; st; st >>= 1) {
            const int32_t e = __shfl_sync(kFull, excl, lo + st);
            if (e <= q) lo += st;
        }
        const int32_t w = __shfl_sync(kFull, w_l, lo);
        const int64_t b = __shfl_sync(kFull, beg_l, lo);
        const int32_t e0 = __shfl_sync(kFull, excl, lo);
        const int32_t v = q < total ? __ldg(p.in_src + b + (q - e0)) : -1;
#pragma unroll 1
        for (int u0 = 0; u0 < LANES; u0 += SUB) {
            int32_t ws[SUB], vs[SUB];
#pragma unroll
            for (int u = 0; u < SUB; ++u) {
                ws[u] = __shfl_sync(kFull, w, gbase + u0 + u);
                vs[u] = __shfl_sync(kFull, v, gbase + u0 + u);
            }
            Row<LANES, VPL> mine[SUB], now[SUB];
#pragma unroll
            for (int u = 0; u < SUB; ++u)
                if (vs[u] >= 0) {
                    row_load(mine[u], rc, ws[u], gl);
                    const uint4 *qn = reinterpret_cast<const uint4 *>(rn) +
                                      (int64_t)vs[u] * (LANES * VPL) + gl;
#pragma unroll
                    for (int k = 0; k < VPL; ++k) now[u].v[k] = __ldcg(qn + k * LANES);
                }
            // first attempts for every word of the round, all in flight
            // together; the values they saw replace `now`, and fl[u] keeps,
            // per 64-bit word i, bit 2i = raised, bit 2i+1 = retry needed
            uint32_t fl[SUB];
#pragma unroll
            for (int u = 0; u < SUB; ++u) {
                fl[u] = 0;
                if (vs[u] >= 0) {
                    unsigned long long *q64 = reinterpret_cast<unsigned long long *>(
                        reinterpret_cast<uint4 *>(rn) + (int64_t)vs[u] * (LANES * VPL) + gl);
#pragma unroll
                    for (int k = 0; k < VPL; ++k) {
                        const uint4 a = now[u].v[k], m4 = mine[u].v[k];
                        const unsigned long long n0 = pack64(a.x, a.y), n1 = pack64(a.z, a.w);
                        const unsigned long long w0 = bmax64(n0, pack64(m4.x, m4.y));
                        const unsigned long long w1 = bmax64(n1, pack64(m4.z, m4.w));
                        unsigned long long s0 = n0, s1 = n1;
                        if (w0 != n0) s0 = atomicCAS(q64 + 2 * k * LANES, n0, w0);
                        if (w1 != n1) s1 = atomicCAS(q64 + 2 * k * LANES + 1, n1, w1);
                        if (w0 != n0) fl[u] |= (s0 == n0 ? 1u : 2u) << (4 * k);
                        if (w1 != n1) fl[u] |= (s1 == n1 ? 1u : 2u) << (4 * k + 2);
                        now[u].v[k] = make_uint4((uint32_t)s0, (uint32_t)(s0 >> 32), (uint32_t)s1,
                                                 (uint32_t)(s1 >> 32));
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < SUB; ++u) {
                uint32_t mask = 0;
                if (vs[u] >= 0) {
                    unsigned long long *q64 = reinterpret_cast<unsigned long long *>(
                        reinterpret_cast<uint4 *>(rn) + (int64_t)vs[u] * (LANES * VPL) + gl);
#pragma unroll
                    for (int k = 0; k < VPL; ++k) {
                        const uint4 a = now[u].v[k], m4 = mine[u].v[k];
                        bool r0 = (fl[u] >> (4 * k)) & 1u, r1 = (fl[u] >> (4 * k + 2)) & 1u;
                        if ((fl[u] >> (4 * k + 1)) & 1u)   // lost a race: retry from what it saw
                            r0 = raise64(q64 + 2 * k * LANES, pack64(a.x, a.y), pack64(m4.x, m4.y), bad);
                        if ((fl[u] >> (4 * k + 3)) & 1u)
                            r1 = raise64(q64 + 2 * k * LANES + 1, pack64(a.z, a.w), pack64(m4.z, m4.w),
                                         bad);
                        if (r0 || r1) mask |= 1u << (((k * LANES + gl) << 4) >> p.b);
                    }
                }
                mask = group_or<LANES>(mask);
                const bool ch = gl == 0 && vs[u] >= 0 && mask != 0;
                const unsigned bal = __ballot_sync(kFull, ch);
                if (bal) {
                    if (ch) {
                        const unsigned long long bit = 1ull << (vs[u] & 63);
                        if ((atomicOr(&p.F[cur ^ 1][vs[u] >> 6], bit) & bit) == 0ull) ++mt.fresh;
                    }
                    tally_runs(p, ch, bal, vs[u], mask, mt);
                }
                if (gl == 0 && vs[u] >= 0) {
                    ++pairs;
                    if (mask) ++raised;
                }
            }
        }
    }
}

// The pushes of a scatter pass: a warp per item, items = the segments listed
// by k_scatter_seed, then the bitmap words of F_t (their nodes of in-degree at
// most p.scatter_inline, 32 entries at a time).
template <int LANES, int VPL>
__global__ void __launch_bounds__(kBlock, min_blocks(VPL)) k_scatter(Plan p)
{
    const DevCtl *ctl = p.ctl;
    if (ctl->done || ctl->mode != kModeScatter) return;
    const int cur = ctl->parity;
    const unsigned long long *Fc = p.F[cur];
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nseg = min((int64_t)ctl->cand_count[0], p.n);   // the list's capacity
    uint32_t pairs = 0, raised = 0;
    MarkTally mt;
    bool bad = false;
    for (int64_t it = warp; it < nseg; it += nwarps) {
        int32_t w = -1, cnt = 0;
        int64_t beg = 0;
        if (lane == 0) {
            w = p.cand_list[0][it];
            const int64_t j = p.cand_list[1][it];
            const int64_t b0 = p.in_off[w], d = p.in_off[w + 1] - b0;
            beg = b0 + j * p.scatter_seg;
            cnt = (int32_t)min((int64_t)p.scatter_seg, d - j * p.scatter_seg);
        }
        scatter_entries<LANES, VPL>(p, cur, w, beg, cnt, mt, pairs, raised, bad);
    }
    // the bitmap words of F_t, 32 per warp iteration (lane l: word i0 + l *
    // nwarps; the warps that finished their segments first take the first
    // ones)
    const int64_t wrank = (warp - nseg % nwarps + nwarps) % nwarps;
    for (int64_t i0 = wrank; i0 < p.nwords; i0 += nwarps * 32) {
        const int64_t iw = i0 + (int64_t)lane * nwarps;
        const unsigned long long mine = iw < p.nwords ? Fc[iw] : 0ull;
        for (unsigned nz = __ballot_sync(kFull, mine != 0ull); nz; nz &= nz - 1u) {
            const int src_lane = __ffs(nz) - 1;
            const int64_t i = i0 + (int64_t)src_lane * nwarps;
            const unsigned long long bits = __shfl_sync(kFull, mine, src_lane);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (((bits >> (32 * h)) & 0xffffffffull) == 0ull) continue;
                const int bit = lane + 32 * h;
                int32_t w = -1, cnt = 0;
                int64_t beg = 0;
                if ((bits >> bit) & 1ull) {
                    w = (int32_t)(i * 64 + bit);
                    beg = p.in_off[w];
                    const int64_t d = p.in_off[w + 1] - beg;
                    if (d <= p.scatter_inline) cnt = (int32_t)d;   // longer lists: by segments
                }
                scatter_entries<LANES, VPL>(p, cur, w, beg, cnt, mt, pairs, raised, bad);
            }
        }
    }
    flush_counters(p, cur, mt, pairs, pairs, pairs, raised);
    if (bad) p.ctl->err = HANF_ESTATE;
}

__global__ void k_slot_T(Plan p)
{
    const DevCtl *c = p.ctl;
    if (c->done) return;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < p.S;
         s += (int64_t)gridDim.x * blockDim.x)
        if (p.slot_T[s] < 0 && p.slot_changed[s] == 0) p.slot_T[s] = c->t;
}

// End of a pass: stop if nothing changed (T = t), otherwise advance t and
// swap the buffers.  In graph mode it also sets the while-node condition.
__global__ void k_post(Plan p, cudaGraphConditionalHandle h, int use_cond)
{
    DevCtl *c = p.ctl;
    unsigned keep = 0;
    if (!c->done && c->err) {
        c->done = 1;   // a scatter pass broke its bound: stop, the host reports it
    } else if (!c->done) {
        const int nxt = c->parity ^ 1;
        const unsigned long long changed = c->changed_count[nxt];
        c->last_changed = changed;
        c->passes += 1;
        if (c->mode == kModePush || c->mode == kModeScatter) c->push_passes += 1;
        if (p.S <= 8)
            for (int r = 0; r < p.S; ++r)
                if (p.slot_T[r] < 0 && p.slot_changed[r] == 0) p.slot_T[r] = c->t;
        if (changed == 0) {
            c->done = 1;
        } else {
            c->t += 1;
            c->parity = nxt;
            if (c->t >= c->max_t || c->t >= p.history_cap) {
                c->err = HANF_ERANGE;
                c->done = 1;
            } else {
                keep = 1;
            }
        }
    }
    if (use_cond) cudaGraphSetConditional(h, keep);
}

// ---------------------------------------------------------------- estimator

// size() of run r of node v (Algorithm 1 with linear counting).  M
// registers a run, known at compile time so that a lane issues all of its
// loads before it adds.
template <int M>
__device__ __forceinline__ double node_size(const Plan &p, const uint8_t *rc, int64_t v, int r)
{
    const uint4 *q = reinterpret_cast<const uint4 *>(rc + v * p.W + (int64_t)r * M);
    uint4 x[M / 16];
#pragma unroll
    for (int k = 0; k < M / 16; ++k) x[k] = q[k];
    unsigned long long S = 0;
    int V = 0;
#pragma unroll
    for (int k = 0; k < M / 16; ++k) vec_sums(x[k], S, V);
    return size_from_sums(p, S, V, M);
}

// Per-node statistics of the sequence E_v(0..T) (the radius distribution and
// closeness centrality of the paper's conclusion): reach E_v(T), the distance
// sum sum_t t (E_v(t) - E_v(t-1)), the last t at which E_v changed, and in a
// replay the first t with E_v(t) >= alpha E_v(T).  Products and sums are
// rounded one by one (no fused multiply-add), as the oracle computes them.
__device__ __forceinline__ void node_stats_update(const Plan &p, int r, int64_t v, double E,
                                                  bool all, int t)
{
    const int64_t i = (int64_t)r * p.n + v;
    if (all) {
        p.ns_prev[i] = E;
        if (p.ns_radius_mode) {
            p.ns_rad[i] = E >= __dmul_rn(p.ns_alpha, p.ns_reach[i]) ? 0 : -1;
        } else {
            p.ns_dist[i] = 0.0;
            p.ns_ecc[i] = 0;
        }
        return;
    }
    const double d = __dsub_rn(E, p.ns_prev[i]);
    if (d != 0.0) {
        if (!p.ns_radius_mode) {
            p.ns_dist[i] = __dadd_rn(p.ns_dist[i], __dmul_rn((double)t, d));
            p.ns_ecc[i] = t;
        }
        p.ns_prev[i] = E;
    }
    if (p.ns_radius_mode && p.ns_rad[i] < 0 && E >= __dmul_rn(p.ns_alpha, p.ns_reach[i]))
        p.ns_rad[i] = t;
}

// Slot of a (run, 64-node block) item: the run, or in a batch graph * R + run.
__device__ __forceinline__ int item_slot(const Plan &p, int r, int64_t blk)
{
    return p.K > 1 ? __ldg(p.blk_graph + blk) * p.R + r : r;
}

// Per 64-node block and run: the exact sum of size() over the block
// (Section 3.3, harmonic partial sums of small blocks), recomputed at t = 0
// and afterwards only for blocks with a counter changed by the last pass;
// the change of each block sum goes into the running sum of its slot.  A warp
// per (run, block); lane 0 keeps the warp's running change and adds it to
// the slot whenever the slot changes.  Not used with the changed-node
// estimate (k_est_first, k_est_changed).
template <int M>
__global__ void __launch_bounds__(kBlock) k_est_blocks(Plan p)
{
    DevCtl *c = p.ctl;
    if (c->done) return;
    const bool all = c->t == 0;
    const uint8_t *rc = p.regs[c->parity];
    const unsigned long long *Fc = p.F[c->parity];
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long cia = 0;   // in-arcs of changed nodes, flushed once
    const int64_t items = p.nwords * p.R;
    Q128 run_q{0ull, 0ull};       // lane 0: change not yet added to slot run_slot
    int run_slot = -1;
    for (int64_t it = warp; it < items; it += nwarps) {
        const int r = (int)(it / p.nwords);
        const int64_t blk = it - (int64_t)r * p.nwords;
        if (!all && Fc[blk] == 0ull) continue;
        const int64_t v0 = blk * 64 + lane, v1 = v0 + 32;
        if (!all && r == 0 && p.in_off) {
            // in-arcs of the nodes that changed: the share of arcs whose
            // successor changed, which picks the next pass's flavour
            const unsigned long long word = Fc[blk];
            unsigned long long d = 0;
            if ((word >> lane) & 1ull) d += (unsigned long long)(p.in_off[v0 + 1] - p.in_off[v0]);
            if ((word >> (lane + 32)) & 1ull) d += (unsigned long long)(p.in_off[v1 + 1] - p.in_off[v1]);
#pragma unroll
            for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(kFull, d, o);
            cia += d;   // warp-uniform after the butterfly
        }
        int64_t lim = p.n;   // padding nodes of a batch do not count
        if (p.K > 1) {
            const int g = __ldg(p.blk_graph + blk);
            lim = p.g_base[g] + p.g_nodes[g];
        }
        const double e0 = v0 < lim ? node_size<M>(p, rc, v0, r) : 0.0;
        const double e1 = v1 < lim ? node_size<M>(p, rc, v1, r) : 0.0;
        if (p.node_stats) {
            if (v0 < lim) node_stats_update(p, r, v0, e0, all, c->t);
            if (v1 < lim) node_stats_update(p, r, v1, e1, all, c->t);
        }
        Q128 s = q_from(e0);
        q_add(s, q_from(e1));
#pragma unroll
        for (int o = 16; o; o >>= 1) q_add(s, q_shfl_xor(s, o));
        const int slot = item_slot(p, r, blk);
        if (lane == 0) {
            unsigned long long *bq = p.blk_q + 2 * it;
            Q128 d = s;
            if (!all) q_sub(d, Q128{bq[0], bq[1]});
            bq[0] = s.lo;
            bq[1] = s.hi;
            if (slot != run_slot) {
                if (run_slot >= 0) q_atomic_add(p.est_acc + 2 * run_slot, run_q);
                run_q = Q128{0ull, 0ull};
                run_slot = slot;
            }
            q_add(run_q, d);
        }
    }
    if (lane == 0) {
        if (run_slot >= 0) q_atomic_add(p.est_acc + 2 * run_slot, run_q);
        if (cia) atomicAdd(&p.ctl->changed_in_arcs, cia);
    }
}

// Changed-node estimate (one graph, byte registers, no per-node
// statistics): after a pass, only the counters it changed (bitmap F_{t+1})
// can change size(), so only they are evaluated, and N changes by their
// size(new) - size(old), size(old) being kept per node and run in a cache.
// The changed nodes of a warp's bitmap words are packed into a queue in
// shared memory and taken 32 at a time, a node per lane, so the
// double-precision work runs on full warps.  Also sums the in-arcs of the
// changed nodes (the share of arcs whose successor changed picks the next
// pass's flavour).
constexpr int kQueue = 96;   // < 32 left over + 64 from one bitmap word

// Changed-node estimate at t = 0: every counter holds its own node only, one
// register at rho+ >= 1 and m - 1 empty, so its raw estimate
// alpha_m m^2 / (m - 1 + 2^-rho+) is below 5m/2 and size() is linear
// counting's m ln(m / (m - 1)) for every node: the cache gets that value and
// N(0) = n m ln(m / (m - 1)), exactly in Q52 (a value below 2 has at most 53
// bits there, and n < 2^31).
__global__ void __launch_bounds__(kBlock) k_est_first(Plan p)
{
    const DevCtl *c = p.ctl;
    if (c->done || !p.est_fused || c->t != 0) return;
    const double E0 = p.lc[p.m - 1];
    const int64_t cells = p.n * p.R;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cells;
         i += (int64_t)gridDim.x * blockDim.x)
        p.ecache[i] = E0;
    if (blockIdx.x == 0 && threadIdx.x < p.R) {
        const Q128 q = q_from(E0);
        const unsigned long long n = (unsigned long long)p.n;
        p.est_acc[2 * threadIdx.x] = q.lo * n;
        p.est_acc[2 * threadIdx.x + 1] = __umul64hi(q.lo, n);
    }
}

template <int M>
__global__ void __launch_bounds__(kBlock) k_est_changed(Plan p)
{
    DevCtl *c = p.ctl;
    if (c->done || !p.est_fused || c->t == 0) return;
    __shared__ int32_t queue[kBlock / 32][kQueue];
    __shared__ unsigned long long wsum[kBlock / 32][kMaxRuns][2];
    const uint8_t *rc = p.regs[c->parity];
    const unsigned long long *Fc = p.F[c->parity];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int32_t *q = queue[wib];
    if (lane < 2 * kMaxRuns) (&wsum[wib][0][0])[lane] = 0ull;
    __syncwarp();
    unsigned long long cia = 0;
    int cnt = 0;   // queued nodes (warp-uniform)
    // nodes q[cnt - k .. cnt), one per lane k > lane
    auto drain = [&](int k) {
        const bool on = lane < k;
        const int32_t v = on ? q[cnt - k + lane] : 0;
        __syncwarp();
        if (on && p.in_off) cia += (unsigned long long)(p.in_off[v + 1] - p.in_off[v]);
        for (int r = 0; r < p.R; ++r) {
            Q128 d{0ull, 0ull};
            if (on) {
                const double E = node_size<M>(p, rc, v, r);
                double *ce = p.ecache + (int64_t)r * p.n + v;
                const double old = *ce;
                if (__double_as_longlong(E) != __double_as_longlong(old)) {
                    d = q_from(E);
                    q_sub(d, q_from(old));
                    *ce = E;
                }
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) q_add(d, q_shfl_xor(d, o));
            if (lane == 0) {
                Q128 t{wsum[wib][r][0], wsum[wib][r][1]};
                q_add(t, d);
                wsum[wib][r][0] = t.lo;
                wsum[wib][r][1] = t.hi;
            }
        }
        cnt -= k;
    };
    // 32 bitmap words per warp iteration (lane l: word i0 + l * nwarps), the
    // non-zero ones in order
    for (int64_t w0 = warp; w0 < p.nwords; w0 += nwarps * 32) {
        const int64_t ww = w0 + (int64_t)lane * nwarps;
        const unsigned long long mine = ww < p.nwords ? Fc[ww] : 0ull;
        for (unsigned nz = __ballot_sync(kFull, mine != 0ull); nz; nz &= nz - 1u) {
            const int src_lane = __ffs(nz) - 1;
            const int64_t w = w0 + (int64_t)src_lane * nwarps;
            const unsigned long long bits = __shfl_sync(kFull, mine, src_lane);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const bool b = (bits >> (32 * h + lane)) & 1ull;
                const unsigned bal = __ballot_sync(kFull, b);
                if (b) q[cnt + __popc(bal & ((1u << lane) - 1u))] = (int32_t)(w * 64 + 32 * h + lane);
                cnt += __popc(bal);
            }
            __syncwarp();
            while (cnt >= 32) drain(32);
        }
    }
    if (cnt > 0) drain(cnt);
    __syncwarp();
    if (lane < p.R) q_atomic_add(p.est_acc + 2 * lane, Q128{wsum[wib][lane][0], wsum[wib][lane][1]});
#pragma unroll
    for (int o = 16; o; o >>= 1) cia += __shfl_xor_sync(kFull, cia, o);
    if (lane == 0 && cia) atomicAdd(&c->changed_in_arcs, cia);
}

// N_s(t) of every slot into the history: its running sum rounded to double.
__global__ void k_est_finalize(Plan p)
{
    const DevCtl *c = p.ctl;
    if (c->done) return;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < p.S;
         s += (int64_t)gridDim.x * blockDim.x)
        p.hist[(int64_t)c->t * p.S + s] =
            q_to_double(Q128{p.est_acc[2 * s], p.est_acc[2 * s + 1]});
}

// ---------------------------------------------------------------- init

// Algorithm 2's initialisation: every counter empty, then node v adds itself
// (Algorithm 1's add): register h_b(v) <- min(rho+(h^b(v)), 31) with
// h = splitmix64(v XOR seed_r).  One thread per 16-byte chunk of the counter
// array.  regs[0] gets c_0; regs[1] (the target of pass 0) only the rows of
// nodes without arcs, which no pass visits: pass 0 stores the row of every
// node it visits.
__global__ void __launch_bounds__(kBlock) k_init(Plan p)
{
    const int64_t cpr = p.W >> 4;
    const int64_t total = p.n * cpr;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // chunk c = v * cpr + j, advanced by the grid stride without a division
    // per chunk
    const int64_t c0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t dv = stride / cpr, dj = stride - dv * cpr;
    int64_t v = c0 / cpr, j = c0 - v * cpr;
    for (int64_t c = c0; c < total; c += stride) {
        const int byte0 = (int)j << 4;
        const int r = byte0 >> p.b;
        const int o = byte0 & (p.m - 1);
        uint64_t item = p.orig_id ? (uint64_t)__ldg(p.orig_id + v) : (uint64_t)v;
        int slot = r;
        if (p.K > 1) {   // a batch: the node's id within its graph, the graph's seeds
            const int g = __ldg(p.blk_graph + (v >> 6));
            item = (uint64_t)(v - p.g_base[g]);
            slot = g * p.R + r;
        }
        const uint64_t h = splitmix64(item ^ p.seeds[slot]);
        const int idx = (int)(h >> (64 - p.b));
        const uint64_t rest = h << p.b;
        int rho = rest ? __clzll((long long)rest) + 1 : 64 - p.b + 1;
        rho = rho > 31 ? 31 : rho;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        const int rel = idx - o;
        if (rel >= 0 && rel < 16) {
            w[rel >> 2] = (uint32_t)rho << ((rel & 3) * 8);
            // the chunk holding the register also records it for pass 0
            if (p.hr) p.hr[v * p.R + r] = (uint16_t)((idx << 8) | rho);
        }
        const uint4 val = make_uint4(w[0], w[1], w[2], w[3]);
        reinterpret_cast<uint4 *>(p.regs[0])[c] = val;
        if (__ldg(p.off + v + 1) == __ldg(p.off + v)) reinterpret_cast<uint4 *>(p.regs[1])[c] = val;
        v += dv;
        j += dj;
        if (j >= cpr) {
            j -= cpr;
            ++v;
        }
    }
}

// CSR validation: offsets start at 0, end at arcs and never decrease; every
// target lies in [0, n).
__global__ void k_validate(Plan p)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool bad = false;
    for (int64_t i = i0; i <= p.n; i += stride) {
        const int64_t o = p.off[i];
        if (i == 0 && o != 0) bad = true;
        if (i == p.n && o != p.arcs) bad = true;
        if (i < p.n && p.off[i + 1] < o) bad = true;
    }
    for (int64_t e = i0; e < p.arcs; e += stride) {
        const int32_t w = p.tgt[e];
        if (w < 0 || (int64_t)w >= p.n) bad = true;
    }
    if (p.K > 1 && !bad) {
        // a batch: arcs stay inside their graph, padding nodes have none
        for (int64_t v = i0; v < p.n; v += stride) {
            const int g = p.blk_graph[v >> 6];
            const int64_t lo = p.g_base[g], hi = lo + p.g_nodes[g];
            const int64_t b = p.off[v], e = p.off[v + 1];
            if (v >= hi && e > b) bad = true;
            for (int64_t k = b; k < e && !bad; ++k) {
                const int32_t w = p.tgt[k];
                if (w < lo || w >= hi) bad = true;
            }
        }
    }
    if (bad) p.ctl->bad_graph = 1;
}

// ---------------------------------------------------------------- scans

constexpr int kScanItems = 16;
constexpr int kScanTile = kBlock * kScanItems;

// Exclusive scan of one value per thread across the block; *total gets the sum.
__device__ __forceinline__ int64_t block_excl_scan(int64_t x, int64_t *total)
{
    __shared__ int64_t warp_tot[kBlock / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t inc = x;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, inc, s);
        if (lane >= s) inc += y;
    }
    __syncthreads();
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    int64_t off = 0, tot = 0;
    for (int w = 0; w < kBlock / 32; ++w) {
        if (w < wid) off += warp_tot[w];
        tot += warp_tot[w];
    }
    if (total) *total = tot;
    return off + inc - x;
}

__global__ void __launch_bounds__(kBlock) k_scan_tile_sums(const int64_t *in, int64_t count,
                                                           int64_t *sums)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < count) s += in[base + k];
    int64_t tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kBlock) k_scan_tile_apply(const int64_t *in, int64_t *out,
                                                            int64_t count,
                                                            const int64_t *tile_offs)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < count ? in[base + k] : 0;
        s += v[k];
    }
    int64_t run = block_excl_scan(s, nullptr) + (tile_offs ? tile_offs[blockIdx.x] : 0);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < count) out[base + k] = run;
        run += v[k];
    }
}

// ---------------------------------------------------------------- preprocessing

constexpr int kClassPerThread = 4;
constexpr int kClassTile = kBlock * kClassPerThread;

__device__ __forceinline__ int node_class(int64_t deg, int32_t d_small, int32_t d_hub)
{
    return deg == 0 ? -1 : (deg <= d_small ? 0 : (deg <= d_hub ? 1 : 2));
}

// Per tile of nodes, how many fall in each class (small, medium, hub);
// counts[c * ntiles + tile].
__global__ void __launch_bounds__(kBlock) k_class_count(Plan p, int32_t d_small, int32_t d_hub,
                                                        int64_t *counts, int64_t ntiles)
{
    int64_t c3[3] = {0, 0, 0};
    const int64_t v0 = (int64_t)blockIdx.x * kClassTile + (int64_t)threadIdx.x * kClassPerThread;
    for (int k = 0; k < kClassPerThread; ++k) {
        const int64_t v = v0 + k;
        if (v < p.n) {
            const int c = node_class(p.off[v + 1] - p.off[v], d_small, d_hub);
            if (c >= 0) c3[c] += 1;
        }
    }
    for (int c = 0; c < 3; ++c) {
        int64_t tot;
        block_excl_scan(c3[c], &tot);
        if (threadIdx.x == 0) counts[c * ntiles + blockIdx.x] = tot;
    }
}

// Scatter node ids into [small | medium | hub] in node order.
__global__ void __launch_bounds__(kBlock) k_class_scatter(Plan p, int32_t d_small, int32_t d_hub,
                                                          const int64_t *offs, int64_t ntiles,
                                                          int32_t *nodes)
{
    int cls[kClassPerThread];
    int64_t c3[3] = {0, 0, 0};
    const int64_t v0 = (int64_t)blockIdx.x * kClassTile + (int64_t)threadIdx.x * kClassPerThread;
    for (int k = 0; k < kClassPerThread; ++k) {
        const int64_t v = v0 + k;
        cls[k] = v < p.n ? node_class(p.off[v + 1] - p.off[v], d_small, d_hub) : -1;
        if (cls[k] >= 0) c3[cls[k]] += 1;
    }
    int64_t pos[3];
    for (int c = 0; c < 3; ++c) pos[c] = block_excl_scan(c3[c], nullptr) + offs[c * ntiles + blockIdx.x];
    for (int k = 0; k < kClassPerThread; ++k)
        if (cls[k] >= 0) nodes[pos[cls[k]]++] = (int32_t)(v0 + k);
}

__global__ void k_hub_seg_count(Plan p, int32_t d_hub, const int32_t *hubs, int64_t n_hub,
                                int64_t *seg_counts)
{
    for (int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; h <= n_hub;
         h += (int64_t)gridDim.x * blockDim.x) {
        if (h == n_hub) {
            seg_counts[h] = 0;
        } else {
            const int32_t v = hubs[h];
            const int64_t deg = p.off[v + 1] - p.off[v];
            seg_counts[h] = (deg + d_hub - 1) / d_hub;
        }
    }
}

__global__ void k_hub_seg_fill(Plan p, int32_t d_hub, const int32_t *hubs, int64_t n_hub,
                               const int64_t *seg_offs, int32_t *seg_node, int64_t *seg_beg,
                               int64_t *seg_end, int32_t *hub_seg_first)
{
    for (int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; h <= n_hub;
         h += (int64_t)gridDim.x * blockDim.x) {
        hub_seg_first[h] = (int32_t)seg_offs[h];
        if (h == n_hub) continue;
        const int32_t v = hubs[h];
        const int64_t b = p.off[v], e = p.off[v + 1];
        int64_t s = seg_offs[h];
        for (int64_t a = b; a < e; a += d_hub, ++s) {
            seg_node[s] = v;
            seg_beg[s] = a;
            seg_end[s] = a + d_hub < e ? a + d_hub : e;
        }
    }
}

__global__ void k_in_degree(Plan p, unsigned long long *cnt)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < p.arcs;
         e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[p.tgt[e]], 1ull);
}

__global__ void k_permute_indeg(const unsigned long long *indeg_in, const int32_t *inv, int64_t n,
                                int64_t *counts)
{
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u <= n;
         u += (int64_t)gridDim.x * blockDim.x)
        counts[u] = u == n ? 0 : (int64_t)indeg_in[inv[u]];
}

__global__ void k_transpose_fill(Plan p, const int64_t *in_off, unsigned long long *cursor,
                                 int32_t *in_src)
{
    constexpr int UF = 4;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < p.n; v += nwarps) {
        const int64_t beg = p.off[v], end = p.off[v + 1];
        for (int64_t e0 = beg + lane; e0 < end; e0 += 32 * UF) {
            int32_t w[UF];
            unsigned long long k[UF];
#pragma unroll
            for (int u = 0; u < UF; ++u) w[u] = e0 + 32 * u < end ? __ldg(p.tgt + e0 + 32 * u) : -1;
#pragma unroll
            for (int u = 0; u < UF; ++u) k[u] = w[u] >= 0 ? atomicAdd(&cursor[w[u]], 1ull) : 0ull;
#pragma unroll
            for (int u = 0; u < UF; ++u)
                if (w[u] >= 0) in_src[in_off[w[u]] + (int64_t)k[u]] = (int32_t)v;
        }
    }
}

// ---------------------------------------------------------------- relabelling

// Popularity class of a node: 0 for the largest in-degrees, 31 for none.
// Nodes are stored hottest class first, so the counters most often gathered
// share cache lines and DRAM pages.
constexpr int kHotClasses = 32;

__device__ __forceinline__ int hot_class(unsigned long long indeg)
{
    return 31 - (63 - __clzll((long long)(indeg + 1)));
}

// counts[c * ntiles + tile] = nodes of class c in the tile.
__global__ void __launch_bounds__(kBlock) k_hot_count(const unsigned long long *indeg, int64_t n,
                                                      int64_t *counts, int64_t ntiles)
{
    __shared__ int hist[kHotClasses];
    if (threadIdx.x < kHotClasses) hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t v0 = (int64_t)blockIdx.x * kClassTile + (int64_t)threadIdx.x * kClassPerThread;
    for (int k = 0; k < kClassPerThread; ++k)
        if (v0 + k < n) atomicAdd(&hist[hot_class(indeg[v0 + k])], 1);
    __syncthreads();
    if (threadIdx.x < kHotClasses) counts[threadIdx.x * ntiles + blockIdx.x] = hist[threadIdx.x];
}

// Stable scatter: new position of every node (class order, then id order).
__global__ void __launch_bounds__(kBlock) k_hot_scatter(const unsigned long long *indeg, int64_t n,
                                                        const int64_t *offs, int64_t ntiles,
                                                        int32_t *perm, int32_t *inv)
{
    const int64_t v0 = (int64_t)blockIdx.x * kClassTile + (int64_t)threadIdx.x * kClassPerThread;
    int cls[kClassPerThread];
    for (int k = 0; k < kClassPerThread; ++k) cls[k] = v0 + k < n ? hot_class(indeg[v0 + k]) : -1;
    for (int c = 0; c < kHotClasses; ++c) {
        int mine = 0;
        for (int k = 0; k < kClassPerThread; ++k) mine += cls[k] == c;
        int64_t pos = block_excl_scan(mine, nullptr) + offs[c * ntiles + blockIdx.x];
        for (int k = 0; k < kClassPerThread; ++k)
            if (cls[k] == c) {
                perm[v0 + k] = (int32_t)pos;
                inv[pos] = (int32_t)(v0 + k);
                ++pos;
            }
    }
}

// Out-degree of every new node (input of the new offsets' scan).
__global__ void k_new_degree(const int64_t *off, const int32_t *inv, int64_t n, int64_t *deg)
{
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u <= n;
         u += (int64_t)gridDim.x * blockDim.x) {
        if (u == n) {
            deg[u] = 0;
        } else {
            const int32_t v = inv[u];
            deg[u] = off[v + 1] - off[v];
        }
    }
}

// Successor lists in the new numbering: a warp per new node.
__global__ void k_relabel_fill(const int64_t *off, const int32_t *tgt, const int32_t *perm,
                               const int32_t *inv, int64_t n, const int64_t *off2, int32_t *tgt2)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < n; u += nwarps) {
        const int32_t v = inv[u];
        const int64_t b = off[v], d = off[v + 1] - b, o = off2[u];
        for (int64_t j = lane; j < d; j += 32) tgt2[o + j] = perm[__ldg(tgt + b + j)];
    }
}

// Rows of nodes (original ids first..first+count) gathered into a staging
// buffer in original order.
__global__ void k_gather_rows(const uint8_t *regs, const int32_t *perm, int64_t first, int64_t count,
                              int W, uint8_t *out)
{
    const int64_t cpr = W >> 4;
    const int64_t total = count * cpr;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < total;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = c / cpr, j = c - i * cpr;
        const int64_t row = perm ? perm[first + i] : first + i;
        reinterpret_cast<uint4 *>(out)[c] = reinterpret_cast<const uint4 *>(regs)[row * cpr + j];
    }
}

// Per-node values of input ids first..first+count (through the relabelling).
template <typename V>
__global__ void k_gather_vals(const V *src, const int32_t *perm, int64_t first, int64_t count,
                              V *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = src[perm ? perm[first + i] : first + i];
}

int grid_for(int64_t work, int per_block, int64_t cap = 152 * 32)
{
    int64_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// ---------------------------------------------------------------- 5-bit bit-sliced layout

// A packed counter of m = 32P registers is five bit-planes of m bits (plane p
// holds bit p of every register; register j is bit j%32 of word j/32):
// 20P bytes instead of m.  The union compares two counters lexicographically
// plane by plane from the top plane down, for 32 registers per word at once
// (the parallel compare of Section 3.3 in bit-sliced form), and keeps the
// larger register of every pair.
template <int P>
struct PRow {
    uint32_t w[5][P];
};

template <int P>
__device__ __forceinline__ void prow_zero(PRow<P> &r)
{
#pragma unroll
    for (int p = 0; p < 5; ++p)
#pragma unroll
        for (int k = 0; k < P; ++k) r.w[p][k] = 0u;
}

template <int P>
__device__ __forceinline__ void prow_load(PRow<P> &r, const uint8_t *base, int64_t row)
{
    const uint8_t *q = base + row * (20 * P);
    if constexpr (P == 1) {
        const uint32_t *s = reinterpret_cast<const uint32_t *>(q);
#pragma unroll
        for (int p = 0; p < 5; ++p) r.w[p][0] = __ldg(s + p);
    } else if constexpr (P == 2) {
        const uint2 *s = reinterpret_cast<const uint2 *>(q);
#pragma unroll
        for (int p = 0; p < 5; ++p) {
            const uint2 x = __ldg(s + p);
            r.w[p][0] = x.x;
            r.w[p][1] = x.y;
        }
    } else {
        const uint4 *s = reinterpret_cast<const uint4 *>(q);
#pragma unroll
        for (int p = 0; p < 5; ++p)
#pragma unroll
            for (int k = 0; k < P / 4; ++k) {
                const uint4 x = __ldg(s + p * (P / 4) + k);
                r.w[p][4 * k] = x.x;
                r.w[p][4 * k + 1] = x.y;
                r.w[p][4 * k + 2] = x.z;
                r.w[p][4 * k + 3] = x.w;
            }
    }
}

template <int P>
__device__ __forceinline__ void prow_store(uint8_t *base, int64_t row, const PRow<P> &r)
{
    uint8_t *q = base + row * (20 * P);
    if constexpr (P == 1) {
        uint32_t *s = reinterpret_cast<uint32_t *>(q);
#pragma unroll
        for (int p = 0; p < 5; ++p) s[p] = r.w[p][0];
    } else if constexpr (P == 2) {
        uint2 *s = reinterpret_cast<uint2 *>(q);
#pragma unroll
        for (int p = 0; p < 5; ++p) s[p] = make_uint2(r.w[p][0], r.w[p][1]);
    } else {
        uint4 *s = reinterpret_cast<uint4 *>(q);
#pragma unroll
        for (int p = 0; p < 5; ++p)
#pragma unroll
            for (int k = 0; k < P / 4; ++k)
                s[p * (P / 4) + k] = make_uint4(r.w[p][4 * k], r.w[p][4 * k + 1], r.w[p][4 * k + 2],
                                                r.w[p][4 * k + 3]);
    }
}

// a <- register-wise max(a, b): lt marks registers where a < b, found at the
// highest plane where they differ; there b's bits are taken.
template <int P>
__device__ __forceinline__ void prow_max(PRow<P> &a, const PRow<P> &b)
{
#pragma unroll
    for (int k = 0; k < P; ++k) {
        uint32_t lt = 0u, eq = 0xffffffffu;
#pragma unroll
        for (int p = 4; p >= 0; --p) {
            const uint32_t x = a.w[p][k], y = b.w[p][k];
            lt |= eq & ~x & y;
            eq &= ~(x ^ y);
        }
#pragma unroll
        for (int p = 0; p < 5; ++p) a.w[p][k] = (a.w[p][k] & ~lt) | (b.w[p][k] & lt);
    }
}

template <int P>
__device__ __forceinline__ bool prow_eq(const PRow<P> &a, const PRow<P> &b)
{
    uint32_t d = 0u;
#pragma unroll
    for (int p = 0; p < 5; ++p)
#pragma unroll
        for (int k = 0; k < P; ++k) d |= a.w[p][k] ^ b.w[p][k];
    return d == 0u;
}

template <int P>
__device__ __forceinline__ void prow_warp_max(PRow<P> &r)
{
#pragma unroll
    for (int s = 16; s; s >>= 1) {
        PRow<P> o;
#pragma unroll
        for (int p = 0; p < 5; ++p)
#pragma unroll
            for (int k = 0; k < P; ++k) o.w[p][k] = __shfl_xor_sync(kFull, r.w[p][k], s);
        prow_max(r, o);
    }
}

// New packed counter of v; the single-run analogue of node_finish (lane-level).
template <int P>
__device__ __forceinline__ uint32_t pnode_finish(const Plan &p, int cur, const PRow<P> &acc,
                                                 bool need, bool inR, int32_t v, uint32_t &c_own,
                                                 uint32_t &c_write, const PRow<P> *pre = nullptr)
{
    if (!need) return 0u;
    PRow<P> own;
    if (pre) own = *pre;
    else prow_load(own, p.regs[cur], v);
    PRow<P> nw = own;
    prow_max(nw, acc);
    const bool changed = !prow_eq(nw, own);
    if (changed || inR) {
        prow_store(p.regs[cur ^ 1], v, nw);
        ++c_write;
    }
    ++c_own;
    return changed ? 1u : 0u;
}

// Small nodes: a lane per node, U arcs in flight per lane.
template <int P>
__global__ void __launch_bounds__(kBlock, P >= 8 ? 1 : min_blocks(P / 2)) k_punion_small(Plan p)
{
    constexpr int U = P == 1 ? 4 : (P == 2 ? 2 : 1);
    const DevCtl *ctl = p.ctl;
    if (ctl->done) return;
    const int cur = ctl->parity;
    const bool first = ctl->t == 0;
    const bool test = ctl->mode != kModeDense;
    const bool push = ctl->mode == kModePush;
    const bool own_early = !test || push;
    const uint8_t *rc = p.regs[cur];
    const unsigned long long *Fc = p.F[cur];
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t *list = push ? p.cand_list[0] : p.nodes;
    const int64_t count = push ? (int64_t)ctl->cand_count[0] : p.n_small;
    uint32_t c_scan = 0, c_gather = 0, c_own = 0, c_write = 0;
    MarkTally mt;
    for (int64_t base = warp * 32; base < count; base += nwarps * 32) {
        const int64_t idx = base + lane;
        const bool valid = idx < count;
        const int32_t v = valid ? __ldg(list + idx) : 0;
        PRow<P> own, acc;
        if (valid && own_early) prow_load(own, rc, v);
        prow_zero(acc);
        bool any = false;
        if (valid) {
            const int64_t beg = __ldg(p.off + v), end = __ldg(p.off + v + 1);
            c_scan += (uint32_t)(end - beg);
            for (int64_t e = beg; e < end; e += U) {
                int32_t w[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    w[u] = e + u < end ? __ldg(p.tgt + e + u) : -1;
                    if (w[u] >= 0 && test && !test_bit(Fc, w[u])) w[u] = -1;
                }
                PRow<P> x[U];
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (w[u] >= 0) prow_load(x[u], rc, w[u]);
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (w[u] >= 0) {
                        prow_max(acc, x[u]);
                        any = true;
                        ++c_gather;
                    }
            }
        }
        const bool inR = valid && !first && test_bit(Fc, v);
        const uint32_t mask = pnode_finish(p, cur, acc, valid && (any || inR), inR, v, c_own,
                                           c_write, own_early ? &own : nullptr);
        warp_mark(p, cur, valid, v, mask, mt);
    }
    flush_counters(p, cur, mt, c_scan, c_gather, c_own, c_write);
}

// Medium nodes and hub segments: a warp per item, lane i merges arcs
// e+i, e+i+32, ... (U per lane in flight), then a warp-wide max.
template <int P>
__global__ void __launch_bounds__(kBlock, P >= 8 ? 1 : min_blocks(P / 2)) k_punion_warp(Plan p)
{
    constexpr int U = P == 1 ? 4 : (P == 2 ? 2 : 1);
    const DevCtl *ctl = p.ctl;
    if (ctl->done) return;
    const int cur = ctl->parity;
    const bool first = ctl->t == 0;
    const bool test = ctl->mode != kModeDense;
    const bool push = ctl->mode == kModePush;
    const uint8_t *rc = p.regs[cur];
    const unsigned long long *Fc = p.F[cur];
    const int32_t *med = push ? p.cand_list[1] : p.nodes + p.n_small;
    const int64_t total = p.n_seg + (push ? (int64_t)ctl->cand_count[1] : p.n_med);
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t c_scan = 0, c_gather = 0, c_own = 0, c_write = 0;
    MarkTally mt;
    for (int64_t it = warp; it < total; it += nwarps) {
        const bool seg = it < p.n_seg;
        const int32_t v = seg ? __ldg(p.seg_node + it) : __ldg(med + (it - p.n_seg));
        const bool take = !seg || !push || test_bit(p.cand, v);
        PRow<P> acc;
        prow_zero(acc);
        bool any = false;
        if (take) {
            const int64_t beg = seg ? __ldg(p.seg_beg + it) : __ldg(p.off + v);
            const int64_t end = seg ? __ldg(p.seg_end + it) : __ldg(p.off + v + 1);
            if (lane == 0) c_scan += (uint32_t)(end - beg);
            for (int64_t e = beg + lane; e < end; e += 32 * U) {
                int32_t w[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    w[u] = e + 32 * u < end ? __ldg(p.tgt + e + 32 * u) : -1;
                    if (w[u] >= 0 && test && !test_bit(Fc, w[u])) w[u] = -1;
                }
                PRow<P> x[U];
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (w[u] >= 0) prow_load(x[u], rc, w[u]);
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (w[u] >= 0) {
                        prow_max(acc, x[u]);
                        any = true;
                        ++c_gather;
                    }
            }
        }
        prow_warp_max(acc);
        any = __any_sync(kFull, any);
        if (seg) {
            if (lane == 0) {
                prow_store(p.hub_part, it, acc);
                p.hub_any[it] = any ? 1 : 0;
            }
        } else {
            const bool inR = take && !first && test_bit(Fc, v);
            const bool need = take && (any || inR) && lane == 0;
            const uint32_t mask = pnode_finish(p, cur, acc, need, inR, v, c_own, c_write);
            warp_mark(p, cur, lane == 0, v, mask, mt);
        }
    }
    flush_counters(p, cur, mt, c_scan, c_gather, c_own, c_write);
}

// Hub nodes: combine the segment partials, a lane per hub.
template <int P>
__global__ void __launch_bounds__(kBlock) k_phub_finish(Plan p)
{
    const DevCtl *ctl = p.ctl;
    if (ctl->done || p.n_hub == 0) return;
    const int cur = ctl->parity;
    const bool first = ctl->t == 0;
    const bool push = ctl->mode == kModePush;
    const unsigned long long *Fc = p.F[cur];
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    uint32_t c_own = 0, c_write = 0;
    MarkTally mt;
    for (int64_t base = tid - (threadIdx.x & 31); base < p.n_hub; base += nthreads) {
        const int64_t h = base + (threadIdx.x & 31);
        const bool valid = h < p.n_hub;
        const int32_t v = valid ? p.nodes[p.n_small + p.n_med + h] : 0;
        const bool take = valid && (!push || test_bit(p.cand, v));
        PRow<P> acc;
        prow_zero(acc);
        bool any = false;
        if (take) {
            for (int32_t s = p.hub_seg_first[h]; s < p.hub_seg_first[h + 1]; ++s) {
                if (p.hub_any[s]) {
                    PRow<P> x;
                    prow_load(x, p.hub_part, s);
                    prow_max(acc, x);
                    any = true;
                }
            }
        }
        const bool inR = take && !first && test_bit(Fc, v);
        const uint32_t mask = pnode_finish(p, cur, acc, take && (any || inR), inR, v, c_own, c_write);
        warp_mark(p, cur, valid, v, mask, mt);
    }
    flush_counters(p, cur, mt, 0u, 0u, c_own, c_write);
}

// size() of a packed counter: V = empty registers; sum_j 2^(31-M[j]) taken
// value by value from the planes.
template <int P>
__device__ __forceinline__ double pnode_size(const Plan &p, const uint8_t *rc, int64_t v)
{
    PRow<P> r;
    prow_load(r, rc, v);
    unsigned long long S = 0;
    int V = 0;
#pragma unroll
    for (int k = 0; k < P; ++k) {
        V += __popc(~(r.w[0][k] | r.w[1][k] | r.w[2][k] | r.w[3][k] | r.w[4][k]));
        for (int M = 0; M < 32; ++M) {
            uint32_t sel = 0xffffffffu;
#pragma unroll
            for (int b = 0; b < 5; ++b) sel &= ((M >> b) & 1) ? r.w[b][k] : ~r.w[b][k];
            S += (unsigned long long)__popc(sel) << (31 - M);
        }
    }
    return size_from_sums(p, S, V, p.m);
}

template <int P>
__global__ void __launch_bounds__(kBlock) k_pest_blocks(Plan p)
{
    DevCtl *c = p.ctl;
    if (c->done) return;
    const bool all = c->t == 0;
    const uint8_t *rc = p.regs[c->parity];
    const unsigned long long *Fc = p.F[c->parity];
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long cia = 0;   // in-arcs of changed nodes, flushed once
    Q128 run_q{0ull, 0ull};       // lane 0: change not yet added to slot run_slot
    int run_slot = -1;
    for (int64_t blk = warp; blk < p.nwords; blk += nwarps) {
        if (!all && Fc[blk] == 0ull) continue;
        const int64_t v0 = blk * 64 + lane, v1 = v0 + 32;
        if (!all && p.in_off) {
            const unsigned long long word = Fc[blk];
            unsigned long long d = 0;
            if ((word >> lane) & 1ull) d += (unsigned long long)(p.in_off[v0 + 1] - p.in_off[v0]);
            if ((word >> (lane + 32)) & 1ull) d += (unsigned long long)(p.in_off[v1 + 1] - p.in_off[v1]);
#pragma unroll
            for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(kFull, d, o);
            cia += d;   // warp-uniform after the butterfly
        }
        int64_t lim = p.n;
        if (p.K > 1) {
            const int g = __ldg(p.blk_graph + blk);
            lim = p.g_base[g] + p.g_nodes[g];
        }
        const double e0 = v0 < lim ? pnode_size<P>(p, rc, v0) : 0.0;
        const double e1 = v1 < lim ? pnode_size<P>(p, rc, v1) : 0.0;
        if (p.node_stats) {
            if (v0 < lim) node_stats_update(p, 0, v0, e0, all, c->t);
            if (v1 < lim) node_stats_update(p, 0, v1, e1, all, c->t);
        }
        Q128 s = q_from(e0);
        q_add(s, q_from(e1));
#pragma unroll
        for (int o = 16; o; o >>= 1) q_add(s, q_shfl_xor(s, o));
        const int slot = item_slot(p, 0, blk);
        if (lane == 0) {
            unsigned long long *bq = p.blk_q + 2 * blk;
            Q128 d = s;
            if (!all) q_sub(d, Q128{bq[0], bq[1]});
            bq[0] = s.lo;
            bq[1] = s.hi;
            if (slot != run_slot) {
                if (run_slot >= 0) q_atomic_add(p.est_acc + 2 * run_slot, run_q);
                run_q = Q128{0ull, 0ull};
                run_slot = slot;
            }
            q_add(run_q, d);
        }
    }
    if (lane == 0) {
        if (run_slot >= 0) q_atomic_add(p.est_acc + 2 * run_slot, run_q);
        if (cia) atomicAdd(&p.ctl->changed_in_arcs, cia);
    }
}

// Algorithm 2's initialisation in the packed layout: node v adds itself.
template <int P>
__global__ void __launch_bounds__(kBlock) k_pinit(Plan p)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < p.n;
         v += (int64_t)gridDim.x * blockDim.x) {
        uint64_t item = p.orig_id ? (uint64_t)__ldg(p.orig_id + v) : (uint64_t)v;
        int slot = 0;
        if (p.K > 1) {
            const int g = __ldg(p.blk_graph + (v >> 6));
            item = (uint64_t)(v - p.g_base[g]);
            slot = g;
        }
        const uint64_t h = splitmix64(item ^ p.seeds[slot]);
        const int idx = (int)(h >> (64 - p.b));
        const uint64_t rest = h << p.b;
        int rho = rest ? __clzll((long long)rest) + 1 : 64 - p.b + 1;
        rho = rho > 31 ? 31 : rho;
        PRow<P> r;
        prow_zero(r);
#pragma unroll
        for (int b = 0; b < 5; ++b)
#pragma unroll
            for (int k = 0; k < P; ++k)
                if (k == (idx >> 5) && ((rho >> b) & 1)) r.w[b][k] = 1u << (idx & 31);
        prow_store(p.regs[0], v, r);
        prow_store(p.regs[1], v, r);
    }
}

// Registers of stored rows perm[first..first+count) (or first.. without a
// permutation) unpacked to one byte each.
template <int P>
__global__ void k_punpack(const uint8_t *regs, const int32_t *perm, int64_t first, int64_t count,
                          uint8_t *out)
{
    constexpr int m = 32 * P;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count * m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t node = i / m;
        const int j = (int)(i - node * m);
        const int64_t row = perm ? perm[first + node] : first + node;
        const uint32_t *q = reinterpret_cast<const uint32_t *>(regs + row * (20 * P));
        uint32_t val = 0;
#pragma unroll
        for (int b = 0; b < 5; ++b) val |= ((q[b * P + (j >> 5)] >> (j & 31)) & 1u) << b;
        out[i] = (uint8_t)val;
    }
}

// Register digest (hanf_digest): for input ids first+i, i < count, FNV-1a-64
// (offset basis 14695981039346656037, prime 2^40 + 2^8 + 0xb3) of the eight
// little-endian bytes of i followed by the m registers of run r, one byte
// each; the values are summed modulo 2^64, which makes the result
// independent of the order the threads add them in.  A thread per node.
__global__ void __launch_bounds__(kBlock) k_digest(Plan p, int32_t r, int64_t first,
                                                   int64_t count, const int32_t *perm,
                                                   unsigned long long *out)
{
    constexpr unsigned long long kBasis = 14695981039346656037ull;
    constexpr unsigned long long kPrime = 1099511628211ull;
    const uint8_t *regs = p.regs[p.ctl->parity];
    unsigned long long acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = perm ? (int64_t)__ldg(perm + first + i) : first + i;
        unsigned long long h = kBasis;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            h ^= ((unsigned long long)i >> (8 * k)) & 0xffull;
            h *= kPrime;
        }
        if (p.layout == 0) {
            const uint4 *q = reinterpret_cast<const uint4 *>(regs + row * p.W + (int64_t)r * p.m);
            for (int k = 0; k < (p.m >> 4); ++k) {
                const uint4 x = q[k];
                const uint32_t w4[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    h ^= (w4[j >> 2] >> (8 * (j & 3))) & 0xffu;
                    h *= kPrime;
                }
            }
        } else {
            // five bit-planes of m bits: register j is bit j%32 of word j/32
            // of every plane
            const int P = p.m >> 5;
            const uint32_t *q = reinterpret_cast<const uint32_t *>(regs + row * p.W);
            for (int j = 0; j < p.m; ++j) {
                uint32_t val = 0;
#pragma unroll
                for (int b = 0; b < 5; ++b) val |= ((q[b * P + (j >> 5)] >> (j & 31)) & 1u) << b;
                h ^= val;
                h *= kPrime;
            }
        }
        acc += h;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

// ---------------------------------------------------------------- node-sharded runs

// Node-sharded runs (the Pregel-style distribution of Algorithm 2 that the
// paper's conclusion proposes): every shard keeps all n counters but holds the
// arcs of its own nodes only, so a pass changes only its own nodes.  Between
// the union kernels and the end of the pass, each shard's changed nodes (the
// bitmap F_{t+1}, restricted to input ids [first, first + count)) and their
// new rows are compacted for the exchange.  A warp per bitmap word; the order
// of the entries depends on timing, which nothing downstream depends on.
__global__ void __launch_bounds__(kBlock) k_shard_collect(Plan p, int64_t first, int64_t count,
                                                          int32_t *ids, uint8_t *rows, int64_t cap)
{
    const DevCtl *c = p.ctl;
    if (c->done) return;
    const int cur = c->parity;
    const unsigned long long *Fn = p.F[cur ^ 1];
    const uint4 *src = reinterpret_cast<const uint4 *>(p.regs[cur ^ 1]);
    uint4 *dst = reinterpret_cast<uint4 *>(rows);
    const int vec = p.W >> 4;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < p.nwords; i += nwarps) {
        const unsigned long long bits = Fn[i];
        if (bits == 0ull) continue;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const int64_t v = i * 64 + 32 * h + lane;
            int32_t id = -1;
            if ((bits >> (32 * h + lane)) & 1ull) {
                id = p.orig_id ? __ldg(p.orig_id + v) : (int32_t)v;
                if (id < first || id >= first + count) id = -1;
            }
            const unsigned bal = __ballot_sync(kFull, id >= 0);
            if (bal == 0u) continue;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&p.ctl->shard_count, (unsigned long long)__popc(bal));
            base = __shfl_sync(kFull, base, 0);
            if (id >= 0) {
                const unsigned long long slot = base + __popc(bal & ((1u << lane) - 1u));
                if (slot < (unsigned long long)cap) {
                    ids[slot] = id;
                    for (int k = 0; k < vec; ++k) dst[(int64_t)slot * vec + k] = src[v * vec + k];
                }
            }
        }
    }
}

// The rows other shards changed in this pass: written into both counter
// buffers (the current one is not read again in this pass, and the next
// pass's target must already hold them, as this shard never visits these
// nodes), marked in F_{t+1}, counted as changed nodes and per run (a run
// counts when its registers differ from the row this shard held).  A warp
// per entry.
__global__ void __launch_bounds__(kBlock) k_shard_apply(Plan p, const int32_t *perm,
                                                        const int32_t *ids, const uint8_t *rows,
                                                        int64_t k)
{
    const DevCtl *c = p.ctl;
    if (c->done) return;
    const int cur = c->parity;
    uint4 *rc = reinterpret_cast<uint4 *>(p.regs[cur]);
    uint4 *rn = reinterpret_cast<uint4 *>(p.regs[cur ^ 1]);
    const uint4 *src = reinterpret_cast<const uint4 *>(rows);
    const int vec = p.W >> 4;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = warp; e < k; e += nwarps) {
        const int32_t id = __ldg(ids + e);
        if (id < 0 || (int64_t)id >= p.n) continue;   // checked by the host as well
        const int64_t v = perm ? (int64_t)__ldg(perm + id) : (int64_t)id;
        uint32_t mask = 0;
        for (int j = lane; j < vec; j += 32) {
            const uint4 nw = src[e * vec + j];
            if (!veq(nw, rc[v * vec + j])) mask |= 1u << ((j << 4) >> p.b);
            rn[v * vec + j] = nw;
            rc[v * vec + j] = nw;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) mask |= __shfl_xor_sync(kFull, mask, o);
        if (lane == 0 && mask) {
            const unsigned long long bit = 1ull << (v & 63);
            if ((atomicOr(&p.F[cur ^ 1][v >> 6], bit) & bit) == 0ull)
                atomicAdd(&p.ctl->changed_count[cur ^ 1], 1ull);
            for (int r = 0; r < p.R; ++r)
                if ((mask >> r) & 1u) atomicAdd(&p.slot_changed[r], 1ull);
        }
    }
}

template <typename F>
cudaError_t with_planes(int m, F &&f)
{
    switch (m) {
    case 32: return f(std::integral_constant<int, 1>());
    case 64: return f(std::integral_constant<int, 2>());
    case 128: return f(std::integral_constant<int, 4>());
    case 256: return f(std::integral_constant<int, 8>());
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------- dispatch on row width

template <int LANES, int VPL>
struct UnionKernels {
    static cudaError_t launch(const Plan &p, cudaStream_t s, const PassFork *fk)
    {
        // persistent grids, but no larger than the work: small graphs launch
        // (and retire) only the blocks they can use
        constexpr int GPW = 32 / LANES;
        constexpr int WPB = kBlock / 32;
        const int64_t persistent = (p.union_warps * 32 + kBlock - 1) / kBlock;
        const int64_t warp_items = p.n_seg + p.n_med;
        const int64_t small_items = (p.n_small + GPW - 1) / GPW;
        const int blocks = (int)std::max<int64_t>(1, std::min(persistent, (warp_items + WPB - 1) / WPB));
        const int sblocks = (int)std::max<int64_t>(1, std::min(persistent, (small_items + WPB - 1) / WPB));
        if (p.in_off && p.scatter_den > 0) {
            // scatter passes (the kernels return at once in every other pass)
            const int64_t scatter_items = p.nwords + p.n;   // words + at most n segments
            k_scatter_seed<<<grid_for(p.nwords, WPB, 152 * 8), kBlock, 0, s>>>(p);
            const int64_t spersistent = (p.scatter_warps * 32 + kBlock - 1) / kBlock;
            k_scatter<LANES, VPL><<<(int)std::max<int64_t>(1, std::min(spersistent,
                                                                        (scatter_items + WPB - 1) / WPB)),
                                    kBlock, 0, s>>>(p);
        }
        // the small-degree kernel runs on the side stream beside the warp
        // kernel (disjoint nodes; bitmap bits and counts by atomics), so each
        // fills the SMs the other drains
        cudaStream_t ss = s;
        if (fk && fk->side && p.W >= 128) {   // measured: a small loss at 64-byte rows
            cudaEventRecord(fk->fork, s);
            cudaStreamWaitEvent(fk->side, fk->fork, 0);
            ss = fk->side;
        }
        if constexpr (VPL <= 2) {
            if (p.first_warps > 0) {   // pass 0 from the c_0 records (other passes: returns)
                const int64_t fpersistent = (p.first_warps * 32 + kBlock - 1) / kBlock;
                const int fw = (int)std::max<int64_t>(1, std::min(fpersistent, (warp_items + WPB - 1) / WPB));
                const int fs = (int)std::max<int64_t>(1, std::min(fpersistent, (small_items + WPB - 1) / WPB));
                k_first_warp<LANES, VPL><<<fw, kBlock, 0, s>>>(p);
                k_first_small<LANES, VPL><<<fs, kBlock, 0, ss>>>(p);
            }
        }
        if constexpr (VPL == 1 && LANES <= 8) {
            if (p.warp_variant == 2) {
                using Cfg = AsyncCfg<LANES>;
                const size_t smem = Cfg::smem_per_block + sizeof(StageMeta) * Cfg::D * (kBlock / 32);
                const int ablocks = (p.union_async_warps * 32 + kBlock - 1) / kBlock;
                k_union_warp_async<LANES><<<ablocks, kBlock, smem, s>>>(p);
            } else {
                k_union_warp<LANES, VPL><<<blocks, kBlock, 0, s>>>(p);
            }
        } else {
            k_union_warp<LANES, VPL><<<blocks, kBlock, 0, s>>>(p);
        }
        bool small_done = false;
        if constexpr (VPL == 1 && LANES <= 8) {
            if (p.small_variant == 3) {
                k_union_small_async<LANES>
                    <<<sblocks, kBlock, SmallAsyncCfg<LANES>::smem_per_block, ss>>>(p);
                small_done = true;
            }
        }
        if (!small_done) k_union_small<LANES, VPL, false><<<sblocks, kBlock, 0, ss>>>(p);
        if constexpr (has_sparse_path<LANES, VPL>())
            k_union_small<LANES, VPL, true><<<sblocks, kBlock, 0, ss>>>(p);
        if (ss != s) {
            cudaEventRecord(fk->join, ss);
            cudaStreamWaitEvent(s, fk->join, 0);
        }
        return cudaGetLastError();
    }
    static cudaError_t launch_hub(const Plan &p, cudaStream_t s)
    {
        constexpr int GPW = 32 / LANES;
        const int blocks = grid_for((p.n_hub + GPW - 1) / GPW, kBlock / 32, 152 * 16);
        k_hub_finish<LANES, VPL><<<blocks, kBlock, 0, s>>>(p);
        return cudaGetLastError();
    }
    static int scatter_occupancy()
    {
        int a = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_scatter<LANES, VPL>, kBlock, 0);
        return a;
    }
    static int occupancy()
    {
        int a = 0, b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_union_small<LANES, VPL, false>, kBlock, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_union_warp<LANES, VPL>, kBlock, 0);
        return a < b ? a : b;
    }
    // Resident blocks of the asynchronous-copy small-degree kernel (0 where
    // it does not apply); also opts it in to more than 48 KB of shared memory.
    static int small_async_occupancy()
    {
        if constexpr (VPL == 1 && LANES <= 8) {
            const size_t smem = SmallAsyncCfg<LANES>::smem_per_block;
            cudaFuncSetAttribute(k_union_small_async<LANES>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            int nb = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_union_small_async<LANES>, kBlock,
                                                          smem);
            return nb;
        } else {
            return 0;
        }
    }
    // Resident blocks of the pass-0 kernels (0 where they do not apply).
    static int first_occupancy()
    {
        if constexpr (VPL <= 2) {
            int a = 0, b = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_first_small<LANES, VPL>, kBlock, 0);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_first_warp<LANES, VPL>, kBlock, 0);
            return a < b ? a : b;
        } else {
            return 0;
        }
    }
    // Resident blocks of the asynchronous-copy warp kernel (0 where it does
    // not apply); also opts it in to more than 48 KB of shared memory.
    static int async_occupancy()
    {
        if constexpr (VPL == 1 && LANES <= 8) {
            using Cfg = AsyncCfg<LANES>;
            const size_t smem = Cfg::smem_per_block + sizeof(StageMeta) * Cfg::D * (kBlock / 32);
            cudaFuncSetAttribute(k_union_warp_async<LANES>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            int nb = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_union_warp_async<LANES>, kBlock,
                                                          smem);
            return nb;
        } else {
            return 0;
        }
    }
};

template <typename F>
cudaError_t with_width(int W, F &&f)
{
    switch (W) {
    case 16: return f(UnionKernels<1, 1>());
    case 32: return f(UnionKernels<2, 1>());
    case 64: return f(UnionKernels<4, 1>());
    case 128: return f(UnionKernels<8, 1>());
    case 256: return f(UnionKernels<16, 1>());
    case 512: return f(UnionKernels<32, 1>());
    case 1024: return f(UnionKernels<32, 2>());
    case 2048: return f(UnionKernels<32, 4>());
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// ---------------------------------------------------------------- launchers

int small_async_blocks(int W)
{
    int nb = 0;
    with_width(W, [&](auto k) {
        nb = decltype(k)::small_async_occupancy();
        return cudaSuccess;
    });
    return nb;
}

int first_pass_warps(int W, int nsm)
{
    int nb = 0;
    with_width(W, [&](auto k) {
        nb = decltype(k)::first_occupancy();
        return cudaSuccess;
    });
    return nb * nsm * (kBlock / 32);
}

int union_async_warps(int W, int nsm)
{
    int nb = 0;
    with_width(W, [&](auto k) {
        nb = decltype(k)::async_occupancy();
        return cudaSuccess;
    });
    return nb * nsm * (kBlock / 32);
}

int packed_occupancy_warps(int m, int nsm)
{
    int nb = 0;
    with_planes(m, [&](auto P) {
        int a = 0, b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_punion_small<decltype(P)::value>, kBlock, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_punion_warp<decltype(P)::value>, kBlock, 0);
        nb = a < b ? a : b;
        return cudaSuccess;
    });
    if (nb < 1) nb = 1;
    return nb * nsm * (kBlock / 32);
}

int scatter_occupancy_warps(int W, int nsm)
{
    int nb = 0;
    with_width(W, [&](auto k) {
        nb = decltype(k)::scatter_occupancy();
        return cudaSuccess;
    });
    if (nb < 1) nb = 1;
    return nb * nsm * (kBlock / 32);
}

int union_occupancy_warps(int W, int nsm)
{
    int nb = 0;
    with_width(W, [&](auto k) {
        nb = decltype(k)::occupancy();
        return cudaSuccess;
    });
    if (nb < 1) nb = 1;
    return nb * nsm * (kBlock / 32);
}

cudaError_t launch_validate(const Plan &p, cudaStream_t s)
{
    k_validate<<<grid_for(p.arcs > p.n ? p.arcs : p.n + 1, kBlock, 152 * 64), kBlock, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_init(const Plan &p, cudaStream_t s)
{
    if (p.layout) {
        return with_planes(p.m, [&](auto P) {
            k_pinit<decltype(P)::value><<<grid_for(p.n, kBlock, 152 * 64), kBlock, 0, s>>>(p);
            return cudaGetLastError();
        });
    }
    k_init<<<grid_for(p.n * (p.W >> 4), kBlock, 152 * 64), kBlock, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_est_changed(const Plan &p, cudaStream_t s);

cudaError_t launch_estimate(const Plan &p, cudaStream_t s, int *nlaunch)
{
    if (p.est_fused) {
        k_est_first<<<grid_for(p.n * p.R, kBlock, 152 * 16), kBlock, 0, s>>>(p);
        const cudaError_t err = launch_est_changed(p, s);
        if (err != cudaSuccess) return err;
    } else if (p.layout) {
        cudaError_t err = with_planes(p.m, [&](auto P) {
            k_pest_blocks<decltype(P)::value><<<grid_for(p.nwords, kBlock / 32, 152 * 64), kBlock, 0, s>>>(p);
            return cudaGetLastError();
        });
        if (err != cudaSuccess) return err;
    } else {
        const int g = grid_for(p.nwords * p.R, kBlock / 32, 152 * 64);
        switch (p.m) {
        case 16: k_est_blocks<16><<<g, kBlock, 0, s>>>(p); break;
        case 32: k_est_blocks<32><<<g, kBlock, 0, s>>>(p); break;
        case 64: k_est_blocks<64><<<g, kBlock, 0, s>>>(p); break;
        case 128: k_est_blocks<128><<<g, kBlock, 0, s>>>(p); break;
        case 256: k_est_blocks<256><<<g, kBlock, 0, s>>>(p); break;
        default: return cudaErrorInvalidValue;
        }
    }
    k_est_finalize<<<grid_for(p.S, kBlock, 152), kBlock, 0, s>>>(p);
    if (nlaunch) *nlaunch += p.est_fused ? 3 : 2;
    return cudaGetLastError();
}

// Changed-node estimate (returns at once at t = 0).
cudaError_t launch_est_changed(const Plan &p, cudaStream_t s)
{
    const int g = grid_for(p.nwords, kBlock / 32, 152 * 8);
    switch (p.m) {
    case 16: k_est_changed<16><<<g, kBlock, 0, s>>>(p); break;
    case 32: k_est_changed<32><<<g, kBlock, 0, s>>>(p); break;
    case 64: k_est_changed<64><<<g, kBlock, 0, s>>>(p); break;
    case 128: k_est_changed<128><<<g, kBlock, 0, s>>>(p); break;
    case 256: k_est_changed<256><<<g, kBlock, 0, s>>>(p); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_pass(const Plan &p, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond,
                        cudaEvent_t ev0, cudaEvent_t ev1, int *nlaunch, const PassFork *fk)
{
    const cudaError_t err = launch_pass_union(p, s, ev0, ev1, nlaunch, fk);
    if (err != cudaSuccess) return err;
    return launch_pass_end(p, s, h, use_cond, nlaunch);
}

cudaError_t launch_pass_union(const Plan &p, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1,
                              int *nlaunch, const PassFork *fk)
{
    k_prep<<<1, 1, 0, s>>>(p);
    k_clear<<<grid_for(std::max<int64_t>(p.nwords, p.S), kBlock, 152 * 16), kBlock, 0, s>>>(p);
    if (p.in_off) k_mark<<<grid_for(p.nwords, kBlock / 32, 152 * 8), kBlock, 0, s>>>(p);
    if (ev0) cudaEventRecord(ev0, s);
    cudaError_t err;
    if (p.layout) {
        err = with_planes(p.m, [&](auto P) {
            constexpr int PP = decltype(P)::value;
            constexpr int WPB = kBlock / 32;
            const int64_t persistent = (p.union_warps * 32 + kBlock - 1) / kBlock;
            const int64_t wi = p.n_seg + p.n_med, si = (p.n_small + 31) / 32;
            const int blocks = (int)std::max<int64_t>(1, std::min(persistent, (wi + WPB - 1) / WPB));
            const int sblocks = (int)std::max<int64_t>(1, std::min(persistent, (si + WPB - 1) / WPB));
            k_punion_warp<PP><<<blocks, kBlock, 0, s>>>(p);
            k_punion_small<PP><<<sblocks, kBlock, 0, s>>>(p);
            if (p.n_hub)
                k_phub_finish<PP><<<grid_for(p.n_hub, kBlock, 152 * 16), kBlock, 0, s>>>(p);
            return cudaGetLastError();
        });
    } else {
        err = with_width(p.W, [&](auto k) { return decltype(k)::launch(p, s, fk); });
        if (err == cudaSuccess && p.n_hub)
            err = with_width(p.W, [&](auto k) { return decltype(k)::launch_hub(p, s); });
    }
    if (err != cudaSuccess) return err;
    if (ev1) cudaEventRecord(ev1, s);
    if (nlaunch)
        *nlaunch += 3 + (p.in_off ? 1 : 0) + (p.n_hub ? 1 : 0) + (!p.layout && p.W <= 128 ? 1 : 0) +
                    (!p.layout && p.in_off && p.scatter_den > 0 ? 2 : 0) +
                    (!p.layout && p.first_warps > 0 ? 2 : 0);
    return cudaGetLastError();
}

cudaError_t launch_pass_end(const Plan &p, cudaStream_t s, cudaGraphConditionalHandle h,
                            int use_cond, int *nlaunch)
{
    if (p.S > 8) k_slot_T<<<grid_for(p.S, kBlock, 152 * 4), kBlock, 0, s>>>(p);
    k_post<<<1, 1, 0, s>>>(p, h, use_cond);
    if (nlaunch) *nlaunch += 2 + (p.S > 8 ? 1 : 0);
    const cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    return launch_estimate(p, s, nlaunch);
}

int64_t scan_tmp_elems(int64_t count)
{
    int64_t total = 0;
    while (count > kScanTile) {
        const int64_t tiles = (count + kScanTile - 1) / kScanTile;
        total += 2 * tiles;
        count = tiles;
    }
    return total + 1;
}

cudaError_t scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t count, int64_t *tmp,
                               int64_t tmp_elems, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    const int64_t tiles = (count + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        k_scan_tile_apply<<<1, kBlock, 0, s>>>(in, out, count, nullptr);
        return cudaGetLastError();
    }
    if (tmp_elems < 2 * tiles) return cudaErrorInvalidValue;
    int64_t *sums = tmp, *offs = tmp + tiles;
    k_scan_tile_sums<<<(unsigned)tiles, kBlock, 0, s>>>(in, count, sums);
    cudaError_t err = scan_exclusive_i64(sums, offs, tiles, tmp + 2 * tiles,
                                         tmp_elems - 2 * tiles, s);
    if (err != cudaSuccess) return err;
    k_scan_tile_apply<<<(unsigned)tiles, kBlock, 0, s>>>(in, out, count, offs);
    return cudaGetLastError();
}

int64_t classify_blocks(int64_t n) { return (n + kClassTile - 1) / kClassTile; }

cudaError_t launch_classify(const Plan &p, int32_t d_small, int32_t d_hub, int64_t *blk_counts,
                            int64_t *blk_offs, int64_t *tmp, int64_t tmp_elems, int32_t *nodes,
                            int64_t *totals_dev, cudaStream_t s)
{
    const int64_t nt = classify_blocks(p.n);
    if (nt == 0) return cudaSuccess;
    k_class_count<<<(unsigned)nt, kBlock, 0, s>>>(p, d_small, d_hub, blk_counts, nt);
    // one scan over [small tiles | medium tiles | hub tiles] lays the three
    // lists out back to back; entry 3*nt is the total
    cudaMemsetAsync(blk_counts + 3 * nt, 0, sizeof(int64_t), s);
    cudaError_t err = scan_exclusive_i64(blk_counts, blk_offs, 3 * nt + 1, tmp, tmp_elems, s);
    if (err != cudaSuccess) return err;
    k_class_scatter<<<(unsigned)nt, kBlock, 0, s>>>(p, d_small, d_hub, blk_offs, nt, nodes);
    // totals: start of medium, start of hub, end
    cudaMemcpyAsync(totals_dev + 0, blk_offs + nt, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(totals_dev + 1, blk_offs + 2 * nt, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(totals_dev + 2, blk_offs + 3 * nt, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    return cudaGetLastError();
}

cudaError_t launch_hub_segments(const Plan &p, int32_t d_hub, int64_t *seg_counts,
                                int64_t *seg_offs, int64_t *tmp, int64_t tmp_elems,
                                int32_t *seg_node, int64_t *seg_beg, int64_t *seg_end,
                                int32_t *hub_seg_first, int64_t *total_dev, cudaStream_t s)
{
    const int32_t *hubs = p.nodes + p.n_small + p.n_med;
    k_hub_seg_count<<<grid_for(p.n_hub + 1, kBlock), kBlock, 0, s>>>(p, d_hub, hubs, p.n_hub,
                                                                     seg_counts);
    cudaError_t err = scan_exclusive_i64(seg_counts, seg_offs, p.n_hub + 1, tmp, tmp_elems, s);
    if (err != cudaSuccess) return err;
    k_hub_seg_fill<<<grid_for(p.n_hub + 1, kBlock), kBlock, 0, s>>>(
        p, d_hub, hubs, p.n_hub, seg_offs, seg_node, seg_beg, seg_end, hub_seg_first);
    cudaMemcpyAsync(total_dev, seg_offs + p.n_hub, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    return cudaGetLastError();
}

cudaError_t launch_transpose(const Plan &p, int64_t *in_off, int32_t *in_src, int64_t *cursor,
                             int64_t *tmp, int64_t tmp_elems, const unsigned long long *indeg_in,
                             const int32_t *inv, int64_t *counts, cudaStream_t s)
{
    cudaError_t err;
    if (indeg_in && inv) {
        // relabelled graph: in-degrees are the input ones, permuted
        k_permute_indeg<<<grid_for(p.n + 1, kBlock, 152 * 64), kBlock, 0, s>>>(indeg_in, inv, p.n,
                                                                              counts);
        err = scan_exclusive_i64(counts, in_off, p.n + 1, tmp, tmp_elems, s);
    } else {
        cudaMemsetAsync(cursor, 0, sizeof(int64_t) * (p.n + 1), s);
        k_in_degree<<<grid_for(p.arcs, kBlock, 152 * 64), kBlock, 0, s>>>(
            p, reinterpret_cast<unsigned long long *>(cursor));
        err = scan_exclusive_i64(cursor, in_off, p.n + 1, tmp, tmp_elems, s);
    }
    if (err != cudaSuccess) return err;
    cudaMemsetAsync(cursor, 0, sizeof(int64_t) * (p.n + 1), s);
    k_transpose_fill<<<152 * 16, kBlock, 0, s>>>(p, in_off,
                                                 reinterpret_cast<unsigned long long *>(cursor),
                                                 in_src);
    return cudaGetLastError();
}

cudaError_t launch_relabel(const int64_t *off, const int32_t *tgt, int64_t n, int64_t arcs,
                           unsigned long long *indeg, int64_t *counts, int64_t *offs,
                           int64_t *tmp, int64_t tmp_elems, int32_t *perm, int32_t *inv,
                           int64_t *deg, int64_t *off2, int32_t *tgt2, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    Plan q{};
    q.n = n;
    q.arcs = arcs;
    q.off = off;
    q.tgt = tgt;
    cudaMemsetAsync(indeg, 0, sizeof(unsigned long long) * (n + 1), s);
    k_in_degree<<<grid_for(arcs, kBlock, 152 * 64), kBlock, 0, s>>>(q, indeg);
    const int64_t nt = classify_blocks(n);
    k_hot_count<<<(unsigned)nt, kBlock, 0, s>>>(indeg, n, counts, nt);
    cudaMemsetAsync(counts + kHotClasses * nt, 0, sizeof(int64_t), s);
    cudaError_t err = scan_exclusive_i64(counts, offs, kHotClasses * nt + 1, tmp, tmp_elems, s);
    if (err != cudaSuccess) return err;
    k_hot_scatter<<<(unsigned)nt, kBlock, 0, s>>>(indeg, n, offs, nt, perm, inv);
    k_new_degree<<<grid_for(n + 1, kBlock, 152 * 64), kBlock, 0, s>>>(off, inv, n, deg);
    err = scan_exclusive_i64(deg, off2, n + 1, tmp, tmp_elems, s);
    if (err != cudaSuccess) return err;
    k_relabel_fill<<<152 * 32, kBlock, 0, s>>>(off, tgt, perm, inv, n, off2, tgt2);
    return cudaGetLastError();
}

int64_t relabel_count_elems(int64_t n) { return kHotClasses * classify_blocks(n) + 1; }

cudaError_t launch_gather_node_values(const void *src, const int32_t *perm, int64_t first,
                                      int64_t count, int elem_bytes, void *out, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    if (elem_bytes == 8)
        k_gather_vals<unsigned long long><<<grid_for(count, kBlock), kBlock, 0, s>>>(
            static_cast<const unsigned long long *>(src), perm, first, count,
            static_cast<unsigned long long *>(out));
    else
        k_gather_vals<uint32_t><<<grid_for(count, kBlock), kBlock, 0, s>>>(
            static_cast<const uint32_t *>(src), perm, first, count, static_cast<uint32_t *>(out));
    return cudaGetLastError();
}

cudaError_t launch_digest(const Plan &p, int32_t run, int64_t first, int64_t count,
                          const int32_t *perm, unsigned long long *out, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    k_digest<<<grid_for(count, kBlock), kBlock, 0, s>>>(p, run, first, count, perm, out);
    return cudaGetLastError();
}

cudaError_t launch_shard_collect(const Plan &p, int64_t first, int64_t count, int32_t *ids,
                                 uint8_t *rows, int64_t cap, cudaStream_t s)
{
    k_shard_collect<<<grid_for(p.nwords, kBlock / 32, 152 * 8), kBlock, 0, s>>>(p, first, count, ids,
                                                                                  rows, cap);
    return cudaGetLastError();
}

cudaError_t launch_shard_apply(const Plan &p, const int32_t *perm, const int32_t *ids,
                               const uint8_t *rows, int64_t k, cudaStream_t s)
{
    if (k <= 0) return cudaSuccess;
    k_shard_apply<<<grid_for(k, kBlock / 32, 152 * 8), kBlock, 0, s>>>(p, perm, ids, rows, k);
    return cudaGetLastError();
}

cudaError_t launch_unpack_rows(const uint8_t *regs, const int32_t *perm, int64_t first,
                               int64_t count, int m, uint8_t *out, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    return with_planes(m, [&](auto P) {
        k_punpack<decltype(P)::value><<<grid_for(count * m, kBlock, 152 * 32), kBlock, 0, s>>>(
            regs, perm, first, count, out);
        return cudaGetLastError();
    });
}

cudaError_t launch_gather_rows(const uint8_t *regs, const int32_t *perm, int64_t first,
                               int64_t count, int W, uint8_t *out, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    k_gather_rows<<<grid_for(count * (W >> 4), kBlock, 152 * 32), kBlock, 0, s>>>(
        regs, perm, first, count, W, out);
    return cudaGetLastError();
}

}  // namespace hanf
