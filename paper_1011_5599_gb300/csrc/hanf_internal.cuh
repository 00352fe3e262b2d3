// Internal declarations of the GB300 HyperANF library: device-side control
// block, the launch plan shared by every kernel, and the launchers that the
// C ABI (hanf_api.cu) drives.  Not installed; the public surface is hanf.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "hanf.h"

namespace hanf {

constexpr int kMaxRuns = 8;       // R <= 8 runs batched in one counter row
constexpr int kBlock = 256;       // threads per block of the streaming kernels

// Mutable iteration state, resident in device memory so that a whole
// HyperANF loop can run as one CUDA graph without the host looking at it.
struct DevCtl {
    int32_t t;           // passes completed since initialisation
    int32_t parity;      // regs[parity] holds c_t, F[parity] the nodes changed into it
    int32_t done;        // 1 once a pass changed no counter
    int32_t mode;        // coming pass: 0 pull + bitmap test, 1 systolic push, 2 dense pull,
                         // 3 scatter (pure push)
    int32_t max_t;       // stop (with err = HANF_ERANGE) after this many passes
    int32_t err;         // HANF_OK, HANF_ERANGE, or HANF_ESTATE (a scatter bound broken)
    int32_t bad_graph;   // set by the CSR validator
    int32_t pad_;
    unsigned long long changed_count[2];     // nodes changed into regs[parity]
    unsigned long long last_changed;         // nodes changed by the last pass
    unsigned long long cand_count[2];        // systolic candidates: small, medium degree
    unsigned long long changed_in_arcs;      // in-degree sum of the nodes the last pass changed
    // work counters since initialisation
    unsigned long long passes, push_passes, arcs_scanned, arcs_gathered, own_reads, writes;
    unsigned long long digest;               // result of the last hanf_digest
    unsigned long long shard_count;          // rows found by the last shard collect
};

// Everything a kernel needs that does not change between passes.  Passed by
// value, so a captured graph replays it unchanged.
struct Plan {
    int64_t n, arcs;
    int32_t b, m, R, W;               // W = bytes per stored node row: R * m (byte
                                      // registers) or 5m/8 (bit-sliced, R = 1)
    int32_t layout;                   // 0 byte registers, 1 five bit-planes
    int64_t nwords;                   // 64-node blocks = bitmap words
    const int64_t *off;
    const int32_t *tgt;
    const int64_t *in_off;            // transpose (systolic mode), or null
    const int32_t *in_src;
    uint8_t *regs[2];                 // ping-pong counter arrays, n x W bytes
    unsigned long long *F[2];         // changed-node bitmaps (parity-indexed)
    unsigned long long *cand;         // systolic candidates of the coming pass
    int32_t *cand_list[2];            // the candidates, small / medium degree (hubs: by bit)
    int32_t d_small, d_hub;           // degree class bounds
    const int32_t *nodes;             // [small | medium | hub] node lists
    int64_t n_small, n_med, n_hub;
    const int32_t *seg_node;          // hub segments: node, arc range
    const int64_t *seg_beg;
    const int64_t *seg_end;
    int64_t n_seg;
    const int32_t *hub_seg_first;     // n_hub + 1 segment offsets
    uint8_t *hub_part;                // n_seg x W partial maxima
    uint8_t *hub_any;                 // n_seg flags: segment merged something
    // N(t) = sum_v size(c_t[v]), kept exactly in signed 128-bit fixed point
    // with 52 fractional bits ("Q52"; two 64-bit words, low first)
    unsigned long long *blk_q;        // R x nwords sums of size() over 64-node blocks
    unsigned long long *est_acc;      // S running sums N_s(t)
    int32_t est_fused;                // 1: after each pass only the changed counters'
                                      // size() is evaluated, its change added to
                                      // est_acc (byte layout, one graph, no per-node
                                      // statistics); 0: blocks with a changed counter
                                      // are summed again
    double *ecache;                   // est_fused: R x n, size() of every counter
    double *hist;                     // history_cap x S values of N(t)
    const double *lc;                 // m+1 linear-counting values m ln(m/V)
    double amm;                       // alpha_m m^2
    const uint64_t *seeds;            // S = K * R slot seeds (slot = graph * R + run)
    // batches of K graphs laid out at 64-aligned node ranges (K = 1: one graph)
    int32_t K, S;
    const int32_t *blk_graph;         // graph of every 64-node block (K > 1)
    const int64_t *g_base;            // K + 1 first stored node of each graph
    const int64_t *g_nodes;           // K real node counts
    int32_t *slot_T;                  // S: first pass that left the slot unchanged
    unsigned long long *slot_changed; // S: nodes changed in the slot this pass
    const int32_t *orig_id;           // input id of every stored node (null: identity)
    uint16_t *hr;                     // c_0 as (index << 8) | rho+ of node v, run r at
                                      // [v * R + r] (byte layout; null otherwise)
    // per-node statistics of the E_v(t) sequence, [run][node] (node_stats)
    double *ns_prev;                  // E_v at the last estimate
    double *ns_dist;                  // sum_t t (E_v(t) - E_v(t-1))
    double *ns_reach;                 // E_v(T) of the previous run (radius replay)
    int32_t *ns_ecc;                  // last t with E_v(t) != E_v(t-1)
    int32_t *ns_rad;                  // first t with E_v(t) >= ns_alpha E_v(T)
    double ns_alpha;
    int32_t node_stats, ns_radius_mode;
    int32_t frontier, push_den, dense_num, dense_den, scatter_den;
    int32_t scatter_seg;              // scatter passes: in-arcs per segment, and the
    int32_t scatter_inline;           // in-degree above which a list is segmented
    int32_t history_cap;
    int32_t union_warps;              // resident warps of the union launch
    int32_t scatter_warps;            // resident warps of the scatter launch
    int32_t union_async_warps;        // resident warps of the asynchronous-copy variant
    int32_t warp_variant;             // medium/hub gathers: 1 register batches, 2 async copies
    int32_t small_variant;            // small-degree dense gathers: 0 registers, 3 async copies
    int32_t first_warps;              // pass 0 from the c_0 records: resident warps of its
                                      // kernels (0 = pass 0 reads rows like the others)
    DevCtl *ctl;
};

// ---- launchers (hanf_kernels.cu); all asynchronous on `s` ----
cudaError_t launch_validate(const Plan &p, cudaStream_t s);
cudaError_t launch_init(const Plan &p, cudaStream_t s);
cudaError_t launch_estimate(const Plan &p, cudaStream_t s, int *nlaunch);
// A second stream for the union kernels of one pass: the small-degree
// kernel runs on `side` beside the warp kernel, joined before the hub combine.
struct PassFork {
    cudaStream_t side;
    cudaEvent_t fork, join;
};
cudaError_t launch_pass(const Plan &p, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond,
                        cudaEvent_t ev_union0, cudaEvent_t ev_union1, int *nlaunch,
                        const PassFork *fk = nullptr);
// The two halves of launch_pass: the pass flavour, marking and union kernels;
// then the stop decision (t, parity, T of each slot) and the estimate.  A
// node-sharded run exchanges the changed counters between them.
cudaError_t launch_pass_union(const Plan &p, cudaStream_t s, cudaEvent_t ev_union0,
                              cudaEvent_t ev_union1, int *nlaunch, const PassFork *fk = nullptr);
cudaError_t launch_pass_end(const Plan &p, cudaStream_t s, cudaGraphConditionalHandle h,
                            int use_cond, int *nlaunch);
// Node-sharded runs: the rows of the nodes a pass changed whose input id lies
// in [first, first + count), compacted (input ids, rows) into caller buffers
// of `cap` entries (ctl->shard_count counts them all); and the rows received
// from other shards written into both counter buffers, marked changed.
cudaError_t launch_shard_collect(const Plan &p, int64_t first, int64_t count, int32_t *ids,
                                 uint8_t *rows, int64_t cap, cudaStream_t s);
cudaError_t launch_shard_apply(const Plan &p, const int32_t *perm, const int32_t *ids,
                               const uint8_t *rows, int64_t k, cudaStream_t s);
int union_occupancy_warps(int W, int nsm);
int small_async_blocks(int W);
int first_pass_warps(int W, int nsm);   // resident warps of the pass-0 kernels (0: none)
int scatter_occupancy_warps(int W, int nsm);
int packed_occupancy_warps(int m, int nsm);
int union_async_warps(int W, int nsm);

// Preprocessing (create time).
cudaError_t scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t count, int64_t *tmp,
                               int64_t tmp_elems, cudaStream_t s);
int64_t scan_tmp_elems(int64_t count);
cudaError_t launch_classify(const Plan &p, int32_t d_small, int32_t d_hub, int64_t *blk_counts,
                            int64_t *blk_offs, int64_t *tmp, int64_t tmp_elems, int32_t *nodes,
                            int64_t *totals_dev, cudaStream_t s);
cudaError_t launch_hub_segments(const Plan &p, int32_t d_hub, int64_t *seg_counts,
                                int64_t *seg_offs, int64_t *tmp, int64_t tmp_elems,
                                int32_t *seg_node, int64_t *seg_beg, int64_t *seg_end,
                                int32_t *hub_seg_first, int64_t *total_dev, cudaStream_t s);
cudaError_t launch_transpose(const Plan &p, int64_t *in_off, int32_t *in_src, int64_t *cursor,
                             int64_t *tmp, int64_t tmp_elems, const unsigned long long *indeg_in,
                             const int32_t *inv, int64_t *counts, cudaStream_t s);
int64_t classify_blocks(int64_t n);

// Node relabelling by in-degree class (create time) and the row gather that
// maps stored rows back to input ids.
cudaError_t launch_relabel(const int64_t *off, const int32_t *tgt, int64_t n, int64_t arcs,
                           unsigned long long *indeg, int64_t *counts, int64_t *offs,
                           int64_t *tmp, int64_t tmp_elems, int32_t *perm, int32_t *inv,
                           int64_t *deg, int64_t *off2, int32_t *tgt2, cudaStream_t s);
int64_t relabel_count_elems(int64_t n);
cudaError_t launch_gather_rows(const uint8_t *regs, const int32_t *perm, int64_t first,
                               int64_t count, int W, uint8_t *out, cudaStream_t s);
cudaError_t launch_gather_node_values(const void *src, const int32_t *perm, int64_t first,
                                      int64_t count, int elem_bytes, void *out, cudaStream_t s);
cudaError_t launch_digest(const Plan &p, int32_t run, int64_t first, int64_t count,
                          const int32_t *perm, unsigned long long *out, cudaStream_t s);
cudaError_t launch_unpack_rows(const uint8_t *regs, const int32_t *perm, int64_t first,
                               int64_t count, int m, uint8_t *out, cudaStream_t s);

// Store the calling thread's message for hanf_last_error().
void record_error(const char *msg);
inline void record_error(const std::string &msg) { record_error(msg.c_str()); }

}  // namespace hanf
