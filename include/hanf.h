/*
 * hanf.h -- C ABI of the GB300 HyperANF library (libhanf.so).
 *
 * HyperANF (Boldi, Rosa, Vigna) approximates the neighbourhood function
 * N(t) = #{(x, y) : d(x, y) <= t} of a directed graph.  Every node keeps a
 * HyperLogLog counter of m = 2^log2m registers (Section 3.1, Algorithm 1);
 * node v starts with itself, and each pass replaces c[v] by the
 * register-wise maximum of c[v] and the counters of its successors
 * (Section 3.2, Algorithm 2).  N(t) is the sum over nodes of the counters'
 * size() estimates.  Passes repeat until one changes no counter
 * (stabilisation, Section 3.2); the last value printed is N(T).
 *
 * Conventions shared by every entry point:
 *   - Graphs are CSR by source: offsets[n+1] (int64, offsets[0] = 0,
 *     non-decreasing), targets[arcs] (int32, each in [0, n)).  Self-loops and
 *     duplicate arcs are legal (max is idempotent).  n < 2^31.
 *   - Register i of run r of node v is one byte, value 0..31 (0 = empty; the
 *     paper's "minus infinity").  rho+ is clamped to 31.
 *   - Hash: h(v) = splitmix64(v XOR seed_r), seed_r = splitmix64(seed + r)
 *     unless explicit seeds are given; the register index is the top log2m
 *     bits of h, rho+ counts the leading zeroes of the remaining bits plus one.
 *   - A context holds K >= 1 graphs (a batch, hanf_opts.num_graphs) and R runs
 *     of each: S = K * R "slots", slot = graph * R + run; per-run outputs
 *     (N(t), T) have one entry per slot.
 *   - size(): E = alpha_m m^2 / sum_j 2^-M[j] with the published alpha_m, and
 *     small-range linear counting E = m ln(m/V) when E <= 5m/2 and V > 0.
 *   - Device memory is never allocated by the library: the caller passes one
 *     device workspace (see hanf_workspace_size) and keeps it alive until
 *     hanf_destroy.  Streams are the caller's (cudaStream_t passed as void*).
 *   - Every function returns HANF_OK (0) or a negative HANF_E* code and never
 *     throws; hanf_last_error() gives a message for the calling thread.
 */
#ifndef HANF_H
#define HANF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Symbols of the public surface; everything else in the library is hidden. */
#if defined(__GNUC__)
#define HANF_API __attribute__((visibility("default")))
#else
#define HANF_API
#endif

#define HANF_OK 0
#define HANF_EINVAL (-1)     /* bad argument: sizes, CSR contents, options */
#define HANF_ENOMEM (-2)     /* workspace smaller than hanf_workspace_size  */
#define HANF_ECUDA (-3)      /* a CUDA runtime call failed                  */
#define HANF_ERANGE (-4)     /* history capacity exhausted before stability */
#define HANF_ESTATE (-5)     /* call not valid in the context's state       */
#define HANF_ETIMEOUT (-6)   /* a wait ran out of time                       */
#define HANF_ECANCELLED (-7) /* the job was cancelled before it started      */

/* Frontier policy (Section 3.3, "tracking modified counters" and "systolic
 * computation"). */
#define HANF_FRONTIER_OFF 0  /* every pass merges every arc                  */
#define HANF_FRONTIER_PULL 1 /* skip successors that did not change          */
#define HANF_FRONTIER_AUTO 2 /* PULL, and systolic push through the transpose
                                when fewer than n/push_den counters changed,
                                or a pure push (scatter) when the changed
                                counters have fewer than arcs/scatter_den
                                in-arcs                                       */

typedef struct hanf_ctx hanf_ctx;

typedef struct hanf_opts {
    int32_t runs;          /* R >= 1 independent seeded runs batched together  */
    int32_t frontier;      /* HANF_FRONTIER_*; default AUTO                    */
    int32_t push_den;      /* systolic switch below n/push_den changes; 4      */
    int32_t small_max_deg; /* degree <= this: a lane group per node; 0 = 256,
                              or 32 for rows of 512 bytes and more           */
    int32_t hub_min_deg;   /* degree > this: split in segments of this many
                              arcs, a warp each; 0 = 16384                     */
    int32_t history_cap;   /* capacity of the device N(t) history; 0 = 4096    */
    int32_t use_graph;     /* hanf_run: 1 = whole loop as one CUDA graph with a
                              device-side while node (no host syncs)           */
    int32_t profile;       /* 1 = time the union kernels of every pass with
                              CUDA events and keep a per-pass trace           */
    int32_t dense_den;     /* while the changed counters' in-arcs are at least
                              arcs/dense_den, a pull pass gathers every
                              successor without testing the changed bitmap;
                              0 = the default: arcs/2, or 15 arcs/16 for rows
                              of 512 bytes and more                           */
    int32_t relabel;       /* 1 = store the counters in decreasing in-degree
                              order (hot counters share cache lines); results
                              and hanf_registers use input ids either way    */
    int32_t gather_variant;/* how rows are gathered: 1 = register batches in
                              every kernel; 2 = asynchronous copies into a
                              shared-memory ring for medium-degree nodes and
                              hub segments; 3 = asynchronous copies into
                              per-lane shared-memory slots in the small-degree
                              kernel's dense passes; 4 = both 2 and 3; 0 = the
                              default, 3 for rows of at most 128 bytes (2, 3
                              and 4 apply to such rows only), 1 otherwise     */
    int32_t layout;        /* 0 = one byte per register; 1 = five bit-planes of
                              m bits (5m/8 bytes per counter; runs = 1 and
                              m >= 32); results are identical               */
    int32_t node_stats;    /* 1 = keep per-node statistics (hanf_node_stats,
                              hanf_node_radius): 32 bytes per node and run    */
    int32_t num_graphs;    /* K >= 1 graphs batched in one context (0 = 1)    */
    const int64_t *graph_base;  /* K > 1: K+1 node offsets (host); graph g owns
                              stored nodes [base[g], base[g+1]); every base[g],
                              g < K, a multiple of 64, base[K] = n             */
    const int64_t *graph_nodes; /* K > 1: K node counts; nodes base[g] ..
                              base[g]+nodes[g]-1 are graph g's nodes 0..; the
                              rest of the range is padding without arcs; arcs
                              stay inside their graph (checked)               */
    const uint64_t *graph_seeds;/* K > 1: run r of graph g hashes with
                              splitmix64(graph_seeds[g] + r); NULL = seed      */
    const uint64_t *seeds; /* R explicit run seeds (host, K = 1), or NULL     */
    void *stream;          /* cudaStream_t for every launch; NULL = default    */
    int32_t scatter_den;   /* frontier AUTO: pure push (scatter) pass while the
                              nodes changed by the last pass have fewer than
                              arcs/scatter_den in-arcs (byte layout); 0 = 8
                              for rows of at most 128 bytes (R*m), never for
                              wider rows; negative = never                   */
    int64_t l2_hot_bytes;  /* > 0: keep up to this many bytes of the hottest
                              counter rows (stored first, by in-degree class)
                              of the buffer a pass reads in the L2's
                              persisting set-aside (an access-policy window on
                              the pass's launches; the context's
                              persisting-L2 limit is raised for the context's
                              lifetime and restored by hanf_destroy, so two
                              such contexts alive at once share it); 0 = 64
                              MiB when the counters take 1 GiB or more, else
                              off; negative = off (served jobs: off)       */
} hanf_opts;

/* Fill *opts with the defaults above. */
HANF_API void hanf_default_opts(hanf_opts *opts);

/* Bytes of device workspace hanf_create needs for a graph of n nodes and
 * `arcs` arcs.  copy_graph = 1 when the CSR will be passed in host memory
 * (the context then keeps its own device copy).  Returns HANF_EINVAL for
 * log2m outside 4..8, n < 0 or n >= 2^31, arcs < 0, runs outside 1..8. */
HANF_API int hanf_workspace_size(int64_t n, int64_t arcs, int32_t log2m, const hanf_opts *opts,
                        int32_t copy_graph, size_t *bytes_out);

/* Create a context and initialise every counter (Algorithm 2: each node adds
 * itself), leaving it at t = 0.
 *   offsets, targets: the CSR (see conventions).  graph_on_device = 0: host
 *     pointers, copied into the workspace (pinned host memory copies
 *     fastest); = 1: device pointers borrowed for the context's lifetime.
 *   workspace: device buffer of at least hanf_workspace_size() bytes, 256-byte
 *     aligned, owned by the caller.
 * The CSR is validated on the device (offsets monotone, targets in range);
 * a bad graph returns HANF_EINVAL and no context.  *out is set only on
 * success. */
HANF_API int hanf_create(hanf_ctx **out, int64_t n, int64_t arcs, const int64_t *offsets,
                const int32_t *targets, int32_t graph_on_device, int32_t log2m,
                uint64_t seed, const hanf_opts *opts, void *workspace,
                size_t workspace_bytes);

/* Algorithm 2, the sum s = sum_v size(c[v]) at the current t, for every slot:
 * N_out (host) receives S = K * R doubles.  Synchronises the stream. */
HANF_API int hanf_estimate(hanf_ctx *ctx, double *N_out);

/* One pass of Algorithm 2's main loop (t -> t+1): every counter becomes the
 * register-wise max of itself and its successors' counters at t (Jacobi).
 * *changed_out (host, nullable) = number of nodes whose counter changed in
 * any run.  Synchronises the stream. */
HANF_API int hanf_iterate(hanf_ctx *ctx, int64_t *changed_out);

/* The whole of Algorithm 2: re-initialise, then print N(t) and run passes
 * until a pass changes no counter of any run (or max_iter passes ran).
 *   N_out (host): S x cap doubles (S = K * R slots), row s holds N_s(0..T_s)
 *     (later entries repeat N_s(T_s) up to the global T).
 *   T_out (host): S ints, T_s = the first pass index that changed no counter
 *     of slot s.
 * Returns HANF_ERANGE if stabilisation needs more than cap values or
 * max_iter passes (N_out then holds what was computed). */
HANF_API int hanf_run(hanf_ctx *ctx, int32_t max_iter, double *N_out, int32_t cap, int32_t *T_out);

/* Copy the registers of nodes [first, first+count) of run r to host memory:
 * count * m bytes, node-major.  Synchronises the stream. */
HANF_API int hanf_registers(hanf_ctx *ctx, int32_t run, int64_t first, int64_t count, uint8_t *out);

/* Digest of the registers of run r for nodes [first, first+count) (input
 * ids): the sum modulo 2^64, over those nodes v, of FNV-1a-64 (Fowler, Noll,
 * Vo; 64-bit offset basis and prime) of the eight little-endian bytes of
 * v - first followed by the m registers of c[v], one byte each, whatever the
 * storage layout.  A check value for Algorithm 2's state (the counters
 * c_t of Section 3.2): two arrays with the same registers give the same
 * digest, and any difference changes it except with probability about
 * 2^-64, so a run can be compared after every pass with another
 * implementation without copying n*m bytes out.  *digest_out (host).  Uses
 * the context's control block as its only scratch.  Synchronises the
 * stream. */
HANF_API int hanf_digest(hanf_ctx *ctx, int32_t run, int64_t first, int64_t count,
                         uint64_t *digest_out);

/* ---- One pass in steps: node-sharded runs ----------------------------------
 * The distribution of Algorithm 2 over several GPUs that the paper's
 * conclusion proposes (Pregel-style: every node computes its new counter from
 * its successors' counters, then the changed counters are exchanged): shard q
 * owns the input ids [lo_q, hi_q) and is a context over all n nodes whose CSR
 * holds the arcs of its own nodes only (other rows empty), so a pass changes
 * only its own counters.  One pass is
 *   hanf_pass_begin   the pass flavour, marking and union kernels (no sync);
 *   hanf_pass_collect its own changed nodes and their new rows, for sending;
 *   hanf_pass_apply   the other shards' changed rows, received;
 *   hanf_pass_end     stop decision and N(t+1), now over every changed node.
 * Every shard then holds all counters of c_{t+1}, and N(t) (hanf_estimate),
 * T and the changed counts are those of the unsharded run.  Byte layout and
 * one graph only (HANF_ESTATE otherwise).  All buffers are device memory. */

/* Start pass t -> t+1 (asynchronous).  *started_out = 0 if the run has
 * already stabilised (nothing launched; then no other step may follow). */
HANF_API int hanf_pass_begin(hanf_ctx *ctx, int32_t *started_out);

/* The nodes with input ids in [first, first+count) that the open pass
 * changed: their input ids into ids[] and their new rows (R*m bytes each,
 * run-major, one byte per register; 16-byte aligned) into rows[], in no
 * particular order, at most `cap` entries; *n_out (host) = how many there are.
 * HANF_ERANGE if more than cap (call again with room for *n_out).
 * Synchronises the stream. */
HANF_API int hanf_pass_collect(hanf_ctx *ctx, int64_t first, int64_t count, int32_t *ids,
                               uint8_t *rows, int64_t cap, int64_t *n_out);

/* Counters other shards changed in the open pass: k input ids (each outside
 * this shard's range, each once) and their new rows, as hanf_pass_collect
 * returns them.  Asynchronous. */
HANF_API int hanf_pass_apply(hanf_ctx *ctx, const int32_t *ids, const uint8_t *rows, int64_t k);

/* Close the pass: *changed_out (host, nullable) = nodes changed in it, over
 * all shards once every shard's rows were applied; 0 means stable.
 * Synchronises the stream. */
HANF_API int hanf_pass_end(hanf_ctx *ctx, int64_t *changed_out);

/* Current pass index t (number of passes run since initialisation). */
HANF_API int hanf_current_t(hanf_ctx *ctx, int32_t *t_out);

/* Work and time counters since the last hanf_run / initialisation:
 * out[0] passes, out[1] arcs scanned, out[2] arcs gathered (successor
 * counters read), out[3] own counters read, out[4] counters written,
 * out[5] union-kernel launches, out[6] union-kernel milliseconds (profile = 1,
 * else 0), out[7] all kernel launches, out[8] estimator milliseconds,
 * out[9] passes run in systolic or scatter (push) mode.  In scatter passes
 * "arcs scanned" and "arcs gathered" count the (changed node, predecessor)
 * pairs pushed, "own counters read" the rows read to push into, and
 * "counters written" the rows copied or raised.  nout = entries wanted
 * (<= 10). */
HANF_API int hanf_counters(hanf_ctx *ctx, double *out, int32_t nout);

/* Per-pass trace of the last run since initialisation (profile = 1 and the
 * host-loop driver): up to max_rows rows of 8 doubles {t, mode (0 pull with
 * the changed-bitmap test, 1 systolic push, 2 pull gathering every
 * successor, 3 scatter: changed nodes push into their predecessors), nodes
 * changed, union milliseconds, arcs scanned, arcs gathered, own counters
 * read, counters written}; *rows_out = rows written. */
HANF_API int hanf_trace(hanf_ctx *ctx, double *out, int32_t max_rows, int32_t *rows_out);

/* Section 4 and 5 statistics of N(0..T) (host arrays, no GPU):
 * out5 = {effective diameter at alpha, interpolated effective diameter, mean
 * distance, variance, spid = variance / mean}, with H(t) = N(t)/max N and
 * h(t) = H(t) - H(t-1); exclude_zero = 1 leaves out the pairs (x, x). */
HANF_API int hanf_stats(const double *N, int32_t T, double alpha, int32_t exclude_zero, double *out5);

/* Allocation-free estimate of N = sum_v size(c[v]) for a register array the
 * caller already holds (the paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory while they run, such as a
 * serving loop whose device memory was all reserved up front, or a process
 * sharing the GPU with an allocator that owns all of it, where cudaMalloc
 * would fail or synchronise the device).
 *   regs: device pointer, 16-byte aligned, to n rows of runs * 2^log2m bytes
 *     (row v holds run 0's registers, then run 1's, ...; values 0..31), the
 *     layout this library keeps.  A register above 31 makes its run's N NaN.
 *   N_out: device pointer, 8-byte aligned, to `runs` doubles, N for each run.
 *   stream: cudaStream_t (NULL = default stream); the call only enqueues work.
 * Its scratch is one fixed array of 2^20 doubles (8 MiB) inside the library,
 * kept by every GPU that loads it until the process exits; runs * (ceil(n/64)
 * + ceil(n/262144)) must not exceed 2^20, otherwise it returns HANF_EINVAL
 * (as it does for a misaligned pointer), before enqueuing anything.
 * The first call in each CUDA context (normally: on each device) looks the
 * array's address up with that context current and remembers it by the
 * context's id, so make that first call before any stream capture; a context
 * created later (after cudaDeviceReset, or another driver-API context) gets
 * its own lookup.  Calls share the array and each overwrites what it reads;
 * calls that overlap on the GPU race and must be serialised by the caller. */
HANF_API int hanf_estimate_static(const uint8_t *regs, int64_t n, int32_t log2m, int32_t runs,
                                  double *N_out, void *stream);

/* Autotuner (the paper has no counterpart; its thread pool needs no tuning):
 * times candidate launch parameters of the union pass on this graph -- the
 * degree split small_max_deg in {32,128,256,1024,4096}, hub_min_deg in
 * {4096,16384,65536} and gather_variant in {1,2,3} (2 and 3 for rows of at
 * most 128 bytes), then on the best of those
 * (frontier AUTO, byte layout, scatter_den 0 in *base) the pass flavour the
 * row width does not default to (scatter_den -1 for rows up to 128 bytes, 8
 * above) -- each with its own context in `workspace`,
 * one warm-up and one timed run of Algorithm 2, and returns the fastest in
 * *best_out (the other fields copied from *base, NULL = defaults) and its
 * time in *best_ms_out (nullable).  cache_path (nullable) names a text file:
 * a result already stored for the same GPU, row width, graph size, frontier
 * policy and relabelling is returned without timing; new results are
 * appended.  Candidates whose workspace does not fit are skipped (size the
 * workspace with hub_min_deg = 4096 to try them all).  Synchronises. */
HANF_API int hanf_autotune(int64_t n, int64_t arcs, const int64_t *offsets,
                           const int32_t *targets, int32_t graph_on_device, int32_t log2m,
                           uint64_t seed, const hanf_opts *base, void *workspace,
                           size_t workspace_bytes, const char *cache_path, hanf_opts *best_out,
                           double *best_ms_out);

/* ---- Serving: continuous batching of HyperANF jobs --------------------------
 * A server owns worker threads, each with its own CUDA stream, and a device
 * arena the caller reserved (the HBM budget).  Jobs are admitted in arrival
 * order as soon as a worker is free and the job's workspace (as sized by
 * hanf_workspace_size) fits in the arena; the admitted job runs the whole of
 * Algorithm 2 as one CUDA graph on its worker's stream, so jobs of different
 * workers overlap on the GPU.  Small jobs (at most 65,536 nodes, default pass
 * limit) admitted together with later queued small jobs of the same m, runs
 * and graph placement share one context (num_graphs > 1, up to 64 jobs and
 * 2^21 stored nodes), so they share launches too.  A job's result is the
 * same whether it runs alone, batched or among others.  (The paper runs one
 * graph at a time; this layer is the serving pattern around its Algorithm
 * 2.) */
typedef struct hanf_server hanf_server;

typedef struct hanf_job {
    int64_t n, arcs;          /* graph size                                       */
    const int64_t *offsets;   /* CSR as for hanf_create; the memory must stay
                                 valid until hanf_server_wait returns for the job */
    const int32_t *targets;
    int32_t graph_on_device;  /* 0: host pointers (copied at admission), 1: device */
    int32_t log2m;            /* 4..8                                               */
    int32_t runs;             /* R, as for hanf_opts.runs                          */
    int32_t max_iter;         /* passes allowed; 0 = 4096                          */
    uint64_t seed;            /* run seeds splitmix64(seed + r)                    */
} hanf_job;

/* Create a server over `arena` (device, 256-byte aligned, arena_bytes long,
 * owned by the caller until hanf_server_destroy) with `workers` worker
 * threads (1..64).  `base` gives the options every job uses (frontier, degree
 * thresholds, relabelling; runs, streams, seeds and drivers are per job);
 * NULL = defaults. */
HANF_API int hanf_server_create(hanf_server **out, void *arena, size_t arena_bytes,
                                int32_t workers, const hanf_opts *base);

/* Queue a job; *id_out identifies it.  HANF_ENOMEM if the job cannot fit even
 * in the empty arena. */
HANF_API int hanf_server_submit(hanf_server *s, const hanf_job *job, uint64_t *id_out);

/* Wait for a job (timeout_ms < 0: no limit; HANF_ETIMEOUT when it runs out, the
 * job stays queued or running).  On success N_out (host, runs x cap, nullable)
 * gets N_r(0..T) with T the job's last pass (entries after T_r repeat
 * N_r(T_r)), T_out (runs, nullable) the T_r, and info_out (5 doubles,
 * nullable) {latency ms from submission to completion, ms queued, ms on a
 * worker, T, workspace bytes}.  The job's own failure code is returned as is.
 * Each job can be waited for once. */
HANF_API int hanf_server_wait(hanf_server *s, uint64_t id, int32_t timeout_ms, double *N_out,
                              int32_t cap, int32_t *T_out, double *info_out);

/* Cancel a job that has not started (HANF_ESTATE if it has). */
HANF_API int hanf_server_cancel(hanf_server *s, uint64_t id);

/* out = {jobs queued, jobs running, completed, failed, largest free arena
 * block, arena bytes, contexts created (a batch of jobs counts once)};
 * nout <= 7. */
HANF_API int hanf_server_stats(hanf_server *s, double *out, int32_t nout);

/* Stop the workers after their current jobs (queued jobs are cancelled) and
 * free the server.  No other call on the server may be in progress. */
HANF_API void hanf_server_destroy(hanf_server *s);

/* Checkpoint and resume (Algorithm 2 keeps its state in the counters and the
 * update file; this is the GPU analogue): the state after any pass -- both
 * counter buffers, the changed-node bitmaps, the N(t) history, the
 * estimator's block partials and the control block -- is copied to a host
 * buffer of hanf_checkpoint_size() bytes, and can be loaded into a context
 * created on the same graph with the same log2m, runs, seeds, layout and
 * relabelling (checked: HANF_EINVAL otherwise).  hanf_continue then runs
 * passes from the current state, like hanf_run without re-initialising; a
 * resumed run gives bit-identical counters, T and N(t).  All synchronise. */
HANF_API int hanf_checkpoint_size(hanf_ctx *ctx, size_t *bytes_out);
HANF_API int hanf_checkpoint_save(hanf_ctx *ctx, void *buf, size_t bytes);
HANF_API int hanf_checkpoint_load(hanf_ctx *ctx, const void *buf, size_t bytes);
HANF_API int hanf_continue(hanf_ctx *ctx, int32_t max_iter, double *N_out, int32_t cap,
                           int32_t *T_out);

/* Per-node statistics (opts.node_stats = 1) -- the radius distribution and
 * closeness centrality that the paper's conclusion proposes to build with
 * HyperANF.  For the last completed run and nodes [first, first+count) of
 * run r (input ids), from the node's estimates E_v(0..T): reach = E_v(T)
 * (nodes reachable from v, v included), dist = sum_t t (E_v(t) - E_v(t-1))
 * (sum of distances to them; closeness = (reach - 1) / dist), ecc = the last
 * t with E_v(t) != E_v(t-1) (eccentricity estimate; never above the true
 * one).  Host outputs, each nullable.  Synchronises. */
HANF_API int hanf_node_stats(hanf_ctx *ctx, int32_t run, int64_t first, int64_t count,
                             double *reach, double *dist, int32_t *ecc);

/* Effective radius of every node (HADI's radius at alpha, e.g. 0.9): the
 * first t with E_v(t) >= alpha E_v(T).  Replays the whole of Algorithm 2 once
 * (deterministic, same counters) after a completed run with node_stats = 1,
 * then copies radius[0..count) of run r for input ids first.. to the host. */
HANF_API int hanf_node_radius(hanf_ctx *ctx, double alpha, int32_t run, int64_t first,
                              int64_t count, int32_t *radius);

/* Algorithm 3 (Section 4, Corollary 2): with each N(t) known to relative
 * error eps, M = max_t N(t), *lo = the largest D- with N(D-)/M <= alpha(1-2eps)
 * and *hi = the smallest D+ with N(D+)/M >= alpha(1+2eps); the effective
 * diameter at alpha lies in [D-..D+] with confidence 1-3 delta.  -1 where no
 * such t exists (no lower end; no upper end within 0..T).  No GPU. */
HANF_API int hanf_ed_interval(const double *N, int32_t T, double alpha, double eps, int32_t *lo,
                              int32_t *hi);

/* Statistics over R runs (Section 4's advice to average many runs; Table 2
 * reports means and standard deviations): N is R x cap row-major with run r's
 * N_r(0..T_r) in row r.  out10 = {mean of ed, ied, mean distance, variance,
 * spid, then their sample standard deviations (0 if R = 1)}.  No GPU. */
HANF_API int hanf_stats_runs(const double *N, int32_t R, int32_t cap, const int32_t *T,
                             double alpha, int32_t exclude_zero, double *out10);

/* Release the context (not the workspace, which belongs to the caller). */
HANF_API void hanf_destroy(hanf_ctx *ctx);

/* Message of the last failing call on this thread ("" if none). */
HANF_API const char *hanf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HANF_H */
