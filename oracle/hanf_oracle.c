/*
 * HyperANF CPU oracle -- TEST INFRASTRUCTURE, not part of the product path.
 *
 * A plain, slow, deliberately literal CPU restatement of what the HyperANF
 * method computes (Boldi, Rosa, Vigna, "HyperANF: Approximating the
 * Neighbourhood Function of Very Large Graphs on a Budget").  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * this file's library.  It shares no code, header, table or constant with the
 * CUDA library: every formula below is written out again from the paper.
 *
 * Readings of points the paper leaves open (each is listed with its reason in
 * the project's design notes):
 *   - hash h(x) = splitmix64(x XOR seed) (standard splitmix64 output step);
 *     h_b(x) = top b bits, h^b(x) = the remaining 64-b bits, left to right;
 *   - an empty register ("set to -infinity", Algorithm 1) is stored as 0:
 *     every added item has rho+ >= 1, so 0 behaves as -infinity under max;
 *   - rho+ is clamped to 31 so that registers fit five bits;
 *   - alpha_m uses the published HyperLogLog constants; size() applies the
 *     small-range linear-counting correction (E <= 5m/2 and V > 0);
 *   - run r of a multi-run job uses seed_r = splitmix64(seed + r);
 *   - the iteration is Jacobi: every new counter of pass t is computed from
 *     the counters of pass t (Algorithm 2 writes <v, m> pairs to an update
 *     file and applies them only after the scan).
 *
 * Parity pins (all in the CPU test suite): published splitmix64 outputs, the
 * paper's rho+ example (Section 3.1), chi-square laws of the index and of
 * rho+, closed-form size() cases, exact ball registers by breadth-first
 * search, the closed-form neighbourhood functions (Section 4 counterexample;
 * paths, cycles, stars, complete digraphs), Theorem 1 / Vysochanskii-Petunin
 * bands over seeds, closed-form distance statistics, Algorithm 3 brackets of
 * exact effective diameters, per-node eccentricity / distance-sum bounds
 * against breadth-first search, per-node statistics of hand-worked E(0..T)
 * sequences, the published FNV-1a-64 test vectors of the register digest, and
 * the threaded per-node sizes summed to exactly ora_sum_sizes' value.
 *
 * Parity unpinned: the spid and effective-diameter values the paper measures
 * on its datasets (Table 2) -- the datasets are absent, so these statistics
 * are pinned only through their definitions on exact distributions.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORA_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------ */
/* Section 3.1: the hash function h.                                   */
/* ------------------------------------------------------------------ */

/* splitmix64 output function: the state is advanced by the golden-ratio
 * increment and then mixed by two xor-shift-multiply rounds. */
ORA_API uint64_t ora_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Seed of run r of a multi-run job. */
ORA_API uint64_t ora_run_seed(uint64_t seed, int32_t r)
{
    return ora_splitmix64(seed + (uint64_t)r);
}

/* Section 3.1: for a hash value h, h_b is the integer made of the leftmost
 * b bits and rho+(h^b) is the number of leading zeroes of the remaining bits
 * plus one.  Written as a bit-by-bit scan so that it can be checked against
 * the definition by eye.  The result is clamped to 31 (five-bit registers). */
ORA_API void ora_place_hash(uint64_t h, int32_t b, int32_t *idx, int32_t *rho)
{
    int32_t i;
    int32_t nrest = 64 - b;
    int32_t r = nrest + 1;             /* all remaining bits are zero */
    *idx = (int32_t)(b == 0 ? 0 : (h >> (64 - b)));
    for (i = 0; i < nrest; ++i) {
        uint64_t bit = (h >> (nrest - 1 - i)) & 1ULL;
        if (bit) { r = i + 1; break; }
    }
    if (r > 31) r = 31;
    *rho = r;
}

/* Placement of item v under seed: register index and value. */
ORA_API void ora_place(uint64_t v, uint64_t seed, int32_t b, int32_t *idx, int32_t *rho)
{
    ora_place_hash(ora_splitmix64(v ^ seed), b, idx, rho);
}

/* ------------------------------------------------------------------ */
/* Algorithm 1: the HyperLogLog counter.                               */
/* ------------------------------------------------------------------ */

/* add(M, x): M[h_b(x)] <- max(M[h_b(x)], rho+(h^b(x))). */
ORA_API void ora_add(uint8_t *M, int32_t b, uint64_t x, uint64_t seed)
{
    int32_t i, r;
    ora_place(x, seed, b, &i, &r);
    if ((int32_t)M[i] < r) M[i] = (uint8_t)r;
}

/* alpha_m: the HyperLogLog bias constants (Flajolet, Fusy, Gandouet, Meunier). */
ORA_API double ora_alpha(int32_t m)
{
    if (m == 16) return 0.673;
    if (m == 32) return 0.697;
    if (m == 64) return 0.709;
    return 0.7213 / (1.0 + 1.079 / (double)m);
}

/* size(M): Z = (sum_j 2^-M[j])^-1, E = alpha_m m^2 Z; if E <= 5m/2 and V,
 * the number of zero registers, is positive, E = m ln(m / V). */
ORA_API double ora_size(const uint8_t *M, int32_t m)
{
    double sum = 0.0, Z, E;
    int32_t j, V = 0;
    for (j = 0; j < m; ++j) {
        sum += ldexp(1.0, -(int)M[j]);
        if (M[j] == 0) ++V;
    }
    Z = 1.0 / sum;
    E = ora_alpha(m) * (double)m * (double)m * Z;
    if (E <= 2.5 * (double)m && V > 0)
        E = (double)m * log((double)m / (double)V);
    return E;
}

/* ------------------------------------------------------------------ */
/* Algorithm 2: HyperANF.                                              */
/* ------------------------------------------------------------------ */

/* Initialisation: every counter starts empty and node v adds itself. */
ORA_API void ora_init(uint8_t *c, int64_t n, int32_t b, uint64_t seed)
{
    int32_t m = 1 << b;
    int64_t v;
    memset(c, 0, (size_t)n * (size_t)m);
    for (v = 0; v < n; ++v)
        ora_add(c + v * m, b, (uint64_t)v, seed);
}

/* One pass of the main loop: for every node v, m <- c[v], then
 * m <- union(c[w], m) for every arc v -> w, and <v, m> goes to the update
 * file (here: c_next).  Returns the number of counters whose value changed.
 * Nodes are independent within a pass (Jacobi), so the node loop may be split
 * across threads, as in the paper's task decomposition, without changing the
 * result. */
ORA_API int64_t ora_union_pass(const int64_t *off, const int32_t *tgt, int64_t n,
                               int32_t m, const uint8_t *c_t, uint8_t *c_next,
                               int32_t threads)
{
    int64_t changed = 0, v;
    (void)threads;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : changed) num_threads(threads > 0 ? threads : 1)
    for (v = 0; v < n; ++v) {
        uint8_t *mv = c_next + v * m;
        int64_t e;
        int32_t i;
        memcpy(mv, c_t + v * m, (size_t)m);
        for (e = off[v]; e < off[v + 1]; ++e) {
            const uint8_t *cw = c_t + (int64_t)tgt[e] * m;
            for (i = 0; i < m; ++i)
                if (cw[i] > mv[i]) mv[i] = cw[i];
        }
        if (memcmp(mv, c_t + v * m, (size_t)m) != 0) ++changed;
    }
    return changed;
}

/* Neumaier-compensated sum of size(c[v]) over all nodes. */
ORA_API double ora_sum_sizes(const uint8_t *c, int64_t n, int32_t m)
{
    double s = 0.0, comp = 0.0;
    int64_t v;
    for (v = 0; v < n; ++v) {
        double x = ora_size(c + v * m, m);
        double t = s + x;
        if (fabs(s) >= fabs(x)) comp += (s - t) + x;
        else comp += (x - t) + s;
        s = t;
    }
    return s + comp;
}

/* size(c[v]) of every node into out[0..n): the nodes are independent, so
 * the loop may be split across threads without changing any value.  With
 * ora_neumaier_sum below it gives exactly ora_sum_sizes' result (same
 * values, same summation order). */
ORA_API void ora_sizes(const uint8_t *c, int64_t n, int32_t m, double *out, int32_t threads)
{
    int64_t v;
    (void)threads;
#pragma omp parallel for schedule(static) num_threads(threads > 0 ? threads : 1)
    for (v = 0; v < n; ++v)
        out[v] = ora_size(c + v * m, m);
}

/* Neumaier-compensated sum of x[0..n), left to right. */
ORA_API double ora_neumaier_sum(const double *x, int64_t n)
{
    double s = 0.0, comp = 0.0;
    int64_t i;
    for (i = 0; i < n; ++i) {
        double t = s + x[i];
        if (fabs(s) >= fabs(x[i])) comp += (s - t) + x[i];
        else comp += (x[i] - t) + s;
        s = t;
    }
    return s + comp;
}

/* ------------------------------------------------------------------ */
/* Register digest (a check value for comparing whole counter arrays;  */
/* not part of the method).                                            */
/* ------------------------------------------------------------------ */

/* FNV-1a, 64-bit (Fowler, Noll, Vo): start from the offset basis; for every
 * byte, xor it into the hash, then multiply by the FNV prime 2^40 + 2^8 +
 * 0xb3, modulo 2^64. */
ORA_API uint64_t ora_fnv1a64(const uint8_t *p, int64_t len)
{
    uint64_t h = 14695981039346656037ULL;
    int64_t i;
    for (i = 0; i < len; ++i) {
        h ^= (uint64_t)p[i];
        h *= 1099511628211ULL;
    }
    return h;
}

/* Digest of the counters of nodes 0..n-1 (m registers each): for node v,
 * FNV-1a-64 of the eight bytes of v (least significant first) followed by
 * the m bytes of c[v]; the digest is the sum of these values modulo 2^64.
 * Addition modulo 2^64 is associative, so the node loop may be split across
 * threads. */
ORA_API uint64_t ora_digest(const uint8_t *c, int64_t n, int32_t m, int32_t threads)
{
    uint64_t total = 0;
    int64_t v;
    (void)threads;
#pragma omp parallel for schedule(static) reduction(+ : total) num_threads(threads > 0 ? threads : 1)
    for (v = 0; v < n; ++v) {
        uint8_t buf[8 + 256];
        int32_t i;
        for (i = 0; i < 8; ++i) buf[i] = (uint8_t)((uint64_t)v >> (8 * i));
        memcpy(buf + 8, c + v * m, (size_t)m);
        total += ora_fnv1a64(buf, 8 + (int64_t)m);
    }
    return total;
}

/* The whole of Algorithm 2 for one run: prints (stores) N(t) before each
 * pass and stops after the first pass that changes no counter.  N_out gets
 * N(0..T); *T_out = T.  Returns 0, or -1 if cap values are not enough (the
 * registers then hold the state after the last completed pass).  If regs is
 * not NULL it receives the final counters (n*m bytes). */
ORA_API int32_t ora_hyperanf(const int64_t *off, const int32_t *tgt, int64_t n,
                             int32_t b, uint64_t seed, double *N_out, int32_t cap,
                             int32_t *T_out, uint8_t *regs, int32_t threads)
{
    int32_t m = 1 << b, t = 0;
    size_t bytes = (size_t)n * (size_t)m;
    uint8_t *c = (uint8_t *)malloc(bytes ? bytes : 1);
    uint8_t *cn = (uint8_t *)malloc(bytes ? bytes : 1);
    int32_t rc = 0;
    if (!c || !cn) { free(c); free(cn); return -2; }
    ora_init(c, n, b, seed);
    for (;;) {
        int64_t changed;
        uint8_t *tmp;
        if (t >= cap) { rc = -1; break; }
        N_out[t] = ora_sum_sizes(c, n, m);
        changed = ora_union_pass(off, tgt, n, m, c, cn, threads);
        tmp = c; c = cn; cn = tmp;           /* read the update file */
        if (changed == 0) break;
        ++t;
    }
    *T_out = t;
    if (regs) memcpy(regs, c, bytes);
    free(c);
    free(cn);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Exact references by breadth-first search (pins, not the method).    */
/* ------------------------------------------------------------------ */

/* Exact neighbourhood function: N_out[t] = #{(x, y) : d(x, y) <= t} for
 * t = 0..cap-1 (saturating at the largest distance).  Returns the largest
 * finite distance D, or -1 if cap <= D. */
ORA_API int32_t ora_exact_nf(const int64_t *off, const int32_t *tgt, int64_t n,
                             int64_t *N_out, int32_t cap)
{
    int32_t *dist = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    int64_t *queue = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    int64_t *cnt = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    int32_t D = 0, t;
    int64_t x;
    for (x = 0; x < n; ++x) {
        int64_t head = 0, tail = 0, i;
        for (i = 0; i < n; ++i) dist[i] = -1;
        dist[x] = 0;
        queue[tail++] = x;
        while (head < tail) {
            int64_t u = queue[head++], e;
            cnt[dist[u]]++;
            if (dist[u] > D) D = dist[u];
            for (e = off[u]; e < off[u + 1]; ++e) {
                int32_t w = tgt[e];
                if (dist[w] < 0) { dist[w] = dist[u] + 1; queue[tail++] = w; }
            }
        }
    }
    {
        int64_t acc = 0;
        for (t = 0; t < cap; ++t) {
            if (t <= n) acc += cnt[t];
            N_out[t] = acc;
        }
    }
    free(dist); free(queue); free(cnt);
    return cap <= D ? -1 : D;
}

/* Registers of the ball B(v, r): the maximum, register by register, of the
 * singleton counters of all nodes at distance <= r from v (r < 0: the whole
 * reachable set).  This is what c[v] must hold after r passes. */
ORA_API void ora_ball_registers(const int64_t *off, const int32_t *tgt, int64_t n,
                                int64_t v, int32_t r, int32_t b, uint64_t seed,
                                uint8_t *out)
{
    int32_t m = 1 << b;
    int32_t *dist = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int64_t *queue = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t head = 0, tail = 0, i;
    memset(out, 0, (size_t)m);
    for (i = 0; i < n; ++i) dist[i] = -1;
    dist[v] = 0;
    queue[tail++] = v;
    while (head < tail) {
        int64_t u = queue[head++], e;
        ora_add(out, b, (uint64_t)u, seed);
        if (r >= 0 && dist[u] >= r) continue;
        for (e = off[u]; e < off[u + 1]; ++e) {
            int32_t w = tgt[e];
            if (dist[w] < 0) { dist[w] = dist[u] + 1; queue[tail++] = w; }
        }
    }
    free(dist);
    free(queue);
}

/* Final sum N(T) of a symmetric graph (every arc u->w has w->u): the ball
 * of v at stabilisation is v's connected component, so c_T[v] is the
 * register-wise maximum of the singleton counters of the component.  The
 * components are found by breadth-first search; the result is the
 * Neumaier-compensated sum of size(c_T[v]) over v = 0..n-1, the same sum
 * Algorithm 2 prints last.  Returns -1.0 on allocation failure. */
ORA_API double ora_symmetric_final_sum(const int64_t *off, const int32_t *tgt, int64_t n,
                                              int32_t b, uint64_t seed)
{
    int32_t m = 1 << b;
    int64_t *comp = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    int64_t *queue = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    uint8_t *creg = NULL;
    double *csize = NULL;
    int64_t ncomp = 0, v;
    double s = 0.0, c = 0.0;
    if (!comp || !queue) { free(comp); free(queue); return -1.0; }
    for (v = 0; v < n; ++v) comp[v] = -1;
    for (v = 0; v < n; ++v) {
        int64_t head = 0, tail = 0;
        if (comp[v] >= 0) continue;
        comp[v] = ncomp;
        queue[tail++] = v;
        while (head < tail) {
            int64_t u = queue[head++], e;
            for (e = off[u]; e < off[u + 1]; ++e) {
                int32_t w = tgt[e];
                if (comp[w] < 0) { comp[w] = ncomp; queue[tail++] = w; }
            }
        }
        ++ncomp;
    }
    creg = (uint8_t *)calloc((size_t)(ncomp ? ncomp : 1) * (size_t)m, 1);
    csize = (double *)malloc((size_t)(ncomp ? ncomp : 1) * sizeof(double));
    if (!creg || !csize) { free(comp); free(queue); free(creg); free(csize); return -1.0; }
    for (v = 0; v < n; ++v) ora_add(creg + comp[v] * m, b, (uint64_t)v, seed);
    for (v = 0; v < ncomp; ++v) csize[v] = ora_size(creg + v * m, m);
    for (v = 0; v < n; ++v) {
        double x = csize[comp[v]], t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    free(comp); free(queue); free(creg); free(csize);
    return s + c;
}

/* ------------------------------------------------------------------ */
/* Section 4 and Section 5: statistics read off N(0..T).               */
/* ------------------------------------------------------------------ */

/* out[0] = effective diameter at alpha (smallest t with H(t) >= alpha),
 * out[1] = interpolated effective diameter (linear interpolation of H between
 * t*-1 and t*), out[2] = mean distance sum_t t h(t), out[3] = variance
 * sum_t t^2 h(t) - mean^2, out[4] = spid = variance / mean, with
 * H(t) = N(t) / max_t N(t) and h(t) = H(t) - H(t-1), H(-1) = 0.  With
 * exclude_zero the pairs (x, x) are left out: N(0) is subtracted from every
 * value before normalising. */
ORA_API void ora_stats(const double *N, int32_t T, double alpha, int32_t exclude_zero,
                       double *out)
{
    double M = -INFINITY, base = exclude_zero ? N[0] : 0.0;
    double prevH = 0.0, mean = 0.0, sq = 0.0;
    int32_t t, tstar = -1;
    for (t = 0; t <= T; ++t)
        if (N[t] > M) M = N[t];
    for (t = 0; t <= T; ++t) {
        double H = (N[t] - base) / (M - base);
        double h = H - prevH;
        mean += (double)t * h;
        sq += (double)t * (double)t * h;
        if (tstar < 0 && H >= alpha) {
            tstar = t;
            out[0] = (double)t;
            out[1] = t == 0 ? 0.0 : (double)(t - 1) + (alpha - prevH) / (H - prevH);
        }
        prevH = H;
    }
    if (tstar < 0) { out[0] = NAN; out[1] = NAN; }
    out[2] = mean;
    out[3] = sq - mean * mean;
    out[4] = out[3] / mean;
}

/* Algorithm 3 (Section 4): M = max_t N(t); D- is the largest t with
 * N(t)/M <= alpha(1-2 eps), D+ the smallest t with N(t)/M >= alpha(1+2 eps);
 * -1 when there is none. */
ORA_API void ora_ed_interval(const double *N, int32_t T, double alpha, double eps, int32_t *lo,
                             int32_t *hi)
{
    double M = -INFINITY;
    int32_t t;
    *lo = -1;
    *hi = -1;
    for (t = 0; t <= T; ++t)
        if (N[t] > M) M = N[t];
    for (t = T; t >= 0; --t)
        if (N[t] / M <= alpha * (1.0 - 2.0 * eps)) { *lo = t; break; }
    for (t = 0; t <= T; ++t)
        if (N[t] / M >= alpha * (1.0 + 2.0 * eps)) { *hi = t; break; }
}

/* Statistics of one node's estimates E(0..T) = size(c_t[v]), t = 0..T, of
 * one run of Algorithm 2 (the radius distribution and closeness centrality
 * proposed in the paper's conclusion): reach = E(T); dist = sum over
 * t = 1..T of t (E(t) - E(t-1)); ecc = the last t with E(t) != E(t-1) (0 if
 * none); rad = the first t with E(t) >= alpha E(T). */
ORA_API void ora_seq_stats(const double *E, int32_t T, double alpha, double *reach,
                           double *dist, int32_t *ecc, int32_t *rad)
{
    double s = 0.0, last = E[T];
    int32_t t, e = 0, r = -1;
    for (t = 0; t <= T; ++t) {
        if (t > 0 && E[t] != E[t - 1]) {
            s = s + (double)t * (E[t] - E[t - 1]);
            e = t;
        }
        if (r < 0 && E[t] >= alpha * last) r = t;
    }
    *reach = last;
    *dist = s;
    *ecc = e;
    *rad = r;
}

/* Per-node statistics (ora_seq_stats) of every node of one run of Algorithm
 * 2.  Keeps every E_v(t): for small graphs.  Returns T, or -1 if cap passes
 * were not enough, -2 on allocation failure. */
ORA_API int32_t ora_node_stats(const int64_t *off, const int32_t *tgt, int64_t n, int32_t b,
                               uint64_t seed, double alpha, int32_t cap, double *reach,
                               double *dist, int32_t *ecc, int32_t *rad)
{
    int32_t m = 1 << b, t, T = -1;
    size_t bytes = (size_t)(n ? n : 1) * (size_t)m;
    uint8_t *c = (uint8_t *)malloc(bytes), *cn = (uint8_t *)malloc(bytes);
    double *E = (double *)malloc(sizeof(double) * (size_t)cap * (size_t)(n ? n : 1));
    double *seq = (double *)malloc(sizeof(double) * (size_t)cap);
    int64_t v;
    if (!c || !cn || !E || !seq) { free(c); free(cn); free(E); free(seq); return -2; }
    ora_init(c, n, b, seed);
    for (t = 0; t < cap; ++t) {
        int64_t changed;
        uint8_t *tmp;
        for (v = 0; v < n; ++v) E[(size_t)t * n + v] = ora_size(c + v * m, m);
        changed = ora_union_pass(off, tgt, n, m, c, cn, 1);
        tmp = c; c = cn; cn = tmp;
        if (changed == 0) { T = t; break; }
    }
    if (T >= 0) {
        for (v = 0; v < n; ++v) {
            for (t = 0; t <= T; ++t) seq[t] = E[(size_t)t * n + v];
            ora_seq_stats(seq, T, alpha, reach + v, dist + v, ecc + v, rad + v);
        }
    }
    free(c); free(cn); free(E); free(seq);
    return T;
}
