"""Pins of the CPU oracle against facts fixed outside of it.

Each test checks the oracle against something the paper or mathematics fixes:
published hash outputs, the paper's rho+ example, distribution laws of the
register placement, closed-form size() values, exact ball registers from
breadth-first search, closed-form neighbourhood functions (Section 4 and
textbook graphs), Theorem 1 / Vysochanskii-Petunin error bands over seeds,
and closed-form distance statistics.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats as sps

from paper_1011_5599_gb300 import graphs as G

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SEED = 0x5EED


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- hash


def test_splitmix64_published_outputs(oracle):
    for x, out in _golden("splitmix64.txt"):
        assert oracle.splitmix64(int(x, 16)) == int(out, 16)


def test_rho_plus_paper_example(oracle):
    for bits, rho in _golden("rho_example.txt"):
        for b in (0, 4, 6, 8):
            idx = (0b1011 << 60) >> (64 - b) if b else 0
            # place w right after the b index bits, rest zero
            h = (idx << (64 - b) if b else 0) | (int(bits, 2) << (64 - b - len(bits)))
            got_idx, got_rho = oracle.place_hash(h, b)
            assert got_idx == idx
            assert got_rho == int(rho)


def test_rho_plus_all_zero_rest_and_clamp(oracle):
    # all 64-b remaining bits zero: rho+ = 64-b+1, clamped to 31
    for b in (4, 6, 8):
        assert oracle.place_hash(0, b) == (0, 31)
    # a one at the 31st remaining position gives exactly 31, the 32nd clamps
    b = 4
    assert oracle.place_hash(1 << (64 - b - 31), b)[1] == 31
    assert oracle.place_hash(1 << (64 - b - 30), b)[1] == 30
    assert oracle.place_hash(1 << (64 - b - 32), b)[1] == 31


def test_seed_enters_by_xor(oracle):
    """h(v) = splitmix64(v XOR seed): the placement of v under seed s is the
    placement of v XOR s under seed 0, and the hash of 0 under seed 0 is the
    first published splitmix64 output."""
    rng = __import__("random").Random(3)
    for _ in range(300):
        v, s = rng.getrandbits(31), rng.getrandbits(64)
        for b in (4, 8):
            assert oracle.place(v, s, b) == oracle.place(v ^ s, 0, b)
    assert oracle.place(0, 0, 4) == oracle.place_hash(0xE220A8397B1DCDAF, 4)


def test_run_seeds_differ_from_shifted_seeds(oracle):
    s = [oracle.run_seed(SEED, r) for r in range(8)]
    assert len(set(s)) == 8
    assert s[0] == oracle.splitmix64(SEED)


@pytest.mark.parametrize("b", [4, 6, 8])
def test_placement_laws(oracle, b):
    """Index uniform over m registers; P(rho+ = k) = 2^-k (chi-square)."""
    n = 1 << 18
    m = 1 << b
    c = oracle.init(n, b, oracle.run_seed(SEED, b))
    assert np.all((c != 0).sum(axis=1) == 1)      # exactly one register set
    idx = c.argmax(axis=1)
    rho = c.max(axis=1).astype(np.int64)
    cnt = np.bincount(idx, minlength=m)
    assert sps.chisquare(cnt).pvalue > 1e-4
    kmax = 12
    obs = np.array([(rho == k).sum() for k in range(1, kmax)] + [(rho >= kmax).sum()])
    p = np.array([2.0 ** -k for k in range(1, kmax)] + [2.0 ** -(kmax - 1)])
    assert sps.chisquare(obs, p * n).pvalue > 1e-4


# ---------------------------------------------------------------- size()


def test_alpha_published_constants(oracle):
    assert oracle.alpha(16) == 0.673
    assert oracle.alpha(32) == 0.697
    assert oracle.alpha(64) == 0.709
    for m in (128, 256):
        assert oracle.alpha(m) == 0.7213 / (1 + 1.079 / m)


@pytest.mark.parametrize("b", [4, 5, 6, 7, 8])
def test_size_closed_forms(oracle, b):
    m = 1 << b
    a = oracle.alpha(m)
    # empty counter: V = m, linear counting gives m ln 1 = 0
    assert oracle.size(np.zeros(m, np.uint8)) == 0.0
    # one register set: raw estimate below 5m/2, V = m-1
    for k in (1, 5, 31):
        M = np.zeros(m, np.uint8)
        M[m // 3] = k
        assert oracle.size(M) == pytest.approx(m * math.log(m / (m - 1)), rel=1e-15)
    # all registers equal k >= 1: V = 0, E = alpha m^2 / (m 2^-k)
    for k in range(1, 32):
        M = np.full(m, k, np.uint8)
        assert oracle.size(M) == pytest.approx(a * m * 2.0 ** k, rel=1e-15)
    # half the registers 0, half 2: raw = a m^2 / (m/2 + m/8) <= 5m/2 -> LC
    M = np.zeros(m, np.uint8)
    M[: m // 2] = 2
    raw = a * m * m / (m / 2 + m / 8)
    assert raw <= 2.5 * m
    assert oracle.size(M) == pytest.approx(m * math.log(2.0), rel=1e-15)


@pytest.mark.parametrize("b,card", [(6, 1000), (8, 5000), (4, 300)])
def test_size_estimates_cardinality(oracle, b, card):
    """HyperLogLog: relative error of a single counter within the standard
    error 1.06/sqrt(m) on average over independent seeds (Section 3.1)."""
    m = 1 << b
    eta = 1.06 / math.sqrt(m)
    S = 300
    # one counter fed with `card` items = the ball registers of a star centre
    off, tgt = G.star(card)
    est = np.array([oracle.size(oracle.ball_registers(off, tgt, 0, 1, b, oracle.run_seed(SEED, s)))
                    for s in range(S)])
    rel = est / card
    assert abs(rel.mean() - 1) < 3 * eta / math.sqrt(S) + 0.01
    assert rel.std() < 1.25 * eta


# ---------------------------------------------------------------- union / Algorithm 2


def _iterate(oracle, off, tgt, b, seed, passes):
    n = off.size - 1
    c = oracle.init(n, b, seed)
    out = [c]
    for _ in range(passes):
        c, _ = oracle.union_pass(off, tgt, c)
        out.append(c)
    return out


@pytest.mark.parametrize("gseed", [1, 2, 3])
def test_counters_equal_ball_registers(oracle, gseed):
    """c_t[v] is exactly the counter of the ball B(v, t) (Section 3.2):
    checked against breadth-first search, register by register."""
    n = 120
    off, tgt = G.er(n, 180 + 40 * gseed, seed=gseed)
    b = 5
    seed = oracle.run_seed(SEED, gseed)
    cs = _iterate(oracle, off, tgt, b, seed, 12)
    for t in (0, 1, 2, 3, 5, 8, 12):
        for v in range(n):
            ball = oracle.ball_registers(off, tgt, v, t, b, seed)
            assert np.array_equal(cs[t][v], ball), (t, v)
    # final counters are the reachable-set counters
    _, T, regs = oracle.hyperanf(off, tgt, b, seed, want_regs=True)
    for v in range(n):
        assert np.array_equal(regs[v], oracle.ball_registers(off, tgt, v, -1, b, seed))


def test_union_includes_own_counter(oracle):
    """A node without successors keeps its own item (m <- c[v] first)."""
    off, tgt = G.path(2)
    c = oracle.init(2, 4, SEED)
    cn, ch = oracle.union_pass(off, tgt, c)
    assert np.array_equal(cn[1], c[1])
    assert np.array_equal(cn[0], np.maximum(c[0], c[1]))


def test_jacobi_not_in_place(oracle):
    """Every counter of pass t+1 is built from the counters of pass t: on the
    path 0->1->2 node 0 must not see node 2 after one pass."""
    off, tgt = G.path(3)
    for s in range(50):
        c = oracle.init(3, 8, oracle.run_seed(SEED, s))
        cn, _ = oracle.union_pass(off, tgt, c)
        assert np.array_equal(cn[0], np.maximum(c[0], c[1]))


def test_registers_monotone_and_fixed_point(oracle):
    off, tgt = G.er(300, 900, seed=5)
    b = 6
    _, T, regs = oracle.hyperanf(off, tgt, b, SEED, want_regs=True)
    cs = _iterate(oracle, off, tgt, b, SEED, T + 1)
    for t in range(T + 1):
        assert np.all(cs[t + 1] >= cs[t])
    assert np.array_equal(cs[T + 1], cs[T])      # the stopping pass changes nothing
    assert np.array_equal(cs[T], regs)
    if T > 0:
        assert not np.array_equal(cs[T], cs[T - 1])
    D = oracle.exact_nf(off, tgt).size - 1
    assert T <= D


def test_empty_and_arcless_graphs(oracle):
    off, tgt = G.empty(0)
    N, T, _ = oracle.hyperanf(off, tgt, 4, SEED)
    assert T == 0 and N[0] == 0.0
    off, tgt = G.empty(50)
    N, T, regs = oracle.hyperanf(off, tgt, 6, SEED, want_regs=True)
    assert T == 0
    assert N[0] == pytest.approx(sum(oracle.size(r) for r in regs), rel=1e-14)


# ---------------------------------------------------------------- exact references


def _path_nf(n, t):
    return sum(n - j for j in range(0, min(t, n - 1) + 1))


def test_exact_nf_closed_forms(oracle):
    for n in (1, 2, 7, 20):
        got = oracle.exact_nf(*G.path(n))
        assert list(got) == [_path_nf(n, t) for t in range(n)]
    for n in (3, 9):
        got = oracle.exact_nf(*G.cycle(n))
        assert list(got) == [n * min(t + 1, n) for t in range(n)]
    for n in (4, 11):
        got = oracle.exact_nf(*G.star(n))
        assert list(got) == [n, 3 * n - 2, n * n]
    for n in (2, 6):
        got = oracle.exact_nf(*G.complete(n))
        assert list(got) == [n, n * n]


def clique_path_nf(k, l, t):
    """Closed form of N_G(t) for two k-cliques joined by a one-way path of l
    nodes (Section 4)."""
    if t == 0:
        return 2 * k + l
    if t <= l:
        return (t + 1) * (2 * k + l - t / 2) - 2 * k + 2 * k * k
    return (l + 1) * (2 * k + l / 2) - 2 * k + 3 * k * k


@pytest.mark.parametrize("k,l", [(5, 3), (7, 4), (3, 1), (20, 2), (35, 3)])
def test_clique_path_closed_form(oracle, k, l):
    got = oracle.exact_nf(*G.clique_path(k, l))
    assert got.size == l + 2
    for t in range(l + 3):
        assert got[min(t, l + 1)] == clique_path_nf(k, l, t)


@pytest.mark.parametrize("l", [2, 3])
def test_clique_path_stabilisation_and_effective_diameter(oracle, l):
    """With k = 2l^2+5l+2 the effective diameter is l+1; stopping one pass
    early reports 1 (Section 4).  HyperANF stops exactly at T = l+1."""
    k = 2 * l * l + 5 * l + 2
    off, tgt = G.clique_path(k, l)
    exact = np.array([clique_path_nf(k, l, t) for t in range(l + 2)], dtype=np.float64)
    assert oracle.stats(exact)["ed"] == l + 1
    assert oracle.stats(exact[: l + 1])["ed"] == 1
    for s in range(20):
        N, T, _ = oracle.hyperanf(off, tgt, 8, oracle.run_seed(SEED, s))
        assert T == l + 1


# ---------------------------------------------------------------- Theorem 1 bands


@pytest.mark.parametrize("name,b", [("er", 6), ("er", 8), ("star", 6), ("cycle", 8)])
def test_theorem1_error_bands(oracle, name, b):
    """N^(t)/N(t): almost unbiased; relative error within k*eta_m with
    frequency at least 1 - 4/(9k^2) (Vysochanskii-Petunin, Section 3.4)."""
    if name == "er":
        off, tgt = G.er(400, 1200, seed=11)
    elif name == "star":
        off, tgt = G.star(500)
    else:
        off, tgt = G.cycle(200)
    exact = oracle.exact_nf(off, tgt).astype(np.float64)
    m = 1 << b
    eta = 1.06 / math.sqrt(m)
    S = 200
    rel = []
    for s in range(S):
        N, T, _ = oracle.hyperanf(off, tgt, b, oracle.run_seed(1000, s))
        full = np.array([N[min(t, T)] for t in range(exact.size)])
        rel.append(full / exact)
    rel = np.array(rel)
    for k in (2, 3):
        frac = np.mean(np.abs(rel - 1) < k * eta)
        assert frac >= 1 - 4 / (9 * k * k)
    mean = rel.mean(axis=0)
    assert np.all(np.abs(mean - 1) < 3 * eta / math.sqrt(S) + 0.01)


# ---------------------------------------------------------------- statistics


@pytest.mark.parametrize("n", [2, 5, 12, 40])
def test_stats_path_closed_form(oracle, n):
    """On the directed path of n nodes n-d pairs lie at distance d, so the
    distance distribution has mean (n-1)/3, variance (n-1)(n+2)/18 and spid
    (n+2)/6 (pairs at distance 0 included)."""
    N = np.array([_path_nf(n, t) for t in range(n)], dtype=np.float64)
    s = oracle.stats(N)
    assert s["mean"] == pytest.approx((n - 1) / 3, rel=1e-12)
    assert s["var"] == pytest.approx((n - 1) * (n + 2) / 18, rel=1e-12)
    assert s["spid"] == pytest.approx((n + 2) / 6, rel=1e-12)
    M = n * (n + 1) / 2
    tstar = next(t for t in range(n) if N[t] / M >= 0.9)
    assert s["ed"] == tstar
    if tstar > 0:
        lo, hi = N[tstar - 1] / M, N[tstar] / M
        assert s["ied"] == pytest.approx(tstar - 1 + (0.9 - lo) / (hi - lo), rel=1e-12)


def test_stats_exclude_zero(oracle):
    """Distances between distinct nodes only: on the path of n nodes,
    n-d pairs at distance d >= 1 give mean (n+1)/3."""
    n = 10
    N = np.array([_path_nf(n, t) for t in range(n)], dtype=np.float64)
    s = oracle.stats(N, exclude_zero=True)
    assert s["mean"] == pytest.approx((n + 1) / 3, rel=1e-12)


def test_stats_star_and_complete(oracle):
    # complete digraph: n pairs at 0, n(n-1) at 1: mean (n-1)/n
    n = 9
    s = oracle.stats(np.array([n, n * n], dtype=np.float64))
    assert s["mean"] == pytest.approx((n - 1) / n)
    assert s["var"] == pytest.approx((n - 1) / n - ((n - 1) / n) ** 2)
    assert s["ed"] == 1
    # all mass at t = 0: effective diameter 0
    s = oracle.stats(np.array([5.0]))
    assert s["ed"] == 0 and s["ied"] == 0 and s["mean"] == 0


@pytest.mark.parametrize("name", ["star", "grid", "er_sym", "two_components"])
def test_symmetric_final_sum_equals_algorithm2(oracle, name):
    """On a symmetric graph the stabilised counters are component unions, so
    the component-based sum equals N(T) of the iteration."""
    if name == "star":
        off, tgt = G.star(50)
    elif name == "grid":
        off, tgt = G.grid2d(12)
    elif name == "er_sym":
        o, t = G.er(200, 300, seed=4)
        src = np.repeat(np.arange(200), np.diff(o))
        off, tgt = G.csr_from_arcs(np.concatenate([src, t]), np.concatenate([t, src]), 200)
    else:
        a, b = G.cycle(30), G.star(20)
        src = np.concatenate([np.repeat(np.arange(30), np.diff(a[0])),
                              30 + np.repeat(np.arange(20), np.diff(b[0]))])
        dst = np.concatenate([a[1], 30 + b[1]])
        src, dst = np.concatenate([src, dst]), np.concatenate([dst, src])
        off, tgt = G.csr_from_arcs(src, dst, 50)
    for s in range(5):
        seed = oracle.run_seed(SEED, s)
        N, T, _ = oracle.hyperanf(off, tgt, 6, seed)
        assert oracle.symmetric_final_sum(off, tgt, 6, seed) == pytest.approx(N[-1], rel=1e-14)


# ---------------------------------------------------------------- Algorithm 3


@pytest.mark.parametrize("n", [5, 12, 40])
def test_ed_interval_exact_bracket(oracle, n):
    """With exact N (eps = 0) Algorithm 3's upper end is the effective
    diameter and the lower end the last t below alpha; a positive eps can only
    widen the bracket."""
    N = np.array([_path_nf(n, t) for t in range(n)], dtype=np.float64)
    ed = oracle.stats(N)["ed"]
    lo, hi = oracle.ed_interval(N, 0.9, 0.0)
    assert hi == ed
    M = N.max()
    assert lo == max(t for t in range(n) if N[t] / M <= 0.9)
    lo2, hi2 = oracle.ed_interval(N, 0.9, 0.02)
    assert lo2 <= lo and (hi2 >= hi or hi2 == -1)


@pytest.mark.parametrize("l", [2, 3])
def test_ed_interval_clique_path(oracle, l):
    """Section 4's graph: the bracket of the exact distribution is [l, l+1];
    stopping one pass early puts the whole bracket at 1 or below."""
    k = 2 * l * l + 5 * l + 2
    exact = np.array([clique_path_nf(k, l, t) for t in range(l + 2)], dtype=np.float64)
    assert oracle.ed_interval(exact, 0.9, 0.0) == (l, l + 1)
    lo, hi = oracle.ed_interval(exact[: l + 1], 0.9, 0.0)
    assert hi == 1


def test_stats_runs_matches_per_run(oracle):
    off, tgt = G.er(300, 900, seed=3)
    runs = [oracle.hyperanf(off, tgt, 6, oracle.run_seed(SEED, r))[0] for r in range(6)]
    agg = oracle.stats_runs(runs)
    spids = [oracle.stats(N)["spid"] for N in runs]
    assert agg["spid"][0] == pytest.approx(np.mean(spids))
    assert agg["spid"][1] == pytest.approx(np.std(spids, ddof=1))


# ---------------------------------------------------------------- per-node statistics


def test_node_eccentricity_never_exceeds_the_true_one(oracle):
    """A counter can only change while its ball still grows, so the estimated
    eccentricity is at most the exact one.  The last step often adds a node or
    two whose hashes raise no register, so the two agree only part of the time."""
    off, tgt = G.er(200, 500, seed=8)
    reach, dsum, ecc = oracle.exact_node_distances(off, tgt)
    agree = 0
    for s in range(5):
        st = oracle.node_stats(off, tgt, 8, oracle.run_seed(SEED, s))
        assert np.all(st["ecc"] <= ecc)
        agree += np.mean(st["ecc"] == ecc)
    assert agree / 5 > 0.5


def test_node_distance_sums_estimate_the_exact_ones(oracle):
    """Averaged over seeds, reach and distance sums are within the
    HyperLogLog error of the exact BFS values; the effective radius of the
    path's first node is the smallest t covering 90% of its n nodes."""
    off, tgt = G.er(300, 1200, seed=9)
    reach, dsum, ecc = oracle.exact_node_distances(off, tgt)
    S = 40
    r_est = np.zeros(reach.size)
    d_est = np.zeros(reach.size)
    for s in range(S):
        st = oracle.node_stats(off, tgt, 8, oracle.run_seed(SEED, s))
        r_est += st["reach"] / S
        d_est += st["dist"] / S
    eta = 1.06 / 16
    live = reach > 50
    assert abs(np.mean(r_est[live] / reach[live]) - 1) < 3 * eta / np.sqrt(S) + 0.01
    assert abs(np.mean(d_est[live] / dsum[live]) - 1) < 3 * eta / np.sqrt(S) + 0.03
    # path of n nodes, node 0: ball of radius t holds t+1 nodes exactly
    n = 30
    rad = np.array([oracle.node_stats(*G.path(n), 8, oracle.run_seed(SEED, s))["radius"][0]
                    for s in range(20)])
    assert abs(np.median(rad) - (int(np.ceil(0.9 * n)) - 1)) <= 2


# ---------------------------------------------------------------- check values and helpers


def test_fnv1a64_published_vectors(oracle):
    for text, out in _golden("fnv1a64.txt"):
        assert oracle.fnv1a64(text.strip('"').encode()) == int(out, 16)


def test_digest_definition_and_sensitivity(oracle):
    """digest = sum over v of FNV-1a-64(8 little-endian bytes of v, then the
    row), modulo 2^64; it sees any single register change and any swap of two
    rows, and does not depend on the thread count."""
    rng = np.random.default_rng(4)
    for m in (16, 64, 256):
        c = rng.integers(0, 32, (37, m)).astype(np.uint8)
        want = sum(oracle.fnv1a64(v.to_bytes(8, "little") + c[v].tobytes())
                   for v in range(c.shape[0])) % 2**64
        assert oracle.digest(c, threads=1) == want
        assert oracle.digest(c, threads=3) == want
        for v, j in ((0, 0), (36, m - 1), (17, m // 2)):
            d = c.copy()
            d[v, j] ^= 1
            assert oracle.digest(d) != want
        d = c.copy()
        d[[3, 4]] = d[[4, 3]]
        assert not np.array_equal(d, c) and oracle.digest(d) != want
    assert oracle.digest(np.zeros((0, 16), np.uint8)) == 0


def test_parallel_sizes_equal_sum_sizes(oracle):
    """The per-node sizes computed on several threads, summed by the
    Neumaier loop, give exactly ora_sum_sizes' value."""
    rng = np.random.default_rng(8)
    for b in (4, 6, 8):
        c = np.minimum(rng.geometric(0.5, (3001, 1 << b)) - 1, 31).astype(np.uint8)
        c[::7] = 0                                  # empty counters: linear counting
        x = oracle.sizes(c, threads=4)
        assert x.shape == (3001,)
        assert x[5] == oracle.size(c[5]) and x[0] == oracle.size(c[0]) and x[-1] == oracle.size(c[-1])
        assert oracle.neumaier_sum(x) == oracle.sum_sizes(c)
        assert oracle.sum_sizes_mt(c, threads=3) == oracle.sum_sizes(c)


def test_neumaier_sum_is_compensated(oracle):
    # plain left-to-right summation gives 0 and 1 here; the exact sums are 1 and 2
    assert oracle.neumaier_sum([1e16, 1.0, -1e16]) == 1.0
    assert oracle.neumaier_sum([1.0, 1e100, 1.0, -1e100]) == 2.0
    x = np.random.default_rng(1).standard_normal(10000) * 1e6
    assert oracle.neumaier_sum(x) == pytest.approx(math.fsum(x), rel=0, abs=1e-6)


# (E(0..T), alpha) -> reach, distance sum, eccentricity, effective radius,
# each worked out by hand from the definitions
SEQUENCES = [
    ([1.0, 3.0, 3.0, 7.0, 10.0], 0.9, 10.0, 1 * 2 + 3 * 4 + 4 * 3, 4, 4),
    ([1.0, 5.0, 9.0, 9.0], 0.9, 9.0, 1 * 4 + 2 * 4, 2, 2),
    ([2.0, 5.0, 10.0], 0.5, 10.0, 1 * 3 + 2 * 5, 2, 1),      # E(1) = alpha E(T) exactly
    ([1.0], 0.9, 1.0, 0.0, 0, 0),
    ([4.0, 4.0, 4.0], 0.9, 4.0, 0.0, 0, 0),
    ([1.0, 2.0, 2.0, 2.0, 3.0, 3.0], 0.6, 3.0, 1 * 1 + 4 * 1, 4, 1),
]


@pytest.mark.parametrize("E,alpha_,reach,dist,ecc,rad", SEQUENCES)
def test_per_node_statistics_of_hand_written_sequences(oracle, E, alpha_, reach, dist, ecc, rad):
    got = oracle.seq_stats(E, alpha_)
    assert got == {"reach": reach, "dist": dist, "ecc": ecc, "radius": rad}
