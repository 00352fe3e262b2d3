"""CUDA path vs the CPU oracle, through the C ABI, on seeded inputs.

The bar: registers bit-exact (after every pass and at stabilisation), the
stopping pass T identical, and N(t) within 1e-12 relative.  Cases cover the
smallest workload (directed ER, n = 10^4, 5*10^4 arcs, m = 16), every
register count m = 16..256, every frontier policy, all three degree classes
(lane group per node, warp per node, hub segments), R-run batching, the
CUDA-graph driver, ragged and degenerate graphs, and invalid input.
"""
import numpy as np
import pytest

from paper_1011_5599_gb300 import graphs as G

pytestmark = pytest.mark.gpu

SEED = 0x5EED
RTOL = 1e-12


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1011_5599_gb300 import build as B
    B.build()
    import paper_1011_5599_gb300.hanf as H
    return H


def check_run(H, O, off, tgt, log2m, seed=SEED, R=1, threads=4, **kw):
    with H.HyperANF(off, tgt, log2m, seed, runs=R, **kw) as h:
        N, T = h.run()
        regs = [h.registers(r) for r in range(R)]
        cnt = h.counters()
    for r in range(R):
        No, To, ro = O.hyperanf(off, tgt, log2m, O.run_seed(seed, r), want_regs=True,
                                threads=threads)
        assert T[r] == To, f"run {r}: T={T[r]} oracle {To}"
        assert np.array_equal(regs[r], ro), f"run {r}: registers differ"
        np.testing.assert_allclose(N[r], No, rtol=RTOL, atol=0)
    return N, T, cnt


def test_smallest_workload_er_m16(H, oracle):
    """Directed ER n=10,000, 50,000 distinct arcs, m=16, one run."""
    off, tgt = G.er(10000, 50000, seed=1)
    for frontier in ("off", "pull", "auto"):
        check_run(H, oracle, off, tgt, 4, frontier=frontier)


@pytest.mark.parametrize("log2m", [4, 5, 6, 7, 8])
@pytest.mark.parametrize("frontier", ["off", "pull", "auto"])
def test_er_every_m_and_frontier(H, oracle, log2m, frontier):
    off, tgt = G.er(3000, 12000, seed=log2m)
    check_run(H, oracle, off, tgt, log2m, frontier=frontier)


def test_every_pass_bit_exact(H, oracle):
    """Step by step: registers and N(t) after every pass."""
    off, tgt = G.web(1 << 13, seed=2)
    log2m = 6
    seed = SEED
    c = oracle.init(off.size - 1, log2m, oracle.run_seed(seed, 0))
    with H.HyperANF(off, tgt, log2m, seed) as h:
        t = 0
        while True:
            assert h.t == t
            assert np.array_equal(h.registers(0), c), f"t={t}"
            np.testing.assert_allclose(h.estimate()[0], oracle.sum_sizes(c), rtol=RTOL)
            changed = h.iterate()
            c_next, ch_o = oracle.union_pass(off, tgt, c)
            assert changed == ch_o, f"t={t}: changed {changed} vs {ch_o}"
            if changed == 0:
                assert np.array_equal(h.registers(0), c_next)
                break
            c = c_next
            t += 1
        assert h.iterate() == 0          # stable: further calls are no-ops


@pytest.mark.parametrize("small,hub", [(1, 2), (1, 4), (2, 8), (4096, 1 << 20), (1, 1 << 20),
                                       (0, 0)])
def test_degree_classes(H, oracle, small, hub):
    """Force nodes into lane-group, warp and hub-segment paths."""
    off, tgt = G.web(1 << 12, seed=5)
    for frontier in ("pull", "auto"):
        check_run(H, oracle, off, tgt, 6, frontier=frontier, small_max_deg=small, hub_min_deg=hub)


def test_rmat_hubs(H, oracle):
    off, tgt = G.rmat(13, seed=3)
    assert np.diff(off).max() > 1024       # has hub segments at this split
    check_run(H, oracle, off, tgt, 6, frontier="auto", hub_min_deg=1024)
    check_run(H, oracle, off, tgt, 6, frontier="auto")
    check_run(H, oracle, off, tgt, 7, frontier="pull", hub_min_deg=64)


@pytest.mark.parametrize("R,log2m", [(2, 4), (4, 6), (8, 6), (8, 8), (2, 8), (8, 4), (4, 8)])
def test_batched_runs(H, oracle, R, log2m):
    off, tgt = G.web(1 << 12, seed=7)
    check_run(H, oracle, off, tgt, log2m, R=R)


def test_explicit_seeds(H, oracle):
    off, tgt = G.er(2000, 6000, seed=9)
    seeds = [11, 0xDEADBEEF, 2**63 + 5, 0]
    with H.HyperANF(off, tgt, 6, 0, runs=4, seeds=seeds) as h:
        N, T = h.run()
        regs = [h.registers(r) for r in range(4)]
    for r, s in enumerate(seeds):
        No, To, ro = oracle.hyperanf(off, tgt, 6, s, want_regs=True)
        assert T[r] == To and np.array_equal(regs[r], ro)
        np.testing.assert_allclose(N[r], No, rtol=RTOL)


def test_graph_driver_matches_host_loop(H, oracle):
    off, tgt = G.web(1 << 13, seed=4)
    a = check_run(H, oracle, off, tgt, 6, R=4, use_graph=False)
    b = check_run(H, oracle, off, tgt, 6, R=4, use_graph=True)
    for r in range(4):
        assert np.array_equal(a[0][r], b[0][r])       # bit-identical N(t)
    assert list(a[1]) == list(b[1])


def test_repeated_runs_identical(H):
    off, tgt = G.rmat(12, seed=8)
    with H.HyperANF(off, tgt, 6, SEED, use_graph=True) as h:
        N1, T1 = h.run()
        N2, T2 = h.run()
    assert list(T1) == list(T2) and np.array_equal(N1[0], N2[0])


@pytest.mark.parametrize("name", ["path", "cycle", "star", "complete", "clique_path", "grid"])
def test_closed_form_fixtures(H, oracle, name):
    g = {"path": lambda: G.path(40), "cycle": lambda: G.cycle(33), "star": lambda: G.star(300),
         "complete": lambda: G.complete(20), "clique_path": lambda: G.clique_path(35, 3),
         "grid": lambda: G.grid2d(30)}[name]()
    for frontier in ("off", "auto"):
        check_run(H, oracle, *g, 8, frontier=frontier)


def test_degenerate_graphs(H, oracle):
    for n in (0, 1, 2, 65, 1000):
        check_run(H, oracle, *G.empty(n), 6)
    # self-loops and duplicate arcs are legal
    off = np.array([0, 3, 5, 6, 6], dtype=np.int64)
    tgt = np.array([0, 1, 1, 2, 2, 0], dtype=np.int32)
    check_run(H, oracle, off, tgt, 4)
    check_run(H, oracle, off, tgt, 8, R=8)


def test_device_resident_graph(H, oracle):
    import torch
    off, tgt = G.er(5000, 20000, seed=12)
    with H.HyperANF(torch.from_numpy(off).cuda(), torch.from_numpy(tgt).cuda(), 6, SEED) as h:
        N, T = h.run()
        regs = h.registers(0)
    No, To, ro = oracle.hyperanf(off, tgt, 6, oracle.run_seed(SEED, 0), want_regs=True)
    assert T[0] == To and np.array_equal(regs, ro)
    np.testing.assert_allclose(N[0], No, rtol=RTOL)


def test_invalid_csr_rejected(H):
    off = np.array([0, 2, 3], dtype=np.int64)
    with pytest.raises(H.HanfError) as e:
        H.HyperANF(off, np.array([0, 5, 1], dtype=np.int32), 6)        # target out of range
    assert e.value.code == H.HANF_EINVAL
    with pytest.raises(H.HanfError) as e:
        H.HyperANF(np.array([0, 2, 1, 3], dtype=np.int64), np.array([0, 1, 2], dtype=np.int32), 6)
    assert e.value.code == H.HANF_EINVAL
    with pytest.raises(H.HanfError) as e:
        H.HyperANF(off, np.array([0, -1, 1], dtype=np.int32), 6)
    assert e.value.code == H.HANF_EINVAL


def test_history_exhausted(H, oracle):
    off, tgt = G.path(50)
    with H.HyperANF(off, tgt, 6, SEED) as h:
        N = np.zeros((1, 10), dtype=np.float64)
        T = np.zeros(1, dtype=np.int32)
        assert h.run_raw(N, T, max_iter=4096) == H.HANF_ERANGE
        No, _, _ = oracle.hyperanf(off, tgt, 6, oracle.run_seed(SEED, 0))
        np.testing.assert_allclose(N[0, :10], No[:10], rtol=RTOL)
        N2, T2 = h.run()                  # the context stays usable
        assert T2[0] == len(No) - 1


@pytest.mark.parametrize("frontier", ["off", "auto"])
def test_input_order_storage(H, oracle, frontier):
    """relabel=False keeps counters in input order; results are identical."""
    off, tgt = G.rmat(12, seed=6)
    check_run(H, oracle, off, tgt, 6, frontier=frontier, relabel=False)
    check_run(H, oracle, off, tgt, 6, R=4, frontier=frontier, relabel=False, use_graph=True)


def test_relabelled_registers_by_input_id(H, oracle):
    """Register reads of arbitrary id ranges map back to input ids."""
    off, tgt = G.rmat(12, seed=9)
    n = off.size - 1
    with H.HyperANF(off, tgt, 6, SEED, runs=2) as h:
        h.run()
        full = [h.registers(r) for r in range(2)]
        for first, count in [(0, 1), (17, 100), (n - 5, 5), (1000, 0)]:
            for r in range(2):
                assert np.array_equal(h.registers(r, first, count), full[r][first:first + count])


@pytest.mark.parametrize("variant", [2, 4])
@pytest.mark.parametrize("log2m", [4, 5, 6, 7, 8])
def test_async_gather_variant(H, oracle, log2m, variant):
    """The asynchronous-copy gathers of the medium-degree and hub kernel (2),
    also with those of the small-degree kernel (4), give the same results
    (rows up to 128 B; wider rows fall back to register batches)."""
    off, tgt = G.rmat(13, seed=10)
    for frontier in ("off", "pull", "auto"):
        check_run(H, oracle, off, tgt, log2m, frontier=frontier, gather_variant=variant,
                  small_max_deg=4, hub_min_deg=256)
    if log2m <= 6:
        # two runs share a row of up to 128 bytes; node degrees straddle the
        # 32-arc stages (31, 32, 33 arcs) and hub segments end mid-stage
        check_run(H, oracle, off, tgt, log2m, R=2, frontier="auto", gather_variant=variant,
                  small_max_deg=31, hub_min_deg=97)
        # many more warps than work items; a web-like graph; an R-MAT graph
        # with arc-less nodes
        for g in (G.star(300), G.web(1 << 12, seed=7), G.rmat(12, seed=8)):
            check_run(H, oracle, *g, log2m, frontier="auto", gather_variant=variant,
                      small_max_deg=8, hub_min_deg=64)


@pytest.mark.parametrize("log2m", [4, 5, 6, 7])
def test_small_async_variant(H, oracle, log2m):
    """Asynchronous row copies in the small-degree kernel (gather_variant 3):
    the same registers, T and N(t); frontier off makes every pass use it."""
    for off, tgt in (G.rmat(13, seed=11), G.web(1 << 12, seed=6), G.empty(70)):
        for frontier in ("off", "auto"):
            check_run(H, oracle, off, tgt, log2m, frontier=frontier, gather_variant=3)


def test_autotune_picks_a_candidate_and_caches_it(H, oracle, tmp_path):
    off, tgt = G.rmat(12, seed=13)
    cache = tmp_path / "tune.txt"
    best, ms = H.autotune(off, tgt, 6, SEED, cache_path=cache)
    assert best["small_max_deg"] in (32, 128, 256, 1024, 4096)
    assert best["hub_min_deg"] in (4096, 16384, 65536)
    assert best["scatter_den"] in (0, -1)          # 64-byte rows: default or pulls only
    assert ms > 0 and cache.read_text().strip()
    again, ms2 = H.autotune(off, tgt, 6, SEED, cache_path=cache)     # from the cache
    assert again == best and ms2 == pytest.approx(ms)
    check_run(H, oracle, off, tgt, 6, **best)


@pytest.mark.parametrize("log2m", [5, 6, 7, 8])
@pytest.mark.parametrize("frontier", ["off", "pull", "auto"])
def test_bit_sliced_layout(H, oracle, log2m, frontier):
    """Five bit-planes per counter give the same registers, T and N(t)."""
    off, tgt = G.rmat(12, seed=14)
    check_run(H, oracle, off, tgt, log2m, frontier=frontier, layout="packed")


def test_bit_sliced_layout_degree_paths(H, oracle):
    off, tgt = G.web(1 << 12, seed=15)
    for small, hub in [(1, 2), (2, 8), (4096, 1 << 20)]:
        check_run(H, oracle, off, tgt, 6, layout="packed", small_max_deg=small, hub_min_deg=hub)
    check_run(H, oracle, off, tgt, 6, layout="packed", relabel=False, use_graph=True)
    check_run(H, oracle, *G.clique_path(35, 3), 8, layout="packed")
    check_run(H, oracle, *G.empty(70), 6, layout="packed")


def test_bit_sliced_every_pass(H, oracle):
    off, tgt = G.er(3000, 12000, seed=16)
    c = oracle.init(off.size - 1, 6, oracle.run_seed(SEED, 0))
    with H.HyperANF(off, tgt, 6, SEED, layout="packed") as h:
        while True:
            assert np.array_equal(h.registers(0), c)
            np.testing.assert_allclose(h.estimate()[0], oracle.sum_sizes(c), rtol=RTOL)
            ch = h.iterate()
            c, ch_o = oracle.union_pass(off, tgt, c)
            assert ch == ch_o
            if ch == 0:
                break


def test_bit_sliced_layout_rejects_unsupported(H):
    off, tgt = G.er(100, 300, seed=1)
    for kw in [dict(layout="packed", runs=2), dict(layout="packed", log2m=4)]:
        log2m = kw.pop("log2m", 6)
        with pytest.raises(H.HanfError) as e:
            H.HyperANF(off, tgt, log2m, **kw)
        assert e.value.code == H.HANF_EINVAL



@pytest.mark.parametrize("layout,R", [("byte", 1), ("byte", 4), ("packed", 1)])
def test_checkpoint_resume_bit_identical(H, oracle, layout, R, tmp_path):
    """Save after some passes, load into a fresh context, resume: counters, T
    and N(t) are the oracle's (and so those of an uninterrupted run)."""
    off, tgt = G.rmat(12, seed=17)
    kw = dict(runs=R, layout=layout)
    ref = [oracle.hyperanf(off, tgt, 6, oracle.run_seed(SEED, r), want_regs=True) for r in range(R)]
    N_ref = [x[0] for x in ref]
    T_ref = [x[1] for x in ref]
    regs_ref = [x[2] for x in ref]
    with H.HyperANF(off, tgt, 6, SEED, **kw) as h:
        N_run, T_run = h.run()
        assert list(T_run) == T_ref
    for stop in (0, 1, 3):
        with H.HyperANF(off, tgt, 6, SEED, **kw) as h:
            for _ in range(stop):
                h.iterate()
            ckp = h.checkpoint()
        path = tmp_path / f"ckp{stop}.bin"
        ckp.tofile(path)
        with H.HyperANF(off, tgt, 6, SEED, use_graph=(stop == 1), **kw) as h2:
            h2.restore(np.fromfile(path, dtype=np.uint8))
            assert h2.t == stop
            N, T = h2.resume()
            assert list(T) == T_ref
            for r in range(R):
                assert np.array_equal(N[r], N_run[r])          # bit-identical to a straight run
                np.testing.assert_allclose(N[r], N_ref[r], rtol=RTOL, atol=0)
                assert np.array_equal(h2.registers(r), regs_ref[r])
                assert h2.digest(r) == oracle.digest(regs_ref[r])


def test_resume_after_pass_limit_and_mismatch(H):
    off, tgt = G.path(40)
    with H.HyperANF(off, tgt, 6, SEED) as h:
        N_full, T_full = h.run()
        Np = np.zeros((1, 4096))
        Tp = np.zeros(1, dtype=np.int32)
        assert h.run_raw(Np, Tp, max_iter=5) == H.HANF_ERANGE
        N2, T2 = h.resume()
        assert list(T2) == list(T_full) and np.array_equal(N2[0], N_full[0])
        ckp = h.checkpoint()
    with H.HyperANF(off, tgt, 6, SEED + 1) as other:
        with pytest.raises(H.HanfError) as e:
            other.restore(ckp)
        assert e.value.code == H.HANF_EINVAL



@pytest.mark.parametrize("kw", [dict(), dict(relabel=False), dict(runs=2), dict(layout="packed"),
                                dict(use_graph=True, frontier="pull")])
def test_node_statistics_match_oracle(H, oracle, kw):
    """Per-node reach, distance sum, eccentricity and effective radius equal
    the oracle's, computed from its own E_v(t) sequence."""
    off, tgt = G.er(2000, 7000, seed=18)
    R = kw.get("runs", 1)
    with H.HyperANF(off, tgt, 6, SEED, node_stats=True, **kw) as h:
        h.run()
        got = [h.node_stats(r) for r in range(R)]
        rad = [h.node_radius(0.9, r) for r in range(R)]
        sub = h.node_stats(0, 100, 50)
    for r in range(R):
        ref = oracle.node_stats(off, tgt, 6, oracle.run_seed(SEED, r), 0.9)
        assert np.array_equal(got[r]["reach"], ref["reach"])
        assert np.array_equal(got[r]["dist"], ref["dist"])
        assert np.array_equal(got[r]["ecc"], ref["ecc"])
        assert np.array_equal(rad[r], ref["radius"])
    assert np.array_equal(sub["dist"], got[0]["dist"][100:150])



def batch_graphs():
    return [G.er(500, 2000, seed=1), G.rmat(10, seed=2), G.grid2d(9), G.empty(0), G.path(64),
            G.clique_path(7, 3), G.er(65, 200, seed=3), G.star(130), G.web(1 << 11, seed=4)]


@pytest.mark.parametrize("R,kw", [(1, dict()), (2, dict()), (4, dict(frontier="pull")),
                                  (1, dict(layout="packed")), (2, dict(use_graph=True)),
                                  (1, dict(frontier="off", small_max_deg=2, hub_min_deg=8))])
def test_batch_of_graphs_matches_each_alone(H, oracle, R, kw):
    """K graphs in one context: every (graph, run) slot has the registers, T
    and N(t) of that graph run alone with its own seeds."""
    graphs = batch_graphs()
    seeds = [100 + 7 * g for g in range(len(graphs))]
    with H.HyperANF.batch(graphs, 6, graph_seeds=seeds, runs=R, **kw) as h:
        N, T = h.run()
        regs = [[h.registers(r, h.graph_base[g], h.graph_nodes[g]) for r in range(R)]
                for g in range(len(graphs))]
        digests = [[h.digest(r, h.graph_base[g], h.graph_nodes[g]) for r in range(R)]
                   for g in range(len(graphs))]
        assert h.estimate().size == len(graphs) * R
    for g, (off, tgt) in enumerate(graphs):
        for r in range(R):
            No, To, ro = oracle.hyperanf(off, tgt, 6, oracle.run_seed(seeds[g], r), want_regs=True)
            s = g * R + r
            assert T[s] == To, (g, r)
            np.testing.assert_allclose(N[s], No, rtol=RTOL, atol=0)
            assert np.array_equal(regs[g][r], ro), (g, r)
            assert digests[g][r] == oracle.digest(ro), (g, r)


def test_batch_checkpoint_and_rejections(H):
    graphs = batch_graphs()[:4]
    with H.HyperANF.batch(graphs, 6, runs=2) as h:
        N_ref, T_ref = h.run()
    with H.HyperANF.batch(graphs, 6, runs=2) as h:
        h.iterate()
        ckp = h.checkpoint()
    with H.HyperANF.batch(graphs, 6, runs=2) as h:
        h.restore(ckp)
        N, T = h.resume()
    assert list(T) == list(T_ref) and all(np.array_equal(a, b) for a, b in zip(N, N_ref))
    # an arc from one graph into another is refused
    off = np.array([0, 1] + [1] * 63, dtype=np.int64)          # graph 0: node 0 -> 70
    off = np.concatenate([off, np.full(64, 1, dtype=np.int64)])  # graph 1: no arcs
    assert off.size == 129
    tgt = np.array([70], dtype=np.int32)
    with pytest.raises(H.HanfError) as e:
        H.HyperANF(off, tgt, 6, graph_base=[0, 64, 128], graph_nodes=[64, 64])
    assert e.value.code == H.HANF_EINVAL
    with pytest.raises(H.HanfError) as e:       # bases must be multiples of 64
        H.HyperANF(*G.empty(100), 6, graph_base=[0, 50, 100], graph_nodes=[50, 50])
    assert e.value.code == H.HANF_EINVAL


@pytest.mark.parametrize("kw", [dict(), dict(relabel=False), dict(layout="packed"), dict(runs=4),
                                dict(runs=2, frontier="off")])
def test_digest_matches_oracle(H, oracle, kw):
    """hanf_digest of the counters after two passes, of the whole array and of
    a ragged node range, equals the oracle's digest of its own counters."""
    off, tgt = G.web(1 << 12, seed=6)
    R = kw.get("runs", 1)
    with H.HyperANF(off, tgt, 6, SEED, **kw) as h:
        h.iterate()
        h.iterate()
        got = [(h.digest(r), h.digest(r, 100, 333), h.digest(r, 4095, 1), h.digest(r, 7, 0))
               for r in range(R)]
    for r in range(R):
        c = oracle.init(off.size - 1, 6, oracle.run_seed(SEED, r))
        for _ in range(2):
            c, _ = oracle.union_pass(off, tgt, c)
        assert got[r] == (oracle.digest(c), oracle.digest(c[100:433]), oracle.digest(c[4095:]), 0)


def test_digest_rejects_bad_ranges(H):
    off, tgt = G.path(10)
    with H.HyperANF(off, tgt, 4, SEED) as h:
        for args in ((1, 0, 5), (0, -1, 3), (0, 8, 3)):
            with pytest.raises(H.HanfError) as e:
                h.digest(*args)
            assert e.value.code == H.HANF_EINVAL
