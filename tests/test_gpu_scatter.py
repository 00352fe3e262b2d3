"""Scatter (pure push) passes vs the CPU oracle, through the C ABI.

A scatter pass pushes the counter of every node changed by the last pass
into its predecessors' new counters (Section 3.3's systolic computation
carried to its end).  It must leave exactly the registers of the Jacobi
pass of Algorithm 2: the tests force scatter passes (scatter_den = 1: any
pass whose changed nodes have fewer in-arcs than the graph has arcs) and
compare registers after every pass, the changed-node counts, T and N(t)
with the oracle, over every row width (16 .. 2048 bytes), in-lists cut
into segments, and batches of graphs.
"""
import numpy as np
import pytest

from paper_1011_5599_gb300 import graphs as G

pytestmark = pytest.mark.gpu

SEED = 0x5EED
RTOL = 1e-12
SCATTER = 3     # pass mode recorded in the trace


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1011_5599_gb300 import build as B
    B.build()
    import paper_1011_5599_gb300.hanf as H
    return H


def fan_in_chain(leaves=5000, chain=12):
    """Node 0 has `leaves` predecessors (in-list of three 2048-arc segments)
    and a chain 0 -> c_1 -> ... -> c_chain, so it changes pass after pass."""
    n = 1 + leaves + chain
    lv = np.arange(1, leaves + 1)
    ch = np.arange(leaves + 1, n)
    src = np.concatenate([lv, [0], ch[:-1]])
    dst = np.concatenate([np.zeros(leaves, np.int64), [ch[0]], ch[1:]])
    return G.csr_from_arcs(src, dst, n)


def run_and_check(H, O, off, tgt, log2m, R=1, expect_scatter=True, **kw):
    with H.HyperANF(off, tgt, log2m, SEED, runs=R, profile=True, **kw) as h:
        N, T = h.run()
        regs = [h.registers(r) for r in range(R)]
        modes = [row["mode"] for row in h.trace()]
    if expect_scatter:
        assert SCATTER in modes, modes
    for r in range(R):
        No, To, ro = O.hyperanf(off, tgt, log2m, O.run_seed(SEED, r), want_regs=True)
        assert T[r] == To, (r, T[r], To)
        assert np.array_equal(regs[r], ro), f"run {r}: registers differ"
        np.testing.assert_allclose(N[r], No, rtol=RTOL, atol=0)
    return modes


def test_scatter_every_pass_bit_exact(H, oracle):
    """Step by step: registers, N(t) and the changed count after every pass."""
    off, tgt = G.web(1 << 13, seed=7)
    log2m = 6
    c = oracle.init(off.size - 1, log2m, oracle.run_seed(SEED, 0))
    with H.HyperANF(off, tgt, log2m, SEED, scatter_den=1) as h:
        t = 0
        while True:
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
        assert h.counters()["push_passes"] > 0


@pytest.mark.parametrize("log2m,R", [(4, 1), (5, 1), (6, 1), (7, 1), (8, 1), (6, 8), (8, 4),
                                     (8, 8)])
def test_scatter_every_row_width(H, oracle, log2m, R):
    """Rows of 16 .. 2048 bytes (one lane .. a warp with four vectors a lane)."""
    off, tgt = G.er(3000, 12000, seed=log2m + R)
    run_and_check(H, oracle, off, tgt, log2m, R=R, scatter_den=1)


def test_scatter_segmented_in_lists(H, oracle):
    off, tgt = fan_in_chain()
    assert np.bincount(tgt, minlength=off.size - 1).max() > 2 * 2048
    for log2m, R in ((6, 1), (4, 2), (8, 8)):
        run_and_check(H, oracle, off, tgt, log2m, R=R, scatter_den=1)


def test_scatter_rmat_hubs_and_default_policy(H, oracle):
    """R-MAT with heavy in-degree hubs: forced scatter, the default policy
    (scatter only late), and scatter disabled all give the oracle's result."""
    off, tgt = G.rmat(13, seed=3)
    run_and_check(H, oracle, off, tgt, 6, scatter_den=1)
    run_and_check(H, oracle, off, tgt, 6, expect_scatter=False)
    modes = run_and_check(H, oracle, off, tgt, 6, expect_scatter=False, scatter_den=-1)
    assert SCATTER not in modes


def test_scatter_with_graph_driver(H, oracle):
    off, tgt = G.web(1 << 12, seed=9)
    with H.HyperANF(off, tgt, 7, SEED, scatter_den=1, use_graph=True) as h:
        N, T = h.run()
        regs = h.registers(0)
    No, To, ro = oracle.hyperanf(off, tgt, 7, oracle.run_seed(SEED, 0), want_regs=True)
    assert T[0] == To and np.array_equal(regs, ro)
    np.testing.assert_allclose(N[0], No, rtol=RTOL, atol=0)


@pytest.mark.parametrize("R", [1, 4])
def test_scatter_batch_of_graphs(H, oracle, R):
    """K graphs in one context with scatter passes: every slot as if alone."""
    graphs = [G.er(500, 2000, seed=1), G.rmat(10, seed=2), G.grid2d(9), G.path(64),
              fan_in_chain(3000, 5), G.web(1 << 11, seed=4), G.empty(0)]
    seeds = [100 + 7 * g for g in range(len(graphs))]
    with H.HyperANF.batch(graphs, 6, graph_seeds=seeds, runs=R, scatter_den=1) as h:
        N, T = h.run()
        regs = [[h.registers(r, h.graph_base[g], h.graph_nodes[g]) for r in range(R)]
                for g in range(len(graphs))]
    for g, (off, tgt) in enumerate(graphs):
        for r in range(R):
            No, To, ro = oracle.hyperanf(off, tgt, 6, oracle.run_seed(seeds[g], r), want_regs=True)
            s = g * R + r
            assert T[s] == To, (g, r)
            np.testing.assert_allclose(N[s], No, rtol=RTOL, atol=0)
            assert np.array_equal(regs[g][r], ro), (g, r)


def sinks_graph(n=1 << 18, arcs=1 << 21, seed=3):
    """Half of the nodes have no out-arcs (they are left out of the degree-
    class lists); the other half point anywhere, so sinks are targets too."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n // 2, arcs)
    dst = rng.integers(0, n, arcs)
    return G.csr_from_arcs(src, dst, n)


@pytest.mark.parametrize("scatter_den", [1, -1])
def test_transpose_with_sinks_and_a_dirty_workspace(H, oracle, scatter_den):
    """The transpose behind systolic and scatter passes must not depend on what
    the workspace held before: fill the allocator's cache with valid-looking
    node ids first, then run with many arc-less nodes."""
    import torch
    off, tgt = sinks_graph()
    n = off.size - 1
    junk = torch.randint(0, n, (1 << 28,), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    del junk          # the caching allocator hands this block out again
    run_and_check(H, oracle, off, tgt, 6, expect_scatter=scatter_den > 0,
                  scatter_den=scatter_den)


@pytest.mark.parametrize("log2m,R", [(4, 1), (7, 1), (6, 8), (8, 8)])
def test_degenerate_graphs_every_flavour(H, oracle, log2m, R):
    """Empty and arc-less graphs, a single node, self-loops and duplicate arcs,
    with scatter passes forced, with them off, and with the pull frontier,
    at rows of 16 to 2048 bytes (the widest also use the second stream)."""
    loops = (np.array([0, 3, 5, 6, 6], dtype=np.int64), np.array([0, 1, 1, 2, 2, 0], dtype=np.int32))
    one_arc = (np.array([0, 1, 1], dtype=np.int64), np.array([1], dtype=np.int32))
    graphs = [G.empty(0), G.empty(1), G.empty(65), loops, one_arc, G.path(3), G.star(70)]
    for off, tgt in graphs:
        for kw in (dict(scatter_den=1), dict(scatter_den=-1), dict(frontier="pull")):
            with H.HyperANF(off, tgt, log2m, SEED, runs=R, **kw) as h:
                N, T = h.run()
                regs = [h.registers(r) for r in range(R)]
            for r in range(R):
                No, To, ro = oracle.hyperanf(off, tgt, log2m, oracle.run_seed(SEED, r),
                                             want_regs=True)
                assert T[r] == To, (off.size - 1, kw, r)
                assert np.array_equal(regs[r], ro), (off.size - 1, kw, r)
                np.testing.assert_allclose(N[r], No, rtol=RTOL, atol=0)
