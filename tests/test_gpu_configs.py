"""CUDA path vs the oracle at the full sizes of the benchmark workloads.

* web-like graph, n = 2^20, m = 64, R = 8 runs batched: the oracle runs all
  eight runs completely; registers, T and N(t) are compared in full.
* symmetrised R-MAT scale 24 (~5e8 arcs), m = 128, and directed R-MAT scale
  27 (~2.1e9 arcs), m = 64, in the launch configuration the benchmark times:
  after every pass t the digest of all n counters (hanf_digest against the
  oracle's digest of its own Jacobi pass), N(t), and the number of changed
  counters are compared, then the whole run through the CUDA-graph driver.
* an R-MAT multigraph of 2^25 nodes and 65 * 2^25 = 2,181,038,080 arcs (past
  2^31; duplicate arcs and self-loops kept), m = 16: the same comparison after
  every pass, for the default pass flavours, with pure-push passes off
  (systolic instead), and with the frontier off (dense passes only).
The large graphs are generated on the GPU and copied to the host for the
oracle; nothing the oracle uses comes from the CUDA path's results.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEED = 0x5EED
RTOL = 1e-12
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1011_5599_gb300 import build as B
    B.build()
    import paper_1011_5599_gb300.hanf as H
    return H


def host_ram_gb():
    try:
        return os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE") / 1e9
    except (ValueError, OSError):
        return 0.0


def test_web_2p20_eight_runs_full(H, oracle):
    from paper_1011_5599_gb300 import graphs as G
    off, tgt = G.web(1 << 20, seed=1)
    R, log2m = 8, 6
    with H.HyperANF(off, tgt, log2m, SEED, runs=R, use_graph=True) as h:
        N, T = h.run()
        regs = [h.registers(r) for r in range(R)]
    for r in range(R):
        No, To, ro = oracle.hyperanf(off, tgt, log2m, oracle.run_seed(SEED, r), want_regs=True,
                                     threads=THREADS)
        assert T[r] == To, (r, T[r], To)
        assert np.array_equal(regs[r], ro), f"run {r}: registers differ"
        np.testing.assert_allclose(N[r], No, rtol=RTOL, atol=0)


def oracle_trajectory(oracle, off, tgt, log2m, seed, threads=THREADS):
    """Algorithm 2 on the oracle, pass by pass: for t = 0..T the tuple
    (N(t), digest of c_t, counters changed by pass t)."""
    c = oracle.init(off.size - 1, log2m, seed)
    traj = []
    while True:
        N = oracle.sum_sizes_mt(c, threads)
        D = oracle.digest(c, threads)
        c, changed = oracle.union_pass(off, tgt, c, threads)
        traj.append((N, D, changed))
        if changed == 0:
            return traj
        assert len(traj) < 200


def check_every_pass(h, traj):
    """Step the context with the host-loop driver and compare each t with the
    oracle's trajectory; returns the pass modes of the trace (profile=True)."""
    for t, (N, D, changed) in enumerate(traj):
        assert h.t == t
        assert h.digest(0) == D, f"t={t}: registers differ"
        np.testing.assert_allclose(h.estimate()[0], N, rtol=RTOL, atol=0, err_msg=f"t={t}")
        assert h.iterate() == changed, f"t={t}: changed counters"
    assert h.iterate() == 0
    return [int(row["mode"]) for row in h.trace()]


def check_graph_driver(h, traj):
    """hanf_run through the CUDA graph: same T, N(0..T) and final registers."""
    N, T = h.run()
    assert T[0] == len(traj) - 1
    np.testing.assert_allclose(N[0], [x[0] for x in traj], rtol=RTOL, atol=0)
    assert h.digest(0) == traj[-1][1]


def test_symmetric_rmat24_m128_every_pass(H, oracle):
    import torch
    from paper_1011_5599_gb300 import graphs as G
    off_d, tgt_d = G.rmat(24, symmetrise=True, seed=1, device="cuda", as_numpy=False)
    off, tgt = off_d.cpu().numpy(), tgt_d.cpu().numpy()
    log2m = 7
    traj = oracle_trajectory(oracle, off, tgt, log2m, oracle.run_seed(SEED, 0))
    assert len(traj) >= 4
    with H.HyperANF(off_d, tgt_d, log2m, SEED, frontier="auto", use_graph=True,
                    profile=True) as h:
        check_every_pass(h, traj)
        check_graph_driver(h, traj)
    del off_d, tgt_d
    torch.cuda.empty_cache()


def test_rmat27_benchmark_configuration_every_pass(H, oracle):
    """Scale 27, m = 64, frontier auto: the benchmark's graph (seed 1) and
    options; every pass against the oracle, then the CUDA-graph driver the
    benchmark times."""
    import torch
    if host_ram_gb() < 48:
        pytest.skip("needs ~48 GB of free host memory for the oracle")
    from paper_1011_5599_gb300 import graphs as G
    off_d, tgt_d = G.rmat(27, seed=1, device="cuda", as_numpy=False)
    off, tgt = off_d.cpu().numpy(), tgt_d.cpu().numpy()
    log2m = 6
    traj = oracle_trajectory(oracle, off, tgt, log2m, oracle.run_seed(SEED, 0))
    with H.HyperANF(off_d, tgt_d, log2m, SEED, frontier="auto", use_graph=True,
                    profile=True) as h:
        modes = check_every_pass(h, traj)
        check_graph_driver(h, traj)
    assert 2 in modes and 3 in modes           # dense and scatter passes both ran
    del off_d, tgt_d
    torch.cuda.empty_cache()


def test_past_2p31_arcs_every_pass(H, oracle):
    """More arcs than int32 can count: offsets past 2^31 reach the degree
    classes, the hub segments, the relabelled CSR, the transpose and every
    pass flavour."""
    import torch
    if host_ram_gb() < 40:
        pytest.skip("needs ~40 GB of free host memory for the oracle")
    from paper_1011_5599_gb300 import graphs as G
    off_d, tgt_d = G.rmat_multigraph(25, 65, seed=5, device="cuda")
    arcs = tgt_d.numel()
    assert arcs == 65 << 25 and arcs > 2**31
    off, tgt = off_d.cpu().numpy(), tgt_d.cpu().numpy()
    assert np.diff(off).max() > 16384           # hub segments
    log2m = 4
    traj = oracle_trajectory(oracle, off, tgt, log2m, oracle.run_seed(SEED, 0))
    del off, tgt
    seen = set()
    for kw in (dict(), dict(scatter_den=-1), dict(frontier="off")):
        with H.HyperANF(off_d, tgt_d, log2m, SEED, use_graph=True, profile=True, **kw) as h:
            seen |= set(check_every_pass(h, traj))
            check_graph_driver(h, traj)
    assert {1, 2, 3} <= seen, seen               # systolic, dense and scatter passes
    del off_d, tgt_d
    torch.cuda.empty_cache()
