"""The continuous-batching server: every job's result is the same alone and in
the mix (and equal to the oracle), admission respects the arena, waits time
out, queued jobs can be cancelled, and failing jobs report their own error."""
import numpy as np
import pytest

from paper_1011_5599_gb300 import graphs as G

pytestmark = pytest.mark.gpu

SEED = 0x5EED


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1011_5599_gb300 import build as B
    B.build()
    import paper_1011_5599_gb300.hanf as H
    return H


def mix():
    jobs = []
    for i in range(24):
        kind = ("er", "rmat", "grid")[i % 3]
        if kind == "er":
            off, tgt = G.er(500 + 300 * i, 4 * (500 + 300 * i), seed=i)
        elif kind == "rmat":
            off, tgt = G.rmat(9 + i % 4, seed=i)
        else:
            off, tgt = G.grid2d(20 + i)
        jobs.append((off, tgt, (4, 6, 8)[i % 3], (1, 4)[i % 2], SEED + i))
    return jobs


def test_results_same_alone_and_in_the_mix(H, oracle):
    jobs = mix()
    alone = []
    for off, tgt, log2m, R, seed in jobs:
        with H.HyperANF(off, tgt, log2m, seed, runs=R, use_graph=True) as h:
            alone.append(h.run())
    with H.Server(1 << 30, workers=4) as srv:
        ids = [srv.submit(off, tgt, log2m, seed, runs=R) for off, tgt, log2m, R, seed in jobs]
        served = [srv.wait(i) for i in ids]
        st = srv.stats()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert st["largest_free"] == st["arena_bytes"]          # every workspace returned
    for (N_a, T_a), (N_s, T_s, info), (off, tgt, log2m, R, seed) in zip(alone, served, jobs):
        assert list(T_a) == list(T_s)
        for r in range(R):
            assert np.array_equal(N_a[r], N_s[r])            # bit-identical
        assert info["latency_ms"] >= info["run_ms"] >= 0
    # and every served result is the oracle's
    for (N_s, T_s, _), (off, tgt, log2m, R, seed) in zip(served, jobs):
        for r in range(R):
            No, To, _ = oracle.hyperanf(off, tgt, log2m, oracle.run_seed(seed, r))
            assert T_s[r] == To
            np.testing.assert_allclose(N_s[r], No, rtol=1e-12)


def test_admission_by_footprint(H):
    """An arena that fits one job at a time still serves them all in order.
    The graphs have more than 65,536 nodes, so no two jobs share a context."""
    from paper_1011_5599_gb300.hanf import make_opts, workspace_size
    off, tgt = G.rmat(17, seed=1)
    need = workspace_size(off.size - 1, tgt.size, 6, make_opts()[0], True)
    with H.Server(need + (1 << 20), workers=4) as srv:
        ids = [srv.submit(off, tgt, 6, SEED + k) for k in range(6)]
        res = [srv.wait(i) for i in ids]
    starts = sorted((r[2]["latency_ms"] - r[2]["run_ms"], r[2]["latency_ms"]) for r in res)
    for (s0, e0), (s1, e1) in zip(starts, starts[1:]):
        assert s1 >= e0 - 1.0                 # one at a time: no overlap in the arena
    with H.Server(need // 2, workers=2) as srv:
        with pytest.raises(H.HanfError) as e:
            srv.submit(off, tgt, 6, SEED)
        assert e.value.code == H.HANF_ENOMEM


def test_timeout_cancel_and_failure(H):
    off, tgt = G.rmat(14, seed=2)
    bad_off = np.array([0, 2, 3], dtype=np.int64)
    bad_tgt = np.array([0, 7, 1], dtype=np.int32)      # target out of range
    from paper_1011_5599_gb300.hanf import make_opts, workspace_size
    need = workspace_size(off.size - 1, tgt.size, 8, make_opts()[0], True)
    with H.Server(need + (1 << 20), workers=1) as srv:
        a = srv.submit(off, tgt, 8, SEED)
        b = srv.submit(off, tgt, 8, SEED + 1)
        c = srv.submit(bad_off, bad_tgt, 6, SEED)
        srv.cancel(b)
        with pytest.raises(H.HanfError) as e:
            srv.wait(b)
        assert e.value.code == H.HANF_ECANCELLED
        with pytest.raises(H.HanfError) as e:
            srv.wait(c)
        assert e.value.code == H.HANF_EINVAL          # the job's own failure
        N, T, info = srv.wait(a)
        assert T[0] > 0
        d = srv.submit(off, tgt, 8, SEED + 2)
        with pytest.raises(H.HanfError) as e:
            srv.wait(d, timeout_ms=0)
        assert e.value.code == H.HANF_ETIMEOUT
        srv.wait(d)                                    # still completes afterwards


def run_queued(H, jobs, on_device):
    """Submit a long job, then `jobs` (graph, log2m, seed) while the only
    worker is busy with it; returns each job's result or error code and the
    server's statistics."""
    import torch
    if on_device:
        jobs = [((torch.from_numpy(off).cuda(), torch.from_numpy(tgt).cuda()), log2m, seed)
                for (off, tgt), log2m, seed in jobs]
        torch.cuda.synchronize()
    with H.Server(1 << 28, workers=1) as srv:
        # a directed path of 3,000 nodes stabilises after 2,999 passes: the
        # worker stays busy with it while every other job is queued
        long_off, long_tgt = G.path(3000)
        first = srv.submit(long_off, long_tgt, 8, SEED)
        ids = [srv.submit(off, tgt, log2m, seed, runs=2) for (off, tgt), log2m, seed in jobs]
        srv.wait(first)
        results = []
        for jid in ids:
            try:
                results.append(srv.wait(jid))
            except H.HanfError as e:
                results.append(e.code)
        return results, srv.stats()


def check_against_oracle(oracle, jobs, results):
    for k, (((off, tgt), log2m, seed), res) in enumerate(zip(jobs, results)):
        if isinstance(res, int):
            continue
        N, T, _ = res
        for r in range(2):
            No, To, _ = oracle.hyperanf(off, tgt, log2m, oracle.run_seed(seed, r))
            assert T[r] == To, (k, r)
            np.testing.assert_allclose(N[r], No, rtol=1e-12, atol=0)


SMALL = [G.er(300 + 97 * i, 1200 + 300 * i, seed=40 + i) for i in range(10)] + \
        [G.grid2d(9), G.path(70), G.empty(5), G.star(65)]
BAD = (np.array([0, 2, 3], dtype=np.int64), np.array([0, 7, 1], dtype=np.int32))


@pytest.mark.parametrize("on_device", [False, True])
def test_small_jobs_share_contexts(H, oracle, on_device):
    """Small queued jobs of one class (m, runs, graph placement) run in shared
    contexts: fewer contexts than jobs, every result the oracle's; a bad graph
    of another class fails on its own."""
    jobs = [(g, 6, SEED + 3 * k) for k, g in enumerate(SMALL)]
    jobs.insert(7, (BAD, 4, SEED))
    results, st = run_queued(H, jobs, on_device)
    assert results[7] == H.HANF_EINVAL
    assert st["contexts"] <= 4, st          # the long job, a batch, the bad job
    assert st["completed"] == len(jobs) and st["failed"] == 1
    check_against_oracle(oracle, jobs, results)


def test_bad_graph_in_a_batch_runs_everything_alone(H, oracle):
    """A batch whose context fails (one graph invalid) puts its jobs back to
    run alone: the bad job reports its own error, the others their results."""
    jobs = [(g, 6, SEED + 3 * k) for k, g in enumerate(SMALL[:6])]
    jobs.insert(3, (BAD, 6, SEED))
    results, st = run_queued(H, jobs, False)
    assert results[3] == H.HANF_EINVAL
    assert all(not isinstance(r, int) for k, r in enumerate(results) if k != 3)
    check_against_oracle(oracle, jobs, results)
