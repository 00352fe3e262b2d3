"""Node-sharded HyperANF (the Pregel-style distribution the paper's
conclusion proposes).

CPU: gloo ranks each hold one shard computed by the oracle (Jacobi over the
shard's own rows, standing in for a GPU) and exchange changed counters with
the same driver and exchange the GPU path uses; N(t) at every t, T and the
final counters equal the single-process oracle.  GPU: several shards of one
graph held by one process on one GPU (library contexts, exchange by device
concatenation; no kernel waits on another), compared with the oracle at every
pass.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1011_5599_gb300 import graphs as G
from paper_1011_5599_gb300 import sharded

SEED = 0x5EED


class OracleShard:
    """A shard computed by the oracle: all n counters, arcs of its own rows."""

    def __init__(self, O, offsets, targets, n, log2m, seed):
        self.O, self.off, self.tgt = O, offsets, targets
        self.c = O.init(n, log2m, seed)
        self.t, self.done = 0, False

    def estimate(self):
        return np.array([self.O.sum_sizes(self.c)])

    def pass_begin(self):
        if self.done:
            return False
        self.cn, self.local = self.O.union_pass(self.off, self.tgt, self.c)
        self.received = 0
        return True

    def pass_collect(self, first, count):
        lo, hi = first, first + count
        ch = np.nonzero((self.cn[lo:hi] != self.c[lo:hi]).any(axis=1))[0] + lo
        return ch.astype(np.int32), self.cn[ch]

    def pass_apply(self, ids, rows):
        self.cn[np.asarray(ids, dtype=np.int64)] = rows
        self.received = len(ids)

    def pass_end(self):
        changed = self.local + self.received
        self.c = self.cn
        if changed == 0:
            self.done = True
        else:
            self.t += 1
        return changed


def test_partition_covers_nodes_in_order():
    off, _ = G.rmat(10, seed=4)
    for parts in (1, 2, 3, 5, 8):
        ranges = sharded.partition(off, parts)
        assert ranges[0][0] == 0 and ranges[-1][1] == off.size - 1
        assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
        share = [off[hi] - off[lo] for lo, hi in ranges]
        assert sum(share) == off[-1]
        assert max(share) <= off[-1] / parts + np.diff(off).max()


def test_local_csr_keeps_only_its_rows():
    off, tgt = G.er(300, 1200, seed=6)
    lo, hi = 70, 190
    lo_off, lo_tgt = sharded.local_csr(off, tgt, lo, hi)
    deg = np.diff(lo_off)
    assert np.all(deg[:lo] == 0) and np.all(deg[hi:] == 0)
    assert np.array_equal(deg[lo:hi], np.diff(off)[lo:hi])
    assert np.array_equal(lo_tgt, tgt[off[lo]:off[hi]])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, size, port, queue):
    import torch.distributed as dist
    from oracle import oracle as O
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=size)
    off, tgt = G.rmat(11, seed=8)
    n = off.size - 1
    ranges = sharded.partition(off, size)
    lo, hi = ranges[rank]
    shard = OracleShard(O, *sharded.local_csr(off, tgt, lo, hi), n, 6, O.run_seed(SEED, 0))
    N, T = sharded.run([shard], [(lo, hi)], exchange=sharded.group_exchange)
    queue.put((rank, [float(x[0]) for x in N], T, O.digest(shard.c)))
    dist.destroy_process_group()


@pytest.mark.parametrize("size", [2, 3])
def test_gloo_ranks_equal_the_single_process_oracle(oracle, size):
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, size, port, queue)) for r in range(size)]
    for p in procs:
        p.start()
    results = []
    while len(results) < size:
        try:
            results.append(queue.get(timeout=5))
        except Exception:
            assert all(p.exitcode in (None, 0) for p in procs), [p.exitcode for p in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    off, tgt = G.rmat(11, seed=8)
    No, To, ro = oracle.hyperanf(off, tgt, 6, oracle.run_seed(SEED, 0), want_regs=True)
    for rank, N, T, dig in results:
        assert T == To, rank
        assert dig == oracle.digest(ro), rank
        np.testing.assert_allclose(N, No, rtol=1e-12, atol=0)


@pytest.mark.gpu
@pytest.mark.parametrize("parts,R,kw", [(1, 1, dict()), (2, 1, dict()), (3, 2, dict()),
                                        (4, 1, dict(frontier="pull")),
                                        (2, 1, dict(relabel=False, scatter_den=-1))])
def test_shards_on_one_gpu_every_pass(oracle, parts, R, kw):
    """Several shards of one graph in one process on one GPU: after every pass
    each shard's counters (digest) and N(t) are the oracle's."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1011_5599_gb300 import build as B
    B.build()
    from paper_1011_5599_gb300.hanf import HyperANF
    off, tgt = G.rmat(14, seed=12)
    n = off.size - 1
    ranges = sharded.partition(off, parts)
    off_d, tgt_d = torch.from_numpy(off).cuda(), torch.from_numpy(tgt).cuda()
    shards = [HyperANF(*sharded.local_csr(off_d, tgt_d, lo, hi), 6, SEED, runs=R, **kw)
              for lo, hi in ranges]
    cs = [oracle.init(n, 6, oracle.run_seed(SEED, r)) for r in range(R)]
    t = 0
    while True:
        for r in range(R):
            N_o = oracle.sum_sizes(cs[r])
            for s in shards:
                assert s.t == t
                assert s.digest(r) == oracle.digest(cs[r]), (t, r)
                np.testing.assert_allclose(s.estimate()[r], N_o, rtol=1e-12, atol=0)
        started = [s.pass_begin() for s in shards]
        assert all(started)
        parts_ = [s.pass_collect(lo, hi - lo) for s, (lo, hi) in zip(shards, ranges)]
        for s, (ids, rows) in zip(shards, sharded.local_exchange(parts_)):
            s.pass_apply(ids, rows)
        changed = [s.pass_end() for s in shards]
        nxt = [oracle.union_pass(off, tgt, cs[r]) for r in range(R)]
        any_changed = np.zeros(n, dtype=bool)
        for r in range(R):
            any_changed |= (nxt[r][0] != cs[r]).any(axis=1)
        assert changed == [int(any_changed.sum())] * parts, (t, changed)
        cs = [x[0] for x in nxt]
        if changed[0] == 0:
            break
        t += 1
    assert not any(s.pass_begin() for s in shards)     # stable: nothing more to run
    for s in shards:
        s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("parts", [2, 5])
def test_sharded_driver_on_one_gpu(oracle, parts):
    """sharded.run with shards held by one process: N(0..T) and T are the
    oracle's, and every shard ends with the oracle's counters."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1011_5599_gb300 import build as B
    B.build()
    from paper_1011_5599_gb300.hanf import HyperANF
    off, tgt = G.web(1 << 13, seed=3)
    ranges = sharded.partition(off, parts)
    shards = [HyperANF(*sharded.local_csr(off, tgt, lo, hi), 6, SEED) for lo, hi in ranges]
    N, T = sharded.run(shards, ranges)
    No, To, ro = oracle.hyperanf(off, tgt, 6, oracle.run_seed(SEED, 0), want_regs=True)
    assert T == To
    np.testing.assert_allclose([x[0] for x in N], No, rtol=1e-12, atol=0)
    for s in shards:
        assert s.digest(0) == oracle.digest(ro)
        s.close()
