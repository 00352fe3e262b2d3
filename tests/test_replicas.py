"""Multi-rank path on the CPU: two gloo ranks shard eight seeded runs, each
computes its share (with the oracle, standing in for a GPU), and the gathered
results equal a single process computing all of them; timing reduces to the
slowest rank and the sum of units."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1011_5599_gb300 import replicas


def test_shard_covers_everything_once():
    for count in (0, 1, 7, 8, 9, 100):
        for size in (1, 2, 3, 8):
            seen = [i for r in range(size) for i in replicas.shard(count, r, size)]
            assert seen == list(range(count))
            lens = [len(replicas.shard(count, r, size)) for r in range(size)]
            assert max(lens) - min(lens) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, size, port, queue):
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_1011_5599_gb300 import graphs as G
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=size)
    off, tgt = G.er(400, 1500, seed=3)
    mine = {}
    for r in replicas.shard(8, rank, size):
        N, T, _ = O.hyperanf(off, tgt, 6, O.run_seed(0x5EED, r))
        mine[r] = (N.tolist(), T)
    allres = replicas.gather(mine)
    t, u = replicas.reduce_max_sum(1.0 + rank, 10.0 * (rank + 1))
    if rank == 0:
        merged = {}
        for part in allres:
            merged.update(part)
        queue.put((merged, t, u))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_runs():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged, t, u = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert t == 2.0 and u == 30.0
    from oracle import oracle as O
    from paper_1011_5599_gb300 import graphs as G
    off, tgt = G.er(400, 1500, seed=3)
    assert sorted(merged) == list(range(8))
    for r in range(8):
        N, T, _ = O.hyperanf(off, tgt, 6, O.run_seed(0x5EED, r))
        assert merged[r][1] == T
        assert np.array_equal(np.array(merged[r][0]), N)
