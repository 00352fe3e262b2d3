"""Replica sharding across ranks (one process per GPU).

HyperANF's work splits into independent units -- the R seeded runs of a
graph, the jobs of a stream, separate graphs -- so N GPUs run N independent
replicas with no exchange on the data path (one graph spread over several
GPUs would need an all-gather of the changed counters after every pass, the
Pregel scheme of the paper's conclusion; not built here).  Only timings and,
optionally, results cross ranks, through torch.distributed.
"""
from __future__ import annotations


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def world() -> tuple[int, int]:
    """(rank, world size); (0, 1) without a process group."""
    d = _dist()
    return (d.get_rank(), d.get_world_size()) if d else (0, 1)


def shard(count: int, rank: int, size: int) -> range:
    """The contiguous share of `count` units that `rank` of `size` owns
    (shares differ by at most one unit)."""
    if size < 1 or not 0 <= rank < size:
        raise ValueError("bad rank / world size")
    base, extra = divmod(count, size)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def reduce_max_sum(elapsed: float, units: float, device=None) -> tuple[float, float]:
    """Whole-job timing: the slowest rank's time and all ranks' units."""
    d = _dist()
    if d is None:
        return float(elapsed), float(units)
    import torch
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    d.all_reduce(t, op=d.ReduceOp.MAX)
    d.all_reduce(u, op=d.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def gather(obj) -> list:
    """Every rank's object, in rank order (on every rank)."""
    d = _dist()
    if d is None:
        return [obj]
    out = [None] * d.get_world_size()
    d.all_gather_object(out, obj)
    return out
