"""Node-sharded HyperANF: one graph's counters computed on several GPUs.

The paper's conclusion proposes distributing Algorithm 2 in the Pregel style:
every node computes its new counter from its successors' counters, and the
counters that changed are exchanged after each pass.  Here:

* Partition: contiguous input-id ranges with about the same number of arcs
  (``partition``).  Shard q is a context over all n nodes whose CSR holds the
  arcs of its own nodes only (``local_csr``); it keeps every counter, so its
  union kernels read local memory only, and a pass changes only its own
  counters.
* One pass: every shard runs its union kernels (``hanf_pass_begin``), collects
  its changed nodes and their new rows (``hanf_pass_collect``), the shards
  exchange them (``exchange``: one all-gather of the counts, then one of the
  ids and one of the rows, padded to the largest count), and each shard
  writes the others' rows into its counters (``hanf_pass_apply``) before it
  closes the pass (``hanf_pass_end``).  After the pass every shard holds all
  of c_{t+1}: N(t+1), T and the changed counts equal those of the unsharded
  run, and every shard computes them itself.

The traffic of a pass is |F_{t+1}| (4 + R m) bytes gathered by every shard.
This module only marshals: the union, the compaction and the application of
received rows run in the library's kernels; the exchange is
``torch.distributed`` (NCCL between GPUs, gloo on CPU).
"""
from __future__ import annotations

import numpy as np


def partition(offsets, parts: int):
    """Contiguous ranges [lo, hi) of node ids, one per part, splitting the
    arcs as evenly as node boundaries allow (ranges may be empty)."""
    off = np.asarray(offsets.cpu() if hasattr(offsets, "cpu") else offsets, dtype=np.int64)
    n = off.size - 1
    arcs = int(off[-1])
    bounds = [0]
    for k in range(1, parts):
        target = (arcs * k) // parts
        b = int(np.searchsorted(off, target, side="left"))
        bounds.append(min(max(b, bounds[-1]), n))
    bounds.append(n)
    return [(bounds[k], bounds[k + 1]) for k in range(parts)]


def local_csr(offsets, targets, lo: int, hi: int):
    """CSR over all n nodes that keeps the rows of [lo, hi) and empties the
    others (numpy arrays or torch tensors, same kind out)."""
    import torch
    if isinstance(offsets, torch.Tensor):
        a0, a1 = int(offsets[lo]), int(offsets[hi])
        off = torch.zeros_like(offsets)
        off[lo + 1:hi + 1] = offsets[lo + 1:hi + 1] - a0
        off[hi + 1:] = a1 - a0
        return off, targets[a0:a1].clone()
    off_in = np.asarray(offsets, dtype=np.int64)
    a0, a1 = int(off_in[lo]), int(off_in[hi])
    off = np.zeros_like(off_in)
    off[lo + 1:hi + 1] = off_in[lo + 1:hi + 1] - a0
    off[hi + 1:] = a1 - a0
    return off, np.asarray(targets)[a0:a1].copy()


def local_exchange(parts):
    """Exchange between shards held by this one process: every shard gets the
    concatenation of the other shards' (ids, rows)."""
    import torch
    out = []
    for q in range(len(parts)):
        others = [parts[j] for j in range(len(parts)) if j != q]
        if not others:
            out.append((parts[q][0][:0], parts[q][1][:0]))
            continue
        if isinstance(parts[q][0], np.ndarray):
            out.append((np.concatenate([o[0] for o in others]),
                        np.concatenate([o[1] for o in others])))
        else:
            out.append((torch.cat([o[0] for o in others]), torch.cat([o[1] for o in others])))
    return out


def group_exchange(parts, group=None):
    """Exchange over a torch.distributed group, one shard per process: counts,
    then ids and rows padded to the largest count, all-gathered; each process
    keeps the other ranks' entries."""
    import torch
    import torch.distributed as dist
    assert len(parts) == 1, "one shard per process"
    ids, rows = parts[0]
    as_numpy = isinstance(ids, np.ndarray)
    if as_numpy:
        ids, rows = torch.from_numpy(np.ascontiguousarray(ids)), torch.from_numpy(
            np.ascontiguousarray(rows))
    world = dist.get_world_size(group)
    me = dist.get_rank(group)
    k = torch.tensor([ids.numel()], dtype=torch.int64, device=ids.device)
    ks = [torch.zeros_like(k) for _ in range(world)]
    dist.all_gather(ks, k, group=group)
    ks = [int(x.item()) for x in ks]
    kmax = max(ks)
    W = rows.shape[1]
    pid = torch.zeros(kmax, dtype=torch.int32, device=ids.device)
    prow = torch.zeros((kmax, W), dtype=torch.uint8, device=ids.device)
    pid[:ids.numel()] = ids
    prow[:ids.numel()] = rows
    gid = [torch.empty_like(pid) for _ in range(world)]
    grow = [torch.empty_like(prow) for _ in range(world)]
    dist.all_gather(gid, pid, group=group)
    dist.all_gather(grow, prow, group=group)
    r_ids = torch.cat([gid[j][:ks[j]] for j in range(world) if j != me])
    r_rows = torch.cat([grow[j][:ks[j]] for j in range(world) if j != me])
    if as_numpy:
        return [(r_ids.numpy(), r_rows.numpy())]
    return [(r_ids, r_rows)]


def run(shards, ranges, exchange=local_exchange, max_iter: int = 4096):
    """Algorithm 2 over node shards: N(0..T) (as every shard computes it) and
    T.  ``shards`` are the shards this process holds (objects with estimate,
    pass_begin, pass_collect, pass_apply, pass_end and t), ``ranges`` their
    (lo, hi), ``exchange`` maps their collected (ids, rows) to what each
    receives."""
    N = [np.asarray(shards[0].estimate(), dtype=np.float64)]
    for _ in range(max_iter):
        started = [s.pass_begin() for s in shards]
        if not all(started):
            if any(started):
                raise RuntimeError("shards disagree on stabilisation")
            break
        parts = [s.pass_collect(lo, hi - lo) for s, (lo, hi) in zip(shards, ranges)]
        received = exchange(parts)
        for s, (ids, rows) in zip(shards, received):
            s.pass_apply(ids, rows)
        changed = [s.pass_end() for s in shards]
        if len(set(changed)) != 1:
            raise RuntimeError(f"shards disagree on the changed count: {changed}")
        if changed[0] == 0:
            break
        N.append(np.asarray(shards[0].estimate(), dtype=np.float64))
    else:
        raise RuntimeError(f"no stabilisation within {max_iter} passes")
    return N, shards[0].t
