"""Seeded synthetic graph generators (CSR by source).

This module only makes inputs: it holds none of HyperANF's arithmetic, so
both the CUDA path and the CPU oracle may be fed from it.  Every generator
returns ``(offsets, targets)`` with int64 offsets of length n+1 and int32
targets, sorted by source and, within a source, by target.

Shapes follow the workloads the paper measures (web graphs with host
locality and skewed degrees, social graphs, a Kronecker/R-MAT graph; Tables 1
and 2), which are not available here and are stood in for by these recipes:

* ``er``       directed Erdos-Renyi with an exact number of distinct arcs;
* ``web``      power-law out-degree (exponent 2.1, mean 16, cap 4096), 80% of
               arcs inside contiguous "host" blocks of 64..4096 ids
               (log-uniform sizes), the rest copied from the target of a
               uniformly chosen earlier arc (preferential attachment on
               in-degree);
* ``rmat``     R-MAT (a, b, c, d) = (0.57, 0.19, 0.19, 0.05), edge factor 16,
               seeded label scramble, self-loops dropped, duplicates removed,
               optional symmetrisation; runs on any torch device (the CUDA
               random stream differs from the CPU one, so a graph is named by
               its recipe, seed and device);
* ``rmat_multigraph`` R-MAT keeping every drawn arc (duplicates and loops),
               for inputs past 2^31 arcs;
* fixtures with closed-form neighbourhood functions: path, cycle, star,
  complete digraph, two cliques joined by a one-way path (Section 4), and a
  4-neighbour grid.
"""
from __future__ import annotations

import math

import numpy as np


# --------------------------------------------------------------------------
# CSR assembly


def csr_from_arcs(src, dst, n: int, dedup: bool = True, drop_loops: bool = True):
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if drop_loops:
        keep = src != dst
        src, dst = src[keep], dst[keep]
    key = src * np.int64(max(n, 1)) + dst
    key = np.unique(key) if dedup else np.sort(key, kind="stable")
    src = key // max(n, 1)
    dst = key % max(n, 1)
    counts = np.bincount(src, minlength=n) if n else np.zeros(0, np.int64)
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    return off, dst.astype(np.int32)


def degrees(offsets):
    return np.diff(np.asarray(offsets, dtype=np.int64))


def transpose(offsets, targets):
    """CSR of the transposed graph (predecessor lists), sorted."""
    off = np.asarray(offsets, dtype=np.int64)
    n = off.size - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(off))
    return csr_from_arcs(np.asarray(targets, np.int64), src, n, dedup=False, drop_loops=False)


# --------------------------------------------------------------------------
# Fixtures with closed forms


def empty(n: int):
    return np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32)


def path(n: int):
    """Directed path 0 -> 1 -> ... -> n-1."""
    s = np.arange(n - 1)
    return csr_from_arcs(s, s + 1, n)


def cycle(n: int):
    s = np.arange(n)
    return csr_from_arcs(s, (s + 1) % n, n)


def star(n: int):
    """Symmetric star: centre 0 <-> leaves 1..n-1."""
    leaves = np.arange(1, n)
    return csr_from_arcs(np.concatenate([np.zeros(n - 1, np.int64), leaves]),
                         np.concatenate([leaves, np.zeros(n - 1, np.int64)]), n)


def complete(n: int):
    """Complete digraph without self-loops."""
    s, d = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return csr_from_arcs(s.ravel(), d.ravel(), n)


def clique_path(k: int, l: int):
    """Two k-cliques joined by a one-way path of l nodes (Section 4).

    Nodes 0..k-1 form clique A, k..k+l-1 the path p_1..p_l, k+l..2k+l-1
    clique B.  Every node of A has an arc to p_1, p_i -> p_{i+1}, and p_l has
    an arc to every node of B.  The cliques are complete digraphs without
    self-loops.
    """
    n = 2 * k + l
    src, dst = [], []
    for base in (0, k + l):
        s, d = np.meshgrid(np.arange(base, base + k), np.arange(base, base + k), indexing="ij")
        src.append(s.ravel()); dst.append(d.ravel())
    src.append(np.arange(k)); dst.append(np.full(k, k))
    src.append(np.arange(k, k + l - 1)); dst.append(np.arange(k + 1, k + l))
    src.append(np.full(k, k + l - 1)); dst.append(np.arange(k + l, 2 * k + l))
    return csr_from_arcs(np.concatenate(src), np.concatenate(dst), n)


def grid2d(side: int):
    """side x side grid, 4-neighbour, symmetric."""
    n = side * side
    v = np.arange(n).reshape(side, side)
    src = [v[:, :-1].ravel(), v[:, 1:].ravel(), v[:-1, :].ravel(), v[1:, :].ravel()]
    dst = [v[:, 1:].ravel(), v[:, :-1].ravel(), v[1:, :].ravel(), v[:-1, :].ravel()]
    return csr_from_arcs(np.concatenate(src), np.concatenate(dst), n)


# --------------------------------------------------------------------------
# Erdos-Renyi


def er(n: int, arcs: int, seed: int = 1):
    """Directed G(n, M): exactly ``arcs`` distinct non-loop arcs, uniform."""
    if arcs > n * (n - 1):
        raise ValueError("too many arcs")
    rng = np.random.default_rng(seed)
    keys = np.zeros(0, dtype=np.int64)
    while keys.size < arcs:
        want = int((arcs - keys.size) * 1.2) + 16
        s = rng.integers(0, n, want, dtype=np.int64)
        d = rng.integers(0, n, want, dtype=np.int64)
        k = s[s != d] * n + d[s != d]
        allk = np.concatenate([keys, k])
        _, first = np.unique(allk, return_index=True)
        keys = allk[np.sort(first)][:arcs]
    return csr_from_arcs(keys // n, keys % n, n)


# --------------------------------------------------------------------------
# Web-like


def _pareto_xmin(mean: float, exponent: float, cap: int) -> float:
    """x_min with E[min(floor(x_min U^(-1/(exponent-1))), cap)] = mean."""
    k = np.arange(1, cap + 1, dtype=np.float64)

    def expect(x):
        return np.minimum(1.0, (x / k) ** (exponent - 1.0)).sum()

    lo, hi = 1e-3, float(cap)
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        if expect(mid) < mean:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def web(n: int = 1 << 20, seed: int = 1, mean_deg: float = 16.0, exponent: float = 2.1,
        cap: int = 4096, p_local: float = 0.8, block_lo: int = 64, block_hi: int = 4096,
        copy_window: float | None = 0.03):
    """Web-like graph: contiguous host blocks of log-uniform size, power-law
    out-degrees, each arc inside its source's host with probability p_local,
    otherwise a copy of the target of an earlier arc.  With copy_window = f
    the copied arc is one of the f * arcs most recent ones (crawl order keeps
    related pages near each other); that gives the broad distance distribution
    of web crawls (spid above 1 at f = 0.03: 2.5 at n = 2^20).  None copies
    from all earlier arcs (a small world, spid about 0.2)."""
    rng = np.random.default_rng(seed)
    # contiguous host blocks, log-uniform sizes
    sizes = np.exp(rng.uniform(math.log(block_lo), math.log(block_hi), n // block_lo + 2))
    sizes = np.maximum(1, sizes.astype(np.int64))
    ends = np.cumsum(sizes)
    nblk = int(np.searchsorted(ends, n)) + 1
    starts = np.concatenate([[0], ends[:nblk - 1]])
    ends = np.minimum(ends[:nblk], n)
    blk_of = np.repeat(np.arange(nblk), ends - starts)[:n]
    bstart = starts[blk_of]
    bsize = (ends - starts)[blk_of]
    # power-law out-degrees
    xmin = _pareto_xmin(mean_deg, exponent, cap)
    u = rng.random(n)
    deg = np.minimum(np.floor(xmin * (1.0 - u) ** (-1.0 / (exponent - 1.0))), cap).astype(np.int64)
    a = int(deg.sum())
    src = np.repeat(np.arange(n, dtype=np.int64), deg)
    local = rng.random(a) < p_local
    tgt = np.full(a, -1, dtype=np.int64)
    li = np.nonzero(local)[0]
    tgt[li] = bstart[src[li]] + np.floor(rng.random(li.size) * bsize[src[li]]).astype(np.int64)
    # copy model: an arc that is not local takes the target of a uniformly
    # chosen earlier arc, among the most recent copy_window * a ones if set
    # (the very first arc takes a uniform node)
    gi = np.nonzero(~local)[0]
    if copy_window is None:
        ptr = np.floor(rng.random(gi.size) * gi).astype(np.int64)
    else:
        span = np.minimum(gi, max(1, int(copy_window * a)))
        ptr = gi - 1 - np.floor(rng.random(gi.size) * span).astype(np.int64)
    first = gi == 0
    tgt[gi[first]] = rng.integers(0, n, int(first.sum()))
    pend, p = gi[~first], ptr[~first]
    link = np.full(a, -1, dtype=np.int64)
    link[pend] = p
    while pend.size:
        ok = tgt[p] >= 0
        tgt[pend[ok]] = tgt[p[ok]]
        pend, p = pend[~ok], p[~ok]
        p = link[p]                       # jump to what the earlier arc copies
    return csr_from_arcs(src, tgt, n)


# --------------------------------------------------------------------------
# R-MAT (torch, any device)


def rmat(scale: int, edge_factor: int = 16, seed: int = 1, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, symmetrise: bool = False, scramble: bool = True,
         device: str = "cpu", chunk: int = 1 << 26, as_numpy: bool = True):
    """R-MAT graph with 2^scale nodes and edge_factor * 2^scale drawn arcs."""
    import torch

    n = 1 << scale
    total = edge_factor * n
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    perm = torch.randperm(n, generator=g, device=device) if scramble else None
    pieces = []
    for s in range(0, total, chunk):
        k = min(chunk, total - s)
        src = torch.zeros(k, dtype=torch.int64, device=device)
        dst = torch.zeros(k, dtype=torch.int64, device=device)
        for _ in range(scale):
            uu = torch.rand(k, generator=g, device=device)
            sb = uu >= (a + b)
            db = ((uu >= a) & (uu < a + b)) | (uu >= (a + b + c))
            src = src * 2 + sb.to(torch.int64)
            dst = dst * 2 + db.to(torch.int64)
            del uu, sb, db
        if perm is not None:
            src = perm[src]
            dst = perm[dst]
        keep = src != dst
        src, dst = src[keep], dst[keep]
        pieces.append((src << scale) | dst)
        if symmetrise:
            pieces.append((dst << scale) | src)
        del src, dst, keep
    keys = torch.cat(pieces)
    del pieces
    keys = torch.unique(keys)
    counts = torch.bincount(keys >> scale, minlength=n)
    off = torch.zeros(n + 1, dtype=torch.int64, device=device)
    torch.cumsum(counts, 0, out=off[1:])
    del counts
    tgt = (keys & (n - 1)).to(torch.int32)
    del keys
    if as_numpy:
        return off.cpu().numpy(), tgt.cpu().numpy()
    return off, tgt


def rmat_multigraph(scale: int, edge_factor: int, seed: int = 1, a: float = 0.57,
                    b: float = 0.19, c: float = 0.19, device: str = "cuda",
                    buckets: int = 16, chunk: int = 1 << 26):
    """R-MAT with every drawn arc kept: duplicate arcs and self-loops stay
    (both are legal inputs, max being idempotent), so the arc count is exactly
    edge_factor * 2^scale and can exceed 2^31.  Labels are scrambled as in
    ``rmat``.  Arcs are binned by the top bits of their source and each bin is
    sorted on its own, so no single sort or count sees 2^31 elements.
    Returns (offsets int64, targets int32) as tensors on ``device``."""
    import torch

    n = 1 << scale
    total = edge_factor * n
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    perm = torch.randperm(n, generator=g, device=device)
    shift = max(scale - max(buckets.bit_length() - 1, 0), 0)
    nb = n >> shift
    bins = [[] for _ in range(nb)]
    for s in range(0, total, chunk):
        k = min(chunk, total - s)
        src = torch.zeros(k, dtype=torch.int64, device=device)
        dst = torch.zeros(k, dtype=torch.int64, device=device)
        for _ in range(scale):
            uu = torch.rand(k, generator=g, device=device)
            sb = uu >= (a + b)
            db = ((uu >= a) & (uu < a + b)) | (uu >= (a + b + c))
            src = src * 2 + sb.to(torch.int64)
            dst = dst * 2 + db.to(torch.int64)
            del uu, sb, db
        src = perm[src]
        dst = perm[dst]
        keys = (src << scale) | dst
        bucket = src >> shift
        order = torch.argsort(bucket, stable=True)
        keys, bucket = keys[order], bucket[order]
        cnt = torch.bincount(bucket, minlength=nb).tolist()
        for i, piece in enumerate(torch.split(keys, cnt)):
            if piece.numel():
                bins[i].append(piece.clone())
        del src, dst, keys, bucket, order
    counts = torch.zeros(n, dtype=torch.int64, device=device)
    tgt = torch.empty(total, dtype=torch.int32, device=device)
    at = 0
    for i in range(nb):
        if not bins[i]:
            continue
        keys = torch.sort(torch.cat(bins[i])).values
        bins[i] = None
        counts += torch.bincount(keys >> scale, minlength=n)
        tgt[at:at + keys.numel()] = (keys & (n - 1)).to(torch.int32)
        at += keys.numel()
        del keys
    assert at == total
    off = torch.zeros(n + 1, dtype=torch.int64, device=device)
    torch.cumsum(counts, 0, out=off[1:])
    return off, tgt


# --------------------------------------------------------------------------
# Served job stream


def job_stream(count: int = 2000, seed: int = 7, rate_per_s: float = 100.0,
               n_lo: float = 1e3, n_hi: float = 1e6):
    """Job descriptors: n log-uniform in [n_lo, n_hi], mean degree U[4, 32],
    type ER / R-MAT / grid equally likely, m in {16, 64, 256}, R in {1, 4},
    Poisson arrivals at ``rate_per_s``."""
    rng = np.random.default_rng(seed)
    jobs = []
    t = 0.0
    for j in range(count):
        t += rng.exponential(1.0 / rate_per_s)
        jobs.append({
            "id": j,
            "arrival_s": t,
            "n": int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi))))),
            "deg": float(rng.uniform(4, 32)),
            "kind": ("er", "rmat", "grid")[int(rng.integers(0, 3))],
            "log2m": (4, 6, 8)[int(rng.integers(0, 3))],
            "R": (1, 4)[int(rng.integers(0, 2))],
            "seed": int(rng.integers(1, 2**31)),
        })
    return jobs


def er_torch(n: int, arcs: int, seed: int = 1, device: str = "cpu"):
    """Directed ER on any torch device: `arcs` uniform draws, loops and
    duplicates removed (so slightly fewer arcs)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    s = torch.randint(0, n, (arcs,), generator=g, device=device, dtype=torch.int64)
    d = torch.randint(0, n, (arcs,), generator=g, device=device, dtype=torch.int64)
    keep = s != d
    keys = torch.unique(s[keep] * n + d[keep])
    counts = torch.bincount(keys // n, minlength=n)
    off = torch.zeros(n + 1, dtype=torch.int64, device=device)
    torch.cumsum(counts, 0, out=off[1:])
    return off, (keys % n).to(torch.int32)


def job_graph_torch(job: dict, device: str = "cuda"):
    """The graph of one job descriptor as device tensors."""
    import torch

    n, kind = job["n"], job["kind"]
    if kind == "er":
        return er_torch(n, int(n * job["deg"]), seed=job["seed"], device=device)
    if kind == "rmat":
        scale = max(4, int(round(math.log2(n))))
        return rmat(scale, edge_factor=max(1, int(round(job["deg"]))), seed=job["seed"],
                    device=device, as_numpy=False)
    off, tgt = grid2d(max(2, int(round(math.sqrt(n)))))
    return torch.from_numpy(off).to(device), torch.from_numpy(tgt).to(device)


def job_graph(job: dict):
    """The graph of one job descriptor (CSR on the host)."""
    n, kind = job["n"], job["kind"]
    if kind == "er":
        return er(n, min(int(n * job["deg"]), n * (n - 1)), seed=job["seed"])
    if kind == "rmat":
        scale = max(4, int(round(math.log2(n))))
        return rmat(scale, edge_factor=max(1, int(round(job["deg"]))), seed=job["seed"])
    side = max(2, int(round(math.sqrt(n))))
    return grid2d(side)
