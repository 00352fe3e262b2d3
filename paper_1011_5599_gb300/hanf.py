"""Thin ctypes binding of ``libhanf.so`` (declared in ``include/hanf.h``).

Argument marshalling only: every step of HyperANF runs in the CUDA library.
PyTorch provides the device workspace the library carves its buffers from and
the stream it launches on.  If the library has not been built, every entry
point raises ``HanfError`` -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libhanf.so")

HANF_OK, HANF_EINVAL, HANF_ENOMEM, HANF_ECUDA, HANF_ERANGE, HANF_ESTATE = 0, -1, -2, -3, -4, -5
HANF_ETIMEOUT, HANF_ECANCELLED = -6, -7
FRONTIER = {"off": 0, "pull": 1, "auto": 2}

# Every function declared in include/hanf.h.
EXPORTS = ("hanf_default_opts", "hanf_workspace_size", "hanf_create", "hanf_estimate",
           "hanf_iterate", "hanf_run", "hanf_registers", "hanf_digest", "hanf_pass_begin",
           "hanf_pass_collect", "hanf_pass_apply", "hanf_pass_end", "hanf_current_t",
           "hanf_counters",
           "hanf_trace", "hanf_checkpoint_size", "hanf_checkpoint_save", "hanf_checkpoint_load",
           "hanf_continue", "hanf_node_stats", "hanf_node_radius", "hanf_stats",
           "hanf_ed_interval", "hanf_stats_runs",
           "hanf_estimate_static", "hanf_autotune",
           "hanf_server_create",
           "hanf_server_submit", "hanf_server_wait", "hanf_server_cancel", "hanf_server_stats",
           "hanf_server_destroy", "hanf_destroy", "hanf_last_error")
TRACE_NAMES = ("t", "mode", "changed", "union_ms", "arcs_scanned", "arcs_gathered", "own_reads",
               "writes")

COUNTER_NAMES = ("passes", "arcs_scanned", "arcs_gathered", "own_reads", "writes",
                 "union_launches", "union_ms", "launches", "estimate_ms", "push_passes")


class HanfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"hanf error {code}: {msg}")
        self.code = code


class Job(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("arcs", ctypes.c_int64),
                ("offsets", ctypes.c_void_p), ("targets", ctypes.c_void_p),
                ("graph_on_device", ctypes.c_int32), ("log2m", ctypes.c_int32),
                ("runs", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


class Opts(ctypes.Structure):
    _fields_ = [("runs", ctypes.c_int32), ("frontier", ctypes.c_int32),
                ("push_den", ctypes.c_int32), ("small_max_deg", ctypes.c_int32),
                ("hub_min_deg", ctypes.c_int32), ("history_cap", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("dense_den", ctypes.c_int32), ("relabel", ctypes.c_int32),
                ("gather_variant", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("node_stats", ctypes.c_int32), ("num_graphs", ctypes.c_int32),
                ("graph_base", ctypes.POINTER(ctypes.c_int64)),
                ("graph_nodes", ctypes.POINTER(ctypes.c_int64)),
                ("graph_seeds", ctypes.POINTER(ctypes.c_uint64)),
                ("seeds", ctypes.POINTER(ctypes.c_uint64)), ("stream", ctypes.c_void_p),
                ("scatter_den", ctypes.c_int32), ("l2_hot_bytes", ctypes.c_int64)]


_lock = threading.Lock()
_lib = None
_vp, _i32, _i64, _u64, _f64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                               ctypes.c_uint64, ctypes.c_double)


def lib():
    """The loaded library (raises HanfError if it was never built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise HanfError(HANF_ESTATE, f"{LIB_PATH} is missing: build it with "
                                         "__graft_entry__.build() (CUDA path only, no fallback)")
        L = ctypes.CDLL(LIB_PATH)
        L.hanf_default_opts.restype = None
        L.hanf_default_opts.argtypes = [ctypes.POINTER(Opts)]
        L.hanf_workspace_size.restype = _i32
        L.hanf_workspace_size.argtypes = [_i64, _i64, _i32, ctypes.POINTER(Opts), _i32,
                                          ctypes.POINTER(ctypes.c_size_t)]
        L.hanf_create.restype = _i32
        L.hanf_create.argtypes = [ctypes.POINTER(_vp), _i64, _i64, _vp, _vp, _i32, _i32, _u64,
                                  ctypes.POINTER(Opts), _vp, ctypes.c_size_t]
        L.hanf_estimate.restype = _i32
        L.hanf_estimate.argtypes = [_vp, ctypes.POINTER(_f64)]
        L.hanf_iterate.restype = _i32
        L.hanf_iterate.argtypes = [_vp, ctypes.POINTER(_i64)]
        L.hanf_run.restype = _i32
        L.hanf_run.argtypes = [_vp, _i32, ctypes.POINTER(_f64), _i32, ctypes.POINTER(_i32)]
        L.hanf_registers.restype = _i32
        L.hanf_registers.argtypes = [_vp, _i32, _i64, _i64, _vp]
        L.hanf_digest.restype = _i32
        L.hanf_digest.argtypes = [_vp, _i32, _i64, _i64, ctypes.POINTER(_u64)]
        L.hanf_pass_begin.restype = _i32
        L.hanf_pass_begin.argtypes = [_vp, ctypes.POINTER(_i32)]
        L.hanf_pass_collect.restype = _i32
        L.hanf_pass_collect.argtypes = [_vp, _i64, _i64, _vp, _vp, _i64, ctypes.POINTER(_i64)]
        L.hanf_pass_apply.restype = _i32
        L.hanf_pass_apply.argtypes = [_vp, _vp, _vp, _i64]
        L.hanf_pass_end.restype = _i32
        L.hanf_pass_end.argtypes = [_vp, ctypes.POINTER(_i64)]
        L.hanf_current_t.restype = _i32
        L.hanf_current_t.argtypes = [_vp, ctypes.POINTER(_i32)]
        L.hanf_counters.restype = _i32
        L.hanf_counters.argtypes = [_vp, ctypes.POINTER(_f64), _i32]
        L.hanf_trace.restype = _i32
        L.hanf_trace.argtypes = [_vp, ctypes.POINTER(_f64), _i32, ctypes.POINTER(_i32)]
        L.hanf_stats.restype = _i32
        L.hanf_stats.argtypes = [ctypes.POINTER(_f64), _i32, _f64, _i32, ctypes.POINTER(_f64)]
        L.hanf_estimate_static.restype = _i32
        L.hanf_estimate_static.argtypes = [_vp, _i64, _i32, _i32, _vp, _vp]
        L.hanf_checkpoint_size.restype = _i32
        L.hanf_checkpoint_size.argtypes = [_vp, ctypes.POINTER(ctypes.c_size_t)]
        L.hanf_checkpoint_save.restype = _i32
        L.hanf_checkpoint_save.argtypes = [_vp, _vp, ctypes.c_size_t]
        L.hanf_checkpoint_load.restype = _i32
        L.hanf_checkpoint_load.argtypes = [_vp, _vp, ctypes.c_size_t]
        L.hanf_continue.restype = _i32
        L.hanf_continue.argtypes = [_vp, _i32, ctypes.POINTER(_f64), _i32, ctypes.POINTER(_i32)]
        L.hanf_node_stats.restype = _i32
        L.hanf_node_stats.argtypes = [_vp, _i32, _i64, _i64, _vp, _vp, _vp]
        L.hanf_node_radius.restype = _i32
        L.hanf_node_radius.argtypes = [_vp, _f64, _i32, _i64, _i64, _vp]
        L.hanf_ed_interval.restype = _i32
        L.hanf_ed_interval.argtypes = [ctypes.POINTER(_f64), _i32, _f64, _f64,
                                       ctypes.POINTER(_i32), ctypes.POINTER(_i32)]
        L.hanf_stats_runs.restype = _i32
        L.hanf_stats_runs.argtypes = [ctypes.POINTER(_f64), _i32, _i32, ctypes.POINTER(_i32), _f64,
                                      _i32, ctypes.POINTER(_f64)]
        L.hanf_autotune.restype = _i32
        L.hanf_autotune.argtypes = [_i64, _i64, _vp, _vp, _i32, _i32, _u64, ctypes.POINTER(Opts),
                                    _vp, ctypes.c_size_t, ctypes.c_char_p, ctypes.POINTER(Opts),
                                    ctypes.POINTER(_f64)]
        L.hanf_server_create.restype = _i32
        L.hanf_server_create.argtypes = [ctypes.POINTER(_vp), _vp, ctypes.c_size_t, _i32,
                                         ctypes.POINTER(Opts)]
        L.hanf_server_submit.restype = _i32
        L.hanf_server_submit.argtypes = [_vp, ctypes.POINTER(Job), ctypes.POINTER(_u64)]
        L.hanf_server_wait.restype = _i32
        L.hanf_server_wait.argtypes = [_vp, _u64, _i32, ctypes.POINTER(_f64), _i32,
                                       ctypes.POINTER(_i32), ctypes.POINTER(_f64)]
        L.hanf_server_cancel.restype = _i32
        L.hanf_server_cancel.argtypes = [_vp, _u64]
        L.hanf_server_stats.restype = _i32
        L.hanf_server_stats.argtypes = [_vp, ctypes.POINTER(_f64), _i32]
        L.hanf_server_destroy.restype = None
        L.hanf_server_destroy.argtypes = [_vp]
        L.hanf_destroy.restype = None
        L.hanf_destroy.argtypes = [_vp]
        L.hanf_last_error.restype = ctypes.c_char_p
        L.hanf_last_error.argtypes = []
        _lib = L
        return L


def torch_int32():
    import torch
    return torch.int32


def check(rc: int):
    if rc != HANF_OK:
        raise HanfError(rc, lib().hanf_last_error().decode())


def default_opts() -> Opts:
    o = Opts()
    lib().hanf_default_opts(ctypes.byref(o))
    return o


def make_opts(runs=1, frontier="auto", push_den=4, small_max_deg=0, hub_min_deg=0,
              history_cap=0, use_graph=False, profile=False, seeds=None, stream=None,
              dense_den=0, relabel=True, gather_variant=0, layout=0, node_stats=False,
              graph_base=None, graph_nodes=None, graph_seeds=None, scatter_den=0,
              l2_hot_bytes=0):
    o = default_opts()
    o.scatter_den = scatter_den
    o.l2_hot_bytes = int(l2_hot_bytes)
    o.runs = runs
    o.frontier = FRONTIER[frontier] if isinstance(frontier, str) else int(frontier)
    o.push_den = push_den
    o.small_max_deg = small_max_deg
    o.hub_min_deg = hub_min_deg
    o.history_cap = history_cap
    o.use_graph = int(bool(use_graph))
    o.profile = int(bool(profile))
    o.dense_den = dense_den
    o.relabel = int(bool(relabel))
    o.gather_variant = gather_variant
    o.node_stats = int(bool(node_stats))
    o.layout = {"byte": 0, "packed": 1}.get(layout, layout) if isinstance(layout, str) else layout
    keep = None
    if seeds is not None:
        keep = (ctypes.c_uint64 * len(seeds))(*[int(s) & (2**64 - 1) for s in seeds])
        o.seeds = ctypes.cast(keep, ctypes.POINTER(ctypes.c_uint64))
    o.stream = stream
    keep = [keep]
    if graph_base is not None:
        K = len(graph_nodes)
        gb = (ctypes.c_int64 * (K + 1))(*[int(x) for x in graph_base])
        gn = (ctypes.c_int64 * K)(*[int(x) for x in graph_nodes])
        o.num_graphs = K
        o.graph_base = ctypes.cast(gb, ctypes.POINTER(ctypes.c_int64))
        o.graph_nodes = ctypes.cast(gn, ctypes.POINTER(ctypes.c_int64))
        keep += [gb, gn]
        if graph_seeds is not None:
            gs = (ctypes.c_uint64 * K)(*[int(x) & (2**64 - 1) for x in graph_seeds])
            o.graph_seeds = ctypes.cast(gs, ctypes.POINTER(ctypes.c_uint64))
            keep.append(gs)
    return o, keep


def workspace_size(n, arcs, log2m, opts: Opts, copy_graph: bool) -> int:
    out = ctypes.c_size_t()
    check(lib().hanf_workspace_size(n, arcs, log2m, ctypes.byref(opts), int(copy_graph),
                                    ctypes.byref(out)))
    return out.value


def stats(N, T=None, alpha=0.9, exclude_zero=False) -> dict:
    N = np.ascontiguousarray(N, dtype=np.float64)
    T = N.size - 1 if T is None else T
    out = np.zeros(5, dtype=np.float64)
    check(lib().hanf_stats(N.ctypes.data_as(ctypes.POINTER(_f64)), T, alpha, int(exclude_zero),
                           out.ctypes.data_as(ctypes.POINTER(_f64))))
    return {"ed": out[0], "ied": out[1], "mean": out[2], "var": out[3], "spid": out[4]}


def estimate_static(regs, n: int, log2m: int, runs: int, out, stream=None) -> None:
    """hanf_estimate_static: N of a device register array without allocating.

    ``regs`` is a CUDA uint8 tensor of n rows of runs * 2^log2m bytes and
    ``out`` a CUDA float64 tensor of ``runs`` values; the call only enqueues
    the work on ``stream`` (default: torch's current stream)."""
    import torch

    if stream is None:
        stream = torch.cuda.current_stream(regs.device)
    check(lib().hanf_estimate_static(regs.data_ptr() if n > 0 else None, n, log2m, runs,
                                     out.data_ptr(), stream.cuda_stream))


def ed_interval(N, alpha=0.9, eps=0.0):
    """Algorithm 3: (D-, D+) bracketing the effective diameter (-1 = none)."""
    N = np.ascontiguousarray(N, dtype=np.float64)
    lo, hi = _i32(), _i32()
    check(lib().hanf_ed_interval(N.ctypes.data_as(ctypes.POINTER(_f64)), N.size - 1, alpha, eps,
                                 ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


def stats_runs(N_runs, alpha=0.9, exclude_zero=False) -> dict:
    """Mean and standard deviation over runs of ed, ied, mean, var, spid."""
    R = len(N_runs)
    cap = max(len(x) for x in N_runs)
    N = np.zeros((R, cap), dtype=np.float64)
    T = np.zeros(R, dtype=np.int32)
    for r, x in enumerate(N_runs):
        N[r, :len(x)] = x
        T[r] = len(x) - 1
    out = np.zeros(10, dtype=np.float64)
    check(lib().hanf_stats_runs(N.ctypes.data_as(ctypes.POINTER(_f64)), R, cap,
                                T.ctypes.data_as(ctypes.POINTER(_i32)), alpha, int(exclude_zero),
                                out.ctypes.data_as(ctypes.POINTER(_f64))))
    keys = ("ed", "ied", "mean", "var", "spid")
    return {k: (out[i], out[5 + i]) for i, k in enumerate(keys)}


class HyperANF:
    """One HyperANF context (Algorithm 2 over R seeded runs) on a CUDA device.

    ``offsets``/``targets`` may be numpy arrays or host tensors (copied into
    the workspace) or CUDA tensors (borrowed; kept referenced here).
    """

    def __init__(self, offsets, targets, log2m: int, seed: int = 0x5EED, *, runs: int = 1,
                 frontier="auto", push_den: int = 4, small_max_deg: int = 0,
                 hub_min_deg: int = 0, history_cap: int = 0, use_graph: bool = False,
                 profile: bool = False, seeds=None, device=None, stream=None,
                 dense_den: int = 0, relabel: bool = True, gather_variant: int = 0,
                 layout=0, node_stats: bool = False, graph_base=None, graph_nodes=None,
                 graph_seeds=None, scatter_den: int = 0, l2_hot_bytes: int = 0):
        import torch

        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        on_dev = isinstance(offsets, torch.Tensor) and offsets.is_cuda
        if on_dev:
            self._off = offsets.to(torch.int64).contiguous()
            self._tgt = targets.to(torch.int32).contiguous()
            off_p, tgt_p = self._off.data_ptr(), self._tgt.data_ptr()
            n, arcs = self._off.numel() - 1, self._tgt.numel()
        else:
            if isinstance(offsets, torch.Tensor):
                self._off = offsets.to(torch.int64).contiguous()
                self._tgt = targets.to(torch.int32).contiguous()
                off_p, tgt_p = self._off.data_ptr(), self._tgt.data_ptr()
                n, arcs = self._off.numel() - 1, self._tgt.numel()
            else:
                self._off = np.ascontiguousarray(offsets, dtype=np.int64)
                self._tgt = np.ascontiguousarray(targets, dtype=np.int32)
                off_p, tgt_p = self._off.ctypes.data, self._tgt.ctypes.data
                n, arcs = self._off.size - 1, self._tgt.size
            if arcs == 0:
                tgt_p = None
        self.n, self.arcs, self.log2m, self.m, self.R = n, arcs, log2m, 1 << log2m, runs
        self._opts, self._seed_keep = make_opts(runs, frontier, push_den, small_max_deg,
                                                hub_min_deg, history_cap, use_graph, profile,
                                                seeds, self.stream.cuda_stream, dense_den,
                                                relabel, gather_variant, layout, node_stats,
                                                graph_base, graph_nodes, graph_seeds,
                                                scatter_den, l2_hot_bytes)
        self.K = 1 if graph_nodes is None else len(graph_nodes)
        self.S = self.K * runs
        self.graph_base = graph_base
        self.graph_nodes = graph_nodes
        size = workspace_size(n, arcs, log2m, self._opts, not on_dev)
        self.workspace_bytes = size
        with torch.cuda.device(self.device):
            self._ws = torch.empty(size, dtype=torch.uint8, device=self.device)
        ctx = ctypes.c_void_p()
        check(lib().hanf_create(ctypes.byref(ctx), n, arcs, off_p, tgt_p, int(on_dev), log2m,
                                seed & (2**64 - 1), ctypes.byref(self._opts),
                                self._ws.data_ptr(), size))
        self._ctx = ctx

    # -- Algorithm 2 -------------------------------------------------------
    @classmethod
    def batch(cls, graphs, log2m: int, seed: int = 0x5EED, *, graph_seeds=None, **kw):
        """Many graphs in one context: their padded disjoint union, each graph
        starting at a multiple of 64 nodes.  N(t) and T come per slot
        (graph g, run r) = g * runs + r; graph g's registers are the node
        range [graph_base[g], graph_base[g] + graph_nodes[g])."""
        degs, tgts, base, nodes = [], [], [0], []
        for off, tgt in graphs:
            off = np.asarray(off, dtype=np.int64)
            n_g = off.size - 1
            span = -(-n_g // 64) * 64
            d = np.zeros(span, dtype=np.int64)
            d[:n_g] = np.diff(off)
            degs.append(d)
            tgts.append(np.asarray(tgt, dtype=np.int64) + base[-1])
            nodes.append(n_g)
            base.append(base[-1] + span)
        offsets = np.zeros(base[-1] + 1, dtype=np.int64)
        if base[-1]:
            np.cumsum(np.concatenate(degs), out=offsets[1:])
        targets = (np.concatenate(tgts) if tgts else np.zeros(0)).astype(np.int32)
        return cls(offsets, targets, log2m, seed, graph_base=base, graph_nodes=nodes,
                   graph_seeds=graph_seeds, **kw)

    def estimate(self) -> np.ndarray:
        out = np.zeros(self.S, dtype=np.float64)
        check(lib().hanf_estimate(self._ctx, out.ctypes.data_as(ctypes.POINTER(_f64))))
        return out

    def iterate(self) -> int:
        ch = ctypes.c_int64()
        check(lib().hanf_iterate(self._ctx, ctypes.byref(ch)))
        return ch.value

    def run(self, max_iter: int = 4096, cap: int = 4096):
        """Whole Algorithm 2.  Returns (list of N_s(0..T_s), array of T_s) for
        every slot s (= run r for one graph)."""
        N = np.zeros((self.S, cap), dtype=np.float64)
        T = np.zeros(self.S, dtype=np.int32)
        check(lib().hanf_run(self._ctx, max_iter, N.ctypes.data_as(ctypes.POINTER(_f64)), cap,
                             T.ctypes.data_as(ctypes.POINTER(_i32))))
        return [N[r, :T[r] + 1].copy() for r in range(self.S)], T

    def run_raw(self, N: np.ndarray, T: np.ndarray, max_iter: int = 4096) -> int:
        """hanf_run into caller arrays (S x cap, S); returns the status code."""
        return lib().hanf_run(self._ctx, max_iter, N.ctypes.data_as(ctypes.POINTER(_f64)),
                              N.shape[1], T.ctypes.data_as(ctypes.POINTER(_i32)))

    def checkpoint(self) -> np.ndarray:
        """The state after the last pass as a host byte array."""
        size = ctypes.c_size_t()
        check(lib().hanf_checkpoint_size(self._ctx, ctypes.byref(size)))
        buf = np.empty(size.value, dtype=np.uint8)
        check(lib().hanf_checkpoint_save(self._ctx, buf.ctypes.data, size.value))
        return buf

    def restore(self, buf: np.ndarray) -> None:
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        check(lib().hanf_checkpoint_load(self._ctx, buf.ctypes.data, buf.size))

    def resume(self, max_iter: int = 4096, cap: int = 4096):
        """Passes from the current state to stabilisation (hanf_continue)."""
        N = np.zeros((self.S, cap), dtype=np.float64)
        T = np.zeros(self.S, dtype=np.int32)
        check(lib().hanf_continue(self._ctx, max_iter, N.ctypes.data_as(ctypes.POINTER(_f64)), cap,
                                  T.ctypes.data_as(ctypes.POINTER(_i32))))
        return [N[r, :T[r] + 1].copy() for r in range(self.S)], T

    def node_stats(self, run: int = 0, first: int = 0, count: int | None = None) -> dict:
        """reach E_v(T), distance sum and eccentricity estimate per node."""
        count = self.n - first if count is None else count
        reach = np.zeros(max(count, 1))
        dist = np.zeros(max(count, 1))
        ecc = np.zeros(max(count, 1), dtype=np.int32)
        check(lib().hanf_node_stats(self._ctx, run, first, count, reach.ctypes.data,
                                    dist.ctypes.data, ecc.ctypes.data))
        return {"reach": reach[:count], "dist": dist[:count], "ecc": ecc[:count]}

    def node_radius(self, alpha: float = 0.9, run: int = 0, first: int = 0,
                    count: int | None = None) -> np.ndarray:
        """First t with E_v(t) >= alpha E_v(T) (replays the run once)."""
        count = self.n - first if count is None else count
        rad = np.zeros(max(count, 1), dtype=np.int32)
        check(lib().hanf_node_radius(self._ctx, alpha, run, first, count, rad.ctypes.data))
        return rad[:count]

    def registers(self, run: int = 0, first: int = 0, count: int | None = None) -> np.ndarray:
        count = self.n - first if count is None else count
        out = np.zeros((max(count, 1), self.m), dtype=np.uint8)
        check(lib().hanf_registers(self._ctx, run, first, count, out.ctypes.data))
        return out[:count]

    def digest(self, run: int = 0, first: int = 0, count: int | None = None) -> int:
        """hanf_digest: check value of run r's registers of input ids
        first..first+count-1 (ids counted from ``first``)."""
        count = self.n - first if count is None else count
        out = _u64()
        check(lib().hanf_digest(self._ctx, run, first, count, ctypes.byref(out)))
        return out.value

    # -- one pass in steps (node-sharded runs) ------------------------------
    def pass_begin(self) -> bool:
        """hanf_pass_begin: False if the run is already stable."""
        started = _i32()
        check(lib().hanf_pass_begin(self._ctx, ctypes.byref(started)))
        return bool(started.value)

    def pass_collect(self, first: int, count: int, cap: int | None = None):
        """hanf_pass_collect: (ids, rows) CUDA tensors of this range's changed
        nodes, rows of R*m bytes."""
        import torch
        cap = 1024 if cap is None else cap
        while True:
            ids = torch.empty(max(cap, 1), dtype=torch.int32, device=self.device)
            rows = torch.empty((max(cap, 1), self.R * self.m), dtype=torch.uint8, device=self.device)
            n = _i64()
            rc = lib().hanf_pass_collect(self._ctx, first, count, ids.data_ptr(), rows.data_ptr(),
                                         cap, ctypes.byref(n))
            if rc == HANF_ERANGE and n.value > cap:
                cap = n.value
                continue
            check(rc)
            return ids[:n.value], rows[:n.value]

    def pass_apply(self, ids, rows) -> None:
        """hanf_pass_apply of CUDA tensors (int32 ids, uint8 rows)."""
        k = int(ids.numel())
        ids = ids.to(device=self.device, dtype=torch_int32()).contiguous()
        rows = rows.to(device=self.device).contiguous()
        check(lib().hanf_pass_apply(self._ctx, ids.data_ptr() if k else None,
                                    rows.data_ptr() if k else None, k))
        self._keep_apply = (ids, rows)     # alive until the stream has used them

    def pass_end(self) -> int:
        """hanf_pass_end: nodes changed in the pass, over all shards."""
        ch = _i64()
        check(lib().hanf_pass_end(self._ctx, ctypes.byref(ch)))
        self._keep_apply = None
        return ch.value

    @property
    def t(self) -> int:
        t = ctypes.c_int32()
        check(lib().hanf_current_t(self._ctx, ctypes.byref(t)))
        return t.value

    def counters(self) -> dict:
        out = np.zeros(len(COUNTER_NAMES), dtype=np.float64)
        check(lib().hanf_counters(self._ctx, out.ctypes.data_as(ctypes.POINTER(_f64)),
                                  len(COUNTER_NAMES)))
        return dict(zip(COUNTER_NAMES, out.tolist()))

    def trace(self) -> list:
        """Per-pass rows of the last run (profile=True, host-loop driver)."""
        rows = ctypes.c_int32()
        out = np.zeros((4096, len(TRACE_NAMES)), dtype=np.float64)
        check(lib().hanf_trace(self._ctx, out.ctypes.data_as(ctypes.POINTER(_f64)), 4096,
                               ctypes.byref(rows)))
        return [dict(zip(TRACE_NAMES, r.tolist())) for r in out[:rows.value]]

    def close(self):
        if getattr(self, "_ctx", None):
            lib().hanf_destroy(self._ctx)
            self._ctx = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def autotune(offsets, targets, log2m: int, seed: int = 0x5EED, cache_path=None, device=None,
             **opts) -> tuple[dict, float]:
    """hanf_autotune on a graph; returns ({small_max_deg, hub_min_deg,
    gather_variant, scatter_den}, best ms).  ``offsets``/``targets`` as for
    HyperANF."""
    import torch

    device = torch.device(device if device is not None else "cuda")
    on_dev = isinstance(offsets, torch.Tensor) and offsets.is_cuda
    if on_dev:
        off, tgt = offsets.to(torch.int64).contiguous(), targets.to(torch.int32).contiguous()
        op, tp, n, arcs = off.data_ptr(), tgt.data_ptr(), off.numel() - 1, tgt.numel()
    else:
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        tgt = np.ascontiguousarray(targets, dtype=np.int32)
        op, tp, n, arcs = off.ctypes.data, (tgt.ctypes.data if tgt.size else None), off.size - 1, tgt.size
    stream = torch.cuda.current_stream(device)
    base, keep = make_opts(stream=stream.cuda_stream, **opts)
    widest, _ = make_opts(hub_min_deg=4096, small_max_deg=32, gather_variant=1, **opts)
    size = workspace_size(n, arcs, log2m, widest, not on_dev)
    ws = torch.empty(size, dtype=torch.uint8, device=device)
    best = Opts()
    ms = _f64()
    path = None if cache_path is None else str(cache_path).encode()
    check(lib().hanf_autotune(n, arcs, op, tp, int(on_dev), log2m, seed & (2**64 - 1),
                              ctypes.byref(base), ws.data_ptr(), size, path, ctypes.byref(best),
                              ctypes.byref(ms)))
    return ({"small_max_deg": best.small_max_deg, "hub_min_deg": best.hub_min_deg,
             "gather_variant": best.gather_variant, "scatter_den": best.scatter_den}, ms.value)


class Server:
    """Continuous-batching HyperANF server (hanf_server_*): jobs are admitted
    in arrival order into a device arena of ``arena_bytes`` (the HBM budget)
    and run on ``workers`` concurrent streams."""

    INFO = ("latency_ms", "queued_ms", "run_ms", "T", "workspace_bytes")

    def __init__(self, arena_bytes: int, workers: int = 4, device=None, **opts):
        import torch

        self.device = torch.device(device if device is not None else "cuda")
        self._opts, self._keep = make_opts(**opts)
        self._arena = torch.empty(arena_bytes, dtype=torch.uint8, device=self.device)
        self._jobs = {}
        srv = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(lib().hanf_server_create(ctypes.byref(srv), self._arena.data_ptr(), arena_bytes,
                                           workers, ctypes.byref(self._opts)))
        self._srv = srv

    def submit(self, offsets, targets, log2m: int, seed: int, runs: int = 1,
               max_iter: int = 0) -> int:
        import torch

        on_dev = isinstance(offsets, torch.Tensor) and offsets.is_cuda
        if on_dev:
            off, tgt = offsets.to(torch.int64).contiguous(), targets.to(torch.int32).contiguous()
            op, tp = off.data_ptr(), tgt.data_ptr()
        else:
            off = np.ascontiguousarray(offsets, dtype=np.int64)
            tgt = np.ascontiguousarray(targets, dtype=np.int32)
            op, tp = off.ctypes.data, (tgt.ctypes.data if tgt.size else None)
        n = (off.numel() if on_dev else off.size) - 1
        arcs = tgt.numel() if on_dev else tgt.size
        job = Job(n, arcs, op, tp, int(on_dev), log2m, runs, max_iter, seed & (2**64 - 1))
        jid = _u64()
        check(lib().hanf_server_submit(self._srv, ctypes.byref(job), ctypes.byref(jid)))
        self._jobs[jid.value] = (off, tgt, runs)     # keep the graph alive until waited
        return jid.value

    def wait(self, jid: int, timeout_ms: int = -1, cap: int = 4097):
        """Returns (list of N_r(0..T_r), array of T_r, info dict)."""
        runs = self._jobs[jid][2]
        N = np.zeros((runs, cap), dtype=np.float64)
        T = np.zeros(runs, dtype=np.int32)
        info = np.zeros(len(self.INFO), dtype=np.float64)
        rc = lib().hanf_server_wait(self._srv, jid, timeout_ms,
                                    N.ctypes.data_as(ctypes.POINTER(_f64)), cap,
                                    T.ctypes.data_as(ctypes.POINTER(_i32)),
                                    info.ctypes.data_as(ctypes.POINTER(_f64)))
        if rc != HANF_ETIMEOUT:
            self._jobs.pop(jid, None)
        check(rc)
        return [N[r, :T[r] + 1].copy() for r in range(runs)], T, dict(zip(self.INFO, info.tolist()))

    def cancel(self, jid: int):
        check(lib().hanf_server_cancel(self._srv, jid))

    def stats(self) -> dict:
        out = np.zeros(7, dtype=np.float64)
        check(lib().hanf_server_stats(self._srv, out.ctypes.data_as(ctypes.POINTER(_f64)), 7))
        return dict(zip(("queued", "running", "completed", "failed", "largest_free",
                         "arena_bytes", "contexts"), out.tolist()))

    def close(self):
        if getattr(self, "_srv", None):
            lib().hanf_server_destroy(self._srv)
            self._srv = None
            self._arena = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
