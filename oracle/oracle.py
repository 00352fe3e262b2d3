"""HyperANF CPU oracle: ctypes binding of ``hanf_oracle.c``.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module.  It shares no code with
the CUDA library: the C source next to this file restates HyperANF
(Algorithms 1 and 2, Sections 3-5 of the paper) on its own.

Every function returns plain numpy values.  The shared object is compiled by
``build()`` with gcc (``-O2 -fopenmp -ffp-contract=off``; no fast-math, so
floating point follows IEEE double rounding step by step).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hanf_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libhanf_oracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle library if it is missing or older than its source."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
           "-shared", "-fvisibility=hidden", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # A test may point at another build of this source (mutation tests).
        path = os.environ.get("HANF_ORACLE_LIB") or build()
        lib = ctypes.CDLL(path)
        lib.ora_splitmix64.restype = ctypes.c_uint64
        lib.ora_splitmix64.argtypes = [ctypes.c_uint64]
        lib.ora_run_seed.restype = ctypes.c_uint64
        lib.ora_run_seed.argtypes = [ctypes.c_uint64, ctypes.c_int32]
        lib.ora_place_hash.restype = None
        lib.ora_place_hash.argtypes = [ctypes.c_uint64, ctypes.c_int32, _i32p, _i32p]
        lib.ora_place.restype = None
        lib.ora_place.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int32, _i32p, _i32p]
        lib.ora_alpha.restype = ctypes.c_double
        lib.ora_alpha.argtypes = [ctypes.c_int32]
        lib.ora_size.restype = ctypes.c_double
        lib.ora_size.argtypes = [_u8p, ctypes.c_int32]
        lib.ora_init.restype = None
        lib.ora_init.argtypes = [_u8p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64]
        lib.ora_union_pass.restype = ctypes.c_int64
        lib.ora_union_pass.argtypes = [_i64p, _i32p, ctypes.c_int64, ctypes.c_int32,
                                       _u8p, _u8p, ctypes.c_int32]
        lib.ora_sum_sizes.restype = ctypes.c_double
        lib.ora_sum_sizes.argtypes = [_u8p, ctypes.c_int64, ctypes.c_int32]
        lib.ora_hyperanf.restype = ctypes.c_int32
        lib.ora_hyperanf.argtypes = [_i64p, _i32p, ctypes.c_int64, ctypes.c_int32,
                                     ctypes.c_uint64, _f64p, ctypes.c_int32, _i32p,
                                     _u8p, ctypes.c_int32]
        lib.ora_exact_nf.restype = ctypes.c_int32
        lib.ora_exact_nf.argtypes = [_i64p, _i32p, ctypes.c_int64, _i64p, ctypes.c_int32]
        lib.ora_ball_registers.restype = None
        lib.ora_ball_registers.argtypes = [_i64p, _i32p, ctypes.c_int64, ctypes.c_int64,
                                           ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                           _u8p]
        lib.ora_symmetric_final_sum.restype = ctypes.c_double
        lib.ora_symmetric_final_sum.argtypes = [_i64p, _i32p, ctypes.c_int64, ctypes.c_int32,
                                                ctypes.c_uint64]
        lib.ora_ed_interval.restype = None
        lib.ora_ed_interval.argtypes = [_f64p, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                        _i32p, _i32p]
        lib.ora_node_stats.restype = ctypes.c_int32
        lib.ora_node_stats.argtypes = [_i64p, _i32p, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_uint64, ctypes.c_double, ctypes.c_int32,
                                       _f64p, _f64p, _i32p, _i32p]
        lib.ora_sizes.restype = None
        lib.ora_sizes.argtypes = [_u8p, ctypes.c_int64, ctypes.c_int32, _f64p, ctypes.c_int32]
        lib.ora_neumaier_sum.restype = ctypes.c_double
        lib.ora_neumaier_sum.argtypes = [_f64p, ctypes.c_int64]
        lib.ora_fnv1a64.restype = ctypes.c_uint64
        lib.ora_fnv1a64.argtypes = [_u8p, ctypes.c_int64]
        lib.ora_digest.restype = ctypes.c_uint64
        lib.ora_digest.argtypes = [_u8p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32]
        lib.ora_seq_stats.restype = None
        lib.ora_seq_stats.argtypes = [_f64p, ctypes.c_int32, ctypes.c_double, _f64p, _f64p,
                                      _i32p, _i32p]
        lib.ora_stats.restype = None
        lib.ora_stats.argtypes = [_f64p, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                  _f64p]
        _lib = lib
        return lib


def _p(arr, typ):
    return arr.ctypes.data_as(typ)


def _csr(offsets, targets):
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    tgt = np.ascontiguousarray(targets, dtype=np.int32)
    if tgt.size == 0:
        tgt = np.zeros(1, dtype=np.int32)      # valid pointer, never read
    return off, tgt, off.size - 1


# --------------------------------------------------------------------------
# Section 3.1: hash, register placement


def splitmix64(x: int) -> int:
    return int(_load().ora_splitmix64(ctypes.c_uint64(x & (2**64 - 1))))


def run_seed(seed: int, r: int) -> int:
    return int(_load().ora_run_seed(seed & (2**64 - 1), r))


def place_hash(h: int, b: int) -> tuple[int, int]:
    i, r = ctypes.c_int32(), ctypes.c_int32()
    _load().ora_place_hash(h & (2**64 - 1), b, ctypes.byref(i), ctypes.byref(r))
    return i.value, r.value


def place(v: int, seed: int, b: int) -> tuple[int, int]:
    i, r = ctypes.c_int32(), ctypes.c_int32()
    _load().ora_place(v & (2**64 - 1), seed & (2**64 - 1), b, ctypes.byref(i), ctypes.byref(r))
    return i.value, r.value


# --------------------------------------------------------------------------
# Algorithm 1


def alpha(m: int) -> float:
    return float(_load().ora_alpha(m))


def size(M) -> float:
    M = np.ascontiguousarray(M, dtype=np.uint8)
    return float(_load().ora_size(_p(M, _u8p), M.size))


# --------------------------------------------------------------------------
# Algorithm 2


def init(n: int, b: int, seed: int) -> np.ndarray:
    c = np.empty((max(n, 1), 1 << b), dtype=np.uint8)
    _load().ora_init(_p(c, _u8p), n, b, seed & (2**64 - 1))
    return c[:n]


def union_pass(offsets, targets, c: np.ndarray, threads: int = 1):
    """One Jacobi pass; returns (c_next, number of changed counters)."""
    off, tgt, n = _csr(offsets, targets)
    c = np.ascontiguousarray(c, dtype=np.uint8)
    cn = np.empty_like(c)
    ch = _load().ora_union_pass(_p(off, _i64p), _p(tgt, _i32p), n, c.shape[1],
                                _p(c, _u8p), _p(cn, _u8p), threads)
    return cn, int(ch)


def sum_sizes(c: np.ndarray) -> float:
    c = np.ascontiguousarray(c, dtype=np.uint8)
    return float(_load().ora_sum_sizes(_p(c, _u8p), c.shape[0], c.shape[1]))


def sizes(c: np.ndarray, threads: int = 1) -> np.ndarray:
    """size(c[v]) of every node (Algorithm 1), nodes split across threads."""
    c = np.ascontiguousarray(c, dtype=np.uint8)
    out = np.empty(max(c.shape[0], 1), dtype=np.float64)
    _load().ora_sizes(_p(c, _u8p), c.shape[0], c.shape[1], _p(out, _f64p), threads)
    return out[:c.shape[0]]


def neumaier_sum(x) -> float:
    """Neumaier-compensated sum, left to right."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(_load().ora_neumaier_sum(_p(x, _f64p), x.size))


def sum_sizes_mt(c: np.ndarray, threads: int = 1) -> float:
    """N = sum_v size(c[v]): the value ora_sum_sizes returns, with the
    per-node sizes computed on several threads."""
    return neumaier_sum(sizes(c, threads))


def fnv1a64(data: bytes) -> int:
    buf = np.frombuffer(bytes(data) or b"\0", dtype=np.uint8)
    return int(_load().ora_fnv1a64(_p(buf, _u8p), len(data)))


def digest(c: np.ndarray, threads: int = 1) -> int:
    """Sum over nodes v (mod 2^64) of FNV-1a-64(v as 8 little-endian bytes,
    then the m register bytes of c[v])."""
    c = np.ascontiguousarray(c, dtype=np.uint8)
    if c.shape[0] == 0:
        return 0
    return int(_load().ora_digest(_p(c, _u8p), c.shape[0], c.shape[1], threads))


def hyperanf(offsets, targets, b: int, seed: int, cap: int = 4096, threads: int = 1,
             want_regs: bool = False):
    """Algorithm 2 for one run.  Returns (N[0..T], T, registers or None)."""
    off, tgt, n = _csr(offsets, targets)
    N = np.zeros(cap, dtype=np.float64)
    T = ctypes.c_int32()
    regs = np.empty((max(n, 1), 1 << b), dtype=np.uint8) if want_regs else None
    rc = _load().ora_hyperanf(_p(off, _i64p), _p(tgt, _i32p), n, b, seed & (2**64 - 1),
                              _p(N, _f64p), cap, ctypes.byref(T),
                              _p(regs, _u8p) if want_regs else None, threads)
    if rc != 0:
        raise RuntimeError(f"oracle hyperanf failed (rc={rc}, cap={cap})")
    return N[:T.value + 1].copy(), T.value, (regs[:n] if want_regs else None)


# --------------------------------------------------------------------------
# Exact references by breadth-first search


def exact_nf(offsets, targets, cap: int | None = None) -> np.ndarray:
    """Exact N(t), t = 0..D (D = largest finite distance)."""
    off, tgt, n = _csr(offsets, targets)
    cap = cap or (n + 1)
    N = np.zeros(cap, dtype=np.int64)
    D = _load().ora_exact_nf(_p(off, _i64p), _p(tgt, _i32p), n, _p(N, _i64p), cap)
    if D < 0:
        raise RuntimeError("cap too small for exact_nf")
    return N[:D + 1].copy()


def ball_registers(offsets, targets, v: int, r: int, b: int, seed: int) -> np.ndarray:
    off, tgt, n = _csr(offsets, targets)
    out = np.zeros(1 << b, dtype=np.uint8)
    _load().ora_ball_registers(_p(off, _i64p), _p(tgt, _i32p), n, v, r, b,
                               seed & (2**64 - 1), _p(out, _u8p))
    return out


def symmetric_final_sum(offsets, targets, b: int, seed: int) -> float:
    """N(T) of a symmetric graph from its connected components."""
    off, tgt, n = _csr(offsets, targets)
    r = _load().ora_symmetric_final_sum(_p(off, _i64p), _p(tgt, _i32p), n, b, seed & (2**64 - 1))
    if r < 0:
        raise MemoryError("oracle allocation failed")
    return float(r)


# --------------------------------------------------------------------------
# Sections 4-5: statistics


def stats(N, alpha_: float = 0.9, exclude_zero: bool = False) -> dict:
    N = np.ascontiguousarray(N, dtype=np.float64)
    out = np.zeros(5, dtype=np.float64)
    _load().ora_stats(_p(N, _f64p), N.size - 1, alpha_, int(exclude_zero), _p(out, _f64p))
    return {"ed": out[0], "ied": out[1], "mean": out[2], "var": out[3], "spid": out[4]}


def hyperanf_runs(offsets, targets, b: int, seed: int, R: int, cap: int = 4096,
                  threads: int = 1):
    """R independent runs with seed_r = splitmix64(seed + r)."""
    return [hyperanf(offsets, targets, b, run_seed(seed, r), cap=cap, threads=threads)[:2]
            for r in range(R)]


def ed_interval(N, alpha_: float = 0.9, eps: float = 0.0):
    """Algorithm 3's bracket [D-, D+] of the effective diameter."""
    N = np.ascontiguousarray(N, dtype=np.float64)
    lo, hi = ctypes.c_int32(), ctypes.c_int32()
    _load().ora_ed_interval(_p(N, _f64p), N.size - 1, alpha_, eps, ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def stats_runs(N_runs, alpha_: float = 0.9, exclude_zero: bool = False) -> dict:
    """Mean and sample standard deviation over runs of each statistic."""
    per = [stats(N, alpha_, exclude_zero) for N in N_runs]
    out = {}
    for k in ("ed", "ied", "mean", "var", "spid"):
        x = np.array([p[k] for p in per])
        out[k] = (float(x.mean()), float(x.std(ddof=1)) if len(x) > 1 else 0.0)
    return out


def seq_stats(E, alpha_: float = 0.9) -> dict:
    """Per-node statistics of one node's estimates E(0..T)."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    reach, dist = ctypes.c_double(), ctypes.c_double()
    ecc, rad = ctypes.c_int32(), ctypes.c_int32()
    _load().ora_seq_stats(_p(E, _f64p), E.size - 1, alpha_, ctypes.byref(reach),
                          ctypes.byref(dist), ctypes.byref(ecc), ctypes.byref(rad))
    return {"reach": reach.value, "dist": dist.value, "ecc": ecc.value, "radius": rad.value}


def node_stats(offsets, targets, b: int, seed: int, alpha_: float = 0.9, cap: int = 512) -> dict:
    """Per-node reach, distance sum, eccentricity and radius estimates."""
    off, tgt, n = _csr(offsets, targets)
    reach = np.zeros(max(n, 1))
    dist = np.zeros(max(n, 1))
    ecc = np.zeros(max(n, 1), dtype=np.int32)
    rad = np.zeros(max(n, 1), dtype=np.int32)
    T = _load().ora_node_stats(_p(off, _i64p), _p(tgt, _i32p), n, b, seed & (2**64 - 1), alpha_,
                               cap, _p(reach, _f64p), _p(dist, _f64p), _p(ecc, _i32p),
                               _p(rad, _i32p))
    if T < 0:
        raise RuntimeError(f"oracle node_stats failed ({T})")
    return {"reach": reach[:n], "dist": dist[:n], "ecc": ecc[:n], "radius": rad[:n], "T": T}


def exact_node_distances(offsets, targets):
    """Exact per-node (reachable count, distance sum, eccentricity) by BFS."""
    off = np.asarray(offsets, dtype=np.int64)
    tgt = np.asarray(targets, dtype=np.int64)
    n = off.size - 1
    reach = np.zeros(n, dtype=np.int64)
    dsum = np.zeros(n, dtype=np.int64)
    ecc = np.zeros(n, dtype=np.int64)
    for x in range(n):
        dist = {x: 0}
        frontier = [x]
        d = 0
        while frontier:
            d += 1
            nxt = []
            for u in frontier:
                for w in tgt[off[u]:off[u + 1]]:
                    w = int(w)
                    if w not in dist:
                        dist[w] = d
                        nxt.append(w)
            frontier = nxt
        reach[x] = len(dist)
        dsum[x] = sum(dist.values())
        ecc[x] = max(dist.values())
    return reach, dsum, ecc
