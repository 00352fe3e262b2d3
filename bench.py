#!/usr/bin/env python
"""Throughput benchmark of HyperANF run to stabilisation on GB300.

One step = the whole hot path on one batch: initialise every counter, then
estimate N(t) and run union passes (frontier-skipping, systolic or pure push
when few counters change) until a pass changes nothing.  The metric is
arcs x registers merged per second of union-kernel time: every successor
counter a pass actually gathers merges m registers per run, so a step counts
(arcs gathered) * m * R, divided by the time of the union launches (measured
with CUDA events in a profiled run of the same context options).  The nominal
rate of Algorithm 2 (every arc merged in every pass, passes * arcs * m * R per
step time) and the gathered merges per step time are reported beside it.

Default workload: directed R-MAT scale 27 (134M nodes, edge factor 16,
~2.1e9 arcs, int64 offsets / int32 targets), m = 64 byte registers, one run.
The timed steps run the whole loop as one CUDA graph (the product's fastest
driver).  Inputs (>= 10 GB of CSR and counters) are far larger than the
129 MB L2, so no flush is needed between steps.

With torchrun (N > 1) every rank runs an independent replica on its own GPU
(the path needs no exchange): value = all ranks' merges / max rank time.
``--impl reference`` times the CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "arcs×registers merged/s per iteration"
METRIC_DEFINITION = ("(successor counters gathered) x m x R per step / union-kernel time per "
                     "step; nominal_rate = passes x arcs x m x R / step time")
UNIT = "arcs*registers/s"

WORKLOADS = {
    "rmat27": dict(kind="rmat", scale=27, ef=16, sym=False, log2m=6, runs=1,
                   text="directed R-MAT scale 27, edge factor 16 (a,b,c,d = .57,.19,.19,.05, "
                        "scrambled labels, loops and duplicate arcs removed), m=64 byte "
                        "registers, 1 run, frontier auto"),
    "rmat22": dict(kind="rmat", scale=22, ef=16, sym=False, log2m=6, runs=1,
                   text="directed R-MAT scale 22, edge factor 16, m=64, 1 run (profiling case)"),
    "rmat24": dict(kind="rmat", scale=24, ef=16, sym=False, log2m=6, runs=1,
                   text="directed R-MAT scale 24, edge factor 16, m=64, 1 run (profiling case)"),
    "rmat24sym": dict(kind="rmat", scale=24, ef=16, sym=True, log2m=7, runs=1,
                      text="symmetrised R-MAT scale 24, edge factor 16, m=128, 1 run"),
    "rmat23sym": dict(kind="rmat", scale=23, ef=16, sym=True, log2m=7, runs=1,
                      text="symmetrised R-MAT scale 23, edge factor 16, m=128, 1 run "
                           "(profiling case)"),
    "web20": dict(kind="web", n=1 << 20, log2m=6, runs=8,
                  text="web-like n=2^20 (power-law out-degree 2.1, mean 16, host blocks), "
                       "m=64, R=8 runs batched"),
    "web18": dict(kind="web", n=1 << 18, log2m=6, runs=8,
                  text="web-like n=2^18, m=64, R=8 runs batched (profiling case)"),
    "er": dict(kind="er", n=10000, arcs=50000, log2m=4, runs=1,
               text="directed ER n=10^4, 5*10^4 arcs, m=16, 1 run"),
}
# bounded CPU samples of the same recipes for the oracle
CPU_SAMPLE = {"rmat27": dict(kind="rmat", scale=22, ef=16, sym=False),
              "rmat22": dict(kind="rmat", scale=18, ef=16, sym=False),
              "rmat24": dict(kind="rmat", scale=19, ef=16, sym=False),
              "rmat24sym": dict(kind="rmat", scale=18, ef=16, sym=True),
              "rmat23sym": dict(kind="rmat", scale=17, ef=16, sym=True),
              "web20": dict(kind="web", n=1 << 16),
              "web18": dict(kind="web", n=1 << 14),
              "er": dict(kind="er", n=10000, arcs=50000)}


def make_graph(spec, seed, device):
    from paper_1011_5599_gb300 import graphs as G
    if spec["kind"] == "rmat":
        return G.rmat(spec["scale"], edge_factor=spec["ef"], seed=seed, symmetrise=spec["sym"],
                      device=device, as_numpy=False)
    import torch
    if spec["kind"] == "web":
        off, tgt = G.web(spec["n"], seed=seed)
    else:
        off, tgt = G.er(spec["n"], spec["arcs"], seed=seed)
    return torch.from_numpy(off).to(device), torch.from_numpy(tgt).to(device)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_index_for(device):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v for v in vis.split(",") if v.strip()]
    if ids and ids[device.index or 0].strip().isdigit():
        return int(ids[device.index or 0])
    return device.index or 0


# ------------------------------------------------------------------ profile summary

def ncu_traffic(workload, layout="byte"):
    """DRAM bytes of a dense pass's union launches (the launch the roofline
    reports) from the committed ncu record of this workload and register
    layout (profiles/traffic.json), or None when there is none or the kernel
    source changed since the capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[workload][layout]
    except (OSError, KeyError, ValueError):
        return None
    src = open(os.path.join(ROOT, "paper_1011_5599_gb300", "csrc", "hanf_kernels.cu"), "rb").read()
    if hashlib.sha256(src).hexdigest() != rec.get("kernel_source_sha256"):
        return None
    return float(rec["traffic_bytes_per_launch"])


def union_bytes(row, n, row_bytes, record_bytes=0):
    """Algorithmic bytes of one pass's union launches from its trace row: 4
    per scanned arc (target id), a row per gathered successor, own counter
    read and counter written, the offsets of every node in a pull pass over
    all nodes (8 n), and the changed-node bitmaps read and written (n / 4).
    Pass 0 reads a c_0 record of record_bytes (2 per run) per successor and
    own counter instead of a row where the library has them (byte layout,
    rows up to 1 KB; record_bytes = 0: rows)."""
    got = record_bytes if (record_bytes and int(row["t"]) == 0) else row_bytes
    b = 4 * row["arcs_scanned"] + got * (row["arcs_gathered"] + row["own_reads"]) + \
        row_bytes * row["writes"]
    if int(row["mode"]) in (0, 2):
        b += 8 * n
    return b + n / 4


def dense_row_passes(rows, n, row_bytes, record_bytes=0):
    """(time ms, algorithmic bytes, count) of the dense pull passes that
    gather rows: the roofline's dominant launches.  Pass 0 reads c_0 records
    instead of rows where the library has them (record_bytes > 0) and is left
    out."""
    ms, nbytes, count = 0.0, 0.0, 0
    for r in rows:
        if int(r["mode"]) == 2 and (int(r["t"]) > 0 or not record_bytes):
            ms += r["union_ms"]
            nbytes += union_bytes(r, n, row_bytes, record_bytes)
            count += 1
    return ms, nbytes, count


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ------------------------------------------------------------------ oracle (CPU) arm

def sample_graph(workload, seed):
    """The bounded CPU sample graph of a workload's recipe."""
    from paper_1011_5599_gb300 import graphs as G
    spec = CPU_SAMPLE[workload]
    if spec["kind"] == "rmat":
        off, tgt = G.rmat(spec["scale"], edge_factor=spec["ef"], seed=seed,
                          symmetrise=spec["sym"], device="cpu")
        desc = (f"R-MAT scale {spec['scale']} ef {spec['ef']}{' symmetrised' if spec['sym'] else ''}"
                f" (same recipe), {tgt.size} arcs")
    elif spec["kind"] == "web":
        off, tgt = G.web(spec["n"], seed=seed)
        desc = f"web-like n={spec['n']}, {tgt.size} arcs"
    else:
        off, tgt = G.er(spec["n"], spec["arcs"], seed=seed)
        desc = f"ER n={spec['n']}, {tgt.size} arcs"
    return off, tgt, desc


_SAMPLES = {}   # (workload, seed) -> (offsets, targets, description), built once


def oracle_sample(workload, seed, threads):
    """Time the oracle (Algorithm 2, all arcs every pass) on a bounded sample
    graph of the same recipe.  Returns (rate, seconds, description)."""
    from oracle import oracle as O
    wl = WORKLOADS[workload]
    if (workload, seed) not in _SAMPLES:
        _SAMPLES[(workload, seed)] = sample_graph(workload, seed)
    off, tgt, desc = _SAMPLES[(workload, seed)]
    m = 1 << wl["log2m"]
    t0 = time.perf_counter()
    merges = 0
    for r in range(wl["runs"]):
        N, T, _ = O.hyperanf(off, tgt, wl["log2m"], O.run_seed(0x5EED, r), threads=threads)
        merges += (T + 1) * tgt.size * m
    dt = time.perf_counter() - t0
    return merges / dt, dt, desc + f", m={m}, R={wl['runs']}, run to stabilisation"


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    threads = os.cpu_count() or 1
    from oracle import oracle as O
    O.build()
    for _ in range(args.warmup):
        oracle_sample(args.workload, 1, threads)
    rates, secs = [], 0.0
    desc = ""
    for _ in range(args.steps):
        r, s, desc = oracle_sample(args.workload, 1, threads)
        rates.append(r)
        secs += s
    value = sum(rates) / len(rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["text"], "sample": desc},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ served stream

def run_serve(args):
    """Served stream: jobs with Poisson arrivals through the continuous-
    batching server vs one job at a time (create + run per job, FIFO), same
    jobs, same GPU, identical results required."""
    import numpy as np
    import torch

    from paper_1011_5599_gb300 import build as B
    from paper_1011_5599_gb300 import graphs as G
    B.build()
    from paper_1011_5599_gb300.hanf import HyperANF, Server

    device = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(device)
    # graph shapes: a pool of seeded graphs drawn from the job recipe; every
    # job takes one of them with its own m, R, HyperLogLog seed and arrival
    shapes = G.job_stream(args.pool, seed=7, rate_per_s=1.0)
    t0 = time.perf_counter()
    pool = [G.job_graph_torch(j, device=str(device)) for j in shapes]
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    picks = np.random.default_rng(9).integers(0, args.pool, args.jobs)
    jobs = G.job_stream(args.jobs, seed=8, rate_per_s=1.0)
    for j, k in zip(jobs, picks):
        j.update(kind=shapes[k]["kind"], n=shapes[k]["n"], shape=int(k))
    graphs = [pool[k] for k in picks]
    arcs = [int(g[1].numel()) for g in graphs]

    # one launch per job: service time of each job alone
    service, plain_N = [], []
    for j, (off, tgt) in zip(jobs, graphs):
        torch.cuda.synchronize()
        a = time.perf_counter()
        with HyperANF(off, tgt, j["log2m"], j["seed"], runs=j["R"], device=device) as h:
            N, T = h.run()
        service.append(time.perf_counter() - a)
        plain_N.append(N)
    capacity = len(jobs) / sum(service)
    by_kind = {}
    for j, sv, N in zip(jobs, service, plain_N):
        d = by_kind.setdefault(j["kind"], {"jobs": 0, "service_s": 0.0, "max_T": 0})
        d["jobs"] += 1
        d["service_s"] += sv
        d["max_T"] = max(d["max_T"], max(len(x) for x in N) - 1)
    results = {}
    for load in args.loads:
        rate = load * capacity
        rng = np.random.default_rng(11)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, len(jobs)))
        # FIFO single server with the measured service times
        fin, lat_plain = 0.0, []
        for arr, sv in zip(arrivals, service):
            fin = max(arr, fin) + sv
            lat_plain.append(fin - arr)
        makespan_plain = fin - arrivals[0]
        # served, in real time
        with Server(args.arena_gb << 30, workers=args.workers, device=device) as srv:
            ids = [None] * len(jobs)
            done = {}

            def collect():
                for k in range(len(jobs)):
                    while ids[k] is None:
                        time.sleep(0.0002)
                    done[k] = srv.wait(ids[k])

            th = threading.Thread(target=collect)
            th.start()
            start = time.perf_counter()
            for k, (j, (off, tgt)) in enumerate(zip(jobs, graphs)):
                delay = start + (arrivals[k] - arrivals[0]) - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                ids[k] = srv.submit(off, tgt, j["log2m"], j["seed"], runs=j["R"])
            th.join()
            makespan = time.perf_counter() - start
        lat = [done[k][2]["latency_ms"] / 1e3 for k in range(len(jobs))]
        same = all(np.array_equal(a, b) for k in range(len(jobs))
                   for a, b in zip(plain_N[k], done[k][0]))
        results[f"{load:g}"] = {
            "arrival_rate_jobs_s": rate,
            "served": {"jobs_s": len(jobs) / makespan, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                       "p99_ms": 1e3 * float(np.percentile(lat, 99))},
            "one_per_job": {"jobs_s": len(jobs) / makespan_plain,
                            "p50_ms": 1e3 * float(np.percentile(lat_plain, 50)),
                            "p99_ms": 1e3 * float(np.percentile(lat_plain, 99))},
            "identical_results": same}
    best = results[f"{max(args.loads):g}"]
    line = {"metric": "served jobs/s (p50/p99 latency)", "value": best["served"]["jobs_s"],
            "unit": "jobs/s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": f"served stream: {len(jobs)} jobs over {args.pool} seeded "
                                   "graphs, n log-uniform in "
                                   "[1e3, 1e6], mean degree U[4, 32], ER / R-MAT / 2D grid, "
                                   "m in {16, 64, 256}, R in {1, 4}, Poisson arrivals at the "
                                   "given fractions of the one-job-at-a-time capacity",
                       "workers": args.workers, "arena_gb": args.arena_gb,
                       "graphs_resident_on_device": True, "graph_gen_s": round(t_gen, 1),
                       "total_arcs": int(sum(arcs))},
            "one_per_job_capacity_jobs_s": capacity, "by_kind": by_kind, "loads": results}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ batched graphs

def run_batch(args):
    """Many small graphs: one context (and one graph-captured launch) for the
    whole batch vs one context per graph, same graphs, identical results."""
    import numpy as np
    import torch

    from paper_1011_5599_gb300 import build as B
    from paper_1011_5599_gb300 import graphs as G
    B.build()
    from paper_1011_5599_gb300.hanf import HyperANF

    device = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(device)
    jobs = G.job_stream(args.jobs, seed=12, rate_per_s=1.0, n_lo=1e3, n_hi=3e4)
    graphs = [G.job_graph(j) for j in jobs]
    seeds = [j["seed"] for j in jobs]
    log2m, R = 6, 4
    arcs = sum(int(t.size) for _, t in graphs)

    def one_per_graph():
        out = []
        for (off, tgt), sd in zip(graphs, seeds):
            with HyperANF(off, tgt, log2m, sd, runs=R, use_graph=True, device=device) as h:
                out.append(h.run())
        return out

    def batched():
        with HyperANF.batch(graphs, log2m, graph_seeds=[s for s in seeds], runs=R, use_graph=True,
                            device=device) as h:
            return h.run()

    for _ in range(2):          # warm-up (allocator, module load)
        one_per_graph()
        batched()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    single = one_per_graph()
    torch.cuda.synchronize()
    t_single = time.perf_counter() - t0
    t0 = time.perf_counter()
    Nb, Tb = batched()
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    # same T and N(t) to 1e-12 (node order and hence summation order differ:
    # batches store graphs in input order, single contexts relabel)
    same = all(single[g][1][r] == Tb[g * R + r]
               and np.allclose(single[g][0][r], Nb[g * R + r], rtol=1e-12, atol=0)
               for g in range(len(graphs)) for r in range(R))
    line = {"metric": "graphs/s (batched in one context vs one context per graph)",
            "value": len(graphs) / t_batch, "unit": "graphs/s", "n_gpus": 1, "steps": 1,
            "warmup": 2, "ms_per_step": 1e3 * t_batch, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": f"{len(graphs)} graphs, n log-uniform in [1e3, 3e4], mean "
                                   "degree U[4, 32], ER / R-MAT / grid, m=64, R=4",
                       "total_arcs": arcs},
            "one_context_per_graph": {"graphs_s": len(graphs) / t_single, "ms": 1e3 * t_single},
            "batched": {"graphs_s": len(graphs) / t_batch, "ms": 1e3 * t_batch},
            "same_T_and_N_within_1e-12": same}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ one graph across ranks

def run_sharded(args):
    """One graph over the ranks: contiguous node shards balanced by arcs, every
    rank holding all counters and its own arcs, changed counters all-gathered
    after each pass (NCCL).  value = all ranks' gathered merges / the slowest
    rank's time per step; the same graph on every N (strong scaling)."""
    import torch
    import torch.distributed as dist

    from paper_1011_5599_gb300 import build as B
    from paper_1011_5599_gb300 import sharded
    B.build()
    from paper_1011_5599_gb300.hanf import HyperANF
    from paper_1011_5599_gb300.replicas import reduce_max_sum

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    device = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(device)
    if world > 1:
        dist.init_process_group("nccl", device_id=device)
    wl = WORKLOADS[args.workload]
    log2m, R = wl["log2m"], wl["runs"]
    m = 1 << log2m
    off, tgt = make_graph(wl, args.seed, device)            # the same graph on every rank
    n, arcs = off.numel() - 1, tgt.numel()
    ranges = sharded.partition(off, world)
    lo, hi = ranges[rank]
    loff, ltgt = sharded.local_csr(off, tgt, lo, hi)
    del off, tgt
    torch.cuda.empty_cache()
    exchange = sharded.group_exchange if world > 1 else sharded.local_exchange

    def step():
        with HyperANF(loff, ltgt, log2m, 0x5EED, runs=R, frontier="auto", device=device,
                      l2_hot_bytes=args.l2_hot_mb << 20) as h:
            N, T = sharded.run([h], [(lo, hi)], exchange=exchange)
            c = h.counters()
        return N, T, c

    for _ in range(args.warmup):
        step()
    gathered, launches = 0.0, 0
    with ClockSampler(gpu_index_for(device)) as clocks:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            N, T, c = step()
            gathered += c["arcs_gathered"] * m * R
            launches += int(c["launches"])
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        elapsed = time.perf_counter() - t0
    step_all, gathered_all = reduce_max_sum(elapsed / args.steps, gathered / args.steps,
                                            device=device)
    line = {"metric": METRIC, "value": gathered_all / step_all, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * step_all,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "metric_definition": "(successor counters gathered) x m x R per step, all ranks / "
                                 "slowest rank's step time (context creation, stepped passes "
                                 "and the exchange included)",
            "config": {"workload": wl["text"], "n": n, "arcs": arcs, "m": m, "runs": R,
                       "parallelism": f"node shards x{world}", "shard_arcs": int(ltgt.numel()),
                       "l2": "inputs larger than L2 (no flush)"},
            "T": int(T), "N_T": float(N[-1][0]), "gpu_launches": launches,
            "clocks": clocks.summary()}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ CUDA arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat27",
                    choices=sorted(WORKLOADS) + ["serve", "batch"])
    ap.add_argument("--jobs", type=int, default=2000, help="served stream: number of jobs")
    ap.add_argument("--pool", type=int, default=100, help="served stream: distinct graphs")
    ap.add_argument("--workers", type=int, default=8, help="served stream: server workers")
    ap.add_argument("--arena-gb", type=int, default=64, help="served stream: HBM budget")
    ap.add_argument("--loads", type=float, nargs="+", default=[0.5, 0.8, 1.5],
                    help="served stream: arrival rate as a fraction of one-at-a-time capacity")
    ap.add_argument("--driver", default="graph", choices=["host", "graph"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--trace", action="store_true", help="per-pass trace of one run on stderr")
    ap.add_argument("--gather-variant", type=int, default=0, choices=[0, 1, 2, 3, 4])
    ap.add_argument("--dense-den", type=int, default=0,
                    help="dense pull passes while the changed nodes' in-arcs are at least "
                         "arcs/dense_den (0 = library default)")
    ap.add_argument("--scatter-den", type=int, default=0,
                    help="pure-push passes below arcs/scatter_den changed in-arcs (0 = library "
                         "default, negative = never)")
    ap.add_argument("--layout", default="byte", choices=["byte", "packed"],
                    help="register layout: one byte each, or five bit-planes")
    ap.add_argument("--autotune", action="store_true",
                    help="pick degree split and gather variant with hanf_autotune first")
    ap.add_argument("--sharded", action="store_true",
                    help="one graph across the ranks (node shards exchanging changed counters "
                         "every pass; strong scaling) instead of one replica per rank")
    ap.add_argument("--l2-hot-mb", type=int, default=0,
                    help="persisting-L2 window over the hottest counter rows, MiB (0 = library "
                         "default, negative = off)")
    ap.add_argument("--profile-steps", type=int, default=2,
                    help="runs of the profiled context that give the union-kernel time")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.sharded:
        return run_sharded(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1011_5599_gb300 import build as B
    B.build()
    from paper_1011_5599_gb300.hanf import HyperANF

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    if world > 1:
        dist.init_process_group("nccl", device_id=device)

    def barrier():
        if world > 1:
            dist.barrier()

    wl = WORKLOADS[args.workload]
    log2m, R = wl["log2m"], wl["runs"]
    m = 1 << log2m
    W = m * R
    row_bytes = 5 * m // 8 if args.layout == "packed" else W   # bytes per stored counter row
    rec_bytes = 2 * R if args.layout == "byte" and W <= 1024 else 0   # pass 0's c_0 records
    t_gen = time.perf_counter()
    off, tgt = make_graph(wl, args.seed + rank, device)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    n, arcs = off.numel() - 1, tgt.numel()
    stream = torch.cuda.current_stream(device)

    tuned = {"gather_variant": args.gather_variant, "layout": args.layout}
    tune_ms = None
    if args.autotune:
        from paper_1011_5599_gb300.hanf import autotune
        cache = os.path.join(ROOT, "paper_1011_5599_gb300", "_lib", "tune_cache.txt")
        t_tune = time.perf_counter()
        tuned, tune_ms = autotune(off, tgt, log2m, 0x5EED, cache_path=cache, device=device,
                                  runs=R, frontier="auto", layout=args.layout)
        tuned["layout"] = args.layout
        print(json.dumps({"autotune": tuned, "best_ms": tune_ms,
                          "tuning_s": time.perf_counter() - t_tune}), file=sys.stderr)
    kw = dict(scatter_den=args.scatter_den, dense_den=args.dense_den,
              l2_hot_bytes=args.l2_hot_mb << 20)
    kw.update(tuned)          # the tuner's choices, where it made one
    h = HyperANF(off, tgt, log2m, 0x5EED, runs=R, frontier="auto", device=device,
                 use_graph=args.driver == "graph", **kw)
    for _ in range(args.warmup):
        h.run()

    nominal = 0
    gathered = 0
    launches = 0
    passes_list, T_list = [], []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_index_for(device)) as clocks:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            N, T = h.run()
            c = h.counters()
            nominal += c["passes"] * arcs * m * R
            gathered += c["arcs_gathered"] * m * R
            launches += int(c["launches"])
            passes_list.append(int(c["passes"]))
            T_list.append(int(max(T)))
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    h.close()
    del h

    # ---- union-kernel time: the same options with per-pass CUDA events ----
    hp = HyperANF(off, tgt, log2m, 0x5EED, runs=R, frontier="auto", device=device,
                  profile=True, **kw)
    hp.run()
    prof_ms, prof_bytes, prof_gathered, rows = 0.0, 0.0, 0, []
    dense_ms, dense_bytes, dense_n = 0.0, 0.0, 0
    for _ in range(max(args.profile_steps, 1)):
        hp.run()
        rows = hp.trace()
        prof_ms += sum(r["union_ms"] for r in rows)
        prof_bytes += sum(union_bytes(r, n, row_bytes, rec_bytes) for r in rows)
        prof_gathered += hp.counters()["arcs_gathered"] * m * R
        d_ms, d_bytes, d_n = dense_row_passes(rows, n, row_bytes, rec_bytes)
        dense_ms += d_ms
        dense_bytes += d_bytes
        dense_n += d_n
    psteps = max(args.profile_steps, 1)
    if prof_gathered != psteps * gathered / args.steps:
        raise RuntimeError("the profiled run gathered a different number of counters")
    if args.trace:
        for row in rows:
            gbs = union_bytes(row, n, row_bytes, rec_bytes) / (row["union_ms"] * 1e6)
            print(json.dumps({**row, "algorithmic_GBps": gbs}), file=sys.stderr)
    union_s = prof_ms / 1e3 / psteps                  # union-kernel seconds per step
    union_launch_ms = prof_ms / max(len(rows) * psteps, 1)
    bytes_per_launch = prof_bytes / max(len(rows) * psteps, 1)
    hp.close()
    del hp

    from paper_1011_5599_gb300.replicas import reduce_max_sum
    step_s = elapsed / args.steps
    step_all, gathered_all = reduce_max_sum(step_s, gathered / args.steps, device=device)
    union_all, _ = reduce_max_sum(union_s, 0.0, device=device)
    _, nominal_all = reduce_max_sum(0.0, nominal / args.steps, device=device)
    value = gathered_all / union_all
    stat = {}
    try:
        from paper_1011_5599_gb300.hanf import stats
        stat = stats(N[0])
    except Exception:
        pass

    # ---- end to end through the C ABI with host buffers (pinned) ----
    e2e = None
    if args.e2e_steps > 0:
        off_h = torch.empty(off.shape, dtype=torch.int64, pin_memory=True)
        tgt_h = torch.empty(tgt.shape, dtype=torch.int32, pin_memory=True)
        off_h.copy_(off)
        tgt_h.copy_(tgt)
        del off, tgt
        torch.cuda.empty_cache()
        e_merges, d2h = 0, 0     # merges counted as for value: counters gathered
        # one untimed warm-up so the workspace is in torch's cache
        HyperANF(off_h, tgt_h, log2m, 0x5EED, runs=R, frontier="auto", device=device).close()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        create_s = 0.0   # of which context creation (upload, validation, relabelling, transpose)
        for _ in range(args.e2e_steps):
            tc = time.perf_counter()
            with HyperANF(off_h, tgt_h, log2m, 0x5EED, runs=R, frontier="auto",
                          device=device, use_graph=args.driver == "graph") as he:
                torch.cuda.synchronize()
                create_s += time.perf_counter() - tc
                Ne, Te = he.run()
                e_merges += he.counters()["arcs_gathered"] * m * R
                d2h += sum(x.nbytes for x in Ne)
        torch.cuda.synchronize()
        e_el = time.perf_counter() - t0
        e_el, e_merges = reduce_max_sum(e_el, e_merges, device=device)
        e2e = {"value": e_merges / e_el, "unit": UNIT,
               "h2d_bytes_per_step": int((n + 1) * 8 + arcs * 4),
               "d2h_bytes_per_step": int(d2h // args.e2e_steps),
               "ms_per_step": 1e3 * e_el / args.e2e_steps,
               "create_ms_per_step": 1e3 * create_s / args.e2e_steps}

    # ---- CPU oracle baseline (rank 0, N = 1 only) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        rate, secs, desc = oracle_sample(args.workload, args.seed, threads)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{desc}; {secs:.1f} s"}

    peak, peak_kind = measured_peak()
    all_gbs = bytes_per_launch / (union_launch_ms / 1e3) / 1e9 if union_launch_ms > 0 else None
    if dense_n:
        launch_bytes, launch_ms = dense_bytes / dense_n, dense_ms / dense_n
        kernel = ("union launches of a dense pull pass that gathers rows, t >= 1 "
                  "(k_union_small_async, k_union_warp, ...)")
    else:
        launch_bytes, launch_ms = bytes_per_launch, union_launch_ms
        kernel = "union launches of one pass (k_union_*, k_scatter*, k_hub_finish)"
    achieved = launch_bytes / (launch_ms / 1e3) / 1e9 if launch_ms > 0 else None
    traffic = ncu_traffic(args.workload, args.layout)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": traffic, "peak_kind": peak_kind, "kernel": kernel,
            "algorithmic_bytes_per_launch": launch_bytes, "avg_launch_ms": launch_ms,
            "all_passes": {"algorithmic_bytes_per_launch": bytes_per_launch,
                           "avg_launch_ms": union_launch_ms, "achieved": all_gbs,
                           "frac": (all_gbs / peak) if all_gbs else None}}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * step_all, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "metric_definition": METRIC_DEFINITION,
            "union_ms_per_step": 1e3 * union_all,
            "nominal_rate": nominal_all / step_all,
            "gathered_per_step_time": gathered_all / step_all,
            "config": {"workload": wl["text"], "n": n, "arcs": arcs, "m": m, "runs": R,
                       "layout": args.layout, "frontier": "auto", "driver": args.driver,
                       "scatter_den": args.scatter_den or "default",
                       "dense_den": args.dense_den or "default",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "l2": "inputs larger than L2 (no flush)", "tuned": tuned,
                       "l2_hot_mb": args.l2_hot_mb or "default",
                       "graph_gen_s": round(t_gen, 2)},
            "T": T_list[-1], "passes_per_step": passes_list[-1],
            "stats": {k: float(v) for k, v in stat.items()},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks.summary()}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
