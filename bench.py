#!/usr/bin/env python
"""Benchmark of the DAWN hot path on B300.

Headline workload (default): single-source DAWN on RMAT scale 20 (2^20
vertices, edge factor 16, a/b/c/d = .57/.19/.19/.05, ids permuted,
symmetrised, duplicates and self-loops removed), 64 seeded sources drawn
from the vertices with out-degree >= 1, run one at a time.  One bench step
is those 64 single-source runs.  Metric: GTEPS = sum over sources of E_r
(arcs out of the reached vertices, the SOVM cost of Sec. 3.3) / device time.

Timing: CUDA events on the launching stream around each source's kernel; the
L2 is flushed (a 512 MiB buffer written) between sources, outside the event
pair.  W >= 3 untimed warm-up steps, then exactly K timed steps bracketed by a
barrier and a device synchronize; the max over ranks is reported.  Multi-GPU
runs are independent replicas (each rank runs the same 64 sources on its own
copy of the graph; no collective on the data path).

``--impl reference`` times the CPU oracle (Alg. 3, single thread) on the same
workload, a bounded sample of sources per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "SSSP GTEPS; batched sources/s and p50/p99 latency vs plain path, bit-exact"
WORKLOAD = "rmat20_sssp_64src"
CONFIG = {
    "workload": WORKLOAD,
    "graph": "RMAT scale 20, edge factor 16, a=.57 b=.19 c=.19 d=.05, permuted, symmetrised, dedup, no self-loops, seed 2",
    "sources": "64 distinct seeded sources (seed 5) with out-degree >= 1, one at a time",
    "dist": "int32, -1 unreachable",
    "l2": "flushed between sources (512 MiB buffer written outside the timed event pairs)",
    "parallelism": "replicas",
}
SSSP_SRC = ROOT / "paper_2208_04514_b300" / "csrc" / "sssp.cu"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def recorded_value(kernel_src: Path, profile: Path, key: str):
    """A figure recorded in a committed ncu summary under `key`, or None when
    absent or taken on a different version of the kernel source."""
    if not profile.exists():
        return None
    text = profile.read_text()
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", text)
    t = re.search(key + r":\s*([0-9.eE+]+)", text)
    if not h or not t:
        return None
    cur = hashlib.sha256(kernel_src.read_bytes()).hexdigest()
    return float(t.group(1)) if h.group(1) == cur[: len(h.group(1))] else None


def recorded_traffic(kernel_src: Path, profile: Path):
    """Per-launch DRAM bytes recorded in a committed ncu summary, or None when
    absent or taken on a different version of the kernel source."""
    if not profile.exists():
        return None
    text = profile.read_text()
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", text)
    t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not h or not t:
        return None
    cur = hashlib.sha256(kernel_src.read_bytes()).hexdigest()
    return float(t.group(1)) if h.group(1) == cur[: len(h.group(1))] else None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.25)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        if not self.lines:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes(n, stats):
    """B_alg of one SSSP: 4 E_r (col_idx of reached rows) + 8 V_r (their
    row_ptr pairs) + 8 V_r (frontier enqueue + dequeue) + 4 n (dist output) +
    pull levels * ceil(n/8) (one pass over the visited bitmap per pull level)."""
    return 4 * stats["edges"] + 16 * stats["reached"] + 4 * n + stats["pull_steps"] * ((n + 7) // 8)


def aggregate_replicas(ms_step: float, edges_per_step: int, world: int, device: str = "cpu"):
    """Whole-job figures of independent replicas: the step time is the MAX
    over ranks, the work is the SUM over ranks (each rank runs its own copy of
    the workload; no collective touches the data path)."""
    import torch
    import torch.distributed as distrib
    t = torch.tensor([ms_step], dtype=torch.float64, device=device)
    e = torch.tensor([edges_per_step], dtype=torch.int64, device=device)
    if world > 1:
        distrib.all_reduce(t, op=distrib.ReduceOp.MAX)
        distrib.all_reduce(e, op=distrib.ReduceOp.SUM)
    return float(t.item()), int(e.item())


def build_workload():
    from paper_2208_04514_b300 import graphgen as gg
    g = gg.rmat(20, 16, 0.57, 0.19, 0.19, seed=2, symmetrise=True)
    srcs = gg.sample_sources(g, 64, seed=5)
    return g, srcs


# ------------------------------------------------------------ reference arm --

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    g, srcs = build_workload()
    deg = g.out_degree()
    budget_s = args.ref_budget_s
    # each step: sources in order until the step's CPU budget is spent
    def one_step(offset):
        t0 = time.perf_counter()
        edges, done = 0, 0
        i = offset
        while True:
            s = int(srcs[i % len(srcs)])
            d = oracle.sssp_sovm(g.row_ptr, g.col_idx, s)
            edges += int(deg[d >= 0].sum())
            done += 1
            i += 1
            if time.perf_counter() - t0 >= budget_s or done >= len(srcs):
                break
        return edges, done, time.perf_counter() - t0
    for w in range(args.warmup):  # warm-up steps: one source each
        s = int(srcs[w % len(srcs)])
        oracle.sssp_sovm(g.row_ptr, g.col_idx, s)
    tot_e, tot_n, tot_t = 0, 0, 0.0
    for k in range(args.steps):
        e, d, t = one_step(args.warmup + k)
        tot_e += e
        tot_n += d
        tot_t += t
    gteps = tot_e / tot_t / 1e9
    sample = (f"{tot_n} single-source runs over {args.steps} steps, taken in order from the 64 sources "
              f"(a step stops after {budget_s:.0f} s or all 64); literal Alg. 3, one core")
    line = {
        "impl": "reference", "metric": METRIC, "value": gteps, "unit": "GTEPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic", "config": CONFIG,
        "cpu_baseline": {"value": gteps, "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": gteps, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- GPU arm --

def cpu_baseline(g, srcs, budget_s):
    import oracle
    deg = g.out_degree()
    t0 = time.perf_counter()
    edges, done = 0, 0
    for s in srcs:
        d = oracle.sssp_sovm(g.row_ptr, g.col_idx, int(s))
        edges += int(deg[d >= 0].sum())
        done += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    t = time.perf_counter() - t0
    # Alg. 2 (FIFO queue BFS), the fairer single-core baseline, on the same sources
    t1 = time.perf_counter()
    e2, d2 = 0, 0
    for s in srcs:
        d = oracle.bfs_queue(g.row_ptr, g.col_idx, int(s))
        e2 += int(deg[d >= 0].sum())
        d2 += 1
        if time.perf_counter() - t1 >= budget_s / 2:
            break
    t2 = time.perf_counter() - t1
    return {"value": edges / t / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"first {done} of the 64 sources, literal Alg. 3 single-threaded, {t:.1f} s",
            "alg2_queue_bfs": {"value": e2 / t2 / 1e9, "unit": "GTEPS", "cores": 1,
                               "sample": f"first {d2} of the 64 sources, Alg. 2 FIFO BFS single-threaded, {t2:.1f} s"},
            "host": host_cpu()}


def host_cpu():
    """nproc and the CPU model of the host the CPU figures ran on."""
    model = ""
    try:
        for line in Path("/proc/cpuinfo").read_text().splitlines():
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    import oracle
    return {"nproc": os.cpu_count(), "model": model, "oracle_build": "gcc " + " ".join(oracle.CFLAGS)}


def _flush(buf, i):
    buf.fill_(i)


def bench_lattice(dawn, torch, flush, nsrc=16, side=4096):
    """4096^2 lattice, bonds deleted with p = 0.1 (seed 3), 16 uniform sources
    (seed 7): GTEPS and microseconds per level of the level loop (AUTO: the
    single-cluster engine on this low-degree graph)."""
    from paper_2208_04514_b300 import graphgen as gg
    g = gg.lattice(side, side, 0.1, seed=3)
    srcs = gg.uniform_vertices(g.n, nsrc, seed=7)
    stream = torch.cuda.current_stream()
    h = dawn.dawn_graph_upload(g.row_ptr, g.col_idx, flags=dawn.DAWN_SYMMETRIC, stream=stream)
    dist = torch.empty(g.n, dtype=torch.int32, device="cuda")
    stats = torch.zeros((nsrc, dawn.STATS_WORDS), dtype=torch.int64, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in srcs]
    dawn.dawn_sssp_async(h, int(srcs[0]), dist, None, stats[0], stream)  # warm-up
    for i, s in enumerate(srcs):
        _flush(flush, i)
        ev[i][0].record(stream)
        dawn.dawn_sssp_async(h, int(s), dist, None, stats[i], stream)
        ev[i][1].record(stream)
    dawn.dawn_graph_sync(h, stream)
    ms = [a.elapsed_time(b) for a, b in ev]
    st = [dawn.stats_from_words(r) for r in stats.cpu().numpy()]
    last = dist.cpu().numpy()
    # the same sources in one dawn_sssp_many call: the sources are independent
    # (Sec. 3.3), so several clusters run side by side, each taking the next
    rows = torch.empty((nsrc, g.n), dtype=torch.int32, device="cuda")
    src_dev = torch.from_numpy(np.ascontiguousarray(srcs, dtype=np.int32)).cuda()
    dawn.dawn_sssp_many(h, src_dev, dist=rows, stream=stream)  # warm-up: sets up the clusters' buffers
    _flush(flush, 99)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    dawn.dawn_sssp_many(h, src_dev, dist=rows, stream=stream)
    e1.record(stream)
    dawn.dawn_graph_sync(h, stream)
    ms_many = e0.elapsed_time(e1)
    same_as_single = bool(np.array_equal(rows[-1].cpu().numpy(), last))
    del rows
    dawn.dawn_graph_free(h)
    edges = sum(x["edges"] for x in st)
    levels = sum(x["levels"] for x in st)
    # CPU: Alg. 2 (FIFO queue BFS, one core) on every source
    import oracle
    t0 = time.perf_counter()
    for s in srcs:
        oracle.bfs_queue(g.row_ptr, g.col_idx, int(s))
    cpu_ms = 1e3 * (time.perf_counter() - t0) / len(srcs)
    return {"workload": f"lattice{side}_p0.1_sssp_{nsrc}src", "n": g.n, "m": g.m,
            "gteps": edges / (sum(ms) * 1e-3) / 1e9, "ms_per_source": sum(ms) / nsrc,
            "us_per_level": 1e3 * sum(ms) / levels, "levels_median": statistics.median(x["levels"] for x in st),
            "l2": "flushed between sources",
            "many_sources_one_call": {"gteps": edges / (ms_many * 1e-3) / 1e9, "ms_total": ms_many,
                                      "speedup_vs_one_at_a_time": sum(ms) / ms_many,
                                      "last_row_equals_single_source_run": same_as_single,
                                      "note": "dawn_sssp_many, device rows: several single-source clusters side "
                                              "by side, each taking the next source; L2 flushed before the call"},
            "cpu_baseline": {"ms_per_source": cpu_ms, "kind": "oracle", "cores": 1,
                             "sample": f"all {len(srcs)} sources, Alg. 2 FIFO BFS (the literal Alg. 3 oracle scans "
                                       "all n vertices per level: ~10^11 checks per source here)"}}


def bench_tree(dawn, torch, flush, g, srcs, peak):
    """Shortest-path tree on the headline graph and sources: microseconds per
    source of dawn_sssp_tree_async (level loop + parent pass) against the
    plain level loop, L2 flushed between sources.  A full parent pass reads
    every in-arc of every reached vertex: 8 E_r (in_idx + the gathered dist)
    + 8 V_r (in_ptr pairs) + 8 n (dist read, parent write) bytes; with rows in
    ascending order it stops at the first qualifying arc, so that figure is
    an upper bound of the bytes it moves and the rate below is an effective
    rate against it, not a roofline fraction."""
    stream = torch.cuda.current_stream()
    h = dawn.dawn_graph_upload(g.row_ptr, g.col_idx, flags=dawn.DAWN_SYMMETRIC, stream=stream)
    dist = torch.empty(g.n, dtype=torch.int32, device="cuda")
    par = torch.empty(g.n, dtype=torch.int32, device="cuda")
    stats = torch.zeros((len(srcs), dawn.STATS_WORDS), dtype=torch.int64, device="cuda")
    deg = g.out_degree()
    times = {}
    for kind in ("sssp", "tree", "sssp", "tree"):  # second round is the measured one
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in srcs]
        for i, sv in enumerate(srcs):
            _flush(flush, i)
            ev[i][0].record(stream)
            if kind == "tree":
                dawn.dawn_sssp_tree_async(h, int(sv), dist, par, stream)
            else:
                dawn.dawn_sssp_async(h, int(sv), dist, None, stats[i], stream)
            ev[i][1].record(stream)
        dawn.dawn_graph_sync(h, stream)
        times[kind] = [a.elapsed_time(b) * 1e3 for a, b in ev]
    st = [dawn.stats_from_words(r) for r in stats.cpu().numpy()]
    dawn.dawn_graph_free(h)
    t_sssp = statistics.median(times["sssp"])
    t_tree = statistics.median(times["tree"])
    e_r = statistics.median(x["edges"] for x in st)
    v_r = statistics.median(x["reached"] for x in st)
    pass_us = max(t_tree - t_sssp, 1e-9)
    balg = 8 * e_r + 8 * v_r + 8 * g.n
    return {"workload": "rmat20_sssp_tree_64src", "us_per_source_tree": t_tree, "us_per_source_sssp": t_sssp,
            "parent_pass_us": pass_us,
            "parent_pass_full_scan_bytes_upper_bound": balg,
            "note": "the pass stops at the first qualifying in-arc of each row, so it moves far fewer bytes than a "
                    "full scan; no rate is derived from the upper bound",
            "l2": "flushed between sources",
            "tie_break": "smallest-id predecessor", "early_stop": "rows in ascending order"}


def bench_weighted(dawn, torch, flush, g, srcs, peak, nsrc=16, cpu_sources=2):
    """Weighted extension ((min, +) rounds of Alg. 3) on the headline graph with
    seeded integer arc weights uniform on [1, 255] (symmetric per edge), the
    first nsrc headline sources, L2 flushed between sources.  GTEPS counts the
    arcs of the reached vertices (E_r), as the unweighted figure does; the
    rounds offer more arcs than that (a vertex is offered again each time its
    distance falls), so relaxations are reported beside it.  Algorithmic
    bytes: 16 per offered arc (col_idx, weight, the head's 8-byte distance)
    + 16 per lowering (the 8-byte write and the head's row bounds) + 8 n (the
    distance vector); roofline fraction against the measured copy bandwidth.
    CPU baseline: the oracle's textbook Dijkstra (single-threaded) on the
    first cpu_sources sources."""
    from paper_2208_04514_b300 import graphgen as gg
    import oracle
    stream = torch.cuda.current_stream()
    w = gg.arc_weights(g, 1, 255, seed=7)
    srcs = [int(s) for s in srcs[:nsrc]]
    h = dawn.dawn_graph_upload(g.row_ptr, g.col_idx, flags=dawn.DAWN_SYMMETRIC, stream=stream)
    dawn.dawn_graph_set_weights(h, w, stream)
    dist = torch.empty((len(srcs), g.n), dtype=torch.int64, device="cuda")
    stats = torch.zeros((len(srcs), dawn.WSTATS_WORDS), dtype=torch.int64, device="cuda")
    for rep in range(2):  # the second pass is the measured one
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in srcs]
        for i, s in enumerate(srcs):
            _flush(flush, i)
            ev[i][0].record(stream)
            dawn.dawn_wsssp_async(h, s, dist[i], stats[i], stream)
            ev[i][1].record(stream)
        dawn.dawn_graph_sync(h, stream)
    us = [a.elapsed_time(b) * 1e3 for a, b in ev]
    st = [dawn.wstats_from_words(r) for r in stats.cpu().numpy()]
    d_host = dist.cpu().numpy()
    dawn.dawn_graph_free(h)
    deg = g.out_degree()
    e_r = [int(deg[d_host[i] >= 0].sum()) for i in range(len(srcs))]
    gteps = [e / (t * 1e-6) / 1e9 for e, t in zip(e_r, us)]
    balg = [16 * x["relaxations"] + 16 * x["improvements"] + 8 * g.n for x in st]
    achieved = [b / (t * 1e-6) / 1e9 for b, t in zip(balg, us)]
    t0 = time.perf_counter()
    ok = True
    for i, s in enumerate(srcs[:cpu_sources]):
        ref = oracle.dijkstra(g.row_ptr, g.col_idx, w, s)
        ok = ok and bool((ref == d_host[i]).all())
    t_cpu = (time.perf_counter() - t0) / max(1, min(cpu_sources, len(srcs)))
    return {"workload": f"rmat20_weighted_1to255_{len(srcs)}src",
            "weights": "int32 uniform on [1, 255] from a hash of the endpoint pair (seed 7), same on both arcs of an edge",
            "us_per_source_median": statistics.median(us), "us_per_source_mean": statistics.fmean(us),
            "gteps_median": statistics.median(gteps),
            "gteps_harmonic_mean": len(gteps) / sum(1.0 / x for x in gteps),
            "rounds_median": statistics.median(x["rounds"] for x in st),
            "relaxations_per_source_median": statistics.median(x["relaxations"] for x in st),
            "relaxations_over_e_r": statistics.median(x["relaxations"] / e for x, e in zip(st, e_r)),
            "roofline": {"bound": "hbm", "achieved_median": statistics.median(achieved), "peak": peak,
                         "unit": "GB/s", "frac": statistics.median(achieved) / peak,
                         "bytes_alg_per_source_median": statistics.median(balg),
                         "kernel": "wsssp_kernel"},
            "bit_exact_vs_oracle_dijkstra": ok,
            "cpu_baseline": {"us_per_source": t_cpu * 1e6, "kind": "oracle", "cores": 1,
                             "sample": f"first {min(cpu_sources, len(srcs))} sources, textbook Dijkstra single-threaded"},
            "l2": "flushed between sources"}


def bench_batched(dawn, torch, flush, plain_sample=4096, k=0, lanes_list=(64, 128, 256)):
    """RMAT scale 16 (seed 4), all 65,536 vertices as sources, int16 distance
    block of each pass kept on the device and reduced to eccentricity and
    distance sum: sources/s per lane width, against the plain path (one
    dawn_sssp launch per source, int32 dist on the device) on a sample."""
    from paper_2208_04514_b300 import graphgen as gg
    g = gg.rmat(16, seed=4)
    n = g.n
    stream = torch.cuda.current_stream()
    h = dawn.dawn_graph_upload(g.row_ptr, g.col_idx, flags=dawn.DAWN_SYMMETRIC, stream=stream)
    k = k or n
    srcs = torch.arange(k, dtype=torch.int32, device="cuda")
    ecc = torch.zeros(k, dtype=torch.int32, device="cuda")
    dsum = torch.zeros(k, dtype=torch.int64, device="cuda")
    out = {"workload": "rmat16_all_sources" if k == n else f"rmat16_{k}_sources", "n": n, "m": g.m, "k": k, "lanes": {}}
    for lanes in lanes_list:
        dawn.dawn_msbfs_ex(h, srcs, k, None, 2, 0, ecc, dsum, None, {"lanes": lanes})  # warm-up
        _flush(flush, lanes)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dawn.dawn_msbfs_ex(h, srcs, k, None, 2, 0, ecc, dsum, None, {"lanes": lanes})
        t = time.perf_counter() - t0
        out["lanes"][str(lanes)] = {"sources_per_s": k / t, "ms": 1e3 * t}
    best = max(out["lanes"].values(), key=lambda x: x["sources_per_s"])
    # plain path: one single-source launch per source
    dist = torch.empty(n, dtype=torch.int32, device="cuda")
    sample = srcs[:plain_sample].cpu().numpy()
    dawn.dawn_sssp_async(h, int(sample[0]), dist, None, None, stream)
    _flush(flush, 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in sample:
        dawn.dawn_sssp_async(h, int(s), dist, None, None, stream)
    e1.record(stream)
    dawn.dawn_graph_sync(h, stream)
    plain = len(sample) / (e0.elapsed_time(e1) * 1e-3)
    dawn.dawn_graph_free(h)
    # L2-bound figure: the graph and the lane words live in L2, so the batched
    # loop is compared with this GPU's L2 read bandwidth, not with HBM
    l2_pass = recorded_value(ROOT / "paper_2208_04514_b300" / "csrc" / "msbfs.cu",
                             ROOT / "profiles" / "msbfs_sliced_kernel_rmat16.md", "l2_bytes_per_pass")
    l2_gbs = dawn.dawn_l2_read_gbs(64 << 20, 50)
    passes = (k + 255) // 256
    t256 = out["lanes"].get("256", best)["ms"] * 1e-3
    out["l2"] = {"measured_l2_read_gbs": l2_gbs,
                 "bytes_per_pass_ncu": l2_pass,
                 "achieved_gbs": (l2_pass * passes / t256 / 1e9) if l2_pass else None,
                 "frac_of_measured_l2": (l2_pass * passes / t256 / 1e9 / l2_gbs) if l2_pass else None,
                 "note": "L2 bytes of one 256-lane pass (ncu, sources 0-255) times the passes of the "
                         "256-lane run over its time; no HBM claim (the 7 MB graph stays in L2)"}
    out["word_ors_per_level_per_pass"] = {"upper_bound": g.m * 4, "note": "m x W word ORs at W = 4 (256 lanes)"}
    import oracle
    sample_c = np.random.default_rng(5).choice(n, 1024, replace=False).astype(np.int32)
    t0 = time.perf_counter()
    oracle.msbfs(g.row_ptr, g.col_idx, sample_c, keep_dist=False)
    t_c = time.perf_counter() - t0
    out["cpu_baseline"] = {"sources_per_s": 1024 / t_c, "kind": "oracle", "cores": 1,
                           "sample": "1,024 sampled sources (seed 5), literal Alg. 3 per source with ecc / sum / "
                                     "reached, single-threaded; all 65,536 extrapolated from it",
                           "extrapolated_all_sources_s": n * t_c / 1024}
    out["best_sources_per_s"] = best["sources_per_s"]
    out["plain_sources_per_s"] = plain
    out["plain_sample"] = f"first {len(sample)} sources, one dawn_sssp launch each, back to back"
    out["speedup_vs_plain"] = best["sources_per_s"] / plain
    out["timing"] = "wall clock of the synchronous dawn_msbfs_ex call (inputs on the device), L2 flushed before"
    return out


def bench_modes(dawn, torch, flush, g_rmat, srcs_rmat, nsrc=16):
    """The paper's two operators alone and the per-level choice, on dense
    low-diameter graphs: SOVM push only (Alg. 3), BOVM pull only (Alg. 1) and
    AUTO, on the headline RMAT scale-20 graph (16 of its sources) and on a
    directed Erdos-Renyi graph with n = 2^18 and mean out-degree 128 (seed 11,
    16 uniform sources).  Median microseconds per source and GTEPS, L2 flushed
    between sources."""
    from paper_2208_04514_b300 import graphgen as gg
    stream = torch.cuda.current_stream()
    out = {}
    er = gg.erdos_renyi(1 << 18, 128.0, seed=11)
    cases = [("rmat20", g_rmat, dawn.DAWN_SYMMETRIC, srcs_rmat[:nsrc]),
             ("er262144_deg128", er, dawn.DAWN_DIRECTED, gg.sample_sources(er, nsrc, seed=12))]
    for name, g, flags, srcs in cases:
        h = dawn.dawn_graph_upload(g.row_ptr, g.col_idx, flags=flags, stream=stream)
        dist = torch.empty(g.n, dtype=torch.int32, device="cuda")
        stats = torch.zeros((len(srcs), dawn.STATS_WORDS), dtype=torch.int64, device="cuda")
        res = {"n": g.n, "m": g.m}
        for mode_name, mode in (("push_sovm", dawn.DAWN_MODE_PUSH), ("pull_bovm", dawn.DAWN_MODE_PULL),
                                ("auto", dawn.DAWN_MODE_AUTO)):
            opts = {"mode": mode}
            dawn.dawn_sssp_async(h, int(srcs[0]), dist, opts, stats[0], stream)  # warm-up
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in srcs]
            for i, sv in enumerate(srcs):
                _flush(flush, i)
                ev[i][0].record(stream)
                dawn.dawn_sssp_async(h, int(sv), dist, opts, stats[i], stream)
                ev[i][1].record(stream)
            dawn.dawn_graph_sync(h, stream)
            us = [a.elapsed_time(b) * 1e3 for a, b in ev]
            st = [dawn.stats_from_words(r) for r in stats.cpu().numpy()]
            edges = sum(x["edges"] for x in st)
            res[mode_name] = {"us_per_source_median": statistics.median(us), "gteps": edges / (sum(us) * 1e-6) / 1e9,
                              "levels_median": statistics.median(x["levels"] for x in st)}
        dawn.dawn_graph_free(h)
        out[name] = res
    out["l2"] = "flushed between sources"
    return out


def bench_many_graph(dawn, torch, g, srcs):
    """dawn_sssp_many with device rows on the headline graph and sources: the
    first call captures the 64 level-loop launches as a CUDA graph, the next
    calls replay it; against the same 64 launches issued one by one (warm L2,
    no flush: a launch-overhead comparison)."""
    stream = torch.cuda.current_stream()
    h = dawn.dawn_graph_upload(g.row_ptr, g.col_idx, flags=dawn.DAWN_SYMMETRIC, stream=stream)
    src_dev = torch.from_numpy(np.ascontiguousarray(srcs, dtype=np.int32)).cuda()
    rows = torch.empty((len(srcs), g.n), dtype=torch.int32, device="cuda")
    stats = torch.zeros((len(srcs), dawn.STATS_WORDS), dtype=torch.int64, device="cuda")
    dawn.dawn_sssp_many(h, src_dev, dist=rows, stats=stats, stream=stream)  # capture
    torch.cuda.synchronize()
    reps = 5
    t0 = time.perf_counter()
    for _ in range(reps):
        dawn.dawn_sssp_many(h, src_dev, dist=rows, stats=stats, stream=stream)  # replays
    torch.cuda.synchronize()
    t_graph = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        for i, s in enumerate(srcs):
            dawn.dawn_sssp_async(h, int(s), rows[i], None, stats[i], stream)
        dawn.dawn_graph_sync(h, stream)
    t_direct = (time.perf_counter() - t0) / reps
    edges = sum(dawn.stats_from_words(r)["edges"] for r in stats.cpu().numpy())
    dawn.dawn_graph_free(h)
    return {"workload": "rmat20_sssp_many_64src_device_rows", "gteps_graph_replay": edges / t_graph / 1e9,
            "gteps_direct_launches": edges / t_direct / 1e9, "us_per_source_graph": 1e6 * t_graph / len(srcs),
            "us_per_source_direct": 1e6 * t_direct / len(srcs), "timing": "wall clock per call, warm L2"}


def bench_centrality(dawn, torch, flush, lanes=256):
    """RMAT scale 16 (seed 4), all 65,536 sources: dawn_centrality (ecc,
    distance sum, reached, closeness, harmonic per source, and the diameter /
    radius summary) with no distance rows stored, against dawn_msbfs_ex with
    its int16 rows, same lanes."""
    from paper_2208_04514_b300 import graphgen as gg
    g = gg.rmat(16, seed=4)
    n = g.n
    stream = torch.cuda.current_stream()
    h = dawn.dawn_graph_upload(g.row_ptr, g.col_idx, flags=dawn.DAWN_SYMMETRIC, stream=stream)
    srcs = torch.arange(n, dtype=torch.int32, device="cuda")
    arrs = [torch.zeros(n, dtype=dt, device="cuda") for dt in (torch.int32, torch.int64, torch.int32,
                                                                   torch.float64, torch.float64)]
    dawn.dawn_centrality(h, srcs, n, *arrs, {"lanes": lanes})  # warm-up
    _flush(flush, 3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    summ = dawn.dawn_centrality(h, srcs, n, *arrs, {"lanes": lanes})
    t = time.perf_counter() - t0
    dawn.dawn_graph_free(h)
    return {"workload": "rmat16_all_sources_centrality", "lanes": lanes, "sources_per_s": n / t, "ms": 1e3 * t,
            "summary": summ, "outputs": "ecc, dsum, reached, closeness, harmonic (device); summary",
            "timing": "wall clock of the synchronous call (inputs on the device), L2 flushed before"}


def bench_serving(dawn, torch, nreq=48, seed=6, rates=(0.3, 0.7, 1.0), ncal=None):
    """Continuous-batching server on 8 resident graphs: RMAT scales 14, 16, 18,
    20, 22 (edge factor 16, symmetrised) and 1024^2, 2048^2, 4096^2 lattices
    (bonds deleted with p = 0.1).  Requests: graph uniform over the 8, k =
    floor(256^U) sources in [1, 256] (log-uniform), sources uniform, int16
    rows written in place into device buffers.  Saturated throughput is
    measured first (ncal requests, default nreq, all at once); then Poisson
    arrival streams of nreq requests at each of `rates` x that throughput
    (0.3x, 0.7x and 1.0x by default).  The plain path serves the 0.3x and 1.0x
    streams FIFO, one dawn_sssp launch per source (int32 rows): its
    per-request service times are measured back to back and its latencies
    follow from the FIFO single-server recursion start = max(arrival, previous
    done)."""
    from paper_2208_04514_b300 import graphgen as gg
    specs = [("rmat14", lambda: gg.rmat(14, seed=114)), ("rmat16", lambda: gg.rmat(16, seed=116)),
             ("rmat18", lambda: gg.rmat(18, seed=118)), ("rmat20", lambda: gg.rmat(20, seed=120)),
             ("rmat22", lambda: gg.rmat(22, seed=122)), ("lattice1024", lambda: gg.lattice(1024, 1024, 0.1, seed=3)),
             ("lattice2048", lambda: gg.lattice(2048, 2048, 0.1, seed=3)),
             ("lattice4096", lambda: gg.lattice(4096, 4096, 0.1, seed=3))]
    import oracle
    handles, ns, csrs = [], [], []
    for name, make in specs:
        g = make()
        handles.append(dawn.dawn_graph_upload(g.row_ptr, g.col_idx, flags=dawn.DAWN_SYMMETRIC))
        ns.append(g.n)
        csrs.append((g.row_ptr, g.col_idx))
        del g
    rng = np.random.default_rng(seed)
    checked = {"rows": 0, "graphs": set()}

    def verify(kept):
        """The first row of the first request on each graph, against Alg. 2
        (FIFO BFS; the int16 row holds the same integers)."""
        for gi, (srcs, out) in kept.items():
            want = oracle.bfs_queue(csrs[gi][0], csrs[gi][1], int(srcs[0])).astype(np.int16)
            got = out[0].cpu().numpy()
            if not np.array_equal(got, want):
                bad = np.nonzero(got != want)[0]
                raise SystemExit(f"bench: served row of graph {specs[gi][0]} source {srcs[0]} differs from the "
                                 f"oracle at {bad.size} vertices (first {bad[:4].tolist()})")
            checked["rows"] += 1
            checked["graphs"].add(specs[gi][0])

    def draw(count):
        reqs = []
        for _ in range(count):
            gi = int(rng.integers(0, len(specs)))
            k = int(min(256, max(1, np.floor(256 ** rng.random()))))
            reqs.append((gi, rng.integers(0, ns[gi], k).astype(np.int32)))
        return reqs

    def serve(reqs, arrivals, check=False):
        s = dawn.dawn_serve_create(handles, 0, 256)
        kept, pending, ids = {}, {}, []  # rows kept for the check; rows freed once their request is done
        t0 = time.perf_counter()
        for (gi, srcs), at in zip(reqs, arrivals):
            while time.perf_counter() - t0 < at:
                for rid in [r for r in pending if dawn.dawn_serve_poll(s, r) >= dawn.DAWN_REQ_DONE]:
                    del pending[rid]
            out = torch.empty((len(srcs), ns[gi]), dtype=torch.int16, device="cuda")
            rid = dawn.dawn_serve_submit(s, gi, srcs, dist_bytes=2, dist_out=out)
            ids.append(rid)
            if check and gi not in kept:
                kept[gi] = (srcs, out)
            else:
                pending[rid] = out
        dawn.dawn_serve_drain(s, 600000)
        t_end = time.perf_counter()
        times = [dawn.dawn_serve_times(s, r) for r in ids]
        dawn.dawn_serve_destroy(s)
        lat = np.array([d - a for a, d in times])
        span = max(d for _, d in times) - min(a for a, _ in times)
        if check:
            verify(kept)
        del kept, pending
        return lat, len(reqs) / span, t_end - t0

    def by_class(reqs, lat):
        """p50 / p99 per graph class (RMAT graphs, lattices) and per request size."""
        out_c = {}
        for cname, pick in (("rmat", lambda gi: specs[gi][0].startswith("rmat")),
                            ("lattice", lambda gi: specs[gi][0].startswith("lattice"))):
            for kname, kpick in (("all_k", lambda k: True), ("k<=4", lambda k: k <= 4), ("k>=64", lambda k: k >= 64)):
                sel = np.array([pick(gi) and kpick(len(srcs)) for gi, srcs in reqs])
                if sel.sum() == 0:
                    continue
                out_c[f"{cname}_{kname}"] = {"requests": int(sel.sum()),
                                             "p50_ms": 1e3 * float(np.percentile(lat[sel], 50)),
                                             "p99_ms": 1e3 * float(np.percentile(lat[sel], 99))}
        return out_c

    out = {"workload": "serve_8graphs", "graphs": [n for n, _ in specs], "requests_per_rate": nreq,
           "dist": "int16 rows written in place into device buffers", "rates": {}}
    ncal = ncal or nreq
    cal = draw(ncal)
    lat, qps_sat, _ = serve(cal, np.zeros(ncal), check=True)
    out["saturated_queries_per_s"] = qps_sat
    out["saturated_sources_per_s"] = sum(len(x[1]) for x in cal) * qps_sat / ncal
    out["calibration_requests"] = ncal
    stream_10 = stream_03 = None
    for frac in rates:
        reqs = draw(nreq)
        arrivals = np.cumsum(rng.exponential(1.0 / (frac * qps_sat), nreq))
        lat, qps, _ = serve(reqs, arrivals, check=True)
        out["rates"][f"{frac:.1f}x"] = {"offered_queries_per_s": frac * qps_sat, "queries_per_s": qps,
                                       "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                                       "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                                       "by_class": by_class(reqs, lat)}
        if frac == 0.3:
            stream_03 = (reqs, arrivals)
        if frac == 1.0:
            stream_10 = (reqs, arrivals)
    # plain path on the 0.3x and 1.0x streams: per-request service times
    # measured back to back, latencies from the FIFO single-server recursion
    stream = torch.cuda.current_stream()
    for tag, stream_x in (("plain_0.3x", stream_03), ("plain_1.0x", stream_10)):
        if stream_x is None:
            continue
        reqs, arrivals = stream_x
        service = []
        for gi, srcs in reqs:
            rows = torch.empty((len(srcs), ns[gi]), dtype=torch.int32, device="cuda")
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i, sv in enumerate(srcs):
                dawn.dawn_sssp_async(handles[gi], int(sv), rows[i], None, None, stream)
            e1.record(stream)
            dawn.dawn_graph_sync(handles[gi], stream)
            service.append(e0.elapsed_time(e1) * 1e-3)
            del rows
        done_prev, lat = 0.0, []
        for at, sv in zip(arrivals, service):
            start = max(at, done_prev)
            done_prev = start + sv
            lat.append(done_prev - at)
        lat = np.array(lat)
        out[tag] = {"queries_per_s": len(reqs) / (done_prev - arrivals[0]),
                    "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                    "busy_s": float(sum(service)), "by_class": by_class(reqs, lat)}
    # lone k = 1 requests on an idle server against the plain single-source
    # call on the same source: low-degree graphs take the server's idle fast
    # path (the cluster engine), the RMAT graph a bit lane of the loop
    lone = {}
    for gi in (3, 5, 6, 7):
        srcs = rng.integers(0, ns[gi], 3).astype(np.int32)
        served, plain = [], []
        s = dawn.dawn_serve_create(handles, 0, 256)
        for sv in srcs:
            out1 = torch.empty((1, ns[gi]), dtype=torch.int16, device="cuda")
            rid = dawn.dawn_serve_submit(s, gi, np.array([sv], dtype=np.int32), dist_bytes=2, dist_out=out1)
            dawn.dawn_serve_drain(s, 600000)
            a_t, d_t = dawn.dawn_serve_times(s, rid)
            served.append(d_t - a_t)
            want = oracle.bfs_queue(csrs[gi][0], csrs[gi][1], int(sv)).astype(np.int16)
            if not np.array_equal(out1[0].cpu().numpy(), want):
                raise SystemExit(f"bench: lone served row of graph {specs[gi][0]} source {sv} differs from the oracle")
            checked["rows"] += 1
            row = torch.empty(ns[gi], dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dawn.dawn_sssp(handles[gi], int(sv), row)
            plain.append(time.perf_counter() - t0)
            del out1, row
        dawn.dawn_serve_destroy(s)
        lone[specs[gi][0]] = {"served_ms_median": 1e3 * statistics.median(served),
                              "plain_ms_median": 1e3 * statistics.median(plain), "sources": len(srcs)}
    out["lone_k1"] = lone
    out["lone_k1_note"] = ("one request at a time on an idle server, submit to done (dawn_serve_times), against a "
                           "synchronous dawn_sssp on the same source (wall clock); rows checked against Alg. 2")
    for h in handles:
        dawn.dawn_graph_free(h)
    out["verified"] = {"rows_checked": checked["rows"], "graphs": sorted(checked["graphs"]),
                       "what": "first row of the first request on each graph in every run, "
                               "against Alg. 2 (oracle FIFO BFS)"}
    return out


def run_gpu(args):
    import torch
    import torch.distributed as distrib
    from paper_2208_04514_b300 import dawn

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        distrib.init_process_group("nccl")

    def barrier():
        if world > 1:
            distrib.barrier()

    g, srcs = build_workload()
    if args.sources:
        srcs = srcs[: args.sources]
    n = g.n
    stream = torch.cuda.current_stream()
    # the upload (validation, symmetry check, degree-ordered pull rows, first2,
    # connected components), host CSR to a ready graph, timed once
    torch.cuda.synchronize()
    t_up = time.perf_counter()
    h = dawn.dawn_graph_upload(g.row_ptr, g.col_idx, flags=dawn.DAWN_SYMMETRIC, stream=stream)
    torch.cuda.synchronize()
    upload_ms = 1e3 * (time.perf_counter() - t_up)
    dist = torch.empty((len(srcs), n), dtype=torch.int32, device="cuda")
    stats = torch.zeros((len(srcs), dawn.STATS_WORDS), dtype=torch.int64, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in srcs]

    def step():
        for i, s in enumerate(srcs):
            flush.fill_(i)
            ev[i][0].record(stream)
            dawn.dawn_sssp_async(h, int(s), dist[i], None, stats[i], stream)
            ev[i][1].record(stream)

    for _ in range(args.warmup):
        step()
    dawn.dawn_graph_sync(h, stream)
    # parity of the warm-up output on the host: the O(n + m) certificate on
    # every source's row, and the literal Alg. 3 oracle on the first four
    verified = None
    if not args.no_verify:
        import oracle
        dh = dist.cpu().numpy()
        for i, s in enumerate(srcs):
            rc = oracle.certificate(g.row_ptr, g.col_idx, int(s), dh[i])
            if rc != (0, -1):
                raise SystemExit(f"bench: certificate failed for source {s}: {rc}")
        n_or = min(4, len(srcs))
        for i in range(n_or):
            if not np.array_equal(dh[i], oracle.sssp_sovm(g.row_ptr, g.col_idx, int(srcs[i]))):
                raise SystemExit(f"bench: source {srcs[i]} differs from the Alg. 3 oracle")
        verified = {"ok": True, "certificate_rows": len(srcs), "oracle_rows": n_or,
                    "what": "warm-up output of the timed call: certificate on every row, literal Alg. 3 on the first rows"}

    barrier()
    torch.cuda.synchronize()
    kernel_ms = 0.0
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step()
            torch.cuda.synchronize()
            kernel_ms += sum(a.elapsed_time(b) for a, b in ev)
        barrier()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    dawn.dawn_graph_sync(h, stream)
    st = [dawn.stats_from_words(r) for r in stats.cpu().numpy()]
    edges_per_step = sum(x["edges"] for x in st)
    ms_step = kernel_ms / args.steps
    # per-source rates of the last timed step: harmonic mean and median
    per_ms = [a.elapsed_time(b) for a, b in ev]
    per_gteps = [x["edges"] / (t * 1e-3) / 1e9 for x, t in zip(st, per_ms)]
    gteps_hm = len(per_gteps) / sum(1.0 / r for r in per_gteps)
    gteps_med = statistics.median(per_gteps)
    # secondary: warm L2 (the same sources back to back, no flush between them).
    # A spacer of flush kernels goes first so that the host has queued every
    # launch before the GPU reaches them: otherwise each event pair would also
    # time the host's launch call (the GPU waiting for it).
    for i in range(len(srcs)):
        _flush(flush, i)
    wev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in srcs]
    for i, s in enumerate(srcs):
        wev[i][0].record(stream)
        dawn.dawn_sssp_async(h, int(s), dist[i], None, None, stream)
        wev[i][1].record(stream)
    dawn.dawn_graph_sync(h, stream)
    warm_ms = [a.elapsed_time(b) for a, b in wev]
    warm = {"gteps": edges_per_step / (sum(warm_ms) * 1e-3) / 1e9, "us_per_source": 1e3 * sum(warm_ms) / len(srcs),
            "note": "one pass over the 64 sources back to back without the L2 flush (queued behind a spacer, so the host's launch calls are not timed), after the timed steps"}
    # max over ranks of the device time
    ms_step_max, edges_all = aggregate_replicas(ms_step, edges_per_step, world, device="cuda")
    value = edges_all / (ms_step_max * 1e-3) / 1e9

    # roofline of the persistent SSSP kernel (one launch = one source)
    peak, peak_kind = measured_peaks()
    balg = sum(algorithmic_bytes(n, x) for x in st) / len(st)
    avg_launch_s = ms_step * 1e-3 / len(srcs)
    achieved = balg / avg_launch_s / 1e9
    traffic = recorded_traffic(SSSP_SRC, ROOT / "profiles" / "sssp_kernel_rmat20.md")

    # end to end through the public call with a pinned host result buffer
    e2e = None
    if not args.no_e2e:
        # the call a user makes for many sources with host results: sources
        # from pinned host memory, one pinned host row per source, copies of
        # each row overlapped with the next source's level loop
        host_src = torch.from_numpy(np.ascontiguousarray(srcs, dtype=np.int32)).pin_memory()
        host_rows = torch.empty((len(srcs), n), dtype=torch.int32, pin_memory=True)
        dawn.dawn_sssp_many(h, host_src, dist=host_rows, stream=stream)  # warm-up
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            dawn.dawn_sssp_many(h, host_src, dist=host_rows, stream=stream)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.steps
        e2e = {"value": world * edges_per_step / e2e_s / 1e9, "unit": "GTEPS",
               "h2d_bytes_per_step": 4 * len(srcs), "d2h_bytes_per_step": 4 * n * len(srcs),
               "note": "dawn_sssp_many: sources from pinned host memory, 64 int32 rows into pinned host "
                       "memory (row copies overlapped with the next source's level loop), synchronous call, "
                       "wall clock; no L2 flush"}

    dawn.dawn_graph_free(h)
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic", "config": dict(CONFIG, n=n, m=g.m),
        "wall_ms_per_step": 1e3 * wall / args.steps,
        "verified": verified,
        "upload_ms": upload_ms,
        "per_source": {"levels_median": statistics.median(x["levels"] for x in st),
                       "reached_median": statistics.median(x["reached"] for x in st),
                       "edges_per_step": edges_per_step,
                       "push_steps": sum(x["push_steps"] for x in st), "pull_steps": sum(x["pull_steps"] for x in st),
                       "us_per_source": 1e3 * ms_step / len(srcs),
                       "gteps_harmonic_mean": gteps_hm, "gteps_median": gteps_med},
        "gteps_graph500_undirected": value / 2,
        "warm_l2": warm,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "sssp_kernel",
                     "peak_kind": f"{peak_kind} hbm_gbs (copy bandwidth)",
                     "bytes_alg_per_launch": balg},
        "e2e": e2e,
        "gpu_launches": args.steps * len(srcs),
        "clocks": clk.summary(),
    }
    if world == 1 and not args.no_secondary:
        line["secondary"] = {"lattice": bench_lattice(dawn, torch, flush),
                             "batched": bench_batched(dawn, torch, flush),
                             "tree": bench_tree(dawn, torch, flush, g, srcs, peak),
                             "weighted": bench_weighted(dawn, torch, flush, g, srcs, peak),
                             "centrality": bench_centrality(dawn, torch, flush),
                             "modes": bench_modes(dawn, torch, flush, g, srcs),
                             "many_graph": bench_many_graph(dawn, torch, g, srcs)}
        del flush
        torch.cuda.empty_cache()
        line["secondary"]["serving"] = bench_serving(dawn, torch, nreq=args.serve_requests)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g, srcs, args.cpu_budget_s)
    print(json.dumps(line), flush=True)
    if world > 1:
        distrib.destroy_process_group()
    return 0


def run_one(args):
    """One secondary workload alone (for profiling): prints its figures."""
    import torch
    from paper_2208_04514_b300 import dawn
    torch.cuda.set_device(0)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    if args.workload == "lattice":
        out = bench_lattice(dawn, torch, flush, nsrc=args.lattice_sources, side=args.lattice_side)
    elif args.workload == "many":
        g, srcs = build_workload()
        out = bench_many_graph(dawn, torch, g, srcs)
    elif args.workload == "modes":
        g, srcs = build_workload()
        out = bench_modes(dawn, torch, flush, g, srcs)
    elif args.workload == "centrality":
        out = bench_centrality(dawn, torch, flush)
    elif args.workload == "tree":
        g, srcs = build_workload()
        out = bench_tree(dawn, torch, flush, g, srcs, measured_peaks()[0])
    elif args.workload == "weighted":
        g, srcs = build_workload()
        out = bench_weighted(dawn, torch, flush, g, srcs, measured_peaks()[0])
    elif args.workload == "batched":
        out = bench_batched(dawn, torch, flush, k=args.batched_k, lanes_list=(args.batched_lanes,) if args.batched_lanes else (64, 128, 256))
    else:
        out = bench_serving(dawn, torch, nreq=args.serve_requests,
                            rates=tuple(float(x) for x in args.serve_rates.split(",")),
                            ncal=args.serve_calibration or None)
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["dawn", "reference"], default="dawn")
    ap.add_argument("--no-verify", action="store_true",
                    help="skip the check of the warm-up output against the certificate and the oracle")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget-s", type=float, default=15.0)
    ap.add_argument("--ref-budget-s", type=float, default=10.0)
    ap.add_argument("--sources", type=int, default=0,
                    help="use only the first N of the 64 sources (small profiling runs; not a bench value)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer pass")
    ap.add_argument("--serve-requests", type=int, default=48, help="requests per arrival rate in the serving mix")
    ap.add_argument("--serve-rates", default="0.3,0.7,1.0",
                    help="with --workload serving: arrival rates as fractions of the saturated throughput")
    ap.add_argument("--serve-calibration", type=int, default=0,
                    help="with --workload serving: requests of the saturated run (0 = --serve-requests)")
    ap.add_argument("--workload", choices=["all", "lattice", "batched", "serving", "tree", "centrality", "modes", "many", "weighted"], default="all",
                    help="run one secondary workload alone and print its figures (profiling runs; not a bench line)")
    ap.add_argument("--batched-k", type=int, default=0, help="with --workload batched: sources (0 = all)")
    ap.add_argument("--lattice-side", type=int, default=4096, help="with --workload lattice: side of the lattice")
    ap.add_argument("--lattice-sources", type=int, default=16, help="with --workload lattice: sources")
    ap.add_argument("--batched-lanes", type=int, default=0, help="with --workload batched: one lane width")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the lattice, batched and serving workloads reported beside the headline")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "all":
        return run_one(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
