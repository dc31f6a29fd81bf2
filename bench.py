"""Benchmark: k-core decomposition throughput on GB300.

One step decomposes the workload graph completely with both methods of the
library, PeelOne (Alg. 4) and HistoCore (Alg. 6), through the C ABI; each
result is a full coreness vector. The metric is coreness edges/s: undirected
edges decomposed per second, summed over the two decompositions of a step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events
on the launching stream with an L2 flush (a 512 MiB write) before it, outside
the events. Every method call is also bracketed by its own events, which give
the per-kernel durations used for the roofline. With N > 1 (torchrun), each
rank decomposes its own replica of the workload (the graphs are independent,
there is no collective on the data path); value = all ranks' edges / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "rmat24": "R-MAT scale 24, edge factor 16, a/b/c/d .57/.19/.19/.05, int32 CSR",
    "rmat22": "R-MAT scale 22, edge factor 16, int64 row_ptr",
    "rmat16": "R-MAT scale 16, edge factor 16, int32 CSR",
    "chunglu24": "Chung-Lu beta 2.1, 2^24 vertices, mean degree 20, planted K_3000",
    "grid4096": "4096 x 4096 4-neighbour grid",
}
# bounded CPU samples of each workload for the oracle timing (same recipe, smaller)
# (the workload itself where one oracle run takes a few seconds)
CPU_SAMPLE = {"rmat24": "rmat24", "rmat22": "rmat22", "rmat16": "rmat16",
              "chunglu24": "chunglu24", "grid4096": "grid4096"}
REF_SAMPLE = {"rmat24": "rmat24", "rmat22": "rmat22", "rmat16": "rmat16",
              "chunglu24": "chunglu24", "grid4096": "grid4096"}


def make_graph(name, device):
    import graphgen as gg
    if name.startswith("grid") and name[4:].isdigit():
        s = int(name[4:])
        return gg.grid_graph(s, s, device)
    if name in ("rmat16", "rmat22", "rmat24", "chunglu24", "grid4096"):
        return gg.workload(name, device)
    if name.startswith("rmat") and name[4:].isdigit():
        return gg.rmat_graph(int(name[4:]), 16, gg.SEED_BASE + 3, device)
    raise ValueError(name)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


KERNEL_SOURCES = {
    "peelone": ("pico_device.cuh", "peelone.cuh", "peelone.cu"),
    "histocore": ("pico_device.cuh", "histocore.cuh", "histocore.cu"),
}


def kernel_source_hash(method: str) -> str:
    """Hash of the sources that define a method's kernel."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[method]:
        with open(os.path.join(ROOT, "paper_2402_15253_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str, method: str, arcs: int, profiles_dir: str | None = None):
    """DRAM bytes per launch from a committed ncu summary of `method`, if it
    was taken on the current kernel sources (its `kernel_source_hash` line
    matches). A capture of a smaller workload of the same family is scaled to
    this one by the arc count (the traffic of both methods grows with the
    arcs they scan). Returns (bytes or None, source description)."""
    best = None
    pdir = profiles_dir or os.path.join(ROOT, "profiles")
    for path in sorted(glob.glob(os.path.join(pdir, f"{method}_*.md"))):
        text = open(path).read()
        m_hash = re.search(r"kernel_source_hash\s*=\s*`?([0-9a-f]+)", text)
        m_bytes = re.search(r"dram_bytes_per_launch\s*=\s*`?([0-9.eE+]+)", text)
        m_wl = re.search(r"workload\s*=\s*(\w+)", text)
        m_arcs = re.search(r"arcs\s*=\s*([0-9]+)", text)
        if not (m_hash and m_bytes and m_wl and m_arcs) or m_hash.group(1) != kernel_source_hash(method):
            continue
        wl = m_wl.group(1)
        if wl == workload:
            return float(m_bytes.group(1)), f"ncu capture of {wl}"
        if wl.rstrip("0123456789") == workload.rstrip("0123456789"):
            best = (float(m_bytes.group(1)) * arcs / int(m_arcs.group(1)),
                    f"ncu capture of {wl}, scaled by arcs")
    return best if best else (None, "no capture of the current kernel sources")


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        if not getattr(self, "lines", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_oracle_time(sample: str, repeats: int = 1, host_csr=None):
    """Single-threaded Batagelj-Zaversnik on a host copy of `sample` (or on
    `host_csr`, a (row_ptr, col_idx) pair of numpy arrays of that graph), and
    the parallel CPU peel (cpu_peel, all host cores) on the same copy, checked
    against it. Returns (edges, oracle s, parallel s, parallel threads)."""
    import numpy as np
    import oracle
    import cpu_peel
    if host_csr is not None:
        rp, ci = host_csr
    else:
        g = make_graph(sample, "cuda")
        rp, ci = g.numpy()
        del g
    oracle.lib()   # load the libraries outside the timing
    cpu_peel.lib()
    times = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        want = oracle.bz_coreness(rp, ci)
        times.append(time.perf_counter() - t0)
    cpu_peel.coreness(rp, ci)   # warm-up (thread pool, pages)
    ptimes = []
    for _ in range(3):
        t0 = time.perf_counter()
        got = cpu_peel.coreness(rp, ci)
        ptimes.append(time.perf_counter() - t0)
    if not np.array_equal(got, want):
        raise AssertionError("the parallel CPU peel disagrees with the oracle")
    edges = int(rp[-1]) // 2
    return edges, statistics.median(times), statistics.median(ptimes), cpu_peel.threads()


def bench_batched(pico, dev, stream, G: int, reps: int = 5):
    """Graphs/s of the batched form on the packed 4,096-graph workload: one
    plain launch, one launch replayed from a CUDA graph, and, as the
    baseline, one single-graph launch per graph (PeelOne throughout; the
    HistoCore batch is timed too). L2 is flushed before every timed launch."""
    import torch
    import graphgen as gg
    pb = gg.batch_graph(G, gg.SEED_BASE + 4, device=dev)
    tv, ta = int(pb.vtx_off[-1]), int(pb.arc_off[-1])
    out = torch.empty(tv, dtype=torch.int32, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def batched(algo):
        rc = pico.pico_coreness_batched(pb.vtx_off, pb.arc_off, G, pb.row_ptr, pb.col_idx, tv, ta,
                                        out, pico.ALGOS[algo], stream)
        if rc != 0:
            raise pico.PicoError(rc, "batched")

    def timed(fn):
        ms = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    from paper_2402_15253_gb300 import autotune
    pico.pico_set_tuning(*autotune.DEFAULT)
    best_peel, timings = autotune.tune_batched(pico, pb.vtx_off, pb.arc_off, pb.row_ptr, pb.col_idx,
                                               "peelone", reps=2, use_cache=False)
    # HistoCore's batch is ~10x slower: only its CTA size and cluster threshold are tuned
    best_histo, _ = autotune.tune_batched(pico, pb.vtx_off, pb.arc_off, pb.row_ptr, pb.col_idx,
                                          "histocore", reps=1, use_cache=False,
                                          cands=[autotune.override(autotune.DEFAULT, o)
                                                 for o in autotune.stages(True)[1]])
    tuned = {"peelone": best_peel, "histocore": best_histo}
    res = {"workload": f"{G} graphs, log-uniform 100..200,000 vertices, half ER (mean degree "
                       f"4-64), half R-MAT (edge factor 8-32); {tv} vertices, {ta} arcs",
           "graphs": G, "vertices": tv, "arcs": ta}
    res["tuning"] = {a: {"small_deg": t[0], "chunk": t[1], "cta_threads": t[2],
                         "cluster_min_arcs": (1 << t[3]) if t[3] < 62 else None}
                     for a, t in tuned.items()}
    res["peelone_default_tuning_ms"] = timings[autotune.DEFAULT]
    for algo in ("peelone", "histocore"):
        pico.pico_set_tuning(*tuned[algo])
        batched(algo)
        if pico.pico_last_device_status(stream) != 0:
            raise RuntimeError("batched warm-up failed")
        ms = timed(lambda: batched(algo))
        res[algo] = {"ms": ms, "graphs_per_s": G / (ms / 1e3), "edges_per_s": ta / 2 / (ms / 1e3)}
    ref = out.clone()

    # the same PeelOne batch replayed from a CUDA graph
    pico.pico_set_tuning(*tuned["peelone"])
    torch.cuda.synchronize()
    cap = torch.cuda.Stream()
    cap.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(cap):
        batched("peelone")          # warm-up on the capture stream
        cap.synchronize()
        with torch.cuda.graph(graph, stream=cap):
            rc = pico.pico_coreness_batched(pb.vtx_off, pb.arc_off, G, pb.row_ptr, pb.col_idx,
                                            tv, ta, out, 0, cap)
    torch.cuda.synchronize()
    if rc != 0:
        raise pico.PicoError(rc, "capture")
    out.zero_()
    graph.replay()
    torch.cuda.synchronize()
    if not torch.equal(out, ref):
        raise AssertionError("graph replay result differs")
    ms_graph = timed(graph.replay)
    res["peelone_graph_replay"] = {"ms": ms_graph, "graphs_per_s": G / (ms_graph / 1e3)}

    # baseline: one single-graph launch per graph, all G graphs once
    single = torch.empty_like(out)
    vo = pb.vtx_off.cpu().tolist()
    ao = pb.arc_off.cpu().tolist()
    views = []
    for g in range(G):
        n = vo[g + 1] - vo[g]
        views.append((pb.row_ptr[vo[g] + g: vo[g + 1] + g + 1], pb.col_idx[ao[g]:ao[g + 1]], n,
                      ao[g + 1] - ao[g], single[vo[g]:vo[g + 1]]))
    flush.zero_()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    for rp, ci, n, m, o in views:
        rc = pico.pico_coreness(rp, ci, n, m, o, 0, stream)
        if rc != 0:
            raise pico.PicoError(rc, "single")
    e1.record(stream)
    e1.synchronize()
    wall = time.perf_counter() - t0
    ms_single = e0.elapsed_time(e1)
    if not torch.equal(single, ref):
        raise AssertionError("per-graph launches differ from the batch")
    res["one_launch_per_graph"] = {"ms": ms_single, "wall_s": wall,
                                   "graphs_per_s": G / (ms_single / 1e3)}
    res["speedup_vs_one_launch_per_graph"] = ms_single / res["peelone"]["ms"]
    res["speedup_graph_replay_vs_one_launch_per_graph"] = ms_single / ms_graph
    return res


def autotune_default():
    from paper_2402_15253_gb300 import autotune
    return autotune.DEFAULT


def bench_serve(pico, dev, requests: int, plain_requests: int = 2000, loads=(0.5, 0.8, 0.95),
                pool_size: int = 256, budget_gb: float = 40.0):
    """Served form: a Poisson stream of requests drawn from the batch size
    distribution (log-uniform 100..200,000 vertices, half ER, half R-MAT)
    plus 5% R-MAT scale 20 outliers, replayed open-loop into the request
    server (continuous batching, 40 GB admission budget) at 0.5/0.8/0.95 of
    its measured capacity, next to the sequential plain path (one
    single-graph call per request, one at a time) at the same offered rates.
    The server takes `requests` requests per run; the plain path, which is
    overloaded at every one of these rates (its latency grows with the
    stream's length), takes the first `plain_requests` of the same stream.
    All server runs come first, then the plain runs.
    Latency = completion - arrival, host clock, including the host-to-device
    copy of each CSR and the copy of its result back; the device-only latency
    of a request is the device time of its micro-batch (copies in, launch,
    copies out), without the wait for admission."""
    import math
    import torch
    import graphgen as gg
    import oracle

    # pool of distinct request graphs on pinned host memory
    specs = gg.batch_specs(pool_size, gg.SEED_BASE + 5)
    n_out = max(1, pool_size // 20)
    graphs = [gg.spec_graph(sp, device=dev) for sp in specs[:pool_size - n_out]]
    graphs += [gg.rmat_graph(20, 16, gg.SEED_BASE + 50 + i, device=dev) for i in range(n_out)]
    pool = []
    for g in graphs:
        rp = g.row_ptr.to(torch.int32).cpu().pin_memory()
        ci = (g.col_idx if g.arcs else torch.zeros(1, dtype=torch.int32, device=dev)).cpu().pin_memory()
        out = torch.zeros(max(g.n, 1), dtype=torch.int32).pin_memory()
        pool.append((g.n, g.arcs, rp, ci, out))
    regular, outliers = list(range(pool_size - n_out)), list(range(pool_size - n_out, pool_size))
    total = max(requests, plain_requests)
    pick = []
    for i in range(total):
        u = gg.unit_int(gg.SEED_BASE + 5, gg.S_SERVE, 2 * i)
        v = gg.unit_int(gg.SEED_BASE + 5, gg.S_SERVE, 2 * i + 1)
        lst = outliers if u < 0.05 else regular
        pick.append(lst[min(len(lst) - 1, int(v * len(lst)))])
    expo = [-math.log(1.0 - gg.unit_int(gg.SEED_BASE + 5, gg.S_SERVE + 1, i))
            for i in range(total)]
    budget = int(budget_gb * (1 << 30))

    def run(rate, single):
        count = plain_requests if single else requests
        cfg = (1, 1, 1) if single else (4, 512, 0)
        srv = pico.pico_server_create(budget, 0, cfg[0], cfg[1], cfg[2])
        if not srv:
            raise RuntimeError("pico_server_create failed")
        t0 = pico.pico_clock_ns() + 2_000_000
        arr, t = [], 0.0
        for i in range(count):
            if rate is not None:
                t += expo[i] / rate
            arr.append(t0 + int(t * 1e9))
        for i, j in enumerate(pick[:count]):
            n, m, rp, ci, out = pool[j]
            if pico.pico_server_submit(srv, rp, ci, n, m, out, arr[i]) < 0:
                raise RuntimeError("submit failed")
        rc = pico.pico_server_drain(srv)
        tk = torch.zeros(count, dtype=torch.int64)
        dn = torch.zeros(count, dtype=torch.int64)
        dv = torch.zeros(count, dtype=torch.int64)
        k = pico.pico_server_poll_device(srv, tk, dn, dv, count)
        pico.pico_server_destroy(srv)
        if rc != 0 or k != count:
            raise RuntimeError(f"server failed rc={rc} done={k}")
        arr_t = torch.tensor(arr, dtype=torch.int64)[tk]
        lat = (dn - arr_t).double() / 1e6
        span = (int(dn.max()) - int(torch.tensor(arr).min())) / 1e9
        dev = dv.double() / 1e6   # the device time of each request's micro-batch
        return {"requests": count, "graphs_per_s": count / span,
                "p50_ms": float(lat.quantile(0.5)), "p99_ms": float(lat.quantile(0.99)),
                "mean_ms": float(lat.mean()),
                "device_p50_ms": float(dev.quantile(0.5)), "device_p99_ms": float(dev.quantile(0.99))}

    pico.pico_set_tuning(*autotune_default())
    run(None, False)   # warm-up: first launches, the memory pool's growth
    capacity = run(None, False)["graphs_per_s"]
    res = {"workload": f"{requests} requests (plain path: the first {plain_requests}), Poisson "
                       f"arrivals, pool of {pool_size} graphs "
                       f"(log-uniform 100..200,000 vertices, half ER, half R-MAT; "
                       f"{n_out} R-MAT scale 20 drawn with probability 0.05)",
           "budget_gb": budget_gb, "capacity_graphs_per_s": capacity, "loads": {}}
    # every request copies its CSR to the device and its result back: at
    # capacity these copies alone need this much of the host link
    io = [4 * (pool[j][0] + 1) + 4 * pool[j][1] + 4 * pool[j][0] for j in pick[:requests]]
    res["copy_bytes_per_request"] = sum(io) / len(io)
    res["copy_gbs_at_capacity"] = capacity * res["copy_bytes_per_request"] / 1e9
    for f in loads:
        res["loads"][str(f)] = {"offered_graphs_per_s": f * capacity,
                                "served": run(f * capacity, False)}
    for f in loads:
        res["loads"][str(f)]["sequential_plain"] = run(f * capacity, True)
    # the result buffer of every requested pool graph (written by the last
    # request for that graph) must hold the oracle's coreness; checked after
    # the timed runs
    from concurrent.futures import ThreadPoolExecutor
    oracle.lib()

    def check(j):
        n, m, rp, ci, out = pool[j]
        want = oracle.bz_coreness(rp.numpy().astype("int64"), ci.numpy()[:m])
        return bool((out[:n].numpy() == want).all())

    asked = sorted(set(pick[:total]))
    with ThreadPoolExecutor(max_workers=16) as ex:
        ok = list(ex.map(check, asked))
    if not all(ok):
        raise AssertionError(f"served results of pool graphs {[j for j, o in zip(asked, ok) if not o]} "
                             "differ from the oracle")
    res["oracle_checked_graphs"] = len(asked)
    return res


BYTES_MODEL = {
    "peelone": "B_PeelOne = B_min + 4 B per successful decrement + 4 B per residual entry scanned, "
               "B_min = w_r(n+1) + 8 B/arc + 4 B/vertex",
    "histocore": "B_HistoCore = B_min + 4(A+n) (histogram build) + 4 B per SumHisto slot "
                 "+ 8 B per arc scanned by UpdateHisto + 8 B per neighbour updated",
}


def method_bytes(algo: str, st: dict, n: int, arcs: int, w_r: int) -> int:
    """Algorithmic bytes of one launch (the per-graph figures of the
    measurement plan), from the launch's own counters."""
    b_min = w_r * (n + 1) + 8 * arcs + 4 * n
    if algo == "peelone":   # successful decrements only: the others are overhead
        return b_min + 4 * (st["atomics"] - st["extra"]) + 4 * st["scanned"]
    # HistoCore: InitHisto scans every arc once (counted in st["arcs"] too);
    # each updated neighbour costs two slot edits (counted in st["atomics"])
    update_arcs = st["arcs"] - arcs
    updated = max(0, (st["atomics"] - arcs) // 2)
    return b_min + 4 * (arcs + n) + 4 * st["slots"] + 8 * update_arcs + 8 * updated


# average speedups the paper reports over its 24 datasets (RTX 3090; Sec. V):
# PeelOne over GPP, CntCore over NbrCore, HistoCore over CntCore
PAPER_AVG_SPEEDUPS = {"peelone_vs_gpp": 1.9, "cntcore_vs_nbrcore": 1.8,
                      "histocore_vs_cntcore": 8.0}


def bench_baselines(pico, rp, ci, n, arcs, ref, tuned, method_ms, stream):
    """The comparison baselines of Sec. V on the same graph (CUDA events, the
    median of up to three runs after one warm-up; one run when a run takes
    over two seconds). Each must return the same coreness as PeelOne."""
    import torch
    fn = pico.pico_coreness if rp.dtype == torch.int32 else pico.pico_coreness_i64
    out = torch.empty(n, dtype=torch.int32, device=rp.device)
    keep = ("levels", "subrounds", "scans", "rounds", "frontier", "active", "arcs",
            "atomics", "extra")
    res = {}
    for name, algo in pico.BASELINES.items():
        peel_like = name in ("gpp", "peel_cas", "peel_addback")
        pico.pico_set_tuning(*tuned["peelone" if peel_like else "histocore"])
        times = []
        for i in range(4):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc = fn(rp, ci, n, arcs, out, algo, stream)
            e1.record(stream)
            if rc != 0:
                raise pico.PicoError(rc, name)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            if times[0] > 2000.0 and len(times) == 2:
                break
        st = pico.pico_last_device_status(stream)
        if st != 0:
            raise pico.PicoError(st, name)
        if not torch.equal(out, ref):
            raise AssertionError(f"{name} disagrees with PeelOne")
        stats = pico.pico_get_stats(stream)
        res[name] = {"ms": statistics.median(times[1:]),
                     "stats": {k: stats[k] for k in keep if stats[k]}}
    ms = {**{k: v["ms"] for k, v in res.items()}, **method_ms}
    speedups = {
        "peelone_vs_gpp": ms["gpp"] / ms["peelone"],
        "peelone_vs_peel_cas": ms["peel_cas"] / ms["peelone"],
        "peelone_vs_peel_addback": ms["peel_addback"] / ms["peelone"],
        "cntcore_vs_nbrcore": ms["nbrcore"] / ms["cntcore"],
        "histocore_vs_cntcore": ms["cntcore"] / ms["histocore"],
        "histocore_vs_nbrcore": ms["nbrcore"] / ms["histocore"],
    }
    return {"runs": res, "speedups": speedups, "paper_average_speedups": PAPER_AVG_SPEEDUPS,
            "note": "same graph, same runtime and tuning; GPP, NbrCore and CntCore as Alg. 3, "
                    "Sec. V and Alg. 5 describe them"}


def bench_auto(pico, rp, ci, n, arcs, ref, stream, reps=3):
    """PICO_ALGO_AUTO on the same graph: the method the selector ran and its
    time (median of `reps` after one warm-up)."""
    import torch
    fn = pico.pico_coreness if rp.dtype == torch.int32 else pico.pico_coreness_i64
    out = torch.empty(n, dtype=torch.int32, device=rp.device)
    times = []
    for i in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = fn(rp, ci, n, arcs, out, pico.PICO_ALGO_AUTO, stream)
        e1.record(stream)
        if rc != 0:
            raise pico.PicoError(rc, "auto")
        e1.synchronize()
        if i:
            times.append(e0.elapsed_time(e1))
    if pico.pico_last_device_status(stream) != 0 or not torch.equal(out, ref):
        raise AssertionError("auto selection failed or disagrees with PeelOne")
    chose = pico.pico_get_stats(stream)["algo"]
    return {"ms": statistics.median(times),
            "method": {v: k for k, v in pico.ALGOS.items()}[chose]}


def bench_configs(pico, dev, stream, names=("rmat16", "rmat22", "chunglu24", "grid4096"),
                  reps: int = 3):
    """Both methods on each of the other single-graph workloads: the
    degree-class tuning is autotuned per graph and method first, then each
    method is timed `reps` times (CUDA events on the launching stream, an L2
    flush before each run, the median kept). The two methods must agree."""
    import torch
    from paper_2402_15253_gb300 import autotune
    peak, peak_kind = peaks()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    res = {}
    for name in names:
        g = make_graph(name, dev)
        rp, ci, n, arcs = g.row_ptr, g.col_idx, g.n, g.arcs
        w_r = rp.element_size()
        fn = pico.pico_coreness if w_r == 4 else pico.pico_coreness_i64
        b_min = w_r * (n + 1) + 8 * arcs + 4 * n
        outs, rec = {}, {"workload": WORKLOADS[name], "n": n, "arcs": arcs,
                         "undirected_edges": arcs // 2}
        for a in ("peelone", "histocore"):
            best, _ = autotune.tune_single(pico, rp, ci, a, reps=2, use_cache=False)
            out = torch.empty(n, dtype=torch.int32, device=dev)
            times = []
            for _ in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rc = fn(rp, ci, n, arcs, out, pico.ALGOS[a], stream)
                e1.record(stream)
                if rc != 0:
                    raise pico.PicoError(rc, f"{name} {a}")
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            st = pico.pico_last_device_status(stream)
            if st != 0:
                raise pico.PicoError(st, f"{name} {a}")
            stats = pico.pico_get_stats(stream)
            ms = statistics.median(times)
            b_alg = method_bytes(a, stats, n, arcs, w_r)
            rec[a] = {"ms": ms, "edges_per_s": arcs / 2 / (ms / 1e3),
                      "alg_frac_of_" + peak_kind: b_alg / (ms / 1e3) / 1e9 / peak,
                      "bmin_frac_of_" + peak_kind: b_min / (ms / 1e3) / 1e9 / peak,
                      "tuning": {"small_deg": best[0], "chunk": best[1]},
                      "stats": {k: stats[k] for k in ("levels", "kmax", "subrounds", "rounds",
                                                      "pull_rounds", "barriers") if stats[k]}}
            outs[a] = out
        if not torch.equal(outs["peelone"], outs["histocore"]):
            raise AssertionError(f"{name}: PeelOne and HistoCore disagree")
        rec["kmax"] = int(outs["peelone"].max().item())
        rec["better"] = min(("peelone", "histocore"), key=lambda a: rec[a]["ms"])
        res[name] = rec
        del g, outs
        torch.cuda.empty_cache()
    return res


def bench_partitioned(pico, g, ref, parts=(2, 4), reps: int = 3):
    """Partitioned HistoCore (pico_coreness_partitioned) on the workload graph
    with P equal vertex ranges on this GPU: wall time of the whole call (it
    synchronises once per phase of every round), the median of `reps` runs
    after one warm-up; the result must equal the single-kernel one."""
    import torch
    rp = g.row_ptr.to(torch.int64)
    res = {"note": "every round: SumHisto in each partition, an exchange of the change "
                   "records, UpdateHisto pulled into each partition's rows; host-driven"}
    for P in parts:
        out, rounds = pico.coreness_partitioned(rp, g.col_idx, P)
        if not torch.equal(out, ref):
            raise AssertionError(f"partitioned HistoCore with {P} parts differs")
        times = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pico.coreness_partitioned(rp, g.col_idx, P, out=out)
            torch.cuda.synchronize()
            times.append(1000.0 * (time.perf_counter() - t0))
        ms = statistics.median(times)
        res[str(P)] = {"ms": ms, "rounds": rounds, "edges_per_s": g.arcs / 2 / (ms / 1e3)}
    del rp
    return res


def bench_maintenance(pico, g, stream, k: int = 10000, seed: int = 0x9C6,
                      update_tuning=None, recompute_tuning=None):
    """Core maintenance on the workload graph: batches of k random edge
    insertions (non-edges), k random deletions (existing edges) and both,
    each timed with CUDA events around pico_dyn_update, against a full
    recomputation (PICO_ALGO_AUTO) of the updated graph. An update rebuilds
    the CSR and then maintains or recomputes the coreness; `speedup` compares
    it with the same rebuild followed by a recomputation, and
    `coreness_step_speedup` the coreness step alone with the recomputation.
    The maintained coreness must equal the recomputed one. The state runs its default
    policy: it recomputes instead of maintaining when its cost model
    predicts that maintenance would take longer ("path"). The tunings (S, C, T, K) are set
    before each update and each recomputation (None: leave as is)."""
    import numpy as np
    import torch
    import graphgen as gg
    kwarm = 256   # edges of the untimed warm-up batch
    n = g.n
    rp_h = g.row_ptr.to(torch.int64).cpu().numpy()
    ci_h = g.col_idx.cpu().numpy()
    deg = np.diff(rp_h)
    idx = np.arange(4 * k, dtype=np.int64)
    # random non-edges (rows are sorted: a binary search rules out existing edges)
    cu = gg.draw_below(seed, 1, torch.from_numpy(idx), n).numpy()
    cv = gg.draw_below(seed, 2, torch.from_numpy(idx), n).numpy()
    ins, seen = [], set()
    for a, b in zip(cu.tolist(), cv.tolist()):
        if a == b:
            continue
        e = (min(a, b), max(a, b))
        row = ci_h[rp_h[e[0]]:rp_h[e[0] + 1]]
        j = np.searchsorted(row, e[1])
        if e in seen or (j < len(row) and row[j] == e[1]):
            continue
        seen.add(e)
        ins.append(e)
        if len(ins) == 2 * k + kwarm:
            break
    # random existing edges (arcs drawn uniformly, each edge once)
    arcs = gg.draw_below(seed, 3, torch.from_numpy(idx), int(rp_h[-1])).numpy()
    src = np.searchsorted(rp_h, arcs, side="right") - 1
    dele, dseen = [], set()
    for a, b in zip(src.tolist(), ci_h[arcs].tolist()):
        e = (min(a, b), max(a, b))
        if e not in dseen:
            dseen.add(e)
            dele.append(e)
        if len(dele) == 2 * k:
            break
    dev = g.row_ptr.device
    if update_tuning:   # the state times its first full computation at creation
        pico.pico_set_tuning(*update_tuning)
    dg = pico.DynamicGraph(g.row_ptr, g.col_idx, capacity_arcs=g.arcs + 4 * k + 1024)
    batches = {"insert": (ins[:k], []), "delete": ([], dele[:k]),
               "mixed": (ins[k:2 * k], dele[k:2 * k])}
    res = {"batch_edges": k, "graph": "the workload graph", "runs": {}}
    # untimed warm-up: insert a few extra non-edges and delete them again, and
    # one recomputation, so that no first-call allocation lands in a timed run
    warm = torch.tensor(ins[2 * k:], dtype=torch.int32, device=dev).reshape(-1, 2)
    for wi, wd in ((warm, None), (None, warm)):
        rc = pico.pico_dyn_update(dg._d, wi, 0 if wi is None else len(warm),
                                  wd, 0 if wd is None else len(warm), stream)
        if rc != pico.PICO_OK:
            raise pico.PicoError(rc, "pico_dyn_update (warm-up)")
    rp2, ci2 = dg.csr()
    pico.coreness(rp2, ci2, "auto")
    torch.cuda.synchronize()
    for name, (bi, bd) in batches.items():
        ti = torch.tensor(bi, dtype=torch.int32, device=dev).reshape(-1, 2) if bi else None
        td = torch.tensor(bd, dtype=torch.int32, device=dev).reshape(-1, 2) if bd else None
        if update_tuning:
            pico.pico_set_tuning(*update_tuning)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = pico.pico_dyn_update(dg._d, ti, len(bi), td, len(bd), stream)
        e1.record(stream)
        e1.synchronize()
        if rc != pico.PICO_OK:
            raise pico.PicoError(rc, "pico_dyn_update")
        st = pico.pico_get_stats(stream)
        rp2, ci2 = dg.csr()
        if recompute_tuning:
            pico.pico_set_tuning(*recompute_tuning)
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        full = pico.coreness(rp2, ci2, "auto")
        r1.record(stream)
        r1.synchronize()
        if not torch.equal(full, dg.coreness()):
            raise AssertionError(f"maintained coreness differs after the {name} batch")
        rebuild_ms, step_ms = dg.last_update_times
        upd_ms, rec_ms = e0.elapsed_time(e1), r0.elapsed_time(r1)
        res["runs"][name] = {"update_ms": upd_ms,
                             "path": ("recomputed" if dg.last_update_kind == pico.PICO_DYN_RECOMPUTED
                                      else "maintained"),
                             "rebuild_ms": rebuild_ms,
                             "coreness_step_ms": step_ms,
                             "recompute_ms": rec_ms,
                             # both ways need the updated CSR: the alternative to
                             # maintenance is the same rebuild plus a recomputation
                             "speedup": (rebuild_ms + rec_ms) / upd_ms,
                             "coreness_step_speedup": rec_ms / step_ms if step_ms > 0 else None,
                             "stats": {x: st[x] for x in ("algo", "rounds", "frontier", "active", "subrounds",
                                                             "barriers", "arcs", "atomics")}}
    dg.close()
    return res


def job_totals(local_ms: float, local_units: int, device=None):
    """Whole-job time and work over the ranks of the current process group
    (or this process alone): the slowest rank's time and the sum of the
    units every rank processed. Each rank works on its own replica, so the
    only communication is this reduction."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return local_ms, local_units
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    u = torch.tensor([local_units], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reference_arm(args):
    """The CPU oracle (single-threaded BZ), as it stands, on a bounded sample."""
    ws, rank, _ = dist_info()
    if rank != 0:
        return 0
    sample = REF_SAMPLE.get(args.workload, "rmat20")
    import oracle
    import torch
    g = make_graph(sample, "cuda" if torch.cuda.is_available() else "cpu")   # not timed
    rp, ci = g.numpy()
    del g
    oracle.lib()
    for _ in range(args.warmup):
        oracle.bz_coreness(rp, ci)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.bz_coreness(rp, ci)
    dt = time.perf_counter() - t0
    edges = int(rp[-1]) // 2
    value = edges * args.steps / dt
    line = {
        "impl": "reference", "metric": "coreness edges/s", "value": value, "unit": "edges/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "sample": sample,
                   "same_config": sample == args.workload,
                   "step": "one BZ decomposition of the sample"},
        "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle",
                         "sample": (f"{sample}: the workload graph itself" if sample == args.workload
                                    else f"{sample}: same recipe at reduced scale") +
                                   f", {edges} undirected edges, single-threaded BZ"},
        "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="rmat24", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="pico", choices=["pico", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-maintenance", action="store_true",
                    help="skip the core-maintenance batches")
    ap.add_argument("--no-baselines", action="store_true",
                    help="skip the comparison baselines of the paper's evaluation")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--tuning", default="auto",
                    help="'auto' (autotune each method on the graph) or S,C,T,K: small_deg, "
                         "chunk, batched CTA threads, cluster log2 arcs, for both methods "
                         "(or PeelOne's/HistoCore's, separated by '/')")
    ap.add_argument("--serve-requests", type=int, default=6000,
                    help="requests of each served-form run (0: skip the served form)")
    ap.add_argument("--plain-requests", type=int, default=2000,
                    help="requests of each run of the sequential plain path beside it")
    ap.add_argument("--no-partitioned", action="store_true",
                    help="skip partitioned HistoCore on the workload graph")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the per-workload record of the other single-graph workloads")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    import torch.distributed as dist

    ws, rank, local = dist_info()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    import __graft_entry__
    if rank == 0 or ws == 1:
        __graft_entry__.build()
    if ws > 1:
        dist.barrier()
    __graft_entry__.build()
    import paper_2402_15253_gb300 as pico

    g = make_graph(args.workload, dev)
    n, arcs = g.n, g.arcs
    m_und = arcs // 2
    rp, ci = g.row_ptr, g.col_idx
    w_r = rp.element_size()
    out = {a: torch.empty(n, dtype=torch.int32, device=dev) for a in ("peelone", "histocore")}
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    # degree-class tuning per method, picked by the library's autotuner on this graph
    from paper_2402_15253_gb300 import autotune
    tuned = {}
    for a in ("peelone", "histocore"):
        if args.tuning == "auto":
            tuned[a], _ = autotune.tune_single(pico, rp, ci, a, reps=2, use_cache=False)
        else:   # S,C,T,K for both methods, or PeelOne's/HistoCore's
            parts = args.tuning.split("/")
            tuned[a] = tuple(int(x) for x in parts[min(len(parts) - 1, 0 if a == "peelone" else 1)]
                             .split(","))
            if not autotune.valid(tuned[a]):
                raise SystemExit(f"invalid --tuning {args.tuning}")

    def step(ev=None):
        for i, a in enumerate(("peelone", "histocore")):
            pico.pico_set_tuning(*tuned[a])
            if ev is not None:
                ev[2 * i].record(stream)
            rc = (pico.pico_coreness if w_r == 4 else pico.pico_coreness_i64)(
                rp, ci, n, arcs, out[a], pico.ALGOS[a], stream)
            if ev is not None:
                ev[2 * i + 1].record(stream)
            if rc != 0:
                raise pico.PicoError(rc, a)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    st = pico.pico_last_device_status(stream)
    if st != 0:
        raise pico.PicoError(st, "warm-up")
    stats = {}
    for a in ("peelone", "histocore"):
        pico.pico_set_tuning(*tuned[a])
        pico.coreness(rp, ci, a, out=out[a])
        stats[a] = pico.pico_get_stats(stream)
    kmax = int(out["peelone"].max().item())
    if not torch.equal(out["peelone"], out["histocore"]):
        raise AssertionError("PeelOne and HistoCore disagree")

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        torch.cuda.nvtx.range_push("timed")
        for k in range(args.steps):
            flush.zero_()
            step_ev[k][0].record(stream)
            step(evs[k])
            step_ev[k][1].record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    st = pico.pico_last_device_status(stream)
    if st != 0:
        raise pico.PicoError(st, "timed steps")

    step_ms = [s.elapsed_time(e) for s, e in step_ev]
    per = {a: [evs[k][2 * i].elapsed_time(evs[k][2 * i + 1]) for k in range(args.steps)]
           for i, a in enumerate(("peelone", "histocore"))}
    total_ms, units = job_totals(sum(step_ms), 2 * m_und * args.steps, dev)
    value = units / (total_ms / 1000.0)

    # roofline of the dominant kernel against its method's algorithmic bytes
    b_min = w_r * (n + 1) + 4 * arcs + 4 * arcs + 4 * n
    b_alg = {a: method_bytes(a, stats[a], n, arcs, w_r) for a in stats}
    peak, peak_kind = peaks()
    mean_ms = {a: statistics.mean(v) for a, v in per.items()}
    dom = max(mean_ms, key=mean_ms.get)
    achieved = b_alg[dom] / (mean_ms[dom] / 1000.0) / 1e9
    traffic, traffic_src = recorded_traffic(args.workload, dom, arcs)
    best = min(mean_ms, key=mean_ms.get)   # the faster method
    best_traffic, best_traffic_src = recorded_traffic(args.workload, best, arcs)
    methods = {a: {"ms_mean": mean_ms[a], "ms_median": statistics.median(per[a]),
                   "alg_bytes": b_alg[a],
                   "alg_gbs": b_alg[a] / (mean_ms[a] / 1000.0) / 1e9,
                   "alg_frac_of_" + peak_kind: b_alg[a] / (mean_ms[a] / 1000.0) / 1e9 / peak,
                   "edges_per_s": m_und / (mean_ms[a] / 1000.0),
                   "bmin_gbs": b_min / (mean_ms[a] / 1000.0) / 1e9,
                   "bmin_frac_of_" + peak_kind: b_min / (mean_ms[a] / 1000.0) / 1e9 / peak,
                   "stats": stats[a]} for a in per}

    line = {
        "metric": "coreness edges/s", "value": value, "unit": "edges/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "n": n,
                   "arcs": arcs, "undirected_edges": m_und, "kmax": kmax,
                   "step": "full decomposition by PeelOne and by HistoCore (2 x edges)",
                   "l2": "inputs larger than L2 (col_idx %.2f GB) and a 512 MiB L2 flush "
                         "before every step, outside its events" % (4 * arcs / 1e9),
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "traffic_source": traffic_src,
                     "bytes_per_launch": b_alg[dom], "peak_kind": peak_kind,
                     "bytes_model": BYTES_MODEL[dom],
                     "bmin_bytes": b_min,
                     "bmin_frac": b_min / (mean_ms[dom] / 1000.0) / 1e9 / peak,
                     "traffic_frac": (traffic / (mean_ms[dom] / 1000.0) / 1e9 / peak
                                      if traffic else None)},
        "tuning": {a: {"small_deg": t[0], "chunk": t[1]} for a, t in tuned.items()},
        "peelone_edges_per_s": methods["peelone"]["edges_per_s"],
        "histocore_edges_per_s": methods["histocore"]["edges_per_s"],
        "roofline_better_method": {
            "kernel": best, "ms": mean_ms[best], "edges_per_s": m_und / (mean_ms[best] / 1e3),
            "bound": "hbm", "peak": peak, "unit": "GB/s", "peak_kind": peak_kind,
            "achieved": b_alg[best] / (mean_ms[best] / 1e3) / 1e9,
            "frac": b_alg[best] / (mean_ms[best] / 1e3) / 1e9 / peak,
            "bytes_per_launch": b_alg[best], "bytes_model": BYTES_MODEL[best],
            "bmin_achieved": b_min / (mean_ms[best] / 1e3) / 1e9,
            "bmin_frac": b_min / (mean_ms[best] / 1e3) / 1e9 / peak,
            "traffic": best_traffic, "traffic_source": best_traffic_src,
            "traffic_frac": (best_traffic / (mean_ms[best] / 1e3) / 1e9 / peak
                             if best_traffic else None)},
        "methods": methods,
        "gpu_launches": 2 * args.steps,
        "clocks": clk.summary(),
    }

    if rank == 0 and not args.no_e2e:
        # end to end through the public API from pinned host buffers: every step
        # copies its CSR to the device, runs both methods and copies both
        # results back. "e2e" overlaps the next step's host-to-device copy (on
        # a copy stream, into the other of two device buffers) with this step's
        # compute; "e2e_serial" runs copy, compute and copy-back in turn.
        h_rp = rp.cpu().pin_memory()
        h_ci = ci.cpu().pin_memory()
        e_steps = max(2, args.steps)
        h_bytes = h_rp.numel() * w_r + h_ci.numel() * 4

        def e2e_run(pipelined):
            bufs = [(torch.empty_like(rp), torch.empty_like(ci)) for _ in range(2)]
            outs = [{a: torch.empty(n, dtype=torch.int32, device=dev) for a in out} for _ in range(2)]
            h_out = [{a: torch.empty(n, dtype=torch.int32).pin_memory() for a in out}
                     for _ in range(2)]
            cs = torch.cuda.Stream() if pipelined else stream
            ev_h2d = [torch.cuda.Event() for _ in range(2)]
            ev_done = [torch.cuda.Event() for _ in range(2)]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cs.wait_event(e0)
            for i in range(e_steps):
                b = i % 2
                with torch.cuda.stream(cs):
                    if i >= 2:
                        cs.wait_event(ev_done[b])   # the step that used buffer b is done
                    bufs[b][0].copy_(h_rp, non_blocking=True)
                    bufs[b][1].copy_(h_ci, non_blocking=True)
                    ev_h2d[b].record(cs)
                stream.wait_event(ev_h2d[b])
                for a in out:
                    pico.pico_set_tuning(*tuned[a])
                    pico.coreness(bufs[b][0], bufs[b][1], a, out=outs[b][a], stream=stream,
                                  check=False)
                    h_out[b][a].copy_(outs[b][a], non_blocking=True)
                ev_done[b].record(stream)
            e1.record(stream)
            torch.cuda.synchronize()
            e_ms = e0.elapsed_time(e1)
            for hb in h_out:
                for a in out:
                    if not torch.equal(hb[a], out["peelone"].cpu()):
                        raise AssertionError("e2e result differs")
            return {"value": 2 * m_und * e_steps / (e_ms / 1000.0), "unit": "edges/s",
                    "h2d_bytes_per_step": h_bytes, "d2h_bytes_per_step": 2 * 4 * n,
                    "steps": e_steps, "wall_s": time.perf_counter() - t0,
                    "h2d_overlapped_with_compute": pipelined}

        line["e2e"] = e2e_run(True)
        line["e2e_serial"] = e2e_run(False)

    if rank == 0:
        pico.pico_set_tuning(*tuned["peelone"])
        line["auto"] = bench_auto(pico, rp, ci, n, arcs, out["peelone"], stream)
    if rank == 0 and not args.no_baselines:
        line["baselines"] = bench_baselines(pico, rp, ci, n, arcs, out["peelone"], tuned,
                                            {a: statistics.median(v) for a, v in per.items()},
                                            stream)
    if rank == 0 and not args.no_maintenance:
        # the updates and the recomputations they are compared with run with
        # the same tuning: the one tuned for the method AUTO picks here
        t_auto = tuned[line["auto"]["method"]]
        line["maintenance"] = bench_maintenance(pico, g, stream, update_tuning=t_auto,
                                                recompute_tuning=t_auto)
    if rank == 0 and not args.no_batched:
        line["batched"] = bench_batched(pico, dev, stream, args.batch_graphs)
    if rank == 0 and not args.no_partitioned:
        line["partitioned"] = bench_partitioned(pico, g, out["histocore"])
    if rank == 0 and args.serve_requests > 0:
        line["served"] = bench_serve(pico, dev, args.serve_requests, args.plain_requests)
    h_csr = None   # host copy of the workload graph for the CPU baseline
    if (rank == 0 and ws == 1 and not args.no_cpu_baseline
            and CPU_SAMPLE.get(args.workload) == args.workload):
        h_csr = g.numpy()
    if rank == 0 and not args.no_configs:
        del g, rp, ci, out
        torch.cuda.empty_cache()
        line["configs"] = bench_configs(pico, dev, stream,
                                        [w for w in ("rmat16", "rmat22", "chunglu24", "grid4096")
                                         if w != args.workload])

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        sample = CPU_SAMPLE.get(args.workload, args.workload)
        edges, secs, psecs, threads = cpu_oracle_time(sample, host_csr=h_csr)
        what = ("the workload graph itself" if sample == args.workload
                else "same recipe at reduced scale")
        line["cpu_baseline"] = {"value": edges / secs, "unit": "edges/s", "cores": 1,
                                "kind": "oracle", "same_config": sample == args.workload,
                                "sample": f"{sample}: {what}, {edges} "
                                          f"undirected edges, one single-threaded "
                                          f"Batagelj-Zaversnik run ({secs:.1f} s)"}
        line["cpu_parallel"] = {"value": edges / psecs, "unit": "edges/s", "cores": threads,
                                "kind": "OpenMP level-synchronous peel (a comparison, not the "
                                        "oracle; its result is checked against the oracle)",
                                "sample": f"{sample}: the same graph, median of 3 runs "
                                          f"({psecs:.2f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
