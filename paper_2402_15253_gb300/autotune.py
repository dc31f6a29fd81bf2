"""Autotuner of the degree-class work assignment.

The kernels assign work by degree class: vertices of degree <= small_deg are
batched 32 per warp, larger ones are split into chunks of `chunk` arcs (one
per warp); the batched kernel gives each graph one CTA of `batched_threads`
threads, or a cluster of 8 CTAs when it has at least 2^cluster_log2 arcs. The
best values depend on the graph mix and the GPU; results never do. This
module times candidate settings on the caller's own workload (CUDA events on
the call's stream, median of several runs after a warm-up) in two stages -
first the degree classes, then the CTA size and cluster threshold - keeps the
fastest, applies it with pico_set_tuning, and caches it in a JSON file keyed
by GPU name, method, call kind and power-of-two size classes, so later runs
of a similar workload start tuned.

Cache file: $PICO_TUNING_CACHE, else ~/.cache/pico_gb300/tuning.json.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import tempfile
from typing import Callable, Iterable, Sequence

SMALL_DEG = (32, 64, 128)
CHUNK = (128, 256, 1024)
THREADS = (256, 512)
CLUSTER = (21, 23, 62)          # 62: no clusters
DEFAULT = (32, 256, 512, 21)


def stages(batched: bool) -> list[list[dict]]:
    """The search: stage 1 varies small_deg x chunk; stage 2 (batched only)
    varies CTA size x cluster threshold around the best of stage 1."""
    s1 = [{"small_deg": s, "chunk": c} for s in SMALL_DEG for c in CHUNK]
    if not batched:
        return [s1]
    s2 = [{"threads": t, "cluster_log2": k} for t in THREADS for k in CLUSTER]
    return [s1, s2]


def candidates(batched: bool) -> list[tuple[int, int, int, int]]:
    """Every setting the staged search can reach (for tests)."""
    out = [override(DEFAULT, o) for st in stages(batched) for o in st]
    return list(dict.fromkeys(out))


_FIELDS = ("small_deg", "chunk", "threads", "cluster_log2")


def override(cand: Sequence[int], changes: dict) -> tuple:
    c = list(cand)
    for k, v in changes.items():
        c[_FIELDS.index(k)] = v
    return tuple(c)


def valid(cand: Sequence[int]) -> bool:
    if len(cand) != 4:
        return False
    s, c, t, k = cand
    return 32 <= s <= 256 and 64 <= c <= 4096 and t in (256, 512) and 10 <= k <= 62


def size_class(x: int) -> int:
    """Power-of-two bucket of a size (0 for 0 and 1)."""
    return int(math.log2(x)) if x > 1 else 0


def cache_key(gpu: str, algo: str, kind: str, n: int, m: int, graphs: int = 1) -> str:
    return f"{gpu}|{algo}|{kind}|G{size_class(graphs)}|n{size_class(n)}|m{size_class(m)}"


def cache_path() -> str:
    return os.environ.get("PICO_TUNING_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "pico_gb300", "tuning.json"))


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(entries: dict, path: str | None = None) -> None:
    """Merges entries into the cache file (written atomically)."""
    path = path or cache_path()
    d = load_cache(path)
    d.update(entries)
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(path) or ".", suffix=".tmp")
    with os.fdopen(fd, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def pick(timings: dict) -> tuple:
    """The candidate with the smallest time (ties: the first in order)."""
    return min(timings, key=lambda c: (timings[c], list(timings).index(c)))


def tune(run: Callable[[tuple], float], cands: Iterable[tuple], reps: int = 3) -> tuple[tuple, dict]:
    """Times every candidate with `run(cand) -> ms` (one warm-up, then the
    median of `reps` runs) and returns (best, {cand: ms})."""
    timings = {}
    for cand in cands:
        if not valid(cand):
            raise ValueError(f"invalid tuning candidate {cand}")
        run(cand)
        timings[tuple(cand)] = statistics.median(run(cand) for _ in range(reps))
    return pick(timings), timings


def tune_staged(run: Callable[[tuple], float], stage_list, start=DEFAULT, reps: int = 3):
    """Coordinate search: each stage tries its overrides on the best setting
    so far. Returns (best, {cand: ms} over all stages)."""
    best, timings = tuple(start), {}
    for st in stage_list:
        cands = list(dict.fromkeys(override(best, o) for o in st))
        b, t = tune(run, cands, reps)
        timings.update(t)
        best = b
    return best, timings


def _timer(pico, stream, call):
    import torch

    def run(cand):
        rc = pico.pico_set_tuning(*cand)
        if rc != pico.PICO_OK:
            raise pico.PicoError(rc, "pico_set_tuning")
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call()
        e1.record(stream)
        e1.synchronize()
        st = pico.pico_last_device_status(stream)
        if st != pico.PICO_OK:
            raise pico.PicoError(st, "tuning run")
        return e0.elapsed_time(e1)

    return run


def tune_batched(pico, vtx_off, arc_off, row_ptr, col_idx, algo="peelone", cands=None,
                 reps: int = 3, use_cache: bool = True, path: str | None = None):
    """Tunes pico_coreness_batched on this packed batch; applies and caches the
    best setting. Returns (best, timings)."""
    import torch
    a = pico.ALGOS[algo]
    G = vtx_off.numel() - 1
    tv, ta = int(vtx_off[-1]), int(arc_off[-1])
    out = torch.empty(tv, dtype=torch.int32, device=row_ptr.device)
    stream = torch.cuda.current_stream()

    def call():
        rc = pico.pico_coreness_batched(vtx_off, arc_off, G, row_ptr, col_idx, tv, ta, out, a,
                                        stream)
        if rc != pico.PICO_OK:
            raise pico.PicoError(rc, "batched")

    run = _timer(pico, stream, call)
    best, timings = tune(run, cands, reps) if cands else tune_staged(run, stages(True), reps=reps)
    pico.pico_set_tuning(*best)
    if use_cache:
        key = cache_key(torch.cuda.get_device_name(), algo, "batched", tv, ta, G)
        save_cache({key: list(best)}, path)
    return best, timings


def tune_single(pico, row_ptr, col_idx, algo="peelone", cands=None, reps: int = 3,
                use_cache: bool = True, path: str | None = None):
    """Tunes the single-graph entry point on this graph; applies and caches the
    best setting. Returns (best, timings)."""
    import torch
    a = pico.ALGOS[algo]
    n, m = row_ptr.numel() - 1, col_idx.numel()
    out = torch.empty(n, dtype=torch.int32, device=row_ptr.device)
    stream = torch.cuda.current_stream()
    fn = pico.pico_coreness if row_ptr.dtype == torch.int32 else pico.pico_coreness_i64

    def call():
        rc = fn(row_ptr, col_idx, n, m, out, a, stream)
        if rc != pico.PICO_OK:
            raise pico.PicoError(rc, "coreness")

    run = _timer(pico, stream, call)
    best, timings = tune(run, cands, reps) if cands else tune_staged(run, stages(False), reps=reps)
    pico.pico_set_tuning(*best)
    if use_cache:
        key = cache_key(torch.cuda.get_device_name(), algo, "single", n, m)
        save_cache({key: list(best)}, path)
    return best, timings


def apply_cached(pico, algo: str, kind: str, n: int, m: int, graphs: int = 1,
                 path: str | None = None):
    """Applies the cached setting for this GPU and size class, if any; returns
    it (or None when the cache has no entry)."""
    import torch
    key = cache_key(torch.cuda.get_device_name(), algo, kind, n, m, graphs)
    cand = load_cache(path).get(key)
    if cand is None or not valid(cand):
        return None
    rc = pico.pico_set_tuning(*cand)
    if rc != pico.PICO_OK:
        raise pico.PicoError(rc, "pico_set_tuning")
    return tuple(cand)
