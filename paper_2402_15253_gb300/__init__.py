"""Python binding of the pico C ABI (libpico.so, declared in include/pico.h).

The functions named ``pico_*`` mirror the C entry points one to one and only
marshal arguments: tensors become device pointers, streams become CUDA
stream handles. :func:`coreness` is a convenience wrapper that allocates the
output, picks the int32- or int64-offset entry point and raises on failure.
Every step of the computation runs in the library's CUDA kernels; there is no
CPU fallback, and importing this module fails if libpico.so is missing.

Build the library with ``paper_2402_15253_gb300.build.build()`` (nvcc,
sm_103a).
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpico.so")

PICO_ALGO_PEELONE = 0
PICO_ALGO_HISTOCORE = 1
PICO_ALGO_GPP = 2
PICO_ALGO_PEEL_CAS = 3
PICO_ALGO_PEEL_ADDBACK = 4
PICO_ALGO_NBRCORE = 5
PICO_ALGO_CNTCORE = 6
PICO_ALGO_AUTO = 7
ALGOS = {"peelone": PICO_ALGO_PEELONE, "histocore": PICO_ALGO_HISTOCORE, "auto": PICO_ALGO_AUTO}
# the comparison baselines of the paper's evaluation (single-graph calls only)
BASELINES = {"gpp": PICO_ALGO_GPP, "peel_cas": PICO_ALGO_PEEL_CAS,
             "peel_addback": PICO_ALGO_PEEL_ADDBACK, "nbrcore": PICO_ALGO_NBRCORE,
             "cntcore": PICO_ALGO_CNTCORE}
METHODS = {**ALGOS, **BASELINES}

PICO_UPDATE_AUTO = 0
PICO_UPDATE_PUSH = 1
PICO_UPDATE_PULL = 2
UPDATES = {"auto": PICO_UPDATE_AUTO, "push": PICO_UPDATE_PUSH, "pull": PICO_UPDATE_PULL}

PICO_OK = 0
PICO_ERR_INVALID_ARG = -1
PICO_ERR_OOM = -2
PICO_ERR_CUDA = -3
PICO_ERR_NOT_CONVERGED = -4
PICO_ERR_TIMEOUT = -5
PICO_ERR_BAD_GRAPH = -6
PICO_ERR_NO_DEVICE = -7


class PicoError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {pico_status_string(status)} ({status})" if what
                         else f"{pico_status_string(status)} ({status})")


PHASES = ("init", "scan", "wave_tiny", "wave_mid", "wave_wide", "inithisto", "sumhisto",
          "updatehisto")
# trace-only kinds: a pulled UpdateHisto round (counted under "updatehisto" in
# pico_stats.phase_ns) and an asynchronous PeelOne level (under "wave_wide")
TRACE_KINDS = PHASES + ("updatehisto_pull", "level")


class pico_stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "algo", "levels", "kmax", "subrounds", "scans", "rounds", "frontier", "barriers",
        "arcs", "atomics", "slots", "blocks", "scanned", "pulled", "pull_rounds", "extra",
        "active")] + [
            ("phase_ns", ctypes.c_int64 * 8),
                                                  ("phase_count", ctypes.c_int64 * 8)]

    def as_dict(self) -> dict:
        d = {f: int(getattr(self, f)) for f, _ in self._fields_ if not f.startswith("phase")}
        d["phases"] = {PHASES[i]: {"ms": self.phase_ns[i] / 1e6, "count": int(self.phase_count[i])}
                       for i in range(8) if self.phase_count[i]}
        return d


class pico_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("algo", ctypes.c_int),
                ("streams", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("single_graph", ctypes.c_int)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libpico.so (raises OSError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it with paper_2402_15253_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.pico_coreness.argtypes = [vp, vp, i64, i64, vp, i32, vp]
    L.pico_coreness_i64.argtypes = [vp, vp, i64, i64, vp, i32, vp]
    L.pico_workspace_bytes.argtypes = [i64, i64, i32]
    L.pico_workspace_bytes.restype = ctypes.c_size_t
    L.pico_status_string.argtypes = [i32]
    L.pico_status_string.restype = ctypes.c_char_p
    L.pico_last_device_status.argtypes = [vp]
    L.pico_get_stats.argtypes = [vp, ctypes.POINTER(pico_stats)]
    for f in (L.pico_coreness, L.pico_coreness_i64, L.pico_last_device_status,
              L.pico_get_stats, L.pico_version):
        f.restype = i32
    L.pico_version.argtypes = []
    L.pico_validate_graph.argtypes = [vp, vp, i64, i64, ctypes.POINTER(ctypes.c_uint32), vp]
    L.pico_validate_graph.restype = i32
    L.pico_validate_graph_i64.argtypes = [vp, vp, i64, i64, ctypes.POINTER(ctypes.c_uint32), vp]
    L.pico_validate_graph_i64.restype = i32
    L.pico_coreness_batched.argtypes = [vp, vp, i32, vp, vp, i64, i64, vp, i32, vp]
    L.pico_coreness_batched.restype = i32
    L.pico_workspace_bytes_batched.argtypes = [i32, i64, i64, i32]
    L.pico_workspace_bytes_batched.restype = ctypes.c_size_t
    L.pico_server_create.argtypes = [ctypes.POINTER(pico_server_config)]
    L.pico_server_create.restype = vp
    L.pico_server_submit.argtypes = [vp, vp, vp, i64, i64, vp, i64]
    L.pico_server_submit.restype = i64
    L.pico_server_poll.argtypes = [vp, vp, vp, i32]
    L.pico_server_poll_device.argtypes = [vp, vp, vp, vp, i32]
    L.pico_server_poll_device.restype = i32
    L.pico_server_poll.restype = i32
    L.pico_server_drain.argtypes = [vp]
    L.pico_server_drain.restype = i32
    L.pico_server_destroy.argtypes = [vp]
    L.pico_server_destroy.restype = i32
    L.pico_clock_ns.argtypes = []
    L.pico_clock_ns.restype = i64
    L.pico_set_tuning.argtypes = [i32, i32, i32, i32]
    L.pico_set_tuning.restype = i32
    L.pico_get_tuning.argtypes = [vp, vp, vp, vp]
    L.pico_get_tuning.restype = i32
    L.pico_dyn_create.argtypes = [vp, vp, i64, i64, i64, vp]
    L.pico_dyn_create.restype = vp
    L.pico_dyn_update.argtypes = [vp, vp, i64, vp, i64, vp]
    L.pico_dyn_update.restype = i32
    L.pico_dyn_coreness.argtypes = [vp, vp, vp]
    L.pico_dyn_coreness.restype = i32
    L.pico_dyn_graph.argtypes = [vp, vp, vp, vp, vp]
    L.pico_dyn_graph.restype = i32
    L.pico_dyn_copy_graph.argtypes = [vp, vp, vp, vp]
    L.pico_dyn_copy_graph.restype = i32
    L.pico_dyn_destroy.argtypes = [vp]
    L.pico_dyn_destroy.restype = None
    L.pico_dyn_set_policy.argtypes = [vp, i32]
    L.pico_dyn_set_policy.restype = i32
    L.pico_dyn_last_update_kind.argtypes = [vp]
    L.pico_dyn_last_update_kind.restype = i32
    L.pico_dyn_last_update_times.argtypes = [vp, vp, vp]
    L.pico_dyn_last_update_times.restype = i32
    L.pico_set_histo_update.argtypes = [i32, i32]
    L.pico_set_histo_update.restype = i32
    L.pico_get_histo_update.argtypes = [vp, vp]
    L.pico_get_histo_update.restype = i32
    L.pico_selftest_wait_timeout.argtypes = [i32, vp]
    L.pico_selftest_wait_timeout.restype = i32
    L.pico_get_trace.argtypes = [vp, vp, i32]
    L.pico_get_trace.restype = i32
    L.pico_coreness_noalloc.argtypes = [vp, vp, i64, i64, vp, vp, vp]
    L.pico_coreness_noalloc.restype = i32
    L.pico_part_create.argtypes = [vp, vp, i64, i64, i64, vp]
    L.pico_part_create.restype = vp
    L.pico_part_sum.argtypes = [vp, vp, vp, vp]
    L.pico_part_sum.restype = i32
    L.pico_part_records.argtypes = [vp]
    L.pico_part_records.restype = vp
    L.pico_part_copy_records.argtypes = [vp, vp, vp]
    L.pico_part_copy_records.restype = i32
    L.pico_part_apply.argtypes = [vp, vp, i64, i32, vp, vp]
    L.pico_part_apply.restype = i32
    L.pico_part_coreness.argtypes = [vp, vp, vp]
    L.pico_part_coreness.restype = i32
    L.pico_part_destroy.argtypes = [vp]
    L.pico_part_destroy.restype = None
    L.pico_coreness_partitioned.argtypes = [vp, vp, i64, i64, vp, i32, vp, vp]
    L.pico_coreness_partitioned.restype = i32
    _lib = L
    return L


def _ptr(t) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(None)
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    """None -> torch's current stream on the current device; an int is taken
    as a raw cudaStream_t; torch.cuda.Stream objects are unwrapped."""
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------------------
# C ABI mirrors
# ---------------------------------------------------------------------------

def pico_coreness(row_ptr, col_idx, n: int, m: int, out_core, algo: int, stream=None) -> int:
    return load().pico_coreness(_ptr(row_ptr), _ptr(col_idx), n, m, _ptr(out_core), algo,
                                _stream(stream))


def pico_coreness_i64(row_ptr, col_idx, n: int, m: int, out_core, algo: int, stream=None) -> int:
    return load().pico_coreness_i64(_ptr(row_ptr), _ptr(col_idx), n, m, _ptr(out_core), algo,
                                    _stream(stream))


# defect bits of pico_validate_graph
PICO_DEFECT_ROWS, PICO_DEFECT_IDS, PICO_DEFECT_LOOP = 1, 2, 4
PICO_DEFECT_ORDER, PICO_DEFECT_ASYMMETRIC = 8, 16


def pico_validate_graph(row_ptr, col_idx, n: int, m: int, stream=None) -> tuple:
    """Returns (status, PICO_DEFECT_* bits)."""
    d = ctypes.c_uint32(0)
    rc = load().pico_validate_graph(_ptr(row_ptr), _ptr(col_idx), n, m, ctypes.byref(d),
                                    _stream(stream))
    return rc, d.value


def pico_validate_graph_i64(row_ptr, col_idx, n: int, m: int, stream=None) -> tuple:
    """Returns (status, PICO_DEFECT_* bits)."""
    d = ctypes.c_uint32(0)
    rc = load().pico_validate_graph_i64(_ptr(row_ptr), _ptr(col_idx), n, m, ctypes.byref(d),
                                        _stream(stream))
    return rc, d.value


def pico_coreness_batched(vtx_off, arc_off, G: int, row_ptr, col_idx, total_vertices: int,
                          total_arcs: int, out_core, algo: int, stream=None) -> int:
    return load().pico_coreness_batched(_ptr(vtx_off), _ptr(arc_off), G, _ptr(row_ptr),
                                        _ptr(col_idx), total_vertices, total_arcs,
                                        _ptr(out_core), algo, _stream(stream))


def pico_workspace_bytes_batched(G: int, total_vertices: int, total_arcs: int, algo: int) -> int:
    return int(load().pico_workspace_bytes_batched(G, total_vertices, total_arcs, algo))


def pico_server_create(hbm_budget_bytes: int, algo: int, streams: int = 4, max_batch: int = 256,
                       single_graph: int = 0):
    cfg = pico_server_config(hbm_budget_bytes, algo, streams, max_batch, single_graph)
    return load().pico_server_create(ctypes.byref(cfg))


def pico_server_submit(server, row_ptr, col_idx, n: int, m: int, out_core, arrival_ns: int) -> int:
    return load().pico_server_submit(server, _ptr(row_ptr), _ptr(col_idx), n, m, _ptr(out_core),
                                     arrival_ns)


def pico_server_poll(server, tickets, done_ns, cap: int) -> int:
    return load().pico_server_poll(server, _ptr(tickets), _ptr(done_ns), cap)


def pico_server_poll_device(server, tickets, done_ns, device_ns, cap: int) -> int:
    return load().pico_server_poll_device(server, _ptr(tickets), _ptr(done_ns), _ptr(device_ns),
                                          cap)


def pico_server_drain(server) -> int:
    return load().pico_server_drain(server)


def pico_server_destroy(server) -> int:
    return load().pico_server_destroy(server)


def pico_clock_ns() -> int:
    return load().pico_clock_ns()


def pico_coreness_noalloc(row_ptr, col_idx, n: int, m: int, out_core, out_status=None,
                          stream=None) -> int:
    """PeelOne through the entry point that allocates no device memory, for
    callers that cannot allocate while they run; graphs up to
    PICO_NOALLOC_MAX_VERTICES vertices and PICO_NOALLOC_MAX_ARCS arcs."""
    return load().pico_coreness_noalloc(_ptr(row_ptr), _ptr(col_idx), n, m, _ptr(out_core),
                                        _ptr(out_status), _stream(stream))


PICO_NOALLOC_MAX_VERTICES = 1 << 20
PICO_NOALLOC_MAX_ARCS = 1 << 24


def pico_coreness_partitioned(row_ptr, col_idx, n: int, m: int, out_core, parts: int,
                              rounds=None, stream=None) -> int:
    return load().pico_coreness_partitioned(_ptr(row_ptr), _ptr(col_idx), n, m, _ptr(out_core),
                                            parts, _ptr(rounds), _stream(stream))


def pico_part_create(row_ptr, col_idx, n: int, lo: int, hi: int, stream=None):
    return load().pico_part_create(_ptr(row_ptr), _ptr(col_idx), n, lo, hi, _stream(stream))


def pico_part_sum(part, n_changed, ymin, stream=None) -> int:
    return load().pico_part_sum(part, n_changed, ymin, _stream(stream))


def pico_part_records(part):
    return load().pico_part_records(part)


def pico_part_copy_records(part, dst, stream=None) -> int:
    return load().pico_part_copy_records(part, _ptr(dst), _stream(stream))


def pico_part_apply(part, records, count: int, ymin: int, next_vcnt, stream=None) -> int:
    return load().pico_part_apply(part, _ptr(records), count, ymin, next_vcnt, _stream(stream))


def pico_part_coreness(part, out_core, stream=None) -> int:
    return load().pico_part_coreness(part, _ptr(out_core), _stream(stream))


def pico_part_destroy(part) -> None:
    load().pico_part_destroy(part)


class Partition:
    """One partition of partitioned HistoCore (pico_part_*): the rows
    [lo, hi) of a graph held on the current device. sum() and apply() are the
    two halves of a round; the exchange of records between partitions happens
    between them (see paper_2402_15253_gb300.distributed)."""

    def __init__(self, row_ptr: torch.Tensor, col_idx: torch.Tensor, lo: int, hi: int,
                 stream=None):
        if row_ptr.dtype != torch.int64 or col_idx.dtype != torch.int32:
            raise TypeError("row_ptr must be int64 and col_idx int32")
        self.device = row_ptr.device
        self.lo, self.hi = lo, hi
        self._keep = (row_ptr, col_idx)
        self._stream = stream
        self._h = pico_part_create(row_ptr, col_idx, row_ptr.numel() - 1, lo, hi, stream)
        if not self._h:
            raise PicoError(PICO_ERR_INVALID_ARG, "pico_part_create")

    def sum(self):
        """SumHisto over the partition's V_cnt: (records, ymin) with records
        an int32 device tensor of 3 * count entries (vertex, old, new)."""
        c, y = ctypes.c_int64(), ctypes.c_int32()
        rc = pico_part_sum(self._h, ctypes.byref(c), ctypes.byref(y), self._stream)
        if rc != PICO_OK:
            raise PicoError(rc, "pico_part_sum")
        count = int(c.value)
        if count == 0:
            return torch.empty(0, dtype=torch.int32, device=self.device), int(y.value)
        recs = torch.empty(3 * count, dtype=torch.int32, device=self.device)
        rc = pico_part_copy_records(self._h, recs, self._stream)
        if rc != PICO_OK:
            raise PicoError(rc, "pico_part_copy_records")
        return recs, int(y.value)

    def apply(self, records: torch.Tensor, ymin: int) -> int:
        """The round's records of all partitions and their smallest new
        estimate: applies the edits to the own rows; returns the next V_cnt
        size."""
        records = records.to(device=self.device, dtype=torch.int32).contiguous()
        nxt = ctypes.c_int64()
        rc = pico_part_apply(self._h, records, records.numel() // 3, ymin, ctypes.byref(nxt),
                             self._stream)
        if rc != PICO_OK:
            raise PicoError(rc, "pico_part_apply")
        return int(nxt.value)

    def coreness(self) -> torch.Tensor:
        out = torch.empty(self.hi - self.lo, dtype=torch.int32, device=self.device)
        rc = pico_part_coreness(self._h, out, self._stream)
        if rc != PICO_OK:
            raise PicoError(rc, "pico_part_coreness")
        torch.cuda.synchronize(self.device)
        return out

    def close(self) -> None:
        if getattr(self, "_h", None):
            pico_part_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def coreness_partitioned(row_ptr: torch.Tensor, col_idx: torch.Tensor, parts: int,
                         out: torch.Tensor | None = None, stream=None):
    """Coreness by partitioned HistoCore with `parts` vertex ranges on the
    current device; returns (coreness, rounds)."""
    row_ptr = row_ptr.to(torch.int64).contiguous()
    col_idx = col_idx.contiguous()
    n = row_ptr.numel() - 1
    if out is None:
        out = torch.empty(max(n, 0), dtype=torch.int32, device=row_ptr.device)
    rounds = torch.zeros(1, dtype=torch.int64)
    with torch.cuda.device(row_ptr.device):
        rc = pico_coreness_partitioned(row_ptr, col_idx, n, col_idx.numel(), out, parts,
                                       rounds.data_ptr(), stream)
        if rc != PICO_OK:
            raise PicoError(rc, "pico_coreness_partitioned")
    return out, int(rounds.item())


def pico_workspace_bytes(n: int, m: int, algo: int) -> int:
    return int(load().pico_workspace_bytes(n, m, algo))


def pico_status_string(status: int) -> str:
    return load().pico_status_string(status).decode()


def pico_last_device_status(stream=None) -> int:
    return load().pico_last_device_status(_stream(stream))


def pico_get_stats(stream=None) -> dict:
    st = pico_stats()
    rc = load().pico_get_stats(_stream(stream), ctypes.byref(st))
    if rc != PICO_OK:
        raise PicoError(rc, "pico_get_stats")
    return st.as_dict()


def pico_get_trace(stream=None, cap: int = 8192) -> list:
    """Phase trace of the last call (needs PICO_TRACE=1 before first use):
    a list of (phase name, work units, device ms)."""
    buf = torch.zeros(3 * cap, dtype=torch.int64)
    k = load().pico_get_trace(_stream(stream), _ptr(buf), cap)
    if k < 0:
        raise PicoError(k, "pico_get_trace")
    b = buf[:3 * k].view(-1, 3).tolist()
    return [(TRACE_KINDS[kind], units, ns / 1e6) for kind, units, ns in b]


PICO_STATS_MAINTENANCE = 100


def pico_dyn_create(row_ptr: torch.Tensor, col_idx: torch.Tensor, n: int, m: int,
                    capacity_arcs: int, stream=None):
    return load().pico_dyn_create(_ptr(row_ptr), _ptr(col_idx), n, m, capacity_arcs,
                                  _stream(stream))


def pico_dyn_update(d, ins: torch.Tensor | None, n_ins: int, dele: torch.Tensor | None,
                    n_del: int, stream=None) -> int:
    return load().pico_dyn_update(d, _ptr(ins) if ins is not None else None, n_ins,
                                  _ptr(dele) if dele is not None else None, n_del, _stream(stream))


def pico_dyn_coreness(d, out: torch.Tensor, stream=None) -> int:
    return load().pico_dyn_coreness(d, _ptr(out), _stream(stream))


def pico_dyn_graph(d):
    rp, ci = ctypes.c_void_p(), ctypes.c_void_p()
    n, m = ctypes.c_int64(), ctypes.c_int64()
    rc = load().pico_dyn_graph(d, ctypes.byref(rp), ctypes.byref(ci), ctypes.byref(n),
                               ctypes.byref(m))
    if rc != PICO_OK:
        raise PicoError(rc, "pico_dyn_graph")
    return rp.value, ci.value, n.value, m.value


def pico_dyn_copy_graph(d, row_ptr: torch.Tensor, col_idx: torch.Tensor, stream=None) -> int:
    return load().pico_dyn_copy_graph(d, _ptr(row_ptr), _ptr(col_idx), _stream(stream))


PICO_DYN_AUTO, PICO_DYN_MAINTAIN, PICO_DYN_RECOMPUTE = 0, 1, 2
PICO_DYN_MAINTAINED, PICO_DYN_RECOMPUTED = 0, 1


def pico_dyn_set_policy(d, policy: int) -> int:
    return load().pico_dyn_set_policy(d, policy)


def pico_dyn_last_update_kind(d) -> int:
    return load().pico_dyn_last_update_kind(d)


def pico_dyn_last_update_times(d) -> tuple:
    """(rebuild ms, coreness-step ms) of the last update (-1 before the first)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    rc = load().pico_dyn_last_update_times(d, ctypes.byref(a), ctypes.byref(b))
    if rc != PICO_OK:
        raise PicoError(rc, "pico_dyn_last_update_times")
    return a.value, b.value


def pico_dyn_destroy(d) -> None:
    load().pico_dyn_destroy(d)


class DynamicGraph:
    """A graph and its coreness kept on the device under batches of edge
    insertions and deletions (pico_dyn_*). ``row_ptr``/``col_idx``: CUDA
    tensors of a CSR; ``capacity_arcs``: room for insertions (arcs)."""

    def __init__(self, row_ptr: torch.Tensor, col_idx: torch.Tensor, capacity_arcs: int | None = None,
                 stream=None):
        self.device = row_ptr.device
        rp = row_ptr.to(torch.int64).contiguous()
        ci = col_idx.to(torch.int32).contiguous()
        self.n = rp.numel() - 1
        m = ci.numel()
        cap = capacity_arcs if capacity_arcs is not None else max(2 * m, 1024)
        with torch.cuda.device(self.device):
            self._d = pico_dyn_create(rp, ci, self.n, m, cap, stream)
        if not self._d:
            raise PicoError(PICO_ERR_INVALID_ARG, "pico_dyn_create")

    def update(self, insert=None, delete=None, stream=None) -> None:
        """insert / delete: int32 CUDA tensors of shape (k, 2), undirected edges."""
        def prep(e):
            if e is None or len(e) == 0:
                return None, 0
            e = torch.as_tensor(e, dtype=torch.int32, device=self.device).contiguous()
            return e, e.shape[0]
        ins, ni = prep(insert)
        dele, nd = prep(delete)
        with torch.cuda.device(self.device):
            rc = pico_dyn_update(self._d, ins, ni, dele, nd, stream)
        if rc != PICO_OK:
            raise PicoError(rc, "pico_dyn_update")

    def set_policy(self, policy: int) -> None:
        """PICO_DYN_AUTO (maintain or recompute by the cost model),
        PICO_DYN_MAINTAIN or PICO_DYN_RECOMPUTE."""
        rc = pico_dyn_set_policy(self._d, policy)
        if rc != PICO_OK:
            raise PicoError(rc, "pico_dyn_set_policy")

    @property
    def last_update_kind(self) -> int:
        """PICO_DYN_MAINTAINED or PICO_DYN_RECOMPUTED for the last update."""
        return pico_dyn_last_update_kind(self._d)

    @property
    def last_update_times(self) -> tuple:
        """(CSR rebuild ms, coreness-step ms) of the last update."""
        return pico_dyn_last_update_times(self._d)

    def coreness(self, stream=None) -> torch.Tensor:
        out = torch.empty(self.n, dtype=torch.int32, device=self.device)
        with torch.cuda.device(self.device):
            rc = pico_dyn_coreness(self._d, out, stream)
            if rc != PICO_OK:
                raise PicoError(rc, "pico_dyn_coreness")
            torch.cuda.current_stream().synchronize()
        return out

    def csr(self):
        """Copies of the current row_ptr (int64) and col_idx (int32)."""
        _, _, n, m = pico_dyn_graph(self._d)
        rp = torch.empty(n + 1, dtype=torch.int64, device=self.device)
        ci = torch.empty(max(m, 1), dtype=torch.int32, device=self.device)
        with torch.cuda.device(self.device):
            rc = pico_dyn_copy_graph(self._d, rp, ci)
            if rc != PICO_OK:
                raise PicoError(rc, "pico_dyn_copy_graph")
            torch.cuda.current_stream().synchronize()
        return rp, ci[:m]

    def close(self) -> None:
        if getattr(self, "_d", None):
            pico_dyn_destroy(self._d)
            self._d = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PULL_PCT_DEFAULT = 50


def pico_set_histo_update(mode: int, pull_pct: int = PULL_PCT_DEFAULT) -> int:
    return load().pico_set_histo_update(mode, pull_pct)


def pico_get_histo_update() -> tuple:
    a, b = ctypes.c_int(), ctypes.c_int()
    rc = load().pico_get_histo_update(ctypes.byref(a), ctypes.byref(b))
    if rc != PICO_OK:
        raise PicoError(rc, "pico_get_histo_update")
    return a.value, b.value


def pico_set_tuning(small_deg: int, chunk: int, batched_threads: int, cluster_log2: int = 21) -> int:
    return load().pico_set_tuning(small_deg, chunk, batched_threads, cluster_log2)


def pico_get_tuning() -> tuple:
    a, b, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    rc = load().pico_get_tuning(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d))
    if rc != PICO_OK:
        raise PicoError(rc, "pico_get_tuning")
    return a.value, b.value, c.value, d.value


def pico_selftest_wait_timeout(limit_ms: int, stream=None) -> int:
    return load().pico_selftest_wait_timeout(limit_ms, _stream(stream))


def pico_version() -> int:
    return load().pico_version()


# ---------------------------------------------------------------------------
# convenience
# ---------------------------------------------------------------------------

def coreness_batched(vtx_off: torch.Tensor, arc_off: torch.Tensor, row_ptr: torch.Tensor,
                     col_idx: torch.Tensor, algo="peelone", total_vertices: int | None = None,
                     total_arcs: int | None = None, out: torch.Tensor | None = None,
                     stream=None, check: bool = True) -> torch.Tensor:
    """Coreness of a packed batch (see pico_coreness_batched). The totals are
    read from the offset tensors unless given (that read synchronises)."""
    a = ALGOS[algo] if isinstance(algo, str) else int(algo)
    G = vtx_off.numel() - 1
    if total_vertices is None:
        total_vertices = int(vtx_off[-1].item())
    if total_arcs is None:
        total_arcs = int(arc_off[-1].item())
    if out is None:
        out = torch.empty(total_vertices, dtype=torch.int32, device=row_ptr.device)
    with torch.cuda.device(row_ptr.device):
        rc = pico_coreness_batched(vtx_off, arc_off, G, row_ptr, col_idx, total_vertices,
                                   total_arcs, out, a, stream)
        if rc != PICO_OK:
            raise PicoError(rc, "pico_coreness_batched")
        if check:
            st = pico_last_device_status(stream)
            if st != PICO_OK:
                raise PicoError(st, "device")
    return out


def coreness(row_ptr: torch.Tensor, col_idx: torch.Tensor, algo="peelone",
             out: torch.Tensor | None = None, stream=None, check: bool = True) -> torch.Tensor:
    """Coreness of a CSR graph held in CUDA tensors (row_ptr int32 or int64,
    col_idx int32). Returns an int32 tensor on the same device. With
    ``check`` the stream is synchronised and device-side errors raise.
    ``algo``: a name of METHODS (the two methods or a baseline) or its value."""
    a = METHODS[algo] if isinstance(algo, str) else int(algo)
    if not (row_ptr.is_cuda and col_idx.is_cuda):
        raise ValueError("row_ptr and col_idx must be CUDA tensors")
    if col_idx.dtype != torch.int32 or row_ptr.dtype not in (torch.int32, torch.int64):
        raise TypeError("row_ptr must be int32/int64 and col_idx int32")
    row_ptr = row_ptr.contiguous()
    col_idx = col_idx.contiguous()
    n = row_ptr.numel() - 1
    m = col_idx.numel()
    if out is None:
        out = torch.empty(max(n, 0), dtype=torch.int32, device=row_ptr.device)
    with torch.cuda.device(row_ptr.device):
        fn = pico_coreness if row_ptr.dtype == torch.int32 else pico_coreness_i64
        rc = fn(row_ptr, col_idx, n, m, out, a, stream)
        if rc != PICO_OK:
            raise PicoError(rc, "pico_coreness")
        if check:
            st = pico_last_device_status(stream)
            if st != PICO_OK:
                raise PicoError(st, "device")
    return out
