"""CPU oracle for k-core decomposition -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The CUDA library never loads it and it
never loads the CUDA library: the two share no code.

What it computes (Sec. I): core(v) = max{k : v is in the k-core}, the k-core
being the maximal subgraph whose minimum degree is >= k; isolated vertices
have core 0. The result is a unique integer vector, so GPU results must match
it bit for bit.

Pure-Python definitions (tiny inputs):
  brute_force_coreness  the definition: for each k delete vertices of degree
                        < k until none is left; core(v) is the last k that v
                        survives.
  hindex                HINDEX of Alg. 2.
  hindex_fixpoint_pass one synchronous round of Alg. 2.

Compiled C (``oracle.c``, built by :func:`build`):
  bz_coreness           Batagelj-Zaversnik bucket peel (Sec. VI).
  bz_coreness_batched   the same over a packed batch.
  hindex_jacobi         Alg. 2 run synchronously to its fixpoint.
  peelone               Alg. 4 run sequentially; level and wave counts.
  histocore             Alg. 6 run sequentially; round counts and the
                        histogram invariant.
  check                 fixpoint / certificate / range checks.

Parity: pinned. BZ is checked against the brute-force definition on every
labelled graph with at most 6 vertices, against closed forms (complete
graphs, cycles, paths, trees, stars, grids, complete bipartite graphs,
hypercubes, disjoint unions, planted cliques) and against the paper's
six-vertex example G1; the three algorithmic renditions (Alg. 2, 4, 6) are
checked against BZ.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (portable C, no intrinsics)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            p64, p32 = ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)
            i64 = ctypes.c_int64
            L.oracle_bz.argtypes = [i64, p64, p32, p32]
            L.oracle_bz_batched.argtypes = [i64, p64, p64, p32, p32, p32]
            L.oracle_hindex_jacobi.argtypes = [i64, p64, p32, p32, p64]
            L.oracle_peelone.argtypes = [i64, p64, p32, p32, p64]
            L.oracle_histocore.argtypes = [i64, p64, p32, p32, p64, ctypes.c_int]
            L.oracle_check.argtypes = [i64, p64, p32, p32, p64]
            for f in (L.oracle_gpp, L.oracle_nbrcore, L.oracle_cntcore):
                f.argtypes = [i64, p64, p32, p32, p64]
                f.restype = ctypes.c_int
            for f in (L.oracle_bz, L.oracle_bz_batched, L.oracle_hindex_jacobi,
                      L.oracle_peelone, L.oracle_histocore, L.oracle_check):
                f.restype = ctypes.c_int
            _lib = L
    return _lib


def _p64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _p32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _csr(row_ptr, col_idx):
    rp = np.ascontiguousarray(np.asarray(row_ptr), dtype=np.int64)
    ci = np.ascontiguousarray(np.asarray(col_idx), dtype=np.int32)
    return rp, ci, len(rp) - 1


def _np(x):
    """Accept numpy arrays or (CPU) torch tensors."""
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return x


# ---------------------------------------------------------------------------
# compiled routines
# ---------------------------------------------------------------------------

def bz_coreness(row_ptr, col_idx) -> np.ndarray:
    rp, ci, n = _csr(_np(row_ptr), _np(col_idx))
    out = np.zeros(max(n, 0), dtype=np.int32)
    if lib().oracle_bz(n, _p64(rp), _p32(ci), _p32(out)) != 0:
        raise MemoryError("oracle_bz")
    return out


def bz_coreness_batched(vtx_off, arc_off, row_ptr, col_idx) -> np.ndarray:
    vo = np.ascontiguousarray(_np(vtx_off), dtype=np.int64)
    ao = np.ascontiguousarray(_np(arc_off), dtype=np.int64)
    rp = np.ascontiguousarray(_np(row_ptr), dtype=np.int32)
    ci = np.ascontiguousarray(_np(col_idx), dtype=np.int32)
    G = len(vo) - 1
    out = np.zeros(int(vo[-1]) if G >= 0 else 0, dtype=np.int32)
    if lib().oracle_bz_batched(G, _p64(vo), _p64(ao), _p32(rp), _p32(ci), _p32(out)) != 0:
        raise MemoryError("oracle_bz_batched")
    return out


def hindex_jacobi(row_ptr, col_idx):
    """Alg. 2 to its fixpoint; returns (core, rounds that changed a value)."""
    rp, ci, n = _csr(_np(row_ptr), _np(col_idx))
    out = np.zeros(n, dtype=np.int32)
    rounds = np.zeros(1, dtype=np.int64)
    if lib().oracle_hindex_jacobi(n, _p64(rp), _p32(ci), _p32(out), _p64(rounds)) != 0:
        raise MemoryError
    return out, int(rounds[0])


def peelone(row_ptr, col_idx):
    """Alg. 4 sequentially; returns (core, stats dict)."""
    rp, ci, n = _csr(_np(row_ptr), _np(col_idx))
    out = np.zeros(n, dtype=np.int32)
    st = np.zeros(5, dtype=np.int64)
    if lib().oracle_peelone(n, _p64(rp), _p32(ci), _p32(out), _p64(st)) != 0:
        raise MemoryError
    keys = ("levels", "kmax", "waves", "decrements", "arcs_scanned")
    return out, dict(zip(keys, (int(x) for x in st)))


def histocore(row_ptr, col_idx, check: bool = False):
    """Alg. 6 sequentially; returns (core, stats dict)."""
    rp, ci, n = _csr(_np(row_ptr), _np(col_idx))
    out = np.zeros(n, dtype=np.int32)
    st = np.zeros(6, dtype=np.int64)
    if lib().oracle_histocore(n, _p64(rp), _p32(ci), _p32(out), _p64(st), int(check)) != 0:
        raise MemoryError
    keys = ("rounds", "frontier", "slots_read", "arcs_scanned", "updates", "violations")
    return out, dict(zip(keys, (int(x) for x in st)))


def gpp(row_ptr, col_idx):
    """Alg. 3 (General Parallel Peel) in synchronous steps; returns
    (core, stats dict)."""
    rp, ci, n = _csr(_np(row_ptr), _np(col_idx))
    out = np.zeros(n, dtype=np.int32)
    st = np.zeros(5, dtype=np.int64)
    if lib().oracle_gpp(n, _p64(rp), _p32(ci), _p32(out), _p64(st)) != 0:
        raise MemoryError
    keys = ("steps", "scans", "decrements", "arcs_scanned", "kmax")
    return out, dict(zip(keys, (int(x) for x in st)))


def _index2core(fn, row_ptr, col_idx):
    rp, ci, n = _csr(_np(row_ptr), _np(col_idx))
    out = np.zeros(n, dtype=np.int32)
    st = np.zeros(5, dtype=np.int64)
    if fn(n, _p64(rp), _p32(ci), _p32(out), _p64(st)) != 0:
        raise MemoryError
    keys = ("rounds", "active", "frontier", "arcs_scanned", "violations")
    return out, dict(zip(keys, (int(x) for x in st)))


def nbrcore(row_ptr, col_idx):
    """NbrCore (neighbours of changed vertices recompute HINDEX), synchronous;
    returns (core, stats dict)."""
    return _index2core(lib().oracle_nbrcore, row_ptr, col_idx)


def cntcore(row_ptr, col_idx):
    """CntCore (Alg. 5), synchronous; returns (core, stats dict)."""
    return _index2core(lib().oracle_cntcore, row_ptr, col_idx)


def check(row_ptr, col_idx, core) -> dict:
    rp, ci, n = _csr(_np(row_ptr), _np(col_idx))
    c = np.ascontiguousarray(_np(core), dtype=np.int32)
    out = np.zeros(3, dtype=np.int64)
    if lib().oracle_check(n, _p64(rp), _p32(ci), _p32(c), _p64(out)) != 0:
        raise MemoryError
    return {"range": int(out[0]), "certificate": int(out[1]), "fixpoint": int(out[2])}


# ---------------------------------------------------------------------------
# pure-Python definitions (tiny inputs only)
# ---------------------------------------------------------------------------

def adjacency(n: int, edges) -> list[set]:
    adj = [set() for _ in range(n)]
    for u, v in edges:
        if u != v:
            adj[u].add(v)
            adj[v].add(u)
    return adj


def brute_force_coreness(n: int, edges) -> list[int]:
    """The definition. For k = 1, 2, ...: starting from the whole graph,
    delete vertices whose degree among the survivors is below k until none
    is; the survivors are the k-core. core(v) is the largest such k."""
    adj = adjacency(n, edges)
    core = [0] * n
    k = 1
    while True:
        alive = set(range(n))
        changed = True
        while changed:
            changed = False
            for v in list(alive):
                if len(adj[v] & alive) < k:
                    alive.discard(v)
                    changed = True
        if not alive:
            return core
        for v in alive:
            core[v] = k
        k += 1


def hindex(values) -> int:
    """HINDEX of Alg. 2: the integer h with at least h values >= h and at
    most h values >= h + 1 (the largest h with #(values >= h) >= h)."""
    h = 0
    for cand in range(1, len(values) + 1):
        if sum(1 for x in values if x >= cand) >= cand:
            h = cand
    return h


def hindex_fixpoint_pass(n: int, edges, core) -> list[int]:
    """One synchronous round of Alg. 2."""
    adj = adjacency(n, edges)
    return [hindex([core[u] for u in adj[v]]) for v in range(n)]


def csr_to_edges(row_ptr, col_idx):
    rp, ci, n = _csr(_np(row_ptr), _np(col_idx))
    edges = []
    for v in range(n):
        for e in range(rp[v], rp[v + 1]):
            if v < ci[e]:
                edges.append((v, int(ci[e])))
    return n, edges
