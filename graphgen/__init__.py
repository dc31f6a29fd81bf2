"""Seeded synthetic graph generators and the CSR builder.

This module is shared by the CPU oracle and the CUDA path: it only draws
random numbers and assembles simple undirected graphs in CSR form. It holds
none of the k-core arithmetic (no degrees are peeled, no h-index is taken).

Every random draw is a counter-based SplitMix64 value: draw ``i`` of stream
``s`` under seed ``seed`` is ``mix(key(seed, s) + (i + 1) * GOLDEN)``, where
``mix`` is the SplitMix64 finaliser (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014). Tensors hold the uint64 bit
pattern in torch.int64; multiplication wraps modulo 2**64 and right shifts
are made logical by masking, so the same draws come out of the CPU and the GPU.
Probabilities are compared as 53-bit (or 62-bit) integers, never as floats, so
the graphs are identical on both devices.

Every graph returned is simple and undirected: self-loops and duplicate edges
are removed, both arc directions are stored, and each neighbour list is sorted
ascending. ``row_ptr[n]`` is the number of arcs (twice the undirected edges).

Workloads (they stand in for the public web/social graphs of the paper's
Table I, which are not available here):
  * R-MAT (Chakrabarti, Zhan, Faloutsos 2004), a/b/c/d = .57/.19/.19/.05;
  * Chung-Lu power law with a planted clique;
  * 2-D 4-neighbour grids;
  * Erdos-Renyi G(n, M);
  * a packed batch of many small/medium graphs;
  * small closed-form families (complete, cycle, path, star, bipartite,
    hypercube) used by the tests.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

_MASK64 = (1 << 64) - 1


def _s64(x: int) -> int:
    """Python int -> signed int64 value with the same low 64 bits."""
    x &= _MASK64
    return x - (1 << 64) if x >= (1 << 63) else x


_GOLDEN_U = 0x9E3779B97F4A7C15
_M1_U = 0xBF58476D1CE4E5B9
_M2_U = 0x94D049BB133111EB
GOLDEN = _s64(_GOLDEN_U)
_M1 = _s64(_M1_U)
_M2 = _s64(_M2_U)

# Stream ids of the generators (any distinct constants would do).
S_RMAT = 0x100
S_ER_SRC, S_ER_DST = 0x200, 0x201
S_CL_SRC, S_CL_DST, S_CL_CLIQUE = 0x300, 0x301, 0x302
S_BATCH = 0x400
S_SERVE = 0x500


def mix64_int(z: int) -> int:
    """SplitMix64 finaliser on a Python int (uint64 semantics)."""
    z &= _MASK64
    z = ((z ^ (z >> 30)) * _M1_U) & _MASK64
    z = ((z ^ (z >> 27)) * _M2_U) & _MASK64
    return z ^ (z >> 31)


def _srl(z: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of an int64 tensor holding uint64 bits."""
    return (z >> s) & ((1 << (64 - s)) - 1)


def mix64(z: torch.Tensor) -> torch.Tensor:
    """SplitMix64 finaliser on an int64 tensor (uint64 bit patterns)."""
    z = (z ^ _srl(z, 30)) * _M1
    z = (z ^ _srl(z, 27)) * _M2
    return z ^ _srl(z, 31)


def stream_key(seed: int, stream: int) -> int:
    """Per-(seed, stream) key, as a signed int64 Python value."""
    return _s64(mix64_int(mix64_int(seed) ^ ((stream + 1) * _GOLDEN_U)))


def draw_bits(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """uint64 draws (int64 bit patterns) for counter values ``idx``."""
    return mix64((idx + 1) * GOLDEN + stream_key(seed, stream))


def draw_bits_int(seed: int, stream: int, i: int) -> int:
    """The same draw as :func:`draw_bits`, as a Python int in [0, 2**64)."""
    return mix64_int(((i + 1) * _GOLDEN_U + (stream_key(seed, stream) & _MASK64)) & _MASK64)


def unit_int(seed: int, stream: int, i: int) -> float:
    """A uniform double in [0, 1) from the top 53 bits of a draw (exact)."""
    return (draw_bits_int(seed, stream, i) >> 11) * (1.0 / (1 << 53))


def draw_below(seed: int, stream: int, idx: torch.Tensor, n: int) -> torch.Tensor:
    """Integers in [0, n) by the multiply-shift map of the top 32 bits (n < 2**31)."""
    hi = _srl(draw_bits(seed, stream, idx), 32)
    return _srl(hi * n, 32)


# ---------------------------------------------------------------------------
# CSR builder
# ---------------------------------------------------------------------------

@dataclass
class Graph:
    """A simple undirected graph in CSR form (tensors on one device)."""
    n: int
    row_ptr: torch.Tensor   # int32 or int64, n + 1 entries
    col_idx: torch.Tensor   # int32, row_ptr[n] entries, sorted per row
    name: str = ""

    @property
    def arcs(self) -> int:
        return int(self.row_ptr[-1].item()) if self.n > 0 else 0

    @property
    def edges(self) -> int:
        return self.arcs // 2

    def to(self, device, off_dtype=None) -> "Graph":
        rp = self.row_ptr.to(device)
        if off_dtype is not None:
            rp = rp.to(off_dtype)
        return Graph(self.n, rp, self.col_idx.to(device), self.name)

    def numpy(self):
        return (self.row_ptr.cpu().numpy().astype(np.int64),
                self.col_idx.cpu().numpy().astype(np.int32))


def csr_from_pairs(src: torch.Tensor, dst: torch.Tensor, n: int,
                   off_dtype=torch.int32, name: str = "") -> Graph:
    """Symmetrise an endpoint-pair list into a sorted simple CSR graph.

    Self-loops and duplicates (in either direction) are dropped.
    """
    device = src.device
    src = src.to(torch.int64)
    dst = dst.to(torch.int64)
    keep = src != dst
    lo = torch.minimum(src, dst)[keep]
    hi = torch.maximum(src, dst)[keep]
    del keep
    und = torch.unique(lo * n + hi)          # sorted unique undirected edges
    del lo, hi
    lo = torch.div(und, n, rounding_mode="floor")
    hi = und - lo * n
    del und
    keys = torch.cat([lo * n + hi, hi * n + lo])
    del lo, hi
    keys, _ = torch.sort(keys)
    s = torch.div(keys, n, rounding_mode="floor")
    col = (keys - s * n).to(torch.int32)
    del keys
    counts = torch.bincount(s, minlength=n)
    del s
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
    if n > 0:
        row_ptr[1:] = torch.cumsum(counts, 0)
    if off_dtype == torch.int32:
        assert n == 0 or int(row_ptr[-1]) < 2 ** 31, "arc count needs int64 offsets"
    return Graph(n, row_ptr.to(off_dtype), col, name)


def from_edge_list(edges, n: int, device="cpu", off_dtype=torch.int32, name="") -> Graph:
    """Graph from a Python list of (u, v) pairs."""
    if len(edges) == 0:
        e = torch.zeros((0, 2), dtype=torch.int64)
    else:
        e = torch.tensor(edges, dtype=torch.int64)
    return csr_from_pairs(e[:, 0].to(device), e[:, 1].to(device), n, off_dtype, name)


# ---------------------------------------------------------------------------
# Random families
# ---------------------------------------------------------------------------

RMAT_ABC = (0.57, 0.19, 0.19)


def rmat_pairs(scale: int, nsamples: int, seed: int, device="cpu",
               abc=RMAT_ABC, first: int = 0) -> tuple[torch.Tensor, torch.Tensor]:
    """Directed R-MAT endpoint samples ``first .. first+nsamples-1``.

    Each sample descends ``scale`` levels of the 2x2 recursive matrix. At level
    l (most significant bit first) one 53-bit draw picks quadrant a, b, c or d:
    b and d set the destination bit, c and d set the source bit.
    """
    a, b, c = abc
    ta = int(a * (1 << 53))
    tab = int((a + b) * (1 << 53))
    tabc = int((a + b + c) * (1 << 53))
    idx = torch.arange(first, first + nsamples, dtype=torch.int64, device=device)
    src = torch.zeros_like(idx)
    dst = torch.zeros_like(idx)
    for lev in range(scale):
        r = _srl(draw_bits(seed, S_RMAT + lev, idx), 11)
        sbit = r >= tab
        dbit = ((r >= ta) & (r < tab)) | (r >= tabc)
        sh = scale - 1 - lev
        src |= sbit.to(torch.int64) << sh
        dst |= dbit.to(torch.int64) << sh
        del r, sbit, dbit
    return src, dst


def rmat_graph(scale: int, edge_factor: int, seed: int, device="cpu",
               off_dtype=torch.int32, chunk: int = 1 << 26) -> Graph:
    """R-MAT graph with 2**scale vertices and edge_factor * 2**scale samples,
    symmetrised, without self-loops or duplicates (no vertex relabelling)."""
    n = 1 << scale
    total = edge_factor * n
    srcs, dsts = [], []
    for first in range(0, total, chunk):
        cnt = min(chunk, total - first)
        s, d = rmat_pairs(scale, cnt, seed, device, first=first)
        lo = torch.minimum(s, d)
        hi = torch.maximum(s, d)
        del s, d
        srcs.append(lo)
        dsts.append(hi)
    src = torch.cat(srcs)
    dst = torch.cat(dsts)
    del srcs, dsts
    return csr_from_pairs(src, dst, n, off_dtype, f"rmat-s{scale}-ef{edge_factor}")


def er_graph(n: int, m_samples: int, seed: int, device="cpu", off_dtype=torch.int32) -> Graph:
    """Erdos-Renyi G(n, M): M uniform endpoint pairs, then dedup (M' <= M)."""
    idx = torch.arange(m_samples, dtype=torch.int64, device=device)
    s = draw_below(seed, S_ER_SRC, idx, n)
    d = draw_below(seed, S_ER_DST, idx, n)
    return csr_from_pairs(s, d, n, off_dtype, f"er-n{n}-M{m_samples}")


def chung_lu_graph(n: int, seed: int, beta: float = 2.1, pairs_per_vertex: int = 10,
                   i0: int = 1, clique: int = 3000, device="cpu",
                   off_dtype=torch.int32, chunk: int = 1 << 26) -> Graph:
    """Chung-Lu power-law graph with a planted clique.

    Weights w_i = (i + i0)^(-1/(beta-1)); ``pairs_per_vertex * n`` endpoint
    pairs are drawn i.i.d. with both ends proportional to w (expected mean
    degree 2 * pairs_per_vertex before dedup). The cumulative weights are
    turned into 62-bit integer thresholds once on the host, so sampling is an
    exact integer search on either device. A clique is planted on ``clique``
    vertices chosen uniformly (the smallest draw keys).
    """
    alpha = 1.0 / (beta - 1.0)
    w = (np.arange(n, dtype=np.float64) + float(i0)) ** (-alpha)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    thr = np.floor(cdf * float(1 << 62)).astype(np.int64)
    thr[-1] = 1 << 62
    thr_t = torch.from_numpy(thr).to(device)
    total = pairs_per_vertex * n
    srcs, dsts = [], []
    for first in range(0, total, chunk):
        cnt = min(chunk, total - first)
        idx = torch.arange(first, first + cnt, dtype=torch.int64, device=device)
        rs = _srl(draw_bits(seed, S_CL_SRC, idx), 2)
        rd = _srl(draw_bits(seed, S_CL_DST, idx), 2)
        srcs.append(torch.searchsorted(thr_t, rs, right=True))
        dsts.append(torch.searchsorted(thr_t, rd, right=True))
        del idx, rs, rd
    if clique > 0:
        keys = draw_bits(seed, S_CL_CLIQUE, torch.arange(n, dtype=torch.int64, device=device))
        members = torch.sort(torch.argsort(keys, stable=True)[:clique]).values
        del keys
        iu = torch.triu_indices(clique, clique, 1, device=device)
        srcs.append(members[iu[0]])
        dsts.append(members[iu[1]])
    src = torch.cat(srcs)
    dst = torch.cat(dsts)
    del srcs, dsts
    g = csr_from_pairs(src, dst, n, off_dtype, f"chunglu-n{n}-b{beta}-clique{clique}")
    return g


def clique_members(n: int, seed: int, clique: int, device="cpu") -> torch.Tensor:
    """The vertices of the clique planted by :func:`chung_lu_graph`."""
    keys = draw_bits(seed, S_CL_CLIQUE, torch.arange(n, dtype=torch.int64, device=device))
    return torch.sort(torch.argsort(keys, stable=True)[:clique]).values


def grid_graph(rows: int, cols: int, device="cpu", off_dtype=torch.int32) -> Graph:
    """rows x cols 4-neighbour grid; vertex (r, c) has id r * cols + c."""
    ids = torch.arange(rows * cols, dtype=torch.int64, device=device).view(rows, cols)
    src = torch.cat([ids[:, :-1].reshape(-1), ids[:-1, :].reshape(-1)])
    dst = torch.cat([ids[:, 1:].reshape(-1), ids[1:, :].reshape(-1)])
    return csr_from_pairs(src, dst, rows * cols, off_dtype, f"grid-{rows}x{cols}")


# ---------------------------------------------------------------------------
# Closed-form families (for tests)
# ---------------------------------------------------------------------------

def complete_graph(n, device="cpu"):
    e = [(i, j) for i in range(n) for j in range(i + 1, n)]
    return from_edge_list(e, n, device, name=f"K{n}")


def cycle_graph(n, device="cpu"):
    return from_edge_list([(i, (i + 1) % n) for i in range(n)], n, device, name=f"C{n}")


def path_graph(n, device="cpu"):
    return from_edge_list([(i, i + 1) for i in range(n - 1)], n, device, name=f"P{n}")


def star_graph(leaves, device="cpu"):
    return from_edge_list([(0, i) for i in range(1, leaves + 1)], leaves + 1, device,
                          name=f"S{leaves}")


def complete_bipartite(a, b, device="cpu"):
    e = [(i, a + j) for i in range(a) for j in range(b)]
    return from_edge_list(e, a + b, device, name=f"K{a},{b}")


def hypercube(d, device="cpu"):
    n = 1 << d
    e = [(v, v ^ (1 << i)) for v in range(n) for i in range(d) if v < v ^ (1 << i)]
    return from_edge_list(e, n, device, name=f"Q{d}")


def random_tree(n, seed, device="cpu"):
    """Random recursive tree: vertex i > 0 attaches to a uniform earlier vertex."""
    e = [(i, int(draw_bits_int(seed, 0x600, i) % i)) for i in range(1, n)]
    return from_edge_list(e, n, device, name=f"tree{n}")


def disjoint_union(graphs, device="cpu", off_dtype=torch.int32) -> Graph:
    """Disjoint union with vertex ids shifted graph by graph."""
    rps, cols, base_v, base_a = [torch.zeros(1, dtype=torch.int64)], [], 0, 0
    for g in graphs:
        rp = g.row_ptr.cpu().to(torch.int64)
        rps.append(rp[1:] + base_a)
        cols.append(g.col_idx.cpu().to(torch.int64) + base_v)
        base_v += g.n
        base_a += int(rp[-1])
    rp = torch.cat(rps).to(off_dtype)
    col = torch.cat(cols).to(torch.int32) if cols else torch.zeros(0, dtype=torch.int32)
    return Graph(base_v, rp.to(device), col.to(device), "union")


# ---------------------------------------------------------------------------
# Packed batch of many graphs
# ---------------------------------------------------------------------------

@dataclass
class BatchSpec:
    kind: str        # "er" or "rmat"
    n: int
    param: float     # ER: mean degree d; R-MAT: edge factor
    seed: int


def batch_specs(G: int, seed: int, nmin: int = 100, nmax: int = 200000) -> list[BatchSpec]:
    """Graph sizes log-uniform in [nmin, nmax]; even indices ER with mean degree
    U[4, 64], odd indices R-MAT with edge factor U{8..32}."""
    out = []
    lmin, lmax = math.log(nmin), math.log(nmax)
    for g in range(G):
        u1 = unit_int(seed, S_BATCH, 2 * g)
        u2 = unit_int(seed, S_BATCH, 2 * g + 1)
        n = int(round(math.exp(lmin + u1 * (lmax - lmin))))
        gseed = mix64_int(seed * 1000003 + g)
        if g % 2 == 0:
            out.append(BatchSpec("er", n, 4.0 + 60.0 * u2, gseed))
        else:
            out.append(BatchSpec("rmat", n, float(8 + min(24, int(u2 * 25))), gseed))
    return out


def spec_graph(sp: BatchSpec, device="cpu") -> Graph:
    """One graph of a batch spec. R-MAT runs at scale ceil(log2 n) with
    edge_factor * n samples, rejecting samples with an endpoint >= n."""
    n = sp.n
    if sp.kind == "er":
        return er_graph(n, int(round(n * sp.param / 2.0)), sp.seed, device)
    scale = max(1, math.ceil(math.log2(n)))
    s, d = rmat_pairs(scale, int(sp.param) * n, sp.seed, device)
    ok = (s < n) & (d < n)
    return csr_from_pairs(s[ok], d[ok], n, torch.int32, f"rmat-n{n}")


@dataclass
class PackedBatch:
    """G graphs packed back to back.

    vtx_off[g], arc_off[g]: int64 prefix offsets (G + 1 entries).
    row_ptr: int32, graph-local (relative to arc_off[g]); graph g's n_g + 1
             entries start at vtx_off[g] + g.
    col_idx: int32 graph-local vertex ids.
    """
    G: int
    vtx_off: torch.Tensor
    arc_off: torch.Tensor
    row_ptr: torch.Tensor
    col_idx: torch.Tensor

    def graph(self, g: int) -> Graph:
        v0, v1 = int(self.vtx_off[g]), int(self.vtx_off[g + 1])
        a0, a1 = int(self.arc_off[g]), int(self.arc_off[g + 1])
        rp = self.row_ptr[v0 + g: v1 + g + 1]
        return Graph(v1 - v0, rp, self.col_idx[a0:a1], f"batch-{g}")


def pack_graphs(graphs: list[Graph], device="cpu") -> PackedBatch:
    G = len(graphs)
    ns = [g.n for g in graphs]
    arcs = [g.arcs for g in graphs]
    vtx_off = torch.zeros(G + 1, dtype=torch.int64)
    arc_off = torch.zeros(G + 1, dtype=torch.int64)
    vtx_off[1:] = torch.cumsum(torch.tensor(ns, dtype=torch.int64), 0)
    arc_off[1:] = torch.cumsum(torch.tensor(arcs, dtype=torch.int64), 0)
    row_ptr = torch.cat([g.row_ptr.to(device=device, dtype=torch.int32) for g in graphs]) \
        if G else torch.zeros(0, dtype=torch.int32, device=device)
    col_idx = torch.cat([g.col_idx.to(device) for g in graphs]) \
        if G else torch.zeros(0, dtype=torch.int32, device=device)
    return PackedBatch(G, vtx_off.to(device), arc_off.to(device), row_ptr, col_idx)


def batch_graph(G: int, seed: int, device="cpu", nmin: int = 100, nmax: int = 200000) -> PackedBatch:
    """The packed batch of :func:`batch_specs` (generated graph by graph)."""
    return pack_graphs([spec_graph(sp, device) for sp in batch_specs(G, seed, nmin, nmax)], device)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

SEED_BASE = 0x9C0


def workload(name: str, device="cpu") -> Graph:
    """The named synthetic workloads, with their fixed seeds.

    rmat16       R-MAT scale 16, edge factor 16, int32 CSR
    rmat22       R-MAT scale 22, edge factor 16, int64 row_ptr
    rmat24       R-MAT scale 24, edge factor 16, int32 CSR
    chunglu24    Chung-Lu beta 2.1, 2**24 vertices, mean degree 20, K_3000 planted
    grid4096     4096 x 4096 grid
    """
    if name == "rmat16":
        return rmat_graph(16, 16, SEED_BASE + 1, device)
    if name == "rmat22":
        return rmat_graph(22, 16, SEED_BASE + 2, device, off_dtype=torch.int64)
    if name == "rmat24":
        return rmat_graph(24, 16, SEED_BASE + 3, device)
    if name == "chunglu24":
        return chung_lu_graph(1 << 24, SEED_BASE + 3, device=device)
    if name == "grid4096":
        return grid_graph(4096, 4096, device)
    m = None
    if name.startswith("rmat"):
        m = name[4:]
        if m.isdigit():
            return rmat_graph(int(m), 16, SEED_BASE + 7, device)
    raise ValueError(f"unknown workload {name!r}")
