"""Pins of the CPU oracle against things other than itself (no GPU needed).

* the definition (brute force) on every labelled graph with <= 6 vertices
  and on random graphs up to 64 vertices;
* closed forms: K_n -> n-1, C_n -> 2, paths/trees/stars -> 1, a x b grids
  -> 2, K_{a,b} -> min(a, b), hypercube Q_d -> d, isolated vertex -> 0,
  disjoint unions -> per component, planted clique K_c -> >= c-1;
* the paper's example G1 (Sec. I) and the h-index example of Fig. 6;
* agreement of BZ with the renditions of Alg. 2, Alg. 4 and Alg. 6, and the
  fixpoint/certificate checks, on synthetic graphs of each workload family.
"""
import itertools

import numpy as np
import pytest

import graphgen as gg
import oracle
from conftest import load_g1, read_golden


def _csr(n, edges):
    g = gg.from_edge_list(edges, n)
    return g.numpy()


def _all_four(rp, ci):
    c = oracle.bz_coreness(rp, ci)
    j, _ = oracle.hindex_jacobi(rp, ci)
    p, _ = oracle.peelone(rp, ci)
    h, st = oracle.histocore(rp, ci)
    return c, j, p, h, st


# --------------------------------------------------------------------------
# the definition
# --------------------------------------------------------------------------

def _pack_numpy(graphs):
    """graphs: list of (n, edges) -> packed batch arrays (numpy)."""
    vtx_off = [0]
    arc_off = [0]
    rps, cis = [], []
    for n, edges in graphs:
        adj = [[] for _ in range(n)]
        for u, v in edges:
            adj[u].append(v)
            adj[v].append(u)
        rp = [0]
        for v in range(n):
            adj[v].sort()
            rp.append(rp[-1] + len(adj[v]))
        rps.extend(rp)
        for v in range(n):
            cis.extend(adj[v])
        vtx_off.append(vtx_off[-1] + n)
        arc_off.append(arc_off[-1] + rp[-1])
    return (np.array(vtx_off, np.int64), np.array(arc_off, np.int64),
            np.array(rps, np.int32), np.array(cis, np.int32))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_bz_equals_definition_on_every_small_graph(n):
    pairs = list(itertools.combinations(range(n), 2))
    graphs = []
    for mask in range(1 << len(pairs)):
        graphs.append((n, [pairs[i] for i in range(len(pairs)) if mask >> i & 1]))
    vo, ao, rp, ci = _pack_numpy(graphs)
    got = oracle.bz_coreness_batched(vo, ao, rp, ci)
    for g, (nn, edges) in enumerate(graphs):
        want = oracle.brute_force_coreness(nn, edges)
        assert list(got[vo[g]:vo[g + 1]]) == want, (n, edges)


def test_bz_equals_definition_on_random_graphs():
    for trial in range(60):
        n = 8 + (trial * 7) % 57
        p = [0.05, 0.1, 0.2, 0.35, 0.5][trial % 5]
        rng = np.random.default_rng(1000 + trial)
        edges = [(u, v) for u in range(n) for v in range(u + 1, n) if rng.random() < p]
        rp, ci = _csr(n, edges)
        want = oracle.brute_force_coreness(n, edges)
        c, j, pe, h, st = _all_four(rp, ci)
        assert list(c) == want
        assert list(j) == want and list(pe) == want and list(h) == want
        assert st["violations"] == 0


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

CLOSED = [
    ("K1", gg.complete_graph(1), lambda n: [0]),
    ("K2", gg.complete_graph(2), lambda n: [1] * 2),
    ("K7", gg.complete_graph(7), lambda n: [6] * 7),
    ("K40", gg.complete_graph(40), lambda n: [39] * 40),
    ("C3", gg.cycle_graph(3), lambda n: [2] * 3),
    ("C50", gg.cycle_graph(50), lambda n: [2] * 50),
    ("P2", gg.path_graph(2), lambda n: [1] * 2),
    ("P33", gg.path_graph(33), lambda n: [1] * 33),
    ("S1", gg.star_graph(1), lambda n: [1] * 2),
    ("S25", gg.star_graph(25), lambda n: [1] * 26),
    ("tree300", gg.random_tree(300, 5), lambda n: [1] * 300),
    ("grid2x2", gg.grid_graph(2, 2), lambda n: [2] * 4),
    ("grid7x13", gg.grid_graph(7, 13), lambda n: [2] * 91),
    ("grid1x9", gg.grid_graph(1, 9), lambda n: [1] * 9),
    ("K3,8", gg.complete_bipartite(3, 8), lambda n: [3] * 11),
    ("K9,9", gg.complete_bipartite(9, 9), lambda n: [9] * 18),
    ("Q1", gg.hypercube(1), lambda n: [1] * 2),
    ("Q5", gg.hypercube(5), lambda n: [5] * 32),
    ("Q8", gg.hypercube(8), lambda n: [8] * 256),
    ("isolated", gg.from_edge_list([], 5), lambda n: [0] * 5),
]


@pytest.mark.parametrize("name,g,want", CLOSED, ids=[c[0] for c in CLOSED])
def test_closed_forms(name, g, want):
    rp, ci = g.numpy()
    expect = want(g.n)
    c, j, p, h, st = _all_four(rp, ci)
    assert list(c) == expect
    assert list(j) == expect and list(p) == expect and list(h) == expect
    if g.n <= 40:
        n, edges = oracle.csr_to_edges(rp, ci)
        assert oracle.brute_force_coreness(n, edges) == expect


def test_disjoint_union_is_per_component():
    parts = [gg.complete_graph(6), gg.cycle_graph(9), gg.from_edge_list([], 3),
             gg.hypercube(4), gg.star_graph(4), gg.complete_bipartite(4, 6)]
    u = gg.disjoint_union(parts)
    rp, ci = u.numpy()
    want = [5] * 6 + [2] * 9 + [0] * 3 + [4] * 16 + [1] * 5 + [4] * 10
    c, j, p, h, _ = _all_four(rp, ci)
    assert list(c) == want and list(j) == want and list(p) == want and list(h) == want


def test_planted_clique():
    n, clique, seed = 1 << 13, 120, 77
    g = gg.chung_lu_graph(n, seed, clique=clique, pairs_per_vertex=3)
    rp, ci = g.numpy()
    c = oracle.bz_coreness(rp, ci)
    members = gg.clique_members(n, seed, clique).numpy()
    assert (c[members] >= clique - 1).all()
    assert c.max() >= clique - 1
    assert oracle.check(rp, ci, c) == {"range": 0, "certificate": 0, "fixpoint": 0}


# --------------------------------------------------------------------------
# the paper's examples
# --------------------------------------------------------------------------

def test_g1_example():
    n, edges, want = load_g1()
    rp, ci = _csr(n, edges)
    assert list(np.diff(rp)) == [1, 1, 2, 3, 2, 5]
    assert oracle.brute_force_coreness(n, edges) == want
    c, j, p, h, st = _all_four(rp, ci)
    assert list(c) == want and list(j) == want and list(p) == want and list(h) == want
    # PeelOne (Sec. III-C): levels k = 1 and k = 2; level 2 runs the frontier
    # {v2, v4}, then the clamped {v3, v5} in a second wave.
    _, pst = oracle.peelone(rp, ci)
    assert pst["levels"] == 2 and pst["kmax"] == 2 and pst["waves"] == 3
    # HistoCore: V_cnt starts as {v3, v5}; one round settles everything.
    _, hst = oracle.histocore(rp, ci, check=True)
    assert hst["rounds"] == 1 and hst["frontier"] == 2 and hst["violations"] == 0


def test_fig6_hindex():
    d = read_golden("fig6_hindex.txt")
    values = [int(x) for x in d["values"][0]]
    histo = {int(a): int(b) for a, b in (t.split(":") for t in d["histo"][0])}
    h = int(d["h"][0][0])
    assert {v: values.count(v) for v in set(values)} == histo
    assert oracle.hindex(values) == h
    # Sec. II-C: starting from core = deg, v5's first re-estimate is 5 -> 2.
    n, edges, _ = load_g1()
    deg = [sum(1 for e in edges if v in e) for v in range(n)]
    frm, to = (int(x) for x in d["change"][0])
    assert deg[5] == frm
    assert [deg[u] for u in (0, 1, 2, 3, 4)] == values
    assert oracle.hindex_fixpoint_pass(n, edges, deg)[5] == to


def test_hindex_definition_small_cases():
    assert oracle.hindex([]) == 0
    assert oracle.hindex([0, 0]) == 0
    assert oracle.hindex([5]) == 1
    assert oracle.hindex([1, 1, 1, 1]) == 1
    assert oracle.hindex([3, 3, 3]) == 3
    assert oracle.hindex([4, 4, 4]) == 3
    assert oracle.hindex([10, 8, 5, 4, 3]) == 4
    assert oracle.hindex([25, 8, 5, 3, 3]) == 3


# --------------------------------------------------------------------------
# synthetic workload families: the four renditions agree, invariants hold
# --------------------------------------------------------------------------

FAMILIES = [
    ("rmat12", lambda: gg.rmat_graph(12, 16, 11)),
    ("rmat14-ef8", lambda: gg.rmat_graph(14, 8, 12)),
    ("er", lambda: gg.er_graph(5000, 60000, 13)),
    ("chunglu", lambda: gg.chung_lu_graph(1 << 13, 14, clique=60)),
    ("grid", lambda: gg.grid_graph(40, 70)),
]


@pytest.mark.parametrize("name,make", FAMILIES, ids=[f[0] for f in FAMILIES])
def test_renditions_agree(name, make):
    g = make()
    rp, ci = g.numpy()
    c, j, p, h, hst = _all_four(rp, ci)
    assert (c == j).all() and (c == p).all() and (c == h).all()
    assert oracle.check(rp, ci, c) == {"range": 0, "certificate": 0, "fixpoint": 0}
    _, hst2 = oracle.histocore(rp, ci, check=True)
    assert hst2["violations"] == 0
    _, pst = oracle.peelone(rp, ci)
    # Non-empty levels are exactly the distinct non-zero coreness values.
    assert pst["levels"] == len(np.unique(c[c > 0]))
    assert pst["kmax"] == c.max()
    # Every arc of a non-isolated vertex is scanned once by its frontier.
    assert pst["arcs_scanned"] == rp[-1]


def test_rmat16_properties():
    g = gg.workload("rmat16")
    rp, ci = g.numpy()
    c = oracle.bz_coreness(rp, ci)
    deg = np.diff(rp)
    assert (c[deg == 0] == 0).all() and (c[deg > 0] >= 1).all()
    assert (c <= deg).all()
    assert oracle.check(rp, ci, c) == {"range": 0, "certificate": 0, "fixpoint": 0}


def test_checker_rejects_wrong_vectors():
    g = gg.rmat_graph(11, 8, 21)
    rp, ci = g.numpy()
    c = oracle.bz_coreness(rp, ci)
    # all zeros is a fixpoint of Alg. 2 (not sufficient) but fails nothing else
    z = np.zeros_like(c)
    r = oracle.check(rp, ci, z)
    assert r["range"] == 0 and r["certificate"] == 0
    # raising one vertex above its coreness breaks the certificate or fixpoint
    v = int(np.argmax(c))
    bad = c.copy()
    bad[v] += 1
    r = oracle.check(rp, ci, bad)
    assert r["certificate"] + r["fixpoint"] + r["range"] > 0
    # lowering one breaks the fixpoint somewhere
    v = int(np.argmax(c > 1))
    bad = c.copy()
    bad[v] -= 1
    assert oracle.check(rp, ci, bad)["fixpoint"] > 0
