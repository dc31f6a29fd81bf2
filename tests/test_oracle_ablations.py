"""Pins of the oracle's ablation renditions (no GPU needed): Alg. 3 (GPP),
NbrCore and CntCore (Alg. 5).

* every rendition gives the definition's coreness (brute force on every
  labelled graph with <= 5 vertices, BZ on the workload families);
* GPP's step structure on closed forms, counted by hand: a path P_n peels
  two endpoints per step (ceil(n/2) steps after one empty scan at k = 0), a
  star takes two steps, K_n and C_n one step after k empty scans; in
  general every empty scan raises k by one, so scans = steps + max coreness;
* NbrCore and CntCore change the same estimates in the same rounds as the
  synchronous h-index iteration of Alg. 2 (Thm. 2), so their round counts
  equal its round count and their changed sets sum to HistoCore's frontier;
  a CntCore frontier vertex always falls (no violations);
* hand-counted active sets and scanned arcs on a star.
"""
import itertools

import numpy as np
import pytest

import graphgen as gg
import oracle
from conftest import load_g1

RENDITIONS = {"gpp": oracle.gpp, "nbrcore": oracle.nbrcore, "cntcore": oracle.cntcore}


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_every_small_graph(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        edges = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        rp, ci = gg.from_edge_list(edges, n).numpy()
        want = oracle.brute_force_coreness(n, edges)
        for name, fn in RENDITIONS.items():
            got, _ = fn(rp, ci)
            assert got.tolist() == want, (name, n, edges)


@pytest.mark.parametrize("n", [2, 3, 4, 7, 10, 101])
def test_gpp_path(n):
    rp, ci = gg.path_graph(n).numpy()
    core, st = oracle.gpp(rp, ci)
    assert (core == 1).all()
    steps = (n + 1) // 2
    assert st["steps"] == steps and st["scans"] == steps + 1
    # an edge decrements unless both ends leave in the same step: only the
    # middle edge of an even path does
    assert st["decrements"] == (n - 2 if n % 2 == 0 else n - 1)
    assert st["arcs_scanned"] == 2 * (n - 1) and st["kmax"] == 1


@pytest.mark.parametrize("leaves", [2, 5, 40])
def test_gpp_star(leaves):
    rp, ci = gg.star_graph(leaves).numpy()
    core, st = oracle.gpp(rp, ci)
    assert st["steps"] == 2 and st["scans"] == 3
    assert st["decrements"] == leaves and st["kmax"] == 1


@pytest.mark.parametrize("name,g,k", [("K9", gg.complete_graph(9), 8), ("C12", gg.cycle_graph(12), 2),
                                      ("Q5", gg.hypercube(5), 5)])
def test_gpp_regular(name, g, k):
    rp, ci = g.numpy()
    core, st = oracle.gpp(rp, ci)
    assert (core == k).all()
    # k empty scans (k = 0 .. k-1), then one step removes every vertex
    assert st["steps"] == 1 and st["scans"] == k + 1 and st["decrements"] == 0


def test_gpp_isolated_vertices_leave_at_zero():
    rp, ci = gg.from_edge_list([(0, 1)], 4).numpy()
    core, st = oracle.gpp(rp, ci)
    assert core.tolist() == [1, 1, 0, 0]
    # k = 0 removes the isolated pair, the rescan at k = 0 is empty, k = 1
    # removes the edge
    assert st["steps"] == 2 and st["scans"] == 3


@pytest.mark.parametrize("leaves", [2, 6, 50])
def test_index2core_star(leaves):
    rp, ci = gg.star_graph(leaves).numpy()
    L = leaves
    c, st = oracle.nbrcore(rp, ci)
    assert (c == 1).all()
    # round 0: all L + 1 vertices, only the centre falls (L -> 1);
    # round 1: its L neighbours recompute, nothing changes
    assert st == {"rounds": 1, "active": 2 * L + 1, "frontier": 1, "arcs_scanned": 3 * L,
                  "violations": 0}
    c, st = oracle.cntcore(rp, ci)
    assert (c == 1).all()
    # round 0: cnt over 2L arcs, the centre (cnt 0 < L) recomputes over L;
    # round 1: the L leaves count again (cnt 1 = estimate 1): empty frontier
    assert st == {"rounds": 1, "active": 2 * L + 1, "frontier": 1, "arcs_scanned": 4 * L,
                  "violations": 0}


@pytest.mark.parametrize("fn", [oracle.nbrcore, oracle.cntcore])
def test_index2core_converged_start(fn):
    # K_n and C_n start at their coreness: one round, no change
    for g, n, d in [(gg.complete_graph(7), 7, 6), (gg.cycle_graph(9), 9, 2)]:
        rp, ci = g.numpy()
        c, st = fn(rp, ci)
        assert (c == d).all()
        assert st["rounds"] == 0 and st["active"] == n and st["frontier"] == 0
        assert st["arcs_scanned"] == n * d


def test_index2core_g1():
    n, edges, want = load_g1()
    rp, ci = gg.from_edge_list(edges, n).numpy()
    for fn in (oracle.nbrcore, oracle.cntcore):
        c, st = fn(rp, ci)
        assert c.tolist() == want
        assert st["rounds"] == 1 and st["frontier"] == 2 and st["violations"] == 0


FAMILIES = [
    ("rmat12", lambda: gg.rmat_graph(12, 16, 11)),
    ("er", lambda: gg.er_graph(3000, 30000, 13)),
    ("chunglu", lambda: gg.chung_lu_graph(1 << 12, 14, clique=50)),
    ("grid", lambda: gg.grid_graph(30, 45)),
    ("path", lambda: gg.path_graph(64)),
]


@pytest.mark.parametrize("name,make", FAMILIES, ids=[f[0] for f in FAMILIES])
def test_families(name, make):
    g = make()
    rp, ci = g.numpy()
    want = oracle.bz_coreness(rp, ci)
    _, jrounds = oracle.hindex_jacobi(rp, ci)
    _, hst = oracle.histocore(rp, ci)
    gc, gst = oracle.gpp(rp, ci)
    assert (gc == want).all()
    assert gst["arcs_scanned"] == rp[-1] and gst["kmax"] == want.max()
    # steps >= non-empty levels; every empty scan raises k by one, from 0
    # to the largest coreness
    assert gst["steps"] >= len(np.unique(want))
    assert gst["scans"] == gst["steps"] + want.max()
    for fn in (oracle.nbrcore, oracle.cntcore):
        c, st = fn(rp, ci)
        assert (c == want).all()
        assert st["rounds"] == jrounds == hst["rounds"]
        assert st["frontier"] == hst["frontier"]
        assert st["violations"] == 0
        assert st["active"] >= st["frontier"]
