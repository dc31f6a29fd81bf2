"""GPU tests of core maintenance (pico_dyn_*): after every batch of edge
insertions and deletions, the maintained coreness must equal the oracle's
(Batagelj-Zaversnik) on the updated graph, and the maintained CSR must hold
exactly the updated edge set."""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pico():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_15253_gb300 as p
    torch.cuda.set_device(0)
    return p


def edges_of(g):
    rp, ci = g.numpy()
    src = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    return {(int(a), int(b)) for a, b in zip(src, ci) if a < b}


def check(pico, dg, n, edges):
    g = gg.from_edge_list(sorted(edges), n)
    rp, ci = g.numpy()
    want = oracle.bz_coreness(rp, ci)
    got = dg.coreness().cpu().numpy()
    assert np.array_equal(got, want)
    drp, dci = dg.csr()
    drp, dci = drp.cpu().numpy(), dci.cpu().numpy()
    assert drp[-1] == 2 * len(edges)
    src = np.repeat(np.arange(n), np.diff(drp))
    got_arcs = set(zip(src.tolist(), dci.tolist()))
    want_arcs = {(a, b) for a, b in edges} | {(b, a) for a, b in edges}
    assert got_arcs == want_arcs


def random_batch(rng, n, edges, k_ins, k_del):
    cur = sorted(edges)
    dele = [cur[i] for i in rng.choice(len(cur), size=min(k_del, len(cur)), replace=False)] \
        if cur and k_del else []
    ins = set()
    while len(ins) < k_ins:
        a, b = (int(x) for x in rng.integers(0, n, size=2))
        if a == b:
            continue
        e = (min(a, b), max(a, b))
        if e not in edges and e not in ins:
            ins.add(e)
    return sorted(ins), dele


def test_closed_forms(pico):
    # a path becomes a cycle (core 1 -> 2); four vertices on a path become K4
    # in one batch (a rise by two, several passes)
    dg = pico.DynamicGraph(gg.path_graph(6).row_ptr.cuda(), gg.path_graph(6).col_idx.cuda())
    dg.update(insert=[(0, 5)])
    assert (dg.coreness().cpu() == 2).all()
    p4 = gg.path_graph(4)
    dg = pico.DynamicGraph(p4.row_ptr.cuda(), p4.col_idx.cuda())
    dg.update(insert=[(0, 2), (1, 3), (0, 3)])
    assert dg.coreness().cpu().tolist() == [3, 3, 3, 3]
    st = pico.pico_get_stats()
    assert st["algo"] == pico.PICO_STATS_MAINTENANCE and st["rounds"] >= 2
    # K6 minus one edge: 5, 5, 4... then every edge removed
    k6 = gg.complete_graph(6)
    dg = pico.DynamicGraph(k6.row_ptr.cuda(), k6.col_idx.cuda())
    dg.update(delete=[(0, 1)])
    assert dg.coreness().cpu().tolist() == [4] * 6
    dg.update(delete=sorted(edges_of(k6) - {(0, 1)}))
    assert (dg.coreness().cpu() == 0).all()


def test_isolated_vertices_join_in_a_mixed_batch(pico):
    # vertices 6..9 start isolated (estimate 0) and gain edges in the same
    # batch that deletes others: the deletion rounds see estimates of 0
    edges = {(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 5), (5, 3)}
    g = gg.from_edge_list(sorted(edges), 10)
    dg = pico.DynamicGraph(g.row_ptr.cuda(), g.col_idx.cuda(), capacity_arcs=200)
    ins = [(6, 0), (6, 1), (7, 6), (7, 0), (8, 9), (9, 3)]
    dele = [(2, 3), (4, 5)]
    dg.update(insert=ins, delete=dele)
    check(pico, dg, 10, (edges - set(dele)) | set(ins))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_small_graphs(pico, seed):
    rng = np.random.default_rng(seed)
    for trial in range(6):
        n = int(rng.integers(5, 60))
        p = [0.05, 0.15, 0.3][trial % 3]
        edges = {(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p}
        g = gg.from_edge_list(sorted(edges), n)
        dg = pico.DynamicGraph(g.row_ptr.cuda(), g.col_idx.cuda(), capacity_arcs=n * n)
        for _ in range(4):
            ins, dele = random_batch(rng, n, edges, int(rng.integers(0, 8)), int(rng.integers(0, 8)))
            dg.update(insert=ins, delete=dele)
            edges = (edges - set(dele)) | set(ins)
            check(pico, dg, n, edges)


@pytest.mark.parametrize("name,make", [("rmat15", lambda: gg.rmat_graph(15, 16, 71)),
                                       ("er-20k", lambda: gg.er_graph(20000, 120000, 72)),
                                       ("grid-120", lambda: gg.grid_graph(120, 120))])
def test_batches_on_larger_graphs(pico, name, make):
    rng = np.random.default_rng(73)
    g = make()
    n = g.n
    edges = edges_of(g)
    dg = pico.DynamicGraph(g.row_ptr.cuda(), g.col_idx.cuda(), capacity_arcs=2 * g.arcs)
    for k_ins, k_del in [(500, 0), (0, 500), (2000, 2000), (50, 3000)]:
        ins, dele = random_batch(rng, n, edges, k_ins, k_del)
        dg.update(insert=ins, delete=dele)
        edges = (edges - set(dele)) | set(ins)
        check(pico, dg, n, edges)


def test_bad_batches_leave_the_state_unchanged(pico):
    g = gg.cycle_graph(10)
    dg = pico.DynamicGraph(g.row_ptr.cuda(), g.col_idx.cuda(), capacity_arcs=100)
    bad = [dict(delete=[(0, 5)]),            # not an edge
           dict(insert=[(0, 1)]),            # already an edge
           dict(insert=[(2, 2)]),            # self-loop
           dict(insert=[(0, 10)]),           # vertex out of range
           dict(insert=[(0, 4), (4, 0)]),    # the same edge twice
           dict(delete=[(0, 1), (1, 0)])]
    for b in bad:
        with pytest.raises(pico.PicoError) as e:
            dg.update(**b)
        assert e.value.status == pico.PICO_ERR_BAD_GRAPH, b
        check(pico, dg, 10, edges_of(g))
    small = pico.DynamicGraph(g.row_ptr.cuda(), g.col_idx.cuda(), capacity_arcs=24)
    with pytest.raises(pico.PicoError) as e:   # 26 arcs > capacity 24
        small.update(insert=[(0, 2), (0, 4), (0, 6)])
    assert e.value.status == pico.PICO_ERR_INVALID_ARG
    small.update(insert=[(0, 2), (0, 4)])     # 24 arcs fit
    check(pico, small, 10, edges_of(g) | {(0, 2), (0, 4)})


@pytest.mark.parametrize("L", [100, 600])
def test_ladder_closes_into_a_prism(pico, L):
    # A 2 x L ladder has coreness 2 (its four corners have degree 2). Closing
    # both rails makes the prism C_L x K2, which is 3-regular: every vertex
    # rises to 3. The region of the first pass spreads from the four endpoints
    # along the rails, about L / 2 levels: within the search's level bound for
    # L = 100, beyond it (every candidate taken instead) for L = 600.
    edges = set()
    for i in range(L):
        edges.add((i, L + i))
        if i + 1 < L:
            edges.add((i, i + 1))
            edges.add((L + i, L + i + 1))
    n = 2 * L
    g = gg.from_edge_list(sorted(edges), n)
    dg = pico.DynamicGraph(g.row_ptr.cuda(), g.col_idx.cuda(), capacity_arcs=2 * len(edges) + 8)
    assert (dg.coreness().cpu() == 2).all()
    ins = [(0, L - 1), (L, 2 * L - 1)]
    dg.update(insert=ins)
    assert (dg.coreness().cpu() == 3).all()
    check(pico, dg, n, edges | set(ins))
    st = pico.pico_get_stats()
    assert st["algo"] == pico.PICO_STATS_MAINTENANCE and st["frontier"] == n


def test_insertions_far_from_other_candidates_stay_local(pico):
    # A 2 x 50 ladder (96 vertices of degree 3 at coreness 2: all candidates
    # to rise) and, apart from it, a path of 10 vertices closed into a cycle by
    # the batch. Only the path's vertices are connected to the inserted edge,
    # so the passes' regions hold at most those 10, and the ladder stays at 2.
    L = 50
    edges = {(i, L + i) for i in range(L)}
    edges |= {(i, i + 1) for i in range(L - 1)} | {(L + i, L + i + 1) for i in range(L - 1)}
    n = 2 * L + 10
    edges |= {(2 * L + i, 2 * L + i + 1) for i in range(9)}
    g = gg.from_edge_list(sorted(edges), n)
    dg = pico.DynamicGraph(g.row_ptr.cuda(), g.col_idx.cuda(), capacity_arcs=2 * len(edges) + 8)
    ins = [(2 * L, 2 * L + 9)]
    dg.update(insert=ins)
    check(pico, dg, n, edges | set(ins))
    assert dg.coreness().cpu().tolist() == [2] * n
    st = pico.pico_get_stats()
    assert st["algo"] == pico.PICO_STATS_MAINTENANCE and st["frontier"] == 10
    assert st["active"] <= 10, st["active"]


def test_consecutive_insertion_batches(pico):
    # Pure insertion batches reuse the neighbour counts the previous passes
    # left (counted once at creation, then kept exact); a deletion batch
    # invalidates them and the next insertion batch counts them again.
    rng = np.random.default_rng(74)
    g = gg.rmat_graph(13, 8, 75)
    n = g.n
    edges = edges_of(g)
    dg = pico.DynamicGraph(g.row_ptr.cuda(), g.col_idx.cuda(), capacity_arcs=2 * g.arcs)
    for k_ins, k_del in [(300, 0), (1, 0), (800, 0), (0, 400), (300, 0), (200, 0), (100, 100),
                         (400, 0)]:
        ins, dele = random_batch(rng, n, edges, k_ins, k_del)
        dg.update(insert=ins, delete=dele)
        edges = (edges - set(dele)) | set(ins)
        check(pico, dg, n, edges)


def test_starting_from_no_edges(pico):
    # An edgeless graph: the neighbour counts start over zero arcs, then a
    # triangle and a pendant edge arrive in two insertion batches.
    n = 6
    g = gg.from_edge_list([], n)
    dg = pico.DynamicGraph(g.row_ptr.cuda(), g.col_idx.cuda(), capacity_arcs=32)
    assert (dg.coreness().cpu() == 0).all()
    dg.update(insert=[(0, 1), (1, 2)])
    check(pico, dg, n, {(0, 1), (1, 2)})
    dg.update(insert=[(0, 2), (2, 3)])
    check(pico, dg, n, {(0, 1), (1, 2), (0, 2), (2, 3)})
    assert dg.coreness().cpu().tolist() == [2, 2, 2, 1, 0, 0]


@pytest.mark.parametrize("policy", ("recompute", "auto"))
def test_recomputation_fallback(pico, policy):
    """The fallback recomputes the coreness from scratch instead of
    maintaining it; every batch must still give the oracle's coreness and
    the exact edge set, and the next insertion batch after a recomputation
    (whose insertion passes must recount their neighbour counts) too."""
    rng = np.random.default_rng(61)
    g = gg.rmat_graph(12, 8, 62)
    n = g.n
    edges = edges_of(g)
    dg = pico.DynamicGraph(g.row_ptr.cuda(), g.col_idx.cuda(), capacity_arcs=2 * len(edges) + 20000)
    pol = {"recompute": pico.PICO_DYN_RECOMPUTE, "auto": pico.PICO_DYN_AUTO}[policy]
    kinds = []
    assert dg.last_update_times == (-1.0, -1.0)
    for step, (ki, kd) in enumerate([(300, 0), (0, 300), (400, 400), (200, 0), (2000, 2000)]):
        dg.set_policy(pol if step != 3 else pico.PICO_DYN_MAINTAIN)
        ins, dele = random_batch(rng, n, edges, ki, kd)
        dg.update(insert=ins, delete=dele)
        edges = (edges - set(dele)) | set(ins)
        check(pico, dg, n, edges)
        kinds.append(dg.last_update_kind)
        rebuild_ms, step_ms = dg.last_update_times   # both phases were timed
        assert rebuild_ms > 0 and step_ms > 0
    assert kinds[3] == pico.PICO_DYN_MAINTAINED   # insertion passes right after a recompute
    if policy == "recompute":
        assert kinds[:3] == [pico.PICO_DYN_RECOMPUTED] * 3 and kinds[4] == pico.PICO_DYN_RECOMPUTED
    else:   # the first batch of each kind is maintained: its cost is not known yet,
        # and so is the last, 5x larger than any earlier one
        assert kinds[0] == pico.PICO_DYN_MAINTAINED and kinds[1] == pico.PICO_DYN_MAINTAINED
        assert kinds[4] == pico.PICO_DYN_MAINTAINED


def test_hub_row_longer_than_two_pieces(pico):
    """A hub of degree 10,300 (its row spans three 4,096-arc pieces of the
    CSR rebuild, and many 1,024-arc steps of a piece) loses arcs spread over
    all of its row and gains new ones in the same batches; the coreness and
    the rebuilt arc set must match the oracle after every batch."""
    rng = np.random.default_rng(63)
    leaves = 10300
    n = leaves + 1 + 300
    edges = {(0, v) for v in range(1, leaves + 1)}
    for _ in range(3000):   # a denser part among the leaves and some outside vertices
        a, b = (int(x) for x in rng.integers(1, n, size=2))
        if a != b:
            edges.add((min(a, b), max(a, b)))
    g = gg.from_edge_list(sorted(edges), n)
    dg = pico.DynamicGraph(g.row_ptr.cuda(), g.col_idx.cuda(), capacity_arcs=2 * len(edges) + 40000)
    dg.set_policy(pico.PICO_DYN_MAINTAIN)
    check(pico, dg, n, edges)
    for step in range(3):
        hub = sorted(e for e in edges if e[0] == 0)
        dele = sorted(set(hub[step::37][:300] + hub[-(5 + step):]))   # the whole row and its end
        ins = set()
        while len(ins) < 400:
            a, b = (int(x) for x in rng.integers(0, n, size=2))
            e = (min(a, b), max(a, b))
            if a != b and e not in edges and e not in ins:
                ins.add(e)
        dg.update(insert=sorted(ins), delete=dele)
        edges = (edges - set(dele)) | ins
        check(pico, dg, n, edges)
