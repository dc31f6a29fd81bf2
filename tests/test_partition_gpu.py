"""GPU parity of partitioned HistoCore (pico_coreness_partitioned and the
per-partition calls pico_part_*) against the oracle.

Splitting the vertices into ranges changes where the rows live, not the
rounds: each round is Alg. 6's synchronous round over all partitions, so the
coreness must equal the oracle's bit for bit and the round count must equal
that of the oracle's sequential rendition of Alg. 6.
"""
import itertools

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from conftest import load_g1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pico():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_15253_gb300 as p
    torch.cuda.set_device(0)
    return p


def check(pico, g, parts):
    rp, ci = g.numpy()
    want = oracle.bz_coreness(rp, ci)
    _, ost = oracle.histocore(rp, ci)
    got, rounds = pico.coreness_partitioned(g.row_ptr.cuda(), g.col_idx.cuda(), parts)
    got = got.cpu().numpy()
    bad = np.nonzero(got != want)[0]
    assert len(bad) == 0, f"{len(bad)} vertices differ, first {bad[:5].tolist()}"
    assert rounds == ost["rounds"]


FAMILIES = [
    ("rmat14", lambda: gg.rmat_graph(14, 16, 71)),
    ("chunglu-2^15", lambda: gg.chung_lu_graph(1 << 15, 72, clique=200)),
    ("grid-150x211", lambda: gg.grid_graph(150, 211)),
    ("er-20k", lambda: gg.er_graph(20001, 160003, 73)),
    ("star-9000", lambda: gg.star_graph(9000)),   # a hub row split into chunks
]


@pytest.mark.parametrize("parts", (1, 2, 3, 4, 7))
@pytest.mark.parametrize("name,make", FAMILIES, ids=[f[0] for f in FAMILIES])
def test_families(pico, name, make, parts):
    check(pico, make(), parts)


@pytest.mark.parametrize("parts", (1, 2, 5))
def test_g1_small_graphs_and_closed_forms(pico, parts):
    n, edges, want = load_g1()
    got, rounds = pico.coreness_partitioned(gg.from_edge_list(edges, n).row_ptr.cuda(),
                                            gg.from_edge_list(edges, n).col_idx.cuda(), parts)
    assert got.cpu().tolist() == want and rounds == 1
    graphs, wants = [], []
    for k in range(1, 6):
        pairs = list(itertools.combinations(range(k), 2))
        for mask in range(1 << len(pairs)):
            es = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
            graphs.append(gg.from_edge_list(es, k))
            wants.extend(oracle.brute_force_coreness(k, es))
    u = gg.disjoint_union(graphs)
    got, _ = pico.coreness_partitioned(u.row_ptr.cuda(), u.col_idx.cuda(), parts)
    assert np.array_equal(got.cpu().numpy(), np.array(wants, dtype=np.int32))
    for g, k in [(gg.complete_graph(64), 63), (gg.cycle_graph(999), 2), (gg.path_graph(3000), 1),
                 (gg.hypercube(9), 9), (gg.complete_bipartite(7, 300), 7)]:
        got, _ = pico.coreness_partitioned(g.row_ptr.cuda(), g.col_idx.cuda(), parts)
        assert (got.cpu().numpy() == k).all()


def test_more_parts_than_vertices_and_isolated(pico):
    g = gg.from_edge_list([(0, 1), (1, 2), (0, 2)], 6)   # a triangle and 3 isolated vertices
    got, rounds = pico.coreness_partitioned(g.row_ptr.cuda(), g.col_idx.cuda(), 16)
    assert got.cpu().tolist() == [2, 2, 2, 0, 0, 0] and rounds == 0
    g = gg.from_edge_list([], 9)
    got, rounds = pico.coreness_partitioned(g.row_ptr.cuda(), g.col_idx.cuda(), 3)
    assert got.cpu().tolist() == [0] * 9 and rounds == 0


def test_per_partition_calls_with_explicit_exchange(pico):
    """Three Partition objects driven like three ranks: each round every one
    runs sum(), the records are concatenated (the all-gather) and every one
    runs apply()."""
    g = gg.rmat_graph(13, 16, 74)
    rp, ci = g.numpy()
    want = oracle.bz_coreness(rp, ci)
    _, ost = oracle.histocore(rp, ci)
    from paper_2402_15253_gb300.distributed import partition_bounds
    drp, dci = g.row_ptr.cuda().to(torch.int64), g.col_idx.cuda()
    ps = [pico.Partition(drp, dci, lo, hi) for lo, hi in partition_bounds(g.n, 3)]
    rounds = 0
    while True:
        outs = [p.sum() for p in ps]
        recs = torch.cat([r for r, _ in outs])
        if recs.numel() == 0:
            break
        ymin = min(y for _, y in outs)
        for p in ps:
            p.apply(recs, ymin)
        rounds += 1
    got = torch.cat([p.coreness() for p in ps]).cpu().numpy()
    for p in ps:
        p.close()
    assert np.array_equal(got, want)
    assert rounds == ost["rounds"]


def test_full_size_rmat22(pico):
    g = gg.workload("rmat22", device="cuda")
    rp, ci = g.numpy()
    want = oracle.bz_coreness(rp, ci)
    got, rounds = pico.coreness_partitioned(g.row_ptr, g.col_idx, 4)
    assert np.array_equal(got.cpu().numpy(), want)
    single = pico.coreness(g.row_ptr, g.col_idx, "histocore")
    assert rounds == pico.pico_get_stats()["rounds"]
    assert torch.equal(single, got)
