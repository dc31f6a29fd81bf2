"""GPU parity of the batched form (pico_coreness_batched) against the oracle.

Each graph of a packed batch must get exactly the coreness the oracle gives
it alone, and the same result as a single-graph call.
"""
import itertools

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

ALGOS = ("peelone", "histocore")


@pytest.fixture(scope="module")
def pico():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_15253_gb300 as p
    torch.cuda.set_device(0)
    return p


def run_batch(pico, pb, algo):
    out = pico.coreness_batched(pb.vtx_off.cuda(), pb.arc_off.cuda(), pb.row_ptr.cuda(),
                                pb.col_idx.cuda(), algo)
    return out.cpu().numpy()


def oracle_batch(pb):
    return oracle.bz_coreness_batched(pb.vtx_off.cpu(), pb.arc_off.cpu(), pb.row_ptr.cpu(),
                                      pb.col_idx.cpu())


@pytest.mark.parametrize("algo", ALGOS)
def test_every_small_graph_as_one_batch(pico, algo):
    graphs, want = [gg.from_edge_list([], 0)], []
    for n in range(1, 6):
        pairs = list(itertools.combinations(range(n), 2))
        for mask in range(1 << len(pairs)):
            edges = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
            graphs.append(gg.from_edge_list(edges, n))
            want.extend(oracle.brute_force_coreness(n, edges))
    graphs.append(gg.from_edge_list([], 7))
    want.extend([0] * 7)
    pb = gg.pack_graphs(graphs)
    got = run_batch(pico, pb, algo)
    assert np.array_equal(got, np.array(want, dtype=np.int32))


@pytest.mark.parametrize("algo", ALGOS)
def test_closed_forms_as_one_batch(pico, algo):
    parts = [(gg.complete_graph(64), 63), (gg.cycle_graph(999), 2), (gg.star_graph(70000), 1),
             (gg.grid_graph(200, 150), 2), (gg.complete_graph(2100), 2099),
             (gg.hypercube(9), 9), (gg.path_graph(3000), 1), (gg.complete_bipartite(7, 300), 7)]
    pb = gg.pack_graphs([g for g, _ in parts])
    got = run_batch(pico, pb, algo)
    want = np.concatenate([np.full(g.n, k, dtype=np.int32) for g, k in parts])
    assert np.array_equal(got, want)


@pytest.mark.parametrize("algo", ALGOS)
def test_mixed_batch_matches_oracle_and_single_calls(pico, algo):
    specs = gg.batch_specs(48, 77, nmin=30, nmax=30000)
    graphs = [gg.spec_graph(s) for s in specs]
    graphs.insert(5, gg.from_edge_list([], 0))          # an empty graph inside the batch
    graphs.insert(9, gg.from_edge_list([], 13))         # isolated vertices only
    pb = gg.pack_graphs(graphs)
    got = run_batch(pico, pb, algo)
    want = oracle_batch(pb)
    assert np.array_equal(got, want)
    vo = pb.vtx_off.numpy()
    for i in (0, 7, 20, len(graphs) - 1):
        g = graphs[i]
        if g.n == 0:
            continue
        single = pico.coreness(g.row_ptr.cuda(), g.col_idx.cuda(), algo).cpu().numpy()
        assert np.array_equal(single, got[vo[i]:vo[i + 1]])


@pytest.mark.parametrize("algo", ALGOS)
def test_batch_on_side_stream(pico, algo):
    pb = gg.pack_graphs([gg.spec_graph(s) for s in gg.batch_specs(16, 78, nmin=100, nmax=5000)])
    want = oracle_batch(pb)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        d = [t.cuda() for t in (pb.vtx_off, pb.arc_off, pb.row_ptr, pb.col_idx)]
        out = pico.coreness_batched(*d, algo, total_vertices=int(pb.vtx_off[-1]),
                                    total_arcs=int(pb.arc_off[-1]), check=False)
    assert pico.pico_last_device_status(s) == 0
    assert np.array_equal(out.cpu().numpy(), want)


def _oracle_every_graph(pb):
    """The oracle's coreness of every graph of a packed batch, one BZ run per
    graph on host threads (the C oracle releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    vo = pb.vtx_off.cpu().numpy()
    ao = pb.arc_off.cpu().numpy()
    rp = pb.row_ptr.cpu().numpy()
    ci = pb.col_idx.cpu().numpy()
    want = np.empty(int(vo[-1]), dtype=np.int32)
    oracle.lib()

    def one(g):
        want[vo[g]:vo[g + 1]] = oracle.bz_coreness(rp[vo[g] + g: vo[g + 1] + g + 1],
                                                   ci[ao[g]:ao[g + 1]])

    order = np.argsort(ao[1:] - ao[:-1])[::-1]        # largest graphs first
    with ThreadPoolExecutor(max_workers=16) as ex:
        list(ex.map(one, order.tolist()))
    return want


def test_full_size_batch(pico):
    """4,096 graphs with log-uniform vertex counts 100..200,000 (half ER, half
    R-MAT; 3.5 G arcs), both methods: every vertex of every graph is compared
    with the oracle run on that graph alone."""
    pb = gg.batch_graph(4096, gg.SEED_BASE + 4, device="cuda")
    got = {}
    for a in ALGOS:
        got[a] = pico.coreness_batched(pb.vtx_off, pb.arc_off, pb.row_ptr, pb.col_idx,
                                       a).cpu().numpy()
    want = _oracle_every_graph(pb)
    vo = pb.vtx_off.cpu().numpy()
    for a in ALGOS:
        bad = np.nonzero(got[a] != want)[0]
        if len(bad):
            g = int(np.searchsorted(vo, bad[0], side="right") - 1)
            raise AssertionError(f"{a}: {len(bad)} vertices differ, first in graph {g}")


@pytest.mark.parametrize("algo", ALGOS)
def test_large_graphs_solved_by_clusters(pico, algo):
    """Graphs with at least 2^21 arcs are solved by a thread-block cluster;
    mixed with small ones, every result must still be the oracle's."""
    graphs = [gg.rmat_graph(17, 16, 61),          # ~3.8 M arcs
              gg.complete_graph(1600),            # 2.56 M arcs, HistoCore CTA walks
              gg.spec_graph(gg.batch_specs(1, 62)[0]),
              gg.grid_graph(800, 800),            # 2.56 M arcs, long peel
              gg.rmat_graph(12, 8, 63)]
    assert sum(g.arcs >= (1 << 21) for g in graphs) == 3
    pb = gg.pack_graphs(graphs)
    got = run_batch(pico, pb, algo)
    assert np.array_equal(got, oracle_batch(pb))


def test_batch_with_pulled_updates(pico):
    """HistoCore with every UpdateHisto pulled, on a batch of small graphs
    (one CTA each) and large ones (one cluster each): same results."""
    graphs = [gg.rmat_graph(17, 16, 64), gg.grid_graph(300, 200)]
    graphs += [gg.spec_graph(s) for s in gg.batch_specs(40, 65, nmin=30, nmax=20000)]
    graphs.insert(7, gg.from_edge_list([], 0))
    pb = gg.pack_graphs(graphs)
    want = oracle_batch(pb)
    assert pico.pico_set_histo_update(pico.PICO_UPDATE_PULL, 25) == 0
    try:
        got = run_batch(pico, pb, "histocore")
        st = pico.pico_get_stats()
    finally:
        pico.pico_set_histo_update(pico.PICO_UPDATE_AUTO, pico.PULL_PCT_DEFAULT)
    assert np.array_equal(got, want)
    assert st["pull_rounds"] > 0 and st["pulled"] > 0
