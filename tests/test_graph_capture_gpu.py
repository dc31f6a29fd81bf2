"""CUDA-graph capture and replay of the compute entry points.

The batched call (and the single-graph call) is recorded once into a CUDA
graph on a side stream, its output is cleared, and the graph is replayed
twice; every replay must give the oracle's coreness bit for bit. The
workspace comes from the stream-ordered allocator, which a capture records
as allocation nodes, so each replay runs on fresh scratch.
"""
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


def _capture(call, warm):
    """Runs `warm` once on a side stream, then captures `call` there."""
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        warm(s)
        s.synchronize()
        with torch.cuda.graph(graph, stream=s):
            rc = call(s)
    torch.cuda.synchronize()
    return graph, rc


@pytest.mark.parametrize("algo", ("peelone", "histocore"))
def test_batched_capture_replays_oracle_result(pico, algo):
    graphs = [gg.spec_graph(s) for s in gg.batch_specs(40, 91, nmin=50, nmax=40000)]
    graphs.insert(3, gg.from_edge_list([], 0))
    graphs.append(gg.rmat_graph(17, 16, 92))          # solved by a cluster
    graphs.append(gg.complete_graph(300))
    pb = gg.pack_graphs(graphs)
    want = oracle.bz_coreness_batched(pb.vtx_off, pb.arc_off, pb.row_ptr, pb.col_idx)
    G = len(graphs)
    tv, ta = int(pb.vtx_off[-1]), int(pb.arc_off[-1])
    d = [t.cuda() for t in (pb.vtx_off, pb.arc_off, pb.row_ptr, pb.col_idx)]
    out = torch.full((tv,), -1, dtype=torch.int32, device="cuda")
    a = pico.ALGOS[algo]

    def call(s):
        return pico.pico_coreness_batched(d[0], d[1], G, d[2], d[3], tv, ta, out, a, s)

    graph, rc = _capture(call, call)
    assert rc == pico.PICO_OK
    for _ in range(2):
        out.fill_(-1)
        graph.replay()
        torch.cuda.synchronize()
        assert pico.pico_last_device_status() == pico.PICO_OK
        got = out.cpu().numpy()
        assert np.array_equal(got, want), f"{int((got != want).sum())} vertices differ"


@pytest.mark.parametrize("algo", ("peelone", "histocore"))
def test_single_graph_capture_replays_oracle_result(pico, algo):
    g = gg.rmat_graph(15, 16, 93).to("cuda")
    want = oracle.bz_coreness(g.row_ptr.cpu().numpy(), g.col_idx.cpu().numpy())
    n, m = g.n, g.arcs   # read before the capture (the arc count is read from the device)
    out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    a = pico.ALGOS[algo]

    def call(s):
        return pico.pico_coreness(g.row_ptr, g.col_idx, n, m, out, a, s)

    graph, rc = _capture(call, call)
    assert rc == pico.PICO_OK
    for _ in range(2):
        out.fill_(-1)
        graph.replay()
        torch.cuda.synchronize()
        assert pico.pico_last_device_status() == pico.PICO_OK
        assert np.array_equal(out.cpu().numpy(), want)
