"""The entry point that allocates no device memory (pico_coreness_noalloc).

Some callers cannot allocate device memory while they run (a service that
reserved its whole budget at start-up, a framework that owns every
allocation); this entry point serves them from a scratch array compiled into
the library. The test calls it through the C ABI twice in a row, on two
different graphs, and checks each result against the regular entry point
(pico_coreness with PeelOne) bit for bit. The file is named so that pytest
collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_15253_gb300 as pico
    torch.cuda.set_device(0)
    return pico, pico.load()


def _regular(pico, g):
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    rc = pico.pico_coreness(g.row_ptr, g.col_idx, g.n, g.arcs, out, pico.PICO_ALGO_PEELONE)
    assert rc == pico.PICO_OK
    assert pico.pico_last_device_status() == pico.PICO_OK
    return out.cpu().numpy()


def test_noalloc_matches_regular_entry_point_twice(lib):
    pico, L = lib
    graphs = [gg.rmat_graph(16, 16, 101).to("cuda"), gg.rmat_graph(15, 24, 102).to("cuda")]
    status = torch.full((1,), -99, dtype=torch.int32, device="cuda")
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    stream = vp(torch.cuda.current_stream().cuda_stream)
    for g in graphs:
        assert g.n <= pico.PICO_NOALLOC_MAX_VERTICES and g.arcs <= pico.PICO_NOALLOC_MAX_ARCS
        want = _regular(pico, g)
        out = torch.full((g.n,), -1, dtype=torch.int32, device="cuda")
        rc = L.pico_coreness_noalloc(vp(g.row_ptr.data_ptr()), vp(g.col_idx.data_ptr()),
                                     i64(g.n), i64(g.arcs), vp(out.data_ptr()),
                                     vp(status.data_ptr()), stream)
        assert rc == pico.PICO_OK
        torch.cuda.synchronize()
        assert int(status.item()) == pico.PICO_OK
        got = out.cpu().numpy()
        assert np.array_equal(got, want), f"{int((got != want).sum())} vertices differ"


def test_noalloc_rejects_graphs_beyond_its_limits(lib):
    pico, L = lib
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    big_n = pico.PICO_NOALLOC_MAX_VERTICES + 1
    big_m = pico.PICO_NOALLOC_MAX_ARCS + 2
    assert L.pico_coreness_noalloc(vp(8), vp(8), i64(big_n), i64(4), vp(8), vp(None),
                                   vp(None)) == pico.PICO_ERR_INVALID_ARG
    assert L.pico_coreness_noalloc(vp(8), vp(8), i64(16), i64(big_m), vp(8), vp(None),
                                   vp(None)) == pico.PICO_ERR_INVALID_ARG
