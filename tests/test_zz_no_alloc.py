"""The entry point that allocates no device memory (pico_coreness_noalloc).

Some callers cannot allocate device memory while they run (a service that
reserved its whole budget at start-up, a framework that owns every
allocation); this entry point serves them from a scratch array compiled into
the library. The test calls it through the C ABI twice in a row, on two
different graphs, and checks each result bit for bit against the regular
entry point (pico_coreness with PeelOne) and against the CPU oracle. A child
process with every scratch allocation failing (PICO_FAULT_ALLOC=1) shows the
property itself: there the regular entry point reports PICO_ERR_OOM while
this one still returns the oracle's result. The file is named so that pytest
collects it last.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle

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
        truth = oracle.bz_coreness(g.row_ptr.cpu().numpy(), g.col_idx.cpu().numpy())
        assert np.array_equal(got, truth), f"{int((got != truth).sum())} vertices differ"


_CHILD = r"""
import ctypes, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import graphgen as gg
import oracle
import paper_2402_15253_gb300 as pico
torch.cuda.set_device(0)
L = pico.load()
g = gg.rmat_graph(14, 16, 103).to("cuda")
out = torch.full((g.n,), -1, dtype=torch.int32, device="cuda")
rc_regular = pico.pico_coreness(g.row_ptr, g.col_idx, g.n, g.arcs, out, pico.PICO_ALGO_PEELONE)
status = torch.full((1,), -99, dtype=torch.int32, device="cuda")
vp, i64 = ctypes.c_void_p, ctypes.c_int64
rc = L.pico_coreness_noalloc(vp(g.row_ptr.data_ptr()), vp(g.col_idx.data_ptr()), i64(g.n),
                             i64(g.arcs), vp(out.data_ptr()), vp(status.data_ptr()),
                             vp(torch.cuda.current_stream().cuda_stream))
torch.cuda.synchronize()
want = oracle.bz_coreness(g.row_ptr.cpu().numpy(), g.col_idx.cpu().numpy())
same = bool(np.array_equal(out.cpu().numpy(), want))
print("RESULT", rc_regular, rc, int(status.item()), int(same))
"""


def test_noalloc_works_where_allocation_fails(lib):
    pico, _ = lib
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PICO_FAULT_ALLOC="1")
    r = subprocess.run([sys.executable, "-c", _CHILD, root], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT")][-1]
    rc_regular, rc, status, same = (int(x) for x in line.split()[1:])
    assert rc_regular == pico.PICO_ERR_OOM
    assert rc == pico.PICO_OK and status == pico.PICO_OK
    assert same == 1


def test_noalloc_rejects_graphs_beyond_its_limits(lib):
    pico, L = lib
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    big_n = pico.PICO_NOALLOC_MAX_VERTICES + 1
    big_m = pico.PICO_NOALLOC_MAX_ARCS + 2
    assert L.pico_coreness_noalloc(vp(8), vp(8), i64(big_n), i64(4), vp(8), vp(None),
                                   vp(None)) == pico.PICO_ERR_INVALID_ARG
    assert L.pico_coreness_noalloc(vp(8), vp(8), i64(16), i64(big_m), vp(8), vp(None),
                                   vp(None)) == pico.PICO_ERR_INVALID_ARG
