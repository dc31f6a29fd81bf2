"""Failure detection without a GPU fault.

* A bounded device-side wait is made to run out (a grid barrier that one CTA
  never reaches): the launch must end by itself with PICO_ERR_TIMEOUT in the
  status word, and the context must stay usable.
* Host-side fault injection (PICO_FAULT_ALLOC=1) makes scratch allocation
  fail: every compute entry point must return PICO_ERR_OOM, and the server
  must report it from drain().
"""
import json
import os
import subprocess
import sys
import time

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from conftest import ROOT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pico():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_15253_gb300 as p
    torch.cuda.set_device(0)
    return p


def test_bounded_wait_times_out_and_context_survives(pico):
    t0 = time.time()
    st = pico.pico_selftest_wait_timeout(300)
    dt = time.time() - t0
    assert st == pico.PICO_ERR_TIMEOUT
    assert dt < 10.0
    assert pico.pico_last_device_status() == pico.PICO_OK   # cleared
    g = gg.rmat_graph(12, 16, 5)
    want = oracle.bz_coreness(*g.numpy())
    for algo in ("peelone", "histocore"):
        got = pico.coreness(g.row_ptr.cuda(), g.col_idx.cuda(), algo).cpu().numpy()
        assert np.array_equal(got, want)


SCRIPT = r"""
import json, sys, torch
sys.path.insert(0, %r)
import graphgen as gg
import paper_2402_15253_gb300 as pico
torch.cuda.set_device(0)
g = gg.rmat_graph(10, 8, 3).to("cuda")
out = torch.empty(g.n, dtype=torch.int32, device="cuda")
res = {"single": [pico.pico_coreness(g.row_ptr, g.col_idx, g.n, g.arcs, out, a) for a in (0, 1)]}
pb = gg.pack_graphs([gg.rmat_graph(8, 8, 4), gg.rmat_graph(9, 8, 5)], device="cuda")
tv, ta = int(pb.vtx_off[-1]), int(pb.arc_off[-1])
bout = torch.empty(tv, dtype=torch.int32, device="cuda")
res["batched"] = pico.pico_coreness_batched(pb.vtx_off, pb.arc_off, pb.G, pb.row_ptr, pb.col_idx,
                                            tv, ta, bout, 0)
srv = pico.pico_server_create(1 << 30, 0, 2, 8, 0)
h = gg.rmat_graph(8, 8, 6)
rp, ci = h.row_ptr.pin_memory(), h.col_idx.pin_memory()
o = torch.zeros(h.n, dtype=torch.int32).pin_memory()
res["submit"] = pico.pico_server_submit(srv, rp, ci, h.n, h.arcs, o, 0)
res["drain"] = pico.pico_server_drain(srv)
res["destroy"] = pico.pico_server_destroy(srv)
print(json.dumps(res))
"""


def test_allocation_fault_injection(pico):
    env = dict(os.environ, PICO_FAULT_ALLOC="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT % ROOT], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["single"] == [pico.PICO_ERR_OOM, pico.PICO_ERR_OOM]
    assert res["batched"] == pico.PICO_ERR_OOM
    assert res["submit"] >= 0
    assert res["drain"] == pico.PICO_ERR_OOM and res["destroy"] == pico.PICO_ERR_OOM
