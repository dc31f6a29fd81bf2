"""GPU tests of the method selection per graph (PICO_ALGO_AUTO).

The selected method must return the oracle's coreness, and the choice must
follow the documented rule: HistoCore when d_max >= 64 m/n and
m^2 <= 2^14 d_max n, PeelOne otherwise (pico_get_stats reports the method
that ran). The batched form runs PeelOne for every graph.
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


def expected_method(rp):
    n, m = len(rp) - 1, int(rp[-1])
    dmax = int(np.diff(rp).max())
    histo = dmax * n >= 64 * m and float(m) * m <= 16384.0 * dmax * n
    return "histocore" if histo else "peelone"


CASES = [
    ("rmat14", lambda: gg.rmat_graph(14, 16, 51), "histocore"),
    ("rmat17-ef4", lambda: gg.rmat_graph(17, 4, 52), "histocore"),
    ("chunglu-2^15", lambda: gg.chung_lu_graph(1 << 15, 53, clique=300), "histocore"),
    ("er-50k-d16", lambda: gg.er_graph(50000, 400000, 54), "peelone"),
    ("grid-300x200", lambda: gg.grid_graph(300, 200), "peelone"),
    ("K400", lambda: gg.complete_graph(400), "peelone"),
    ("star-30k", lambda: gg.star_graph(30000), "histocore"),
]


@pytest.mark.parametrize("name,make,want_method", CASES, ids=[c[0] for c in CASES])
def test_auto_picks_by_rule_and_matches_oracle(pico, name, make, want_method):
    g = make()
    rp, ci = g.numpy()
    assert expected_method(rp) == want_method
    out = pico.coreness(g.row_ptr.cuda(), g.col_idx.cuda(), "auto")
    st = pico.pico_get_stats()
    assert st["algo"] == pico.ALGOS[want_method]
    assert np.array_equal(out.cpu().numpy(), oracle.bz_coreness(rp, ci))
    if want_method == "histocore":
        _, ost = oracle.histocore(rp, ci)
        assert st["rounds"] == ost["rounds"] and st["frontier"] == ost["frontier"]
    else:
        _, ost = oracle.peelone(rp, ci)
        assert st["levels"] == ost["levels"] and st["arcs"] == ost["arcs_scanned"]
        assert st["atomics"] - st["extra"] == ost["decrements"]


def test_auto_int64_offsets(pico):
    g = gg.rmat_graph(15, 16, 55)
    rp, ci = g.numpy()
    out = pico.coreness(g.row_ptr.cuda().to(torch.int64), g.col_idx.cuda(), "auto")
    assert np.array_equal(out.cpu().numpy(), oracle.bz_coreness(rp, ci))
    assert pico.pico_get_stats()["algo"] == pico.ALGOS[expected_method(rp)]


def test_auto_batched_runs_peelone(pico):
    pb = gg.pack_graphs([gg.spec_graph(s) for s in gg.batch_specs(24, 56, nmin=50, nmax=20000)])
    d = [t.cuda() for t in (pb.vtx_off, pb.arc_off, pb.row_ptr, pb.col_idx)]
    out = pico.coreness_batched(*d, "auto")
    assert pico.pico_get_stats()["algo"] == pico.PICO_ALGO_PEELONE
    want = oracle.bz_coreness_batched(pb.vtx_off, pb.arc_off, pb.row_ptr, pb.col_idx)
    assert np.array_equal(out.cpu().numpy(), want)
