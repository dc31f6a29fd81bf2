"""GPU parity of the comparison baselines of Sec. V (PICO_ALGO_GPP,
PEEL_CAS, PEEL_ADDBACK, NBRCORE, CNTCORE) against the oracle.

Every baseline returns the definition's coreness, and its iteration
structure equals the oracle's rendition of the same algorithm: GPP's steps,
scans and decrements (Alg. 3); the PeelOne variants' levels and
successful decrements (Alg. 4, whatever the clamp); NbrCore's and CntCore's
rounds, active sets, frontiers and scanned arcs.
"""
import itertools

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from conftest import load_g1

pytestmark = pytest.mark.gpu

BASELINES = ("gpp", "peel_cas", "peel_addback", "nbrcore", "cntcore")


@pytest.fixture(scope="module")
def pico():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_15253_gb300 as p
    torch.cuda.set_device(0)
    return p


def run(pico, g, algo, off_dtype=None):
    rp = g.row_ptr.cuda()
    if off_dtype is not None:
        rp = rp.to(off_dtype)
    out = pico.coreness(rp, g.col_idx.cuda(), algo)
    st = pico.pico_get_stats()
    if g.arcs:   # a graph without arcs launches nothing
        assert st["algo"] == pico.METHODS[algo]
    return out.cpu().numpy(), st


def check_stats(algo, rp, ci, st):
    if algo == "gpp":
        _, o = oracle.gpp(rp, ci)
        assert (st["subrounds"], st["scans"]) == (o["steps"], o["scans"])
        assert st["atomics"] == o["decrements"] and st["arcs"] == o["arcs_scanned"]
        assert st["kmax"] == o["kmax"]
    elif algo in ("peel_cas", "peel_addback"):
        _, o = oracle.peelone(rp, ci)
        assert (st["levels"], st["kmax"]) == (o["levels"], o["kmax"])
        assert st["arcs"] == o["arcs_scanned"]
        assert st["atomics"] - st["extra"] == o["decrements"]
    else:
        _, o = (oracle.nbrcore if algo == "nbrcore" else oracle.cntcore)(rp, ci)
        assert st["rounds"] == o["rounds"] and st["active"] == o["active"]
        assert st["frontier"] == o["frontier"] and st["arcs"] == o["arcs_scanned"]


@pytest.mark.parametrize("algo", BASELINES)
def test_every_small_graph(pico, algo):
    for n in range(1, 6):
        pairs = list(itertools.combinations(range(n), 2))
        for mask in range(1 << len(pairs)):
            edges = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
            g = gg.from_edge_list(edges, n)
            got, _ = run(pico, g, algo)
            assert got.tolist() == oracle.brute_force_coreness(n, edges), (algo, n, edges)


@pytest.mark.parametrize("algo", BASELINES)
def test_g1_and_closed_forms(pico, algo):
    n, edges, want = load_g1()
    got, _ = run(pico, gg.from_edge_list(edges, n), algo)
    assert got.tolist() == want
    for g, k in [(gg.complete_graph(300), 299), (gg.cycle_graph(1001), 2),
                 (gg.star_graph(5000), 1), (gg.grid_graph(70, 90), 2), (gg.hypercube(10), 10),
                 (gg.path_graph(777), 1), (gg.complete_bipartite(9, 400), 9)]:
        got, st = run(pico, g, algo)
        assert (got == k).all(), (algo, g.name)
        check_stats(algo, *g.numpy(), st)


FAMILIES = [
    ("rmat14", lambda: gg.rmat_graph(14, 16, 41)),
    ("er-30k", lambda: gg.er_graph(30001, 240007, 42)),
    ("chunglu-2^15", lambda: gg.chung_lu_graph(1 << 15, 43, clique=200)),
    ("grid-150x211", lambda: gg.grid_graph(150, 211)),
]


@pytest.mark.parametrize("algo", BASELINES)
@pytest.mark.parametrize("name,make", FAMILIES, ids=[f[0] for f in FAMILIES])
def test_families_match_oracle(pico, algo, name, make):
    g = make()
    rp, ci = g.numpy()
    got, st = run(pico, g, algo)
    assert np.array_equal(got, oracle.bz_coreness(rp, ci)), (algo, name)
    check_stats(algo, rp, ci, st)


@pytest.mark.parametrize("algo", BASELINES)
def test_int64_offsets_and_isolated(pico, algo):
    g = gg.rmat_graph(13, 16, 44)   # R-MAT leaves isolated vertices
    rp, ci = g.numpy()
    assert (np.diff(rp) == 0).any()
    got, _ = run(pico, g, algo, off_dtype=torch.int64)
    assert np.array_equal(got, oracle.bz_coreness(rp, ci))
    # no arcs at all, and no vertices
    got = pico.coreness(torch.zeros(6, dtype=torch.int32, device="cuda"),
                        torch.zeros(0, dtype=torch.int32, device="cuda"), algo)
    assert got.numel() == 5 and (got.cpu() == 0).all()
    empty = pico.coreness(torch.zeros(1, dtype=torch.int32, device="cuda"),
                          torch.zeros(0, dtype=torch.int32, device="cuda"), algo)
    assert empty.numel() == 0


@pytest.mark.parametrize("algo", BASELINES)
def test_rmat18_matches_peelone(pico, algo):
    """R-MAT scale 18 (about 8 M arcs): the same coreness as PeelOne, checked
    against the oracle."""
    g = gg.rmat_graph(18, 16, 45)
    want = oracle.bz_coreness(*g.numpy())
    got, _ = run(pico, g, algo)
    assert np.array_equal(got, want)


def test_batched_form_rejects_baselines(pico):
    pb = gg.pack_graphs([gg.complete_graph(5)])
    d = [t.cuda() for t in (pb.vtx_off, pb.arc_off, pb.row_ptr, pb.col_idx)]
    out = torch.empty(5, dtype=torch.int32, device="cuda")
    for a in pico.BASELINES.values():
        assert pico.pico_coreness_batched(d[0], d[1], 1, d[2], d[3], 5, int(pb.arc_off[-1]), out,
                                          a, None) == pico.PICO_ERR_INVALID_ARG
