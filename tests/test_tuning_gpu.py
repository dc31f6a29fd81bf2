"""Tuning changes the speed only: every candidate setting gives the oracle's
coreness, for single graphs and batches; the autotuner applies and caches."""
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
    yield p
    p.pico_set_tuning(32, 256, 512, 21)


def test_every_candidate_gives_the_same_coreness(pico):
    from paper_2402_15253_gb300 import autotune as at
    g = gg.rmat_graph(15, 16, 41)
    want = oracle.bz_coreness(*g.numpy())
    pb = gg.pack_graphs([gg.spec_graph(s) for s in gg.batch_specs(12, 42, nmin=50, nmax=20000)])
    bwant = oracle.bz_coreness_batched(pb.vtx_off, pb.arc_off, pb.row_ptr, pb.col_idx)
    rp, ci = g.row_ptr.cuda(), g.col_idx.cuda()
    d = [t.cuda() for t in (pb.vtx_off, pb.arc_off, pb.row_ptr, pb.col_idx)]
    for cand in at.candidates(True) + [(64, 128, 256, 12), (32, 1024, 512, 14)]:
        assert pico.pico_set_tuning(*cand) == 0
        assert pico.pico_get_tuning() == cand
        for algo in ("peelone", "histocore"):
            got = pico.coreness(rp, ci, algo).cpu().numpy()
            assert np.array_equal(got, want), (cand, algo)
            bgot = pico.coreness_batched(*d, algo).cpu().numpy()
            assert np.array_equal(bgot, bwant), (cand, algo)
    assert pico.pico_set_tuning(16, 256, 512, 21) == pico.PICO_ERR_INVALID_ARG
    assert pico.pico_set_tuning(32, 256, 384, 21) == pico.PICO_ERR_INVALID_ARG
    assert pico.pico_set_tuning(32, 256, 512, 70) == pico.PICO_ERR_INVALID_ARG


def test_autotuner_applies_and_caches(pico, tmp_path):
    from paper_2402_15253_gb300 import autotune as at
    path = str(tmp_path / "tuning.json")
    pb = gg.pack_graphs([gg.spec_graph(s) for s in gg.batch_specs(32, 43, nmin=100, nmax=30000)],
                        device="cuda")
    cands = [(32, 256, 512, 21), (64, 128, 256, 62), (128, 1024, 512, 12)]
    best, timings = at.tune_batched(pico, pb.vtx_off, pb.arc_off, pb.row_ptr, pb.col_idx,
                                    "peelone", cands=cands, reps=2, path=path)
    assert best in cands and set(timings) == set(cands)
    assert pico.pico_get_tuning() == best
    pico.pico_set_tuning(32, 256, 512, 21)
    tv, ta = int(pb.vtx_off[-1]), int(pb.arc_off[-1])
    assert at.apply_cached(pico, "peelone", "batched", tv, ta, pb.G, path=path) == best
    assert pico.pico_get_tuning() == best
    g = gg.rmat_graph(14, 16, 44).to("cuda")
    best1, _ = at.tune_single(pico, g.row_ptr, g.col_idx, "histocore",
                              cands=[(32, 256, 512, 21), (64, 1024, 512, 21)], reps=2, path=path)
    assert at.apply_cached(pico, "histocore", "single", g.n, g.arcs, path=path) == best1
