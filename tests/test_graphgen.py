"""The seeded input generators: determinism and structure (no GPU needed)."""
import numpy as np
import torch

import graphgen as gg


def _np_splitmix(seed, stream, count):
    key = np.uint64(gg.stream_key(seed, stream) & ((1 << 64) - 1))
    with np.errstate(over="ignore"):
        z = (np.arange(count, dtype=np.uint64) + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15) + key
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def test_draws_match_uint64_rendition():
    for seed, stream in [(0, 0), (5, 7), (2 ** 40 + 3, gg.S_RMAT + 9)]:
        t = gg.draw_bits(seed, stream, torch.arange(4096, dtype=torch.int64)).numpy().view(np.uint64)
        assert (t == _np_splitmix(seed, stream, 4096)).all()
        assert gg.draw_bits_int(seed, stream, 17) == int(t[17])


def test_draw_below_range_and_spread():
    x = gg.draw_below(3, 1, torch.arange(100000, dtype=torch.int64), 1000)
    assert int(x.min()) == 0 and int(x.max()) == 999
    counts = np.bincount(x.numpy(), minlength=1000)
    assert counts.min() > 50 and counts.max() < 160


def _assert_simple_symmetric(g):
    rp, ci = g.numpy()
    n = g.n
    assert rp[0] == 0 and (np.diff(rp) >= 0).all()
    src = np.repeat(np.arange(n), np.diff(rp))
    assert (src != ci).all(), "self-loop"
    assert (ci >= 0).all() and (ci < n).all()
    for v in range(0, n, max(1, n // 200)):
        row = ci[rp[v]:rp[v + 1]]
        assert (np.diff(row) > 0).all(), "unsorted or duplicate neighbours"
    fwd = set(zip(src.tolist(), ci.tolist()))
    assert all((b, a) in fwd for a, b in list(fwd)[:20000])


def test_rmat_is_deterministic_and_simple():
    a = gg.rmat_graph(12, 16, 99)
    b = gg.rmat_graph(12, 16, 99, chunk=5000)      # chunking must not matter
    assert torch.equal(a.row_ptr, b.row_ptr) and torch.equal(a.col_idx, b.col_idx)
    c = gg.rmat_graph(12, 16, 100)
    assert not torch.equal(a.col_idx[:1000], c.col_idx[:1000])
    _assert_simple_symmetric(a)
    # R-MAT with a = .57 favours low ids: vertex 0 is a hub
    deg = np.diff(a.numpy()[0])
    assert deg[0] == deg.max()


def test_structured_families():
    g = gg.grid_graph(30, 40)
    assert g.arcs == 2 * (30 * 39 + 29 * 40)
    _assert_simple_symmetric(g)
    assert gg.complete_graph(9).arcs == 72
    assert gg.hypercube(6).arcs == 6 * 64
    _assert_simple_symmetric(gg.er_graph(3000, 20000, 4))
    cl = gg.chung_lu_graph(1 << 12, 5, clique=50, pairs_per_vertex=4)
    _assert_simple_symmetric(cl)
    m = gg.clique_members(1 << 12, 5, 50).numpy()
    rp, ci = cl.numpy()
    for v in m[:10]:
        assert set(m) - {v} <= set(ci[rp[v]:rp[v + 1]].tolist())


def test_int64_offsets():
    g = gg.rmat_graph(10, 8, 3, off_dtype=torch.int64)
    assert g.row_ptr.dtype == torch.int64
    h = gg.rmat_graph(10, 8, 3)
    assert torch.equal(g.row_ptr.to(torch.int32), h.row_ptr)


def test_batch_specs_and_packing():
    specs = gg.batch_specs(64, 11)
    ns = np.array([s.n for s in specs])
    assert ns.min() >= 100 and ns.max() <= 200000
    assert all(s.kind == ("er" if i % 2 == 0 else "rmat") for i, s in enumerate(specs))
    assert all(4 <= s.param <= 64 for s in specs if s.kind == "er")
    assert all(8 <= s.param <= 32 and s.param == int(s.param) for s in specs if s.kind == "rmat")
    assert specs == gg.batch_specs(64, 11)
    small = gg.batch_specs(6, 11, nmin=50, nmax=400)
    pb = gg.pack_graphs([gg.spec_graph(s) for s in small])
    assert pb.vtx_off.dtype == torch.int64 and pb.arc_off.dtype == torch.int64
    assert pb.row_ptr.numel() == int(pb.vtx_off[-1]) + pb.G
    for i, s in enumerate(small):
        g = pb.graph(i)
        ref = gg.spec_graph(s)
        assert g.n == s.n
        assert torch.equal(g.row_ptr.to(torch.int64), ref.row_ptr.to(torch.int64))
        assert torch.equal(g.col_idx, ref.col_idx)
        _assert_simple_symmetric(g)
