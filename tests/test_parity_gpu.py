"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle.

Coreness is a unique integer vector, so every comparison is exact (bit for
bit). The renditions of Alg. 4 and Alg. 6 in the oracle also fix the
iteration structure: the GPU's non-empty levels, arcs walked and successful
decrements (PeelOne) and rounds (HistoCore) must equal theirs. PeelOne
processes each level's dynamic frontier asynchronously, so the waves of the
sequential rendition are not a GPU quantity there: Thm. 1 and Cor. 1 make
the result independent of the order within a level. The per-wave form (every
wave ended by a grid barrier, switched on with PICO_PEEL_WAVES=1) must match
the waves too.
"""
import os
import subprocess
import sys

import itertools

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from conftest import load_g1

pytestmark = pytest.mark.gpu

ALGOS = ("peelone", "histocore")


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
    return out.cpu().numpy(), pico.pico_get_stats()


def assert_same(got, want, what):
    if not np.array_equal(got, want):
        bad = np.nonzero(got != want)[0]
        raise AssertionError(f"{what}: {len(bad)} vertices differ, first {bad[:8].tolist()} "
                             f"got {got[bad[:8]].tolist()} want {want[bad[:8]].tolist()}")


# --------------------------------------------------------------------------
# small exact cases
# --------------------------------------------------------------------------

@pytest.mark.parametrize("algo", ALGOS)
def test_g1(pico, algo):
    n, edges, want = load_g1()
    got, st = run(pico, gg.from_edge_list(edges, n), algo)
    assert got.tolist() == want
    if algo == "peelone":
        assert st["levels"] == 2 and st["kmax"] == 2
        # level 1 lowers v5 twice (v0, v1); level 2 lowers v3 and v5 once each
        assert st["arcs"] == 14 and st["atomics"] - st["extra"] == 4
    else:
        assert st["rounds"] == 1 and st["frontier"] == 2


@pytest.mark.parametrize("algo", ALGOS)
def test_every_graph_up_to_5_vertices(pico, algo):
    """All labelled graphs on 1..5 vertices, as one disjoint union."""
    parts, wants = [], []
    for n in range(1, 6):
        pairs = list(itertools.combinations(range(n), 2))
        for mask in range(1 << len(pairs)):
            edges = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
            parts.append(gg.from_edge_list(edges, n))
            wants.extend(oracle.brute_force_coreness(n, edges))
    u = gg.disjoint_union(parts)
    got, _ = run(pico, u, algo)
    assert_same(got, np.array(wants, dtype=np.int32), f"union of small graphs ({algo})")


CLOSED = [
    ("K2", lambda: gg.complete_graph(2), 1),
    ("K64", lambda: gg.complete_graph(64), 63),
    ("K2100", lambda: gg.complete_graph(2100), 2099),   # HistoCore CTA walk (K > 2048)
    ("C1000", lambda: gg.cycle_graph(1000), 2),
    ("P5000", lambda: gg.path_graph(5000), 1),           # ~2500 frontier waves
    ("star70000", lambda: gg.star_graph(70000), 1),      # hub split into 69 chunks
    ("grid300x200", lambda: gg.grid_graph(300, 200), 2),
    ("K40,3000", lambda: gg.complete_bipartite(40, 3000), 40),
    ("Q10", lambda: gg.hypercube(10), 10),
    ("tree20000", lambda: gg.random_tree(20000, 3), 1),
]


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("name,make,k", CLOSED, ids=[c[0] for c in CLOSED])
def test_closed_forms(pico, algo, name, make, k):
    g = make()
    got, _ = run(pico, g, algo)
    assert (got == k).all(), f"{name}: values {np.unique(got)[:10]}"


@pytest.mark.parametrize("algo", ALGOS)
def test_isolated_and_empty(pico, algo):
    g = gg.from_edge_list([], 1000)
    got, _ = run(pico, g, algo)
    assert (got == 0).all()
    g = gg.from_edge_list([(3, 7)], 10)
    got, _ = run(pico, g, algo)
    assert got.tolist() == [0, 0, 0, 1, 0, 0, 0, 1, 0, 0]
    import paper_2402_15253_gb300 as p
    rp = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = p.coreness(rp, torch.zeros(0, dtype=torch.int32, device="cuda"), algo)
    assert out.numel() == 0


@pytest.mark.parametrize("algo", ALGOS)
def test_random_small_graphs(pico, algo):
    rng = np.random.default_rng(5)
    parts, wants = [], []
    for t in range(200):
        n = int(rng.integers(2, 65))
        p = [0.03, 0.08, 0.15, 0.3, 0.6][t % 5]
        edges = [(u, v) for u in range(n) for v in range(u + 1, n) if rng.random() < p]
        parts.append(gg.from_edge_list(edges, n))
        wants.extend(oracle.brute_force_coreness(n, edges))
    got, _ = run(pico, gg.disjoint_union(parts), algo)
    assert_same(got, np.array(wants, dtype=np.int32), "random small graphs")


# --------------------------------------------------------------------------
# synthetic families, several tiles and ragged tails, against BZ and the
# iteration structure of the sequential renditions
# --------------------------------------------------------------------------

FAMILIES = [
    ("rmat16", lambda: gg.workload("rmat16")),
    ("rmat14-ef8", lambda: gg.rmat_graph(14, 8, 31)),
    ("er-50k", lambda: gg.er_graph(50001, 400003, 32)),
    ("chunglu-2^16", lambda: gg.chung_lu_graph(1 << 16, 33, clique=300)),
    ("grid-257x333", lambda: gg.grid_graph(257, 333)),
]


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("name,make", FAMILIES, ids=[f[0] for f in FAMILIES])
def test_families_match_oracle(pico, algo, name, make):
    g = make()
    rp, ci = g.numpy()
    want = oracle.bz_coreness(rp, ci)
    got, st = run(pico, g, algo)
    assert_same(got, want, f"{name} {algo}")
    if algo == "peelone":
        _, ost = oracle.peelone(rp, ci)
        assert st["levels"] == ost["levels"]
        assert st["kmax"] == ost["kmax"]
        assert st["arcs"] == ost["arcs_scanned"]
        assert st["atomics"] - st["extra"] == ost["decrements"]
    else:
        _, ost = oracle.histocore(rp, ci)
        assert st["rounds"] == ost["rounds"]
        assert st["frontier"] == ost["frontier"]
        assert st["slots"] == ost["slots_read"]
        # InitHisto's arcs and edits, then the rounds' (either direction)
        assert st["arcs"] == g.arcs + ost["arcs_scanned"]
        assert st["atomics"] == g.arcs + 2 * ost["updates"]


# --------------------------------------------------------------------------
# PeelOne's level structure: many consecutive levels, gaps between levels
# (empty levels skipped), a hub whose residual degree falls through many
# values before its level, thousands of vertices reaching one value, and a
# dense R-MAT core; int32 and int64 offsets (arc-range and (vertex, chunk)
# entries for large vertices)
# --------------------------------------------------------------------------

def _cliques(sizes):
    """Disjoint union of complete graphs K_s (coreness s - 1 each)."""
    return gg.disjoint_union([gg.complete_graph(s) for s in sizes])


def _hub_over_cliques(n_cliques, s, leaves):
    """K_s copies whose vertex 0 all join one hub, which also has `leaves`
    leaves: the hub's residual degree falls through many values."""
    edges, base = [], 0
    for _ in range(n_cliques):
        edges += [(base + i, base + j) for i in range(s) for j in range(i + 1, s)]
        base += s
    hub = base
    edges += [(hub, c * s) for c in range(n_cliques)]
    edges += [(hub, hub + 1 + i) for i in range(leaves)]
    return gg.from_edge_list(edges, hub + 1 + leaves)


LEVEL_CASES = [
    ("consecutive-1..40", lambda: _cliques(list(range(2, 42)) * 3)),
    ("gaps", lambda: _cliques([2, 4, 8, 20, 21, 56, 57, 91, 130] * 4)),
    ("hub-over-cliques", lambda: _hub_over_cliques(60, 12, 30)),
    ("many-at-one-value", lambda: gg.disjoint_union([gg.path_graph(10)] +
                                                  [gg.complete_graph(5)] * 5000)),
    ("rmat12-ef32", lambda: gg.rmat_graph(12, 32, 41)),
]


@pytest.mark.parametrize("off", [None, torch.int64], ids=["int32", "int64"])
@pytest.mark.parametrize("name,make", LEVEL_CASES, ids=[c[0] for c in LEVEL_CASES])
def test_peelone_level_structure(pico, name, make, off):
    g = make()
    rp, ci = g.numpy()
    want = oracle.bz_coreness(rp, ci)
    got, st = run(pico, g, "peelone", off)
    assert_same(got, want, f"{name} peelone")
    _, ost = oracle.peelone(rp, ci)
    assert st["levels"] == ost["levels"]
    assert st["kmax"] == ost["kmax"]
    assert st["arcs"] == ost["arcs_scanned"]
    assert st["atomics"] - st["extra"] == ost["decrements"]


@pytest.fixture
def update_mode(pico):
    """Sets the UpdateHisto direction for one test, then restores auto."""
    def set_mode(name):
        assert pico.pico_set_histo_update(pico.UPDATES[name], 25) == 0
        assert pico.pico_get_histo_update() == (pico.UPDATES[name], 25)
    yield set_mode
    assert pico.pico_set_histo_update(pico.PICO_UPDATE_AUTO, pico.PULL_PCT_DEFAULT) == 0


@pytest.mark.parametrize("mode", ["push", "pull"])
@pytest.mark.parametrize("name,make", FAMILIES, ids=[f[0] for f in FAMILIES])
def test_histocore_update_directions(pico, update_mode, mode, name, make):
    """Pushed and pulled UpdateHisto apply the same edits: the result, the
    rounds, the frontier and the edit count all equal the oracle's Alg. 6."""
    g = make()
    rp, ci = g.numpy()
    update_mode(mode)
    got, st = run(pico, g, "histocore")
    assert_same(got, oracle.bz_coreness(rp, ci), f"{name} {mode}")
    _, ost = oracle.histocore(rp, ci)
    assert st["rounds"] == ost["rounds"]
    assert st["frontier"] == ost["frontier"]
    assert st["slots"] == ost["slots_read"]
    assert st["arcs"] == g.arcs + ost["arcs_scanned"]
    assert st["atomics"] == g.arcs + 2 * ost["updates"]
    if mode == "pull":
        assert st["pull_rounds"] == st["rounds"] and st["pulled"] > 0
    else:
        assert st["pull_rounds"] == 0 and st["pulled"] == 0


@pytest.mark.parametrize("mode", ["push", "pull"])
def test_histocore_wide_estimates(pico, update_mode, mode):
    """Hubs of degree above 65,534: their {old, new} records do not fit the
    packed 16-bit form that pull rounds gather, so readers fall back to the
    full record. Two hubs (70,000 and 66,000 leaves, triangles through the
    first) each touch 10 members of a K_30, whose rows their drop edits."""
    edges = [(0, i) for i in range(1, 70001)]
    edges += [(1 + 2 * i, 2 + 2 * i) for i in range(500)]          # triangles with hub 0
    hub1 = 70001
    edges += [(hub1, i) for i in range(70002, 70002 + 66000)]
    base = 70002 + 66000
    edges += [(base + a, base + b) for a in range(30) for b in range(a + 1, 30)]
    edges += [(0, base + a) for a in range(10)] + [(hub1, base + 10 + a) for a in range(10)]
    n = base + 30
    g = gg.from_edge_list(edges, n)
    rp, ci = g.numpy()
    update_mode(mode)
    got, st = run(pico, g, "histocore")
    assert_same(got, oracle.bz_coreness(rp, ci), f"wide estimates {mode}")
    _, ost = oracle.histocore(rp, ci)
    assert ost["updates"] > 0
    assert st["rounds"] == ost["rounds"] and st["frontier"] == ost["frontier"]
    assert st["atomics"] == g.arcs + 2 * ost["updates"]
    if mode == "pull":
        assert st["pull_rounds"] == st["rounds"]


def test_histocore_auto_pulls_large_rounds(pico, update_mode):
    """R-MAT scale 18 (8.4 M arcs): the auto mode pulls the first rounds,
    whose changed vertices hold most arcs, and pushes the later ones."""
    g = gg.rmat_graph(18, 16, 36)
    assert g.arcs >= 1 << 22
    rp, ci = g.numpy()
    update_mode("auto")
    got, st = run(pico, g, "histocore")
    assert_same(got, oracle.bz_coreness(rp, ci), "rmat18 auto")
    assert 0 < st["pull_rounds"] < st["rounds"]
    _, ost = oracle.histocore(rp, ci)
    assert st["rounds"] == ost["rounds"]
    assert st["atomics"] == g.arcs + 2 * ost["updates"]


@pytest.mark.parametrize("algo", ALGOS)
def test_int64_offsets(pico, algo):
    g = gg.rmat_graph(15, 16, 34)
    want = oracle.bz_coreness(*g.numpy())
    got, _ = run(pico, g, algo, off_dtype=torch.int64)
    assert_same(got, want, "int64 row_ptr")


@pytest.mark.parametrize("algo", ALGOS)
def test_side_stream_and_repeat(pico, algo):
    g = gg.rmat_graph(14, 16, 35)
    want = oracle.bz_coreness(*g.numpy())
    rp, ci = g.row_ptr.cuda(), g.col_idx.cuda()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        outs = [pico.coreness(rp, ci, algo, check=False) for _ in range(3)]
    assert pico.pico_last_device_status(s) == 0
    for o in outs:
        assert_same(o.cpu().numpy(), want, "side stream")


# --------------------------------------------------------------------------
# full-size workloads (the launch configuration the benchmark times)
# --------------------------------------------------------------------------

FULL = ["rmat22", "rmat24", "chunglu24", "grid4096"]


@pytest.mark.parametrize("name", FULL)
def test_full_size_workloads(pico, name):
    g = gg.workload(name, device="cuda")
    rp, ci = g.numpy()
    want = oracle.bz_coreness(rp, ci)
    for algo in ALGOS:
        out = pico.coreness(g.row_ptr, g.col_idx, algo)
        assert_same(out.cpu().numpy(), want, f"{name} {algo}")
    if name == "chunglu24":
        members = gg.clique_members(g.n, gg.SEED_BASE + 3, 3000).numpy()
        assert (want[members] >= 2999).all()
    if name == "grid4096":
        assert (want == 2).all()


_WAVES_CHILD = r"""
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import torch
import graphgen as gg
import oracle
import paper_2402_15253_gb300 as pico
torch.cuda.set_device(0)
bad = 0
for g in (gg.workload("rmat16"), gg.chung_lu_graph(1 << 16, 33, clique=300),
          gg.grid_graph(257, 333), gg.path_graph(5000)):
    rp, ci = g.numpy()
    out = pico.coreness(g.row_ptr.cuda(), g.col_idx.cuda(), "peelone").cpu().numpy()
    st = pico.pico_get_stats()
    _, ost = oracle.peelone(rp, ci)
    ok = (np.array_equal(out, oracle.bz_coreness(rp, ci)) and st["levels"] == ost["levels"]
          and st["subrounds"] == ost["waves"] and st["arcs"] == ost["arcs_scanned"])
    bad += not ok
print("BAD", bad)
"""


def test_peelone_per_wave_form_matches_oracle_waves():
    """PICO_PEEL_WAVES=1 selects the form that ends every wave of the dynamic
    frontier with a grid barrier: results, levels and waves are the oracle's."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _WAVES_CHILD, root],
                       env=dict(os.environ, PICO_PEEL_WAVES="1"), capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "BAD 0" in r.stdout, r.stdout[-2000:]
