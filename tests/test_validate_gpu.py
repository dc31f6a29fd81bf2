"""Input validation (pico_validate_graph, PICO_VALIDATE=1) on the GPU.

Valid graphs of every family report no defect; each kind of malformed CSR
(row offsets that do not start at 0, fall, or end elsewhere than at m;
neighbour ids outside [0, n); self-loops; duplicate arcs; unsorted rows;
an arc without its reverse) is reported with its own defect bit. With
PICO_VALIDATE=1 the compute entry point refuses a malformed graph and still
computes the oracle's coreness of a valid one.
"""
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
def pico():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_15253_gb300 as p
    torch.cuda.set_device(0)
    return p


def csr(rows, off=torch.int32):
    """CSR of a list of neighbour lists, taken as given (no cleaning)."""
    rp = np.zeros(len(rows) + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.array([u for r in rows for u in r] or [0], dtype=np.int32)
    return torch.from_numpy(rp).to(off).cuda(), torch.from_numpy(ci).cuda(), len(rows), int(rp[-1])


def validate(pico, rp, ci, n, m):
    f = pico.pico_validate_graph_i64 if rp.dtype == torch.int64 else pico.pico_validate_graph
    return f(rp, ci, n, m)


def rows_of(g):
    rp, ci = g.numpy()
    return [ci[rp[v]:rp[v + 1]].tolist() for v in range(g.n)]


# a small valid graph: a triangle 0-1-2, a pendant 3 on 2, an isolated 4
BASE = [[1, 2], [0, 2], [0, 1, 3], [2], []]


@pytest.mark.parametrize("off", [torch.int32, torch.int64], ids=["int32", "int64"])
@pytest.mark.parametrize("name,make", [
    ("rmat14", lambda: gg.rmat_graph(14, 16, 71)),
    ("grid-100x77", lambda: gg.grid_graph(100, 77)),
    ("chunglu-2^14", lambda: gg.chung_lu_graph(1 << 14, 72, clique=120)),
    ("isolated-only", lambda: gg.from_edge_list([], 7)),
], ids=lambda x: x if isinstance(x, str) else "")
def test_valid_graphs_have_no_defect(pico, name, make, off):
    g = make()
    rp = g.row_ptr.to(off).cuda()
    ci = g.col_idx.cuda() if g.arcs else torch.zeros(1, dtype=torch.int32, device="cuda")
    assert validate(pico, rp, ci, g.n, g.arcs) == (pico.PICO_OK, 0)


def defect_cases(pico):
    D = pico
    # (name, rows, m override or None, row_ptr edit or None, expected bits);
    # an unsorted row may also hide a reverse arc from the binary search,
    # so ASYMMETRIC may come with ORDER there
    cases = [
        ("base", BASE, None, None, 0),
        ("id-n", [[1, 2], [0, 2], [0, 1, 3, 5], [2], []], None, None, D.PICO_DEFECT_IDS),
        ("id-negative", [[-1, 1, 2], [0, 2], [0, 1, 3], [2], []], None, None, D.PICO_DEFECT_IDS),
        ("self-loop", [[0, 1, 2], [0, 2], [0, 1, 3], [2], []], None, None,
         D.PICO_DEFECT_LOOP),
        ("duplicate", [[1, 1, 2], [0, 0, 2], [0, 1, 3], [2], []], None, None,
         D.PICO_DEFECT_ORDER),
        ("unsorted", [[2, 1], [0, 2], [0, 1, 3], [2], []], None, None, D.PICO_DEFECT_ORDER),
        ("asymmetric", [[1, 2], [0, 2], [0, 1, 3], [], []], None, None,
         D.PICO_DEFECT_ASYMMETRIC),
        ("m-mismatch", BASE, 7, None, D.PICO_DEFECT_ROWS),
        ("first-offset", BASE, None, (0, 1), D.PICO_DEFECT_ROWS),
        ("falling-offset", BASE, None, (2, 1), D.PICO_DEFECT_ROWS),
        ("offset-past-m", BASE, None, (3, 9), D.PICO_DEFECT_ROWS),
    ]
    return cases


@pytest.mark.parametrize("off", [torch.int32, torch.int64], ids=["int32", "int64"])
def test_each_defect_is_reported(pico, off):
    for name, rows, m_over, edit, want in defect_cases(pico):
        rp, ci, n, m = csr(rows, off)
        if edit is not None:
            rp[edit[0]] = edit[1]
        if m_over is not None:
            m = m_over
        rc, bits = validate(pico, rp, ci, n, m)
        extra = pico.PICO_DEFECT_ASYMMETRIC if name == "unsorted" else 0
        assert bits & ~extra == want, (name, bits, want)
        assert rc == (pico.PICO_OK if want == 0 else pico.PICO_ERR_BAD_GRAPH), (name, rc)


def test_defects_in_a_large_graph(pico):
    """One defect hidden in an R-MAT graph of 2^16 vertices is found."""
    g = gg.rmat_graph(16, 16, 73)
    rows = rows_of(g)
    v = max(range(g.n), key=lambda x: len(rows[x]))   # the largest row
    u = rows[v][len(rows[v]) // 2]
    bad = [list(r) for r in rows]
    bad[u].remove(v)                                  # drop one direction of (v, u)
    rp, ci, n, m = csr(bad)
    assert validate(pico, rp, ci, n, m) == (pico.PICO_ERR_BAD_GRAPH, pico.PICO_DEFECT_ASYMMETRIC)
    rp, ci, n, m = csr(rows)
    assert validate(pico, rp, ci, n, m) == (pico.PICO_OK, 0)


_CHILD = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import graphgen as gg
import oracle
import paper_2402_15253_gb300 as pico
torch.cuda.set_device(0)
g = gg.rmat_graph(13, 16, 74).to("cuda")
out = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
rc_good = pico.pico_coreness(g.row_ptr, g.col_idx, g.n, g.arcs, out, pico.PICO_ALGO_HISTOCORE)
torch.cuda.synchronize()
want = oracle.bz_coreness(g.row_ptr.cpu().numpy(), g.col_idx.cpu().numpy())
same = bool(np.array_equal(out.cpu().numpy(), want))
ci = g.col_idx.clone()
ci[0] = g.n   # an id outside [0, n)
out2 = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
rc_bad, untouched = -999, 0
# the compute call is made only once the validator is known to refuse this
# graph, so that it never runs on it
if pico.pico_validate_graph(g.row_ptr, ci, g.n, g.arcs)[0] == pico.PICO_ERR_BAD_GRAPH:
    rc_bad = pico.pico_coreness(g.row_ptr, ci, g.n, g.arcs, out2, pico.PICO_ALGO_PEELONE)
    torch.cuda.synchronize()
    untouched = int(bool((out2 == -7).all().item()))
print("RESULT", rc_good, int(same), rc_bad, untouched)
"""


def test_validate_env_guards_the_compute_entry_point(pico):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PICO_VALIDATE="1")
    r = subprocess.run([sys.executable, "-c", _CHILD, root], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT")][-1]
    rc_good, same, rc_bad, untouched = (int(x) for x in line.split()[1:])
    assert rc_good == pico.PICO_OK and same == 1
    assert rc_bad == pico.PICO_ERR_BAD_GRAPH and untouched == 1
