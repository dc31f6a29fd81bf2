"""The C ABI library builds, loads and exports every declared symbol; host-side
argument checks answer without a GPU."""
import ctypes
import glob
import os
import re

import pytest

from conftest import ROOT

from paper_2402_15253_gb300 import build as libbuild


@pytest.fixture(scope="module")
def lib():
    path = libbuild.build()
    import paper_2402_15253_gb300 as pico
    return pico, ctypes.CDLL(path)


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(pico_\w+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    _, L = lib
    names = declared_functions()
    assert "pico_coreness" in names and "pico_coreness_i64" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings(lib):
    pico, _ = lib
    assert pico.pico_status_string(pico.PICO_OK) == "ok"
    for code in range(-7, 0):
        s = pico.pico_status_string(code)
        assert s and s != "unknown status"
    assert pico.pico_status_string(12345) == "unknown status"
    assert pico.pico_version() >= 100


def test_workspace_bytes(lib):
    pico, _ = lib
    a = pico.pico_workspace_bytes(1 << 20, 1 << 24, pico.PICO_ALGO_PEELONE)
    b = pico.pico_workspace_bytes(1 << 20, 1 << 24, pico.PICO_ALGO_HISTOCORE)
    assert a > 3 * 4 * (1 << 20)            # two residual lists and the queue
    assert b > 4 * (1 << 24)                # the histogram has one slot per arc
    assert pico.pico_workspace_bytes(-1, 5, 0) == 0
    assert pico.pico_workspace_bytes(5, 5, 9) == 0


def test_argument_checks_need_no_gpu(lib):
    pico, L = lib
    vp = ctypes.c_void_p
    # negative sizes, unknown method, null pointers: rejected before any CUDA call
    assert L.pico_coreness(vp(None), vp(None), ctypes.c_int64(-1), ctypes.c_int64(0), vp(None),
                           0, vp(None)) == pico.PICO_ERR_INVALID_ARG
    for bad_algo in (-1, 8, 99):
        assert L.pico_coreness(vp(8), vp(8), ctypes.c_int64(4), ctypes.c_int64(4), vp(8),
                               bad_algo, vp(None)) == pico.PICO_ERR_INVALID_ARG
    assert L.pico_coreness(vp(None), vp(8), ctypes.c_int64(4), ctypes.c_int64(4), vp(8),
                           0, vp(None)) == pico.PICO_ERR_INVALID_ARG
    assert L.pico_coreness_i64(vp(8), vp(8), ctypes.c_int64(1 << 31), ctypes.c_int64(4), vp(8),
                               1, vp(None)) == pico.PICO_ERR_INVALID_ARG
    # int32 offsets cannot address 2^31 arcs
    assert L.pico_coreness(vp(8), vp(8), ctypes.c_int64(4), ctypes.c_int64(1 << 31), vp(8),
                           0, vp(None)) == pico.PICO_ERR_INVALID_ARG
    # an empty graph is a no-op
    assert L.pico_coreness(vp(None), vp(None), ctypes.c_int64(0), ctypes.c_int64(0), vp(None),
                           0, vp(None)) == pico.PICO_OK
    # validation: sizes and pointers are checked on the host; an empty graph
    # is valid iff it has no arcs, and nothing is read
    d = ctypes.c_uint32(99)
    i64 = ctypes.c_int64

    def val(f, rp, ci, n, m):
        d.value = 99
        return f(vp(rp), vp(ci), i64(n), i64(m), ctypes.byref(d), vp(None)), d.value

    assert val(L.pico_validate_graph, None, None, -1, 0) == (pico.PICO_ERR_INVALID_ARG, 0)
    assert val(L.pico_validate_graph, None, None, 0, 0) == (pico.PICO_OK, 0)
    assert val(L.pico_validate_graph, None, None, 0, 3) == (pico.PICO_ERR_BAD_GRAPH,
                                                            pico.PICO_DEFECT_ROWS)
    assert val(L.pico_validate_graph, None, 8, 4, 4)[0] == pico.PICO_ERR_INVALID_ARG
    assert val(L.pico_validate_graph_i64, 8, None, 4, 4)[0] == pico.PICO_ERR_INVALID_ARG
    # UpdateHisto direction: unknown modes and thresholds outside 1..100
    for mode, pct in ((-1, 25), (3, 25), (pico.PICO_UPDATE_AUTO, 0), (pico.PICO_UPDATE_PULL, 101)):
        assert L.pico_set_histo_update(mode, pct) == pico.PICO_ERR_INVALID_ARG
    assert L.pico_get_histo_update(vp(None), vp(None)) == pico.PICO_ERR_INVALID_ARG


def test_binding_names_mirror_the_abi(lib):
    pico, _ = lib
    for name in declared_functions():
        assert hasattr(pico, name), name


def test_server_rejects_invalid_configs_without_gpu(lib):
    pico, _ = lib
    assert not pico.pico_server_create(1 << 30, 5, 4, 64, 0)     # unknown method
    assert not pico.pico_server_create(1 << 30, 0, 0, 64, 0)     # no streams
    assert not pico.pico_server_create(1 << 30, 0, 4, 0, 0)      # empty batches
    assert pico.pico_server_submit(None, None, None, 1, 0, None, 0) == pico.PICO_ERR_INVALID_ARG
    assert pico.pico_server_drain(None) == pico.PICO_ERR_INVALID_ARG
