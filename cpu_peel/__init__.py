"""Parallel CPU comparison for the benchmark: a level-synchronous OpenMP
peel over all host cores (``cpu_peel.c``). It is neither the oracle nor the
product path; ``bench.py`` times it beside the single-threaded oracle, and
its results are checked against the oracle."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpu_peel.c")
_LIB = os.path.join(_HERE, "libcpu_peel.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile cpu_peel.c into libcpu_peel.so (gcc, OpenMP, portable C)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", tmp,
                               _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.cpu_peel_coreness.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                            ctypes.c_void_p]
            L.cpu_peel_coreness.restype = ctypes.c_int
            L.cpu_peel_threads.argtypes = []
            L.cpu_peel_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def threads() -> int:
    """OpenMP threads the peel uses."""
    return int(lib().cpu_peel_threads())


def coreness(rp, ci) -> np.ndarray:
    """Coreness of a CSR graph held in numpy arrays (rp: n + 1 offsets, ci:
    neighbour ids)."""
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    n = len(rp) - 1
    out = np.empty(max(n, 0), dtype=np.int32)
    rc = lib().cpu_peel_coreness(rp.ctypes.data, ci.ctypes.data, n, out.ctypes.data)
    if rc != 0:
        raise MemoryError("cpu_peel: out of memory")
    return out
