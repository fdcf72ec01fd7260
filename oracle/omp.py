"""Test infrastructure: the OpenMP build of the oracle's mode-1 contraction
loop (contract_omp.c), the all-cores column of the benchmark's CPU
baseline.  Only tests and the benchmark's CPU-baseline leg use it.

``build()`` compiles contract_omp.c with gcc (-O2 -fopenmp) into
liboracle_omp.so next to it; ``mode1_omp`` evaluates unfold_1 of
A.(X,Y)_{2,3} (Algorithm 3 step (i)) with it, in FP64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "contract_omp.c")
LIB = os.path.join(HERE, "liboracle_omp.so")
_lib = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp"
    r = subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", SRC, "-o", tmp],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"gcc failed for {SRC}:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        i64, vp, ci = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
        L.oracle_mode1_omp.argtypes = [i64, i64, vp, vp, vp, vp, vp, ci, vp, ci, vp, ci]
        L.oracle_mode1_omp.restype = None
        L.oracle_omp_threads.argtypes = []
        L.oracle_omp_threads.restype = ci
        _lib = L
    return _lib


def threads() -> int:
    """Threads the OpenMP loop uses: every processor of the host."""
    return int(_load().oracle_omp_threads())


def csr_rowptr(A) -> np.ndarray:
    """Row pointers of a stored tensor (entries sorted by (i, j, k))."""
    return np.searchsorted(A.i, np.arange(A.m + 1), side="left").astype(np.int64)


def mode1_omp(A, X: np.ndarray, Y: np.ndarray, rowptr: np.ndarray | None = None) -> np.ndarray:
    """unfold_1 of A.(X,Y)_{2,3}: m x (p q), column a + p b, FP64."""
    L = _load()
    X = np.asfortranarray(X, dtype=np.float64)
    Y = np.asfortranarray(Y, dtype=np.float64)
    p, q = X.shape[1], Y.shape[1]
    assert p * q <= 64
    rp = csr_rowptr(A) if rowptr is None else rowptr
    j = np.ascontiguousarray(A.j, dtype=np.int32)
    k = np.ascontiguousarray(A.k, dtype=np.int32)
    v = np.ascontiguousarray(A.v, dtype=np.float64)
    out = np.empty((A.m, p * q), order="F")
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data)
    L.oracle_mode1_omp(A.m, A.n, ptr(rp), ptr(j), ptr(k), ptr(v), ptr(X), p, ptr(Y), q, ptr(out),
                       threads())
    return out
