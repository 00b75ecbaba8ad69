"""Python access to O2, the dense bounded simplex in ``simplex.c``.

Test infrastructure only (see ``oracle/__init__``).  ``build()`` compiles the
C file with gcc into ``_simplex.so`` next to it (no CUDA, no product code).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "simplex.c")
_LIB = os.path.join(_HERE, "_simplex.so")
_lib = None

STATUS = {0: "optimal", 1: "infeasible", 2: "unbounded", 3: "iteration_limit", -1: "error"}


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        f = lib.oracle_simplex
        P = ctypes.POINTER
        f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                      P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_double),
                      P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
                      ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double),
                      P(ctypes.c_double), P(ctypes.c_int)]
        f.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclasses.dataclass
class SimplexResult:
    status: str
    x: np.ndarray
    y: np.ndarray
    obj: float          # c.x (without any objective constant)
    iters: int


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def solve(A, q, c, l, u, m_eq: int, max_iter: int = 10_000_000) -> SimplexResult:
    lib = _load()
    A = sp.csc_matrix(A)
    A.sort_indices()
    m, n = A.shape
    cp = np.ascontiguousarray(A.indptr, np.int32)
    ri = np.ascontiguousarray(A.indices, np.int32)
    av = np.ascontiguousarray(A.data, np.float64)
    q = np.ascontiguousarray(q, np.float64)
    c = np.ascontiguousarray(c, np.float64)
    l = np.ascontiguousarray(l, np.float64)
    u = np.ascontiguousarray(u, np.float64)
    x = np.zeros(n)
    y = np.zeros(m)
    obj = ctypes.c_double(0.0)
    it = ctypes.c_int(0)
    rc = lib.oracle_simplex(m, n, m_eq, _ptr(cp, ctypes.c_int), _ptr(ri, ctypes.c_int),
                            _ptr(av, ctypes.c_double), _ptr(q, ctypes.c_double),
                            _ptr(c, ctypes.c_double), _ptr(l, ctypes.c_double),
                            _ptr(u, ctypes.c_double), int(max_iter), _ptr(x, ctypes.c_double),
                            _ptr(y, ctypes.c_double), ctypes.byref(obj), ctypes.byref(it))
    return SimplexResult(status=STATUS.get(rc, "error"), x=x, y=y, obj=obj.value, iters=it.value)


def solve_lp(lp, max_iter: int = 10_000_000) -> SimplexResult:
    """Solve an ``oracle.lp.LP``; ``obj`` then includes ``lp.obj_const``."""
    r = solve(lp.A, lp.q, lp.c, lp.l, lp.u, lp.m_eq, max_iter)
    r.obj += lp.obj_const
    return r
