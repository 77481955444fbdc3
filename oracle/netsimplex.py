"""O1: exact transportation optimum by the plain network simplex in ``netsimplex.c``.

Test infrastructure only (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import build as _build
from .costs import KINDS, Cost

_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        f = _lib.ot_oracle_netsimplex
        P = ctypes.c_void_p
        f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P, P, P, P, P,
                      P, P, P, P, P, P, P, P, ctypes.c_int64, ctypes.c_int64]
        f.restype = ctypes.c_int
    return _lib


@dataclass
class SimplexResult:
    obj: float            # sum c_ij p_ij at the optimal vertex
    I: np.ndarray         # tree arcs (sources)
    J: np.ndarray         # tree arcs (targets)
    P: np.ndarray         # flows on the tree arcs
    u: np.ndarray         # potentials: c_ij - u_i - v_j >= 0, = 0 on the tree
    v: np.ndarray
    pivots: int


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def solve(cost: Cost, a: np.ndarray, b: np.ndarray, block: int = 0,
          max_pivots: int = 1 << 40) -> SimplexResult:
    lib = _load()
    m, n = cost.m, cost.n
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    ti = np.zeros(m + n, dtype=np.int32)
    tj = np.zeros(m + n, dtype=np.int32)
    tp = np.zeros(m + n, dtype=np.float64)
    nt = ctypes.c_int(0)
    u = np.zeros(m)
    v = np.zeros(n)
    obj = ctypes.c_double(0.0)
    piv = ctypes.c_int64(0)
    C = cost.C if cost.kind == "dense" else None
    rc = lib.ot_oracle_netsimplex(m, n, KINDS[cost.kind], _ptr(C), _ptr(cost.sx), _ptr(cost.sy),
                                  _ptr(cost.tx), _ptr(cost.ty), _ptr(a), _ptr(b), _ptr(ti), _ptr(tj),
                                  _ptr(tp), ctypes.byref(nt), _ptr(u), _ptr(v), ctypes.byref(obj),
                                  ctypes.byref(piv), block, max_pivots)
    if rc != 0:
        raise RuntimeError(f"network simplex failed with code {rc}")
    k = nt.value
    # gauge (u - t, v + t) leaves every reduced cost unchanged; remove the big-M offset
    t = float(np.floor(u.mean()))
    u -= t
    v += t
    return SimplexResult(obj.value, ti[:k].copy(), tj[:k].copy(), tp[:k].copy(), u, v, piv.value)
