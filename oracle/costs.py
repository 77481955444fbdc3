"""Cost definitions for the oracle (Section 5.1 distances plus the squared-Euclidean cost).

Test infrastructure only (see ``oracle/__init__.py``).

A ``Cost`` is either dense (an explicit m x n matrix, for brute-force cases) or a pixel
distance between source points (sx, sy) and target points (tx, ty):
  sqeuclid  (dx^2 + dy^2)       -- the cost of the workloads measured here
  euclid    sqrt(dx^2 + dy^2)   -- the paper's "2-distance"
  l1        |dx| + |dy|
  linf      max(|dx|, |dy|)
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

KINDS = {"sqeuclid": 0, "euclid": 1, "l1": 2, "linf": 3, "dense": 4}


@dataclass
class Cost:
    kind: str
    m: int
    n: int
    C: np.ndarray | None = None          # dense m x n (row-major), kind == "dense"
    sx: np.ndarray | None = None
    sy: np.ndarray | None = None
    tx: np.ndarray | None = None
    ty: np.ndarray | None = None

    @staticmethod
    def dense(C: np.ndarray) -> "Cost":
        C = np.ascontiguousarray(C, dtype=np.float64)
        return Cost("dense", C.shape[0], C.shape[1], C=C)

    @staticmethod
    def points(sx, sy, tx, ty, kind: str = "sqeuclid") -> "Cost":
        f = lambda z: np.ascontiguousarray(z, dtype=np.float64)
        return Cost(kind, len(sx), len(tx), sx=f(sx), sy=f(sy), tx=f(tx), ty=f(ty))

    def block(self, i0: int, i1: int) -> np.ndarray:
        """Rows i0..i1-1 of the cost matrix, float64."""
        if self.kind == "dense":
            return self.C[i0:i1].copy()
        dx = self.sx[i0:i1, None] - self.tx[None, :]
        dy = self.sy[i0:i1, None] - self.ty[None, :]
        if self.kind == "sqeuclid":
            return dx * dx + dy * dy
        if self.kind == "euclid":
            return np.sqrt(dx * dx + dy * dy)
        if self.kind == "l1":
            return np.abs(dx) + np.abs(dy)
        return np.maximum(np.abs(dx), np.abs(dy))

    def full(self) -> np.ndarray:
        return self.block(0, self.m)

    def pairs(self, I: np.ndarray, J: np.ndarray) -> np.ndarray:
        """c_ij for index arrays I, J."""
        if self.kind == "dense":
            return self.C[I, J]
        dx = self.sx[I] - self.tx[J]
        dy = self.sy[I] - self.ty[J]
        if self.kind == "sqeuclid":
            return dx * dx + dy * dy
        if self.kind == "euclid":
            return np.sqrt(dx * dx + dy * dy)
        if self.kind == "l1":
            return np.abs(dx) + np.abs(dy)
        return np.maximum(np.abs(dx), np.abs(dy))

    def max_cost(self) -> float:
        if self.kind == "dense":
            return float(self.C.max())
        best = 0.0
        step = max(1, (1 << 22) // max(self.n, 1))
        for i0 in range(0, self.m, step):
            best = max(best, float(self.block(i0, min(self.m, i0 + step)).max()))
        return best


def square_grid(k: int, kind: str = "sqeuclid") -> Cost:
    """Two k x k pixel grids; pixel i at (i mod k, i div k)."""
    i = np.arange(k * k)
    x = (i % k).astype(np.float64)
    y = (i // k).astype(np.float64)
    return Cost.points(x, y, x, y, kind)


def line_grid(k: int, kind: str = "sqeuclid") -> Cost:
    """Two 1 x k images (points 0..k-1 on a line)."""
    x = np.arange(k, dtype=np.float64)
    z = np.zeros(k)
    return Cost.points(x, z, x, z, kind)
