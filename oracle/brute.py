"""O3: brute-force optima for tiny transportation problems (pins for O1 and O2).

Test infrastructure only (see ``oracle/__init__.py``).

* ``vertex_enumeration``: an LP attains its optimum at a vertex of the feasible region;
  every vertex of {A p = f, p >= 0} with A of rank m+n-1 (Section 2.1) is a basic solution
  on m+n-1 columns.  Enumerate all column subsets of that size, keep the nonsingular
  nonnegative ones, take the cheapest.
* ``assignment``: with a = b = 1/n, Birkhoff-von Neumann makes the permutation matrices
  the vertices, so OPT = min over permutations of sum_i c_{i,pi(i)} / n.
* ``monotone_1d``: on a line with a convex cost of the difference, the monotone
  (north-west corner on sorted positions) coupling is optimal; its cost is the closed form.
"""
from __future__ import annotations

import itertools

import numpy as np


def constraint_matrix(m: int, n: int) -> np.ndarray:
    """A = [e_n^T (x) I_m ; I_n (x) e_m^T] acting on column-major vec(P) (Section 2.1)."""
    A1 = np.kron(np.ones((1, n)), np.eye(m))
    A2 = np.kron(np.eye(n), np.ones((1, m)))
    return np.vstack([A1, A2])


def vertex_enumeration(C: np.ndarray, a: np.ndarray, b: np.ndarray) -> tuple[float, np.ndarray]:
    m, n = C.shape
    A = constraint_matrix(m, n)
    f = np.concatenate([a, b])
    c = C.reshape(-1, order="F")            # column-major, like vec(P)
    best, bestp = np.inf, None
    r = m + n - 1
    for cols in itertools.combinations(range(m * n), r):
        B = A[:, cols]
        if np.linalg.matrix_rank(B) < r:
            continue
        pB, *_ = np.linalg.lstsq(B, f, rcond=None)
        if np.abs(B @ pB - f).max() > 1e-10 or pB.min() < -1e-12:
            continue
        val = float(c[list(cols)] @ pB)
        if val < best:
            best = val
            bestp = np.zeros(m * n)
            bestp[list(cols)] = pB
    return best, bestp.reshape((m, n), order="F")


def assignment(C: np.ndarray) -> float:
    n = C.shape[0]
    best = np.inf
    rows = np.arange(n)
    for perm in itertools.permutations(range(n)):
        val = C[rows, perm].sum()
        if val < best:
            best = val
    return float(best) / n


def monotone_1d(x: np.ndarray, a: np.ndarray, y: np.ndarray, b: np.ndarray,
                cost=lambda d: d * d) -> float:
    """North-west corner rule on positions sorted ascending (both sides)."""
    ia, ib = np.argsort(x, kind="stable"), np.argsort(y, kind="stable")
    ra, rb = a[ia].astype(np.float64).copy(), b[ib].astype(np.float64).copy()
    i = j = 0
    total = 0.0
    while i < len(ra) and j < len(rb):
        q = min(ra[i], rb[j])           # one of the two becomes exactly zero
        total += q * cost(x[ia[i]] - y[ib[j]])
        ra[i] -= q
        rb[j] -= q
        if ra[i] <= 0.0:
            i += 1
        if rb[j] <= 0.0:
            j += 1
    return total
