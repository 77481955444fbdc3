"""LP certificates for transportation solutions (Sections 2.1-2.2).

Test infrastructure only (see ``oracle/__init__.py``).

* Weak duality: for any v, u_i = min_j (c_ij - v_j) (the c-transform) makes (u, v) dual
  feasible, so a^T u + b^T v <= OPT.  With a feasible p, c^T p >= OPT.  Equal values
  certify optimality.
* Section 2.2: a vertex of the feasible region is acyclic as a bipartite graph, hence has
  at most m+n-1 nonzeros.
"""
from __future__ import annotations

import numpy as np

from .costs import Cost


def c_transform_lower_bound(cost: Cost, a: np.ndarray, b: np.ndarray, v: np.ndarray) -> float:
    ubar = np.empty(cost.m)
    step = max(1, (1 << 22) // max(cost.n, 1))
    for i0 in range(0, cost.m, step):
        i1 = min(cost.m, i0 + step)
        ubar[i0:i1] = (cost.block(i0, i1) - v[None, :]).min(axis=1)
    return float(a @ ubar + b @ v)


def min_reduced_cost(cost: Cost, u: np.ndarray, v: np.ndarray) -> float:
    best = np.inf
    step = max(1, (1 << 22) // max(cost.n, 1))
    for i0 in range(0, cost.m, step):
        i1 = min(cost.m, i0 + step)
        best = min(best, float(((cost.block(i0, i1) - u[i0:i1, None]) - v[None, :]).min()))
    return best


def marginal_residual_l1(m: int, n: int, I, J, P, a, b) -> float:
    ra = a - np.bincount(I, weights=P, minlength=m)
    rb = b - np.bincount(J, weights=P, minlength=n)
    return float(np.abs(ra).sum() + np.abs(rb).sum())


def is_forest(m: int, n: int, I, J) -> bool:
    """Union-find over the bipartite graph of the given edges: True iff no cycle."""
    parent = list(range(m + n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for i, j in zip(np.asarray(I).tolist(), np.asarray(J).tolist()):
        ri, rj = find(i), find(m + j)
        if ri == rj:
            return False
        parent[ri] = rj
    return True
