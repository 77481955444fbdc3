"""Incomplete Cholesky factor of the Schur complement with a drop tolerance (Section 4.2).

Test infrastructure only (see ``oracle/__init__.py``).

The paper preconditions CG in its iterative phase with an incomplete Cholesky factor whose drop
tolerance is lowered when CG needs many iterations.  The reading used here (and by the library):

  * order: the targets are coloured greedily in index order (each takes the smallest colour that
    none of its earlier neighbours in the graph of S_M holds); the new order lists the colours in
    sequence, targets in index order within a colour;
  * pattern: the entries of S_M that pass the drop test on their own value,
    |S_rs| >= tau * sqrt(S_rr S_ss), strictly lower in that order (no fill); the colouring is
    made on this pattern;
  * factor S ~ L D L^T, L unit lower, row by row in the new order, entries in increasing column:
        l_rs = (S_rs - sum_{t < s} l_rt l_st d_t) / d_s,   d_r = S_rr - sum_s l_rs^2 d_s,
    where the sums run over the pattern; an entry is dropped (set to 0) when
    |l_rs d_s| < tau * sqrt(S_rr S_ss); a pivot d_r <= eps * S_rr becomes +infinity, and every
    term carrying a +infinity pivot is zero;
  * apply: x = L^-T D^-1 L^-1 b in the new order, 1/inf = 0.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def greedy_coloring(S: sp.csr_matrix) -> np.ndarray:
    """Colour of every vertex: the smallest colour no earlier neighbour holds (index order)."""
    S = sp.csr_matrix(S)
    n = S.shape[0]
    color = np.full(n, -1, dtype=np.int64)
    for v in range(n):
        used = {int(color[u]) for u in S.indices[S.indptr[v]:S.indptr[v + 1]] if u != v and color[u] >= 0}
        c = 0
        while c in used:
            c += 1
        color[v] = c
    return color


def multicolor_order(color: np.ndarray) -> np.ndarray:
    """perm[new] = old: colours in sequence, indices increasing within a colour."""
    return np.lexsort((np.arange(len(color)), color))


def drop_pattern(S: sp.csr_matrix, diag: np.ndarray, tau: float) -> sp.csr_matrix:
    """The off-diagonal entries with |S_rs| >= tau * sqrt(S_rr S_ss)."""
    C = sp.coo_matrix(S)
    keep = (C.row != C.col) & (np.abs(C.data) >= tau * np.sqrt(diag[C.row] * diag[C.col]))
    return sp.csr_matrix((C.data[keep], (C.row[keep], C.col[keep])), shape=S.shape)


def factor(S: sp.csr_matrix, diag: np.ndarray, tau: float, eps: float = 1e-12):
    """Returns (perm, L rows as {s: l_rs} dicts in the new order, D in the new order).  S holds the
    off-diagonal entries (its diagonal is ignored), diag the diagonal S_jj."""
    S = drop_pattern(S, np.asarray(diag, np.float64), tau)
    n = S.shape[0]
    perm = multicolor_order(greedy_coloring(S))
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    rows = []
    D = np.zeros(n)
    for r in range(n):
        v = perm[r]
        ent = []
        for k in range(S.indptr[v], S.indptr[v + 1]):
            u = S.indices[k]
            if u != v and iperm[u] < r:
                ent.append((int(iperm[u]), float(S.data[k])))
        ent.sort()
        srr = float(diag[v])
        lrow = {}
        dsum = 0.0
        for s, a_rs in ent:
            acc = a_rs
            lrs_row = rows[s]
            for t, l_rt in lrow.items():
                if t < s and t in lrs_row and D[t] < np.inf:
                    acc -= l_rt * lrs_row[t] * D[t]
            ds = D[s]
            l = acc / ds if ds < np.inf else 0.0
            if l != 0.0 and abs(l * ds) < tau * np.sqrt(srr * float(diag[perm[s]])):
                l = 0.0
            lrow[s] = l
            if ds < np.inf:
                dsum += l * l * ds
        d = srr - dsum
        D[r] = d if d > eps * srr else np.inf
        rows.append(lrow)
    return perm, rows, D


def apply(perm: np.ndarray, rows, D: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x = L^-T D^-1 L^-1 b (b and x in the original order)."""
    n = len(perm)
    y = np.zeros(n)
    for r in range(n):
        acc = float(b[perm[r]])
        for s, l in rows[r].items():
            acc -= l * y[s]
        y[r] = acc
    z = np.where(D < np.inf, y / np.where(D < np.inf, D, 1.0), 0.0)
    xn = z.copy()
    for r in range(n - 1, -1, -1):
        for s, l in rows[r].items():
            xn[s] -= l * xn[r]
    x = np.zeros(n)
    x[perm] = xn
    return x
