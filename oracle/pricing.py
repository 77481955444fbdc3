"""Pricing rule of Section 3.4 with an exact selection contract.

Test infrastructure only (see ``oracle/__init__.py``).

Section 3.4: the reduced cost of column (i, j) is c_ij - y_{k1j} - y_{k2j}, i.e. with the
duals y = (u, v) of the row and column constraints, d_ij = c_ij - u_i - v_j.  Section 3.2
(support enlargement) adds the most negative reduced costs to the support, at most m per
iteration (end of Section 3.2).

Exact contract (the reading used everywhere in this project):
  * d_ij = (c_ij - u_i) - v_j evaluated in IEEE-754 float64, round to nearest, in exactly
    that order (no fused multiply-add);
  * candidates: (i, j) not in the support with d_ij < 0;
  * order by (d_ij, jlin) ascending with jlin = i + j*m, the 0-based column-major position
    of p_ij in vec(P) (Section 2.1); keep the first min(kmax, #candidates).
The set kept is unique; tests compare sets bit for bit.

Heuristic set J (Section 3.4): with ``cmax`` given, only the pairs with c_ij < cmax are
candidates (J is fixed before the iterations start; a full pricing refreshes the support every
few iterations).
"""
from __future__ import annotations

import numpy as np

from .costs import Cost


def reduced_costs(cost: Cost, u: np.ndarray, v: np.ndarray, i0: int = 0, i1: int | None = None) -> np.ndarray:
    """Rows i0..i1-1 of d = (c - u) - v in float64."""
    i1 = cost.m if i1 is None else i1
    c = cost.block(i0, i1)
    return (c - u[i0:i1, None]) - v[None, :]


def select(cost: Cost, u: np.ndarray, v: np.ndarray, support_i: np.ndarray,
           support_j: np.ndarray, kmax: int, rows_per_chunk: int | None = None, cmax: float | None = None):
    """Return (I, J, d) of the selected columns, ordered by (d, jlin); candidates restricted to
    c_ij < cmax when cmax is given."""
    m, n = cost.m, cost.n
    sup_key = np.sort(np.asarray(support_i, np.int64) * n + np.asarray(support_j, np.int64))
    if rows_per_chunk is None:
        rows_per_chunk = max(1, (1 << 23) // max(n, 1))
    Is, Js, Ds = [], [], []
    for i0 in range(0, m, rows_per_chunk):
        i1 = min(m, i0 + rows_per_chunk)
        c = cost.block(i0, i1)
        d = (c - u[i0:i1, None]) - v[None, :]
        neg = d < 0.0
        if cmax is not None:
            neg &= c < cmax
        ii, jj = np.nonzero(neg)
        if ii.size == 0:
            continue
        gi = ii + i0
        key = gi.astype(np.int64) * n + jj
        pos = np.searchsorted(sup_key, key)
        member = (pos < len(sup_key)) & (sup_key[np.minimum(pos, len(sup_key) - 1)] == key) \
            if len(sup_key) else np.zeros(len(key), bool)
        keep = ~member
        Is.append(gi[keep]); Js.append(jj[keep]); Ds.append(d[ii[keep], jj[keep]])
    if not Is:
        e = np.zeros(0, dtype=np.int64)
        return e, e.copy(), np.zeros(0)
    I = np.concatenate(Is).astype(np.int64)
    J = np.concatenate(Js).astype(np.int64)
    D = np.concatenate(Ds)
    jlin = I + J * m
    order = np.lexsort((jlin, D))[:kmax]
    return I[order], J[order], D[order]


def select_bruteforce(C: np.ndarray, u, v, support: set, kmax: int, cmax: float | None = None):
    """Pure-Python loops over every pair; for tiny inputs only."""
    m, n = C.shape
    cand = []
    for j in range(n):
        for i in range(m):
            if (i, j) in support:
                continue
            if cmax is not None and not float(C[i, j]) < cmax:
                continue
            d = (float(C[i, j]) - float(u[i])) - float(v[j])
            if d < 0.0:
                cand.append((d, i + j * m, i, j))
    cand.sort()
    return [(i, j) for _, _, i, j in cand[:kmax]]


def _chunk_topk(args):
    cost, u, v, sup_key, i0, i1, kmax, cmax, rows_per_chunk = args
    m, n = cost.m, cost.n
    best_I = np.zeros(0, np.int64)
    best_J = np.zeros(0, np.int64)
    best_D = np.zeros(0)
    for r0 in range(i0, i1, rows_per_chunk):
        r1 = min(i1, r0 + rows_per_chunk)
        c = cost.block(r0, r1)
        d = (c - u[r0:r1, None]) - v[None, :]
        neg = d < 0.0
        if cmax is not None:
            neg &= c < cmax
        ii, jj = np.nonzero(neg)
        if ii.size == 0:
            continue
        gi = (ii + r0).astype(np.int64)
        jj = jj.astype(np.int64)
        key = gi * n + jj
        if len(sup_key):
            pos = np.searchsorted(sup_key, key)
            member = (pos < len(sup_key)) & (sup_key[np.minimum(pos, len(sup_key) - 1)] == key)
            keep = ~member
            gi, jj = gi[keep], jj[keep]
            dd = d[ii[keep], jj]
        else:
            dd = d[ii, jj]
        I = np.concatenate([best_I, gi])
        J = np.concatenate([best_J, jj])
        D = np.concatenate([best_D, dd])
        o = np.lexsort((I + J * m, D))[:kmax]
        best_I, best_J, best_D = I[o], J[o], D[o]
    return best_I, best_J, best_D


def select_streaming(cost: Cost, u: np.ndarray, v: np.ndarray, support_i, support_j, kmax: int,
                     cmax: float | None = None, rows_per_chunk: int | None = None, workers: int = 1):
    """The same selection as ``select`` for inputs too large to hold every candidate: each block of
    rows keeps its own first kmax candidates in (d, jlin) order, and the blocks' lists are merged
    the same way (the overall first kmax are among the blocks' first kmax).  ``workers`` > 1 runs
    the blocks in a process pool started with 'spawn'."""
    m, n = cost.m, cost.n
    sup_key = np.sort(np.asarray(support_i, np.int64) * n + np.asarray(support_j, np.int64))
    if rows_per_chunk is None:
        rows_per_chunk = max(1, (1 << 22) // max(n, 1))
    nblk = max(1, workers * 4)
    edges = np.linspace(0, m, nblk + 1).astype(int)
    jobs = [(cost, u, v, sup_key, int(edges[b]), int(edges[b + 1]), kmax, cmax, rows_per_chunk)
            for b in range(nblk) if edges[b + 1] > edges[b]]
    if workers > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            parts = pool.map(_chunk_topk, jobs)
    else:
        parts = [_chunk_topk(j) for j in jobs]
    I = np.concatenate([p[0] for p in parts])
    J = np.concatenate([p[1] for p in parts])
    D = np.concatenate([p[2] for p in parts])
    o = np.lexsort((I + J * m, D))[:kmax]
    return I[o], J[o], D[o]
