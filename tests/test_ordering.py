"""Host symbolic analysis of the direct branch (Sections 4.1-4.3), on the CPU.

* the pattern of L from the elimination tree equals brute-force symbolic elimination;
* both orderings are permutations;
* Theorem 2 / its corollary: when the support is a forest, V^T V is chordal and minimum degree
  eliminates it with zero fill."""
from __future__ import annotations

import os
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2206_11009_gb300 import build as libbuild
from paper_2206_11009_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def driver():
    d = tempfile.mkdtemp()
    exe = os.path.join(d, "ordering_driver")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I" + libbuild.CSRC, os.path.join(HERE, "csrc", "ordering_driver.cpp"),
                    "-o", exe], check=True)
    return exe


def run(exe, mode, n, pairs):
    inp = f"{mode} {n} {len(pairs)}\n" + "\n".join(f"{r} {c}" for r, c in pairs) + "\n"
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    perm = np.array(out[0].split(), int)
    Lp = np.array(out[1].split(), int)
    Li = np.array(out[2].split(), int) if out[2].strip() else np.zeros(0, int)
    return perm, Lp, Li


def brute_pattern(n, pairs, perm):
    """Symbolic elimination on a dense boolean matrix in the order perm."""
    iperm = np.empty(n, int)
    iperm[perm] = np.arange(n)
    B = np.zeros((n, n), bool)
    for r, c in pairs:
        B[iperm[r], iperm[c]] = True
    for q in range(n):
        nb = np.nonzero(B[q + 1:, q])[0] + q + 1
        B[np.ix_(nb, nb)] = True
    return [set(np.nonzero(B[q + 1:, q])[0] + q + 1) for q in range(n)]


def schur_pattern(n_cols, I, J):
    """Off-diagonal pattern of V^T V (columns sharing a row)."""
    rows = {}
    for i, j in zip(I, J):
        rows.setdefault(i, []).append(j)
    pairs = set()
    for js in rows.values():
        for a in js:
            for b in js:
                if a != b:
                    pairs.add((a, b))
    return sorted(pairs)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("seed", range(4))
def test_symbolic_matches_bruteforce(driver, mode, seed):
    n = 40
    r = synth.uniform01(seed, n * n).reshape(n, n) < 0.08
    r = r | r.T
    np.fill_diagonal(r, False)
    pairs = [(int(a), int(b)) for a, b in zip(*np.nonzero(r))]
    perm, Lp, Li = run(driver, mode, n, pairs)
    assert sorted(perm.tolist()) == list(range(n))
    want = brute_pattern(n, pairs, perm)
    for q in range(n):
        got = Li[Lp[q]:Lp[q + 1]]
        assert list(got) == sorted(want[q])


def random_bipartite_forest(m, n, seed, drop=0):
    """A random spanning tree of K_{m,n} (each new node joins a placed node of the other side),
    minus `drop` edges (a forest)."""
    u = synth.uniform01(seed, 4 * (m + n))
    placed = {0: [], 1: [0]}       # side 0 = sources, side 1 = targets; start with target 0
    left = {0: m, 1: n - 1}
    I, J = [], []
    t = 0
    while left[0] + left[1] > 0:
        side = 0 if (left[1] == 0 or (left[0] > 0 and u[t] < left[0] / (left[0] + left[1]))) else 1
        other = placed[1 - side]
        if not other:
            side = 1 - side
            other = placed[1 - side]
        new = (m - left[0]) if side == 0 else (n - left[1])
        nb = other[int(u[t + 1] * len(other)) % len(other)]
        if side == 0:
            I.append(new); J.append(nb)
        else:
            I.append(nb); J.append(new)
        placed[side].append(new)
        left[side] -= 1
        t += 2
    return I[drop:], J[drop:]


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("drop", [0, 5])
def test_forest_support_has_zero_fill(driver, seed, drop):
    """Corollary of Theorem 2: for an acyclic support V^T V is chordal, and a perfect elimination
    ordering (reverse maximum cardinality search) factors it with zero fill."""
    m, n = 30, 25
    I, J = random_bipartite_forest(m, n, seed, drop)
    from oracle.certificate import is_forest
    assert is_forest(m, n, I, J)
    pairs = schur_pattern(n, I, J)
    perm, Lp, Li = run(driver, 2, n, pairs)
    lower = len(pairs) // 2
    assert len(Li) == lower
    assert sorted(perm.tolist()) == list(range(n))


def test_cycle_support_is_not_chordal(driver):
    """An 8-cycle in the bipartite graph (4 sources, 4 targets) gives a chordless 4-cycle in
    V^T V: no ordering is fill-free (Theorem 1), so reverse MCS must create fill."""
    I = [0, 0, 1, 1, 2, 2, 3, 3]
    J = [0, 1, 1, 2, 2, 3, 3, 0]
    pairs = schur_pattern(4, I, J)
    perm, Lp, Li = run(driver, 2, 4, pairs)
    assert len(Li) > len(pairs) // 2


def test_grid_support_nested_dissection_reduces_fill(driver):
    # S_M pattern of the initial 3x3 support on a 48x48 grid (a 5x5 stencil)
    k = 48
    I, J = [], []
    for i in range(k * k):
        for j in range(k * k):
            if abs(i % k - j % k) <= 1 and abs(i // k - j // k) <= 1:
                I.append(i); J.append(j)
    pairs = schur_pattern(k * k, I, J)
    _, _, Li_nd = run(driver, 1, k * k, pairs)
    # natural (banded) order fills the whole band: about n * 2k entries
    assert len(Li_nd) < (k * k) * 2 * k
