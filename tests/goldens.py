"""Readers for the hand-computed fixtures under tests/golden/."""
from __future__ import annotations

import os

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _pairs(tokens):
    out = []
    for t in tokens:
        i, j = t.split(",")
        out.append((int(i), int(j)))
    return out


def pricing_cases():
    lines = open(os.path.join(HERE, "pricing_tiny.txt")).read().splitlines()
    lines = [ln for ln in lines if not ln.startswith("#")]
    cases, cur = [], []
    for ln in lines + [""]:
        if ln.strip() == "":
            if cur:
                cases.append(cur)
                cur = []
            continue
        cur.append(ln)
    out = []
    for blk in cases:
        m, n = map(int, blk[0].split())
        C = np.array([[float(x) for x in blk[1 + r].split()] for r in range(m)])
        rest = blk[1 + m:]
        u = np.array([float(x) for x in rest[0].split()[1:]])
        v = np.array([float(x) for x in rest[1].split()[1:]])
        sup = _pairs(rest[2].split()[1:])
        kmax = int(rest[3].split()[1])
        exp = _pairs(rest[4].split()[1:])
        out.append(dict(C=C, u=u, v=v, support=sup, kmax=kmax, expect=exp))
    return out
