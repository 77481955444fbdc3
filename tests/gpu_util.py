"""Shared helpers of the GPU tests: seeded duals and supports, golden optima, device tensors."""
from __future__ import annotations

import os

import numpy as np

from paper_2206_11009_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def opt_value(k: int, seed: int, spike: float = 0.0) -> float:
    for ln in open(os.path.join(GOLDEN, "opt_values.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        kk, ss, sp, val, _ = ln.split()
        if int(kk) == k and int(ss) == seed and float(sp) == spike:
            return float(val)
    raise KeyError((k, seed, spike))


def rect_coords(w: int, h: int, x0: int = 0, y0: int = 0):
    i = np.arange(w * h)
    return (i % w + x0).astype(np.int32), (i // w + y0).astype(np.int32)


def banded_duals(sx, sy, tx, ty, seed: int, amp: float, noise: float):
    """Duals with the structure of IPM iterates: u_i = phi(x_i), v_j = -phi(y_j) + noise, phi a
    tilted smooth field of gradient about `amp`; the negative reduced costs then form a disc of
    radius about amp/2 around each source (|d| grows away from it)."""
    a = synth.normal(seed, 4)
    t = a[:2] / np.linalg.norm(a[:2])

    def phi(x, y):
        x = x.astype(float)
        y = y.astype(float)
        return amp * (t[0] * x + t[1] * y) + 2.0 * np.sin(0.13 * x + a[2]) * np.cos(0.09 * y + a[3])
    u = phi(sx, sy)
    v = -phi(tx, ty) + noise * (synth.uniform01(seed + 99, len(tx)) - 0.5)
    return u, v


def random_support(m: int, n: int, frac: float, seed: int):
    r = synth.uniform01(seed, m * n)
    key = np.nonzero(r < frac)[0].astype(np.int64)
    return (key // n).astype(np.int32), (key % n).astype(np.int32)


def neighbourhood_support(sx, sy, tx, ty, radius2: int = 2):
    """Pairs with squared distance <= radius2 (the initial support of the solver on grids)."""
    I, J = [], []
    for i in range(len(sx)):
        d = (sx[i] - tx) ** 2 + (sy[i] - ty) ** 2
        jj = np.nonzero(d <= radius2)[0]
        I.append(np.full(len(jj), i))
        J.append(jj)
    I = np.concatenate(I).astype(np.int32)
    J = np.concatenate(J).astype(np.int32)
    o = np.lexsort((J, I))
    return I[o], J[o]


def cuda_tensors(*arrays):
    import torch
    dev = torch.device("cuda:0")
    out = []
    for a in arrays:
        a = np.ascontiguousarray(a)
        dt = torch.int32 if a.dtype.kind in "iu" else torch.float64
        out.append(torch.as_tensor(a.astype(np.int32 if dt == torch.int32 else np.float64), dtype=dt, device=dev))
    return out
