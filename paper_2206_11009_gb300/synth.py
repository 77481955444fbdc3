"""Seeded synthetic OT workloads (image-marginal pairs) shared by tests, bench and smoke.

This module holds no arithmetic of the solver: it only draws inputs.  Both the CUDA
path and the CPU oracle receive the arrays it returns.

The paper evaluates on DOTmark grayscale images (Section 5.1), square grids of
k x k pixels whose intensities are the masses.  That collection is not available
here, so inputs are seeded stand-ins with the same shape and structure:

* white noise N(0,1) on the k x k grid, drawn from SplitMix64 (Steele, Lea & Flood,
  "Fast splittable pseudorandom number generators", OOPSLA 2014) through the
  Box-Muller transform;
* a separable Gaussian blur of standard deviation k/8 pixels (mirror boundary);
* standardisation to zero mean / unit variance, then ``exp`` (a log-normal field,
  strictly positive);
* optional sparse bright spikes: ceil(frac*m) distinct pixels get +amp x median;
* normalisation to total mass 1 in float64.

Pixel i sits at column alpha_i = i mod k and row beta_i = i div k.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """``count`` successive SplitMix64 outputs for the given 64-bit seed (uint64 array)."""
    with np.errstate(over="ignore"):
        idx = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int) -> np.ndarray:
    """Uniform doubles in the open interval (0, 1) from the top 53 bits of SplitMix64."""
    z = splitmix64(seed, count) >> np.uint64(11)
    return (z.astype(np.float64) + 0.5) * (2.0 ** -53)


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normal samples (Box-Muller, cosine branch)."""
    u = uniform01(seed, 2 * count)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def _blur_1d(x: np.ndarray, sigma: float, axis: int) -> np.ndarray:
    r = max(1, int(math.ceil(3.0 * sigma)))
    t = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-0.5 * (t / sigma) ** 2)
    w /= w.sum()
    pad = [(0, 0), (0, 0)]
    pad[axis] = (r, r)
    xp = np.pad(x, pad, mode="symmetric")
    out = np.zeros_like(x)
    n = x.shape[axis]
    for s, ws in enumerate(w):
        sl = [slice(None), slice(None)]
        sl[axis] = slice(s, s + n)
        out += ws * xp[tuple(sl)]
    return out


def grf_image(k: int, seed: int, spike_frac: float = 0.0, spike_amp: float = 20.0,
              sigma_frac: float = 0.125) -> np.ndarray:
    """One k x k positive image flattened to k*k masses summing to 1 (float64)."""
    g = normal(seed, k * k).reshape(k, k)
    sigma = max(sigma_frac * k, 0.5)
    g = _blur_1d(_blur_1d(g, sigma, 0), sigma, 1)
    g = (g - g.mean()) / max(g.std(), 1e-300)
    a = np.exp(g).reshape(-1)
    if spike_frac > 0.0:
        cnt = int(math.ceil(spike_frac * a.size))
        keys = splitmix64(seed ^ 0x5DEECE66D, a.size)
        pick = np.argsort(keys, kind="stable")[:cnt]
        a[pick] += spike_amp * float(np.median(a))
    return a / a.sum()


def grid_coords(k: int) -> tuple[np.ndarray, np.ndarray]:
    """Integer pixel coordinates (alpha, beta) = (i mod k, i div k) as int32 arrays."""
    i = np.arange(k * k, dtype=np.int64)
    return (i % k).astype(np.int32), (i // k).astype(np.int32)


@dataclass
class Instance:
    """A square-grid OT instance with squared-Euclidean pixel cost."""
    k: int
    a: np.ndarray
    b: np.ndarray
    seed: int

    @property
    def m(self) -> int:
        return self.k * self.k

    @property
    def n(self) -> int:
        return self.k * self.k


def image_pair(k: int, s: int, spike_frac: float = 0.0) -> Instance:
    """Instance number ``s`` at side ``k``: seed 2s for the source, 2s+1 for the target."""
    a = grf_image(k, 2 * s, spike_frac)
    b = grf_image(k, 2 * s + 1, spike_frac)
    return Instance(k=k, a=a, b=b, seed=s)


def batch_sides(count: int = 64, lo: int = 24, hi: int = 96, seed: int = 1234) -> np.ndarray:
    """Seeded uneven grid sides, uniform on [lo, hi], for a batch of instances."""
    u = uniform01(seed, count)
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64).clip(lo, hi)


def random_int_costs(m: int, n: int, seed: int, hi: int = 20) -> np.ndarray:
    """Dense m x n integer cost matrix in [0, hi] (float64), for brute-force cases."""
    u = uniform01(seed, m * n)
    return np.floor(u * (hi + 1)).reshape(m, n).astype(np.float64)


def random_masses(count: int, seed: int, integer: bool = False) -> np.ndarray:
    """Positive masses summing to 1; with ``integer`` they are small integers / total."""
    u = uniform01(seed, count)
    if integer:
        w = 1.0 + np.floor(u * 5.0)
    else:
        w = 0.1 + u
    return w / w.sum()
