"""Autotuner for the launch shapes the solver exposes (ot_options.scan_rows, dense32_max_n).

For each problem size bucket a grid search solves one seeded instance per candidate
configuration, times it with the solver's own device clock (CUDA events inside ot_ipm_solve) and
keeps the fastest.  Results are cached in JSON keyed by "m x n"; ``lookup`` answers with the entry
of the nearest cached size (by m * n) so that a batch of uneven sizes can be tuned on a few
buckets.

    python -m paper_2206_11009_gb300.autotune --sides 24 40 56 72 88 96 [--cache PATH]
"""
from __future__ import annotations

import argparse
import json
import os
import time

CACHE = os.environ.get("OT_TUNE_CACHE",
                       os.path.join(os.path.expanduser("~"), ".cache", "paper_2206_11009_gb300", "tuning.json"))
SCAN_ROWS = (0, 32, 64)           # 0: the library's own rule
TUNE_SEED = 777                      # instances used for tuning (not the evaluation seeds)

_cache_mem: dict | None = None


def _load(path: str = CACHE) -> dict:
    global _cache_mem
    if _cache_mem is None:
        try:
            with open(path) as f:
                _cache_mem = json.load(f)
        except (OSError, ValueError):
            _cache_mem = {}
    return _cache_mem


def _save(cache: dict, path: str = CACHE):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    with open(path, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)


def candidates(n: int):
    """The grid: scan tile rows x (dense FP32 preconditioner on / off where it applies)."""
    dense = (0, -1) if n <= 8192 else (0,)
    return [{"scan_rows": r, "dense32_max_n": d} for r in SCAN_ROWS for d in dense]


def tune_side(k: int, repeats: int = 1, verbose: bool = True) -> dict:
    """Grid search for k x k pixel grids; returns the winning options and every timing."""
    from . import synth
    from .api import Solver
    inst = synth.image_pair(k, TUNE_SEED)
    best, table = None, []
    for opts in candidates(k * k):
        secs = []
        for _ in range(repeats):
            with Solver(inst.a, inst.b, grid=(k, k), **opts) as s:
                r = s.solve(raise_on_error=False)
            secs.append(r.seconds if r.status == 0 else float("inf"))
        t = min(secs)
        table.append({**opts, "seconds": t})
        if best is None or t < best[1]:
            best = (opts, t)
    if verbose:
        print(f"  k={k}: best {best[0]} {best[1] * 1e3:.1f} ms of {len(table)} configurations", flush=True)
    return {"options": best[0], "seconds": best[1], "grid": table}


def tune(sides, path: str = CACHE, verbose: bool = True) -> dict:
    cache = _load(path)
    t0 = time.time()
    for k in sides:
        cache[f"{k * k}x{k * k}"] = tune_side(k, verbose=verbose)
    _save(cache, path)
    if verbose:
        print(f"  tuned {len(sides)} sizes in {time.time() - t0:.1f} s -> {path}", flush=True)
    return cache


def lookup(m: int, n: int, path: str = CACHE) -> dict:
    """Options of the cached size nearest to m * n (empty when nothing is cached)."""
    cache = _load(path)
    if not cache:
        return {}
    def size(key):
        a, b = key.split("x")
        return int(a) * int(b)
    key = min(cache, key=lambda kk: abs(size(kk) - m * n))
    return dict(cache[key]["options"])


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--sides", type=int, nargs="+", default=[24, 40, 56, 72, 88, 96])
    ap.add_argument("--cache", default=CACHE)
    args = ap.parse_args(argv)
    tune(args.sides, args.cache)


if __name__ == "__main__":
    main()
