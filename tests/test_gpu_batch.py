"""Batched solve (many uneven instances through one work queue) and the autotuner."""
import json

import numpy as np
import pytest


@pytest.mark.gpu
def test_batch_matches_individual_solves():
    from paper_2206_11009_gb300 import Solver, synth
    from paper_2206_11009_gb300.api import solve_batch
    sides = synth.batch_sides(12, 12, 28, seed=99)
    pairs = []
    for s, k in enumerate(sides):
        inst = synth.image_pair(int(k), 500 + s)
        pairs.append((inst.a, inst.b, int(k)))
    res = solve_batch(pairs, workers=4)
    assert len(res) == len(pairs)
    for (a, b, k), r in zip(pairs, res):
        assert r.status == 0
        with Solver(a, b, grid=(k, k)) as s:
            one = s.solve()
        # same deterministic path: identical iteration counts and objective
        assert r.iters == one.iters
        assert abs(r.obj - one.obj) <= 1e-12 * abs(one.obj)


def test_batch_rejects_bad_arguments():
    from paper_2206_11009_gb300 import _lib
    lib = _lib.load()
    assert lib.ot_ipm_solve_batch(None, 1, None, 1) == _lib.OT_ERR_ARG


@pytest.mark.gpu
def test_autotune_cache_roundtrip(tmp_path):
    from paper_2206_11009_gb300 import autotune
    path = str(tmp_path / "tune.json")
    autotune._cache_mem = None
    cache = autotune.tune([16], path=path, verbose=False)
    entry = cache["256x256"]
    assert entry["options"] in autotune.candidates(256)
    assert entry["seconds"] == min(g["seconds"] for g in entry["grid"])
    assert json.load(open(path)) == cache
    assert autotune.lookup(300, 300, path=path) == entry["options"]
    autotune._cache_mem = None
