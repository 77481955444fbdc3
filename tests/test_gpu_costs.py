"""Pricing and solves for the distances of Section 5.1 (L1, Euclidean, L-infinity), an explicit
cost matrix, the heuristic pricing set J of Section 3.4, and an explicit scan tile height: the CUDA
path against the oracle's exact selection rule (bit for bit) and against the exact optimum of the
oracle network simplex."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import costs, netsimplex, pricing
from paper_2206_11009_gb300 import synth
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

KINDS = ["euclid", "l1", "linf"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _price(kind, sx, sy, tx, ty, u, v, si, sj, kmax, precision, **kw):
    from paper_2206_11009_gb300 import price_topk
    T = U.cuda_tensors(sx, sy, tx, ty, u, v, si, sj)
    gi, gj, gd = price_topk(*T, kmax=kmax, precision=precision, cost=kind, **kw)
    return gi.cpu().numpy(), gj.cpu().numpy(), gd.cpu().numpy()


def _check(kind, sx, sy, tx, ty, u, v, si, sj, kmax, precision, cmax=None, **kw):
    gi, gj, gd = _price(kind, sx, sy, tx, ty, u, v, si, sj, kmax, precision,
                        jset_cmax=cmax if cmax else 0.0, **kw)
    c = costs.Cost.points(sx, sy, tx, ty, kind)
    oi, oj, od = pricing.select(c, u, v, si.astype(np.int64), sj.astype(np.int64), kmax, cmax=cmax)
    assert len(gi) == len(oi)
    assert np.array_equal(gi, oi) and np.array_equal(gj, oj)
    assert np.array_equal(gd, od)          # bit-exact float64 reduced costs
    return len(oi)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("shape", [((13, 11), (9, 17), (-3, 5)), ((37, 29), (31, 41), (100, -50)),
                                   ((1, 1), (1, 7), (0, 0)), ((80, 70), (75, 66), (-200, 300))])
@pytest.mark.parametrize("kmax_mode", ["one", "m", "huge"])
def test_other_costs_selection_bit_exact(precision, kind, shape, kmax_mode):
    """Several tiles, ragged edges, shifted coordinates; the FP32 direct-form scan (with its own
    proven error window) and the FP64 scan select the oracle's set."""
    (ws, hs), (wt, ht), (x0, y0) = shape
    sx, sy = U.rect_coords(ws, hs, x0, y0)
    tx, ty = U.rect_coords(wt, ht, x0 + 2, y0 - 1)
    m, n = len(sx), len(tx)
    amp = {"euclid": 0.6, "l1": 0.8, "linf": 0.5}[kind]
    u, v = U.banded_duals(sx, sy, tx, ty, seed=ws * 7 + wt, amp=amp, noise=0.7)
    si, sj = U.random_support(m, n, 0.05, seed=m + n)
    kmax = {"one": 1, "m": m, "huge": m * n}[kmax_mode]
    _check(kind, sx, sy, tx, ty, u, v, si, sj, kmax, precision)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kind", KINDS)
def test_other_costs_exact_ties(precision, kind):
    """Integer costs and integer duals: many exactly equal reduced costs, ordered by jlin."""
    sx, sy = U.rect_coords(12, 12)
    u = np.floor(U.banded_duals(sx, sy, sx, sy, 3, 0.7, 0.0)[0])
    v = -u + 1.0
    assert _check(kind, sx, sy, sx, sy, u, v, np.zeros(0, np.int32), np.zeros(0, np.int32), 100, precision) == 100


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kind,cmax", [("sqeuclid", 10.0), ("sqeuclid", 37.5), ("euclid", 3.2), ("euclid", 5.0),
                                       ("l1", 4.0), ("linf", 2.5)])
def test_jset_selection_bit_exact(precision, kind, cmax):
    """Section 3.4's J = {c_ij < C_max}: the listed-pair scan selects the oracle's restricted set,
    including C_max exactly on a cost value (5.0 = sqrt(25), 4 for L1)."""
    sx, sy = U.rect_coords(45, 38, 3, -2)
    tx, ty = U.rect_coords(41, 40, 5, -4)
    m, n = len(sx), len(tx)
    amp = 4.0 if kind == "sqeuclid" else 0.6
    u, v = U.banded_duals(sx, sy, tx, ty, seed=11, amp=amp, noise=1.0)
    si, sj = U.random_support(m, n, 0.02, seed=5)
    for kmax in (1, m, m * n):
        _check(kind, sx, sy, tx, ty, u, v, si, sj, kmax, precision, cmax=cmax)


@pytest.mark.parametrize("precision", [0, 1])
def test_jset_empty_and_full(precision):
    sx, sy = U.rect_coords(20, 20)
    tx, ty = U.rect_coords(20, 20, 100, 0)            # every cost >= 81^2
    u, v = U.banded_duals(sx, sy, tx, ty, seed=2, amp=3.0, noise=1.0)
    v = v + 20000.0                                    # every reduced cost negative
    si = np.zeros(0, np.int32)
    # C_max below every cost: J is empty
    assert _check("sqeuclid", sx, sy, tx, ty, u, v, si, si, 400, precision, cmax=50.0) == 0
    # C_max above every cost: same as the full scan
    full = _price("sqeuclid", sx, sy, tx, ty, u, v, si, si, 400, precision)
    capped = _price("sqeuclid", sx, sy, tx, ty, u, v, si, si, 400, precision, jset_cmax=1e6)
    assert len(full[0]) == 400
    assert all(np.array_equal(x, y) for x, y in zip(full, capped))


@pytest.mark.parametrize("precision", [0, 1])
def test_dense_cost_selection_bit_exact(precision):
    """An explicit m x n cost matrix (always scanned in FP64), with and without J."""
    import torch
    from paper_2206_11009_gb300 import price_topk
    m, n = 70, 2500                      # two column tiles of 2048, the second ragged
    C = synth.random_int_costs(m, n, 9, hi=40).astype(np.float64) + 0.25
    rng = synth.uniform01(31, m + n)
    u, v = rng[:m] * 20, rng[m:] * 20
    si, sj = U.random_support(m, n, 0.1, seed=4)
    dev = torch.device("cuda:0")
    Cd = torch.as_tensor(C, device=dev)
    uu, vv, ssi, ssj = U.cuda_tensors(u, v, si, sj)
    for cmax in (None, 15.0):
        for kmax in (1, m, m * n):
            gi, gj, gd = price_topk(None, None, None, None, uu, vv, ssi, ssj, kmax=kmax, precision=precision, C=Cd,
                                    jset_cmax=cmax or 0.0)
            oi, oj, od = pricing.select(costs.Cost.dense(C), u, v, si.astype(np.int64), sj.astype(np.int64), kmax,
                                        cmax=cmax)
            assert np.array_equal(gi.cpu().numpy(), oi) and np.array_equal(gj.cpu().numpy(), oj)
            assert np.array_equal(gd.cpu().numpy(), od)


@pytest.mark.parametrize("rows", [256, 8, 40])
def test_scan_tile_height_128x128(rows):
    """The 128x128 pair (268M pairs) with the tile height forced: 256 rows is the shape the
    256x256 bench measures, 8 the smallest, 40 a non-power of two."""
    k = 128
    sx, sy = U.rect_coords(k, k)
    u, v = U.banded_duals(sx, sy, sx, sy, seed=k, amp=6.0, noise=2.0)
    si, sj = U.neighbourhood_support(sx, sy, sx, sy)
    assert _check("sqeuclid", sx, sy, sx, sy, u, v, si, sj, k * k, 1, scan_rows=rows) == k * k


# --------------------------------------------------------------------------------- solves

def _opt(cost, a, b):
    return netsimplex.solve(cost, a, b).obj


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("k,seed", [(12, 3), (16, 0)])
def test_other_costs_reach_exact_optimum(precision, kind, k, seed):
    from paper_2206_11009_gb300 import Solver
    inst = synth.image_pair(k, seed)
    opt = _opt(costs.square_grid(k, kind), inst.a, inst.b)
    with Solver(inst.a, inst.b, grid=(k, k), cost=kind, tol=1e-8, precision=precision) as s:
        r = s.solve(raise_on_error=False)
    assert r.status == 0, r
    assert abs(r.obj - opt) <= 1e-6 * opt and r.r1_l1 <= 1e-8 and r.rel_gap <= 1e-8


@pytest.mark.parametrize("precision", [0, 1])
def test_dense_cost_reaches_exact_optimum(precision):
    from paper_2206_11009_gb300 import Solver
    m, n = 40, 55
    C = synth.random_int_costs(m, n, 21, hi=30).astype(np.float64)
    a, b = synth.random_masses(m, 22), synth.random_masses(n, 23)
    opt = _opt(costs.Cost.dense(C), a, b)
    with Solver(a, b, C=C, tol=1e-8, precision=precision, init_cost=3.0) as s:
        r = s.solve(raise_on_error=False)
        I, J, P, u, v = s.solution()
    assert r.status == 0, r
    assert abs(r.obj - opt) <= 1e-6 * max(opt, 1.0) and r.r1_l1 <= 1e-8
    assert abs(C[I, J] @ P - r.obj) <= 1e-12 * max(1.0, r.obj)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kind,cmax", [("sqeuclid", 9.0), ("euclid", 3.0), ("l1", 4.0)])
def test_jset_solve_reaches_exact_optimum(precision, kind, cmax):
    """Pricing on J with a full refresh every 3rd iteration (Section 3.4)."""
    from paper_2206_11009_gb300 import Solver
    k = 16
    inst = synth.image_pair(k, 0)
    opt = _opt(costs.square_grid(k, kind), inst.a, inst.b)
    with Solver(inst.a, inst.b, grid=(k, k), cost=kind, tol=1e-8, precision=precision, jset_cmax=cmax) as s:
        r = s.solve(raise_on_error=False)
    assert r.status == 0, r
    assert abs(r.obj - opt) <= 1e-6 * opt and r.r1_l1 <= 1e-8


def test_one_iteration_with_jset_matches_oracle():
    """One GPU iteration that prices on J (iteration index 0: not a refresh) from the oracle's
    starting point reproduces the oracle's new support."""
    from oracle import ipm
    from paper_2206_11009_gb300 import Solver
    k = 10
    inst = synth.image_pair(k, 1)
    opt = ipm.Options(tol=1e-8, jset_cmax=5.0)
    prob = ipm.Problem(costs.square_grid(k), inst.a, inst.b)
    I, J = ipm.initial_support(prob, opt)
    st = ipm.initial_point(prob, I, J)
    tr = ipm.Tracker()
    _, res, _ = ipm.stop_test(prob, st, opt, tr)
    new, lg, _, (aI, aJ, _), _ = ipm.one_iteration(prob, st, res, opt, tr, 0)
    c = costs.square_grid(k)
    assert np.all(c.pairs(aI, aJ) < 5.0) and len(aI) > 0
    with Solver(inst.a, inst.b, grid=(k, k), tol=1e-8, precision=0, cg_tol_pred=1e-13, cg_tol_corr=1e-13,
                max_cg=20000, jset_cmax=5.0) as s:
        s.set_state(st.I, st.J, st.p, st.s, st.u, st.v, reset_mu0=True)
        info = s.step()
        gI, gJ, *_ = s.state()
    assert info["added"] == lg.added
    assert np.array_equal(gI, new.I) and np.array_equal(gJ, new.J)
