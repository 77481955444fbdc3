"""Input handling of the C ABI: zero masses (presolve), non-square and different grids (m != n),
general point clouds, and inputs given as device pointers -- each solved on the GPU and checked
against the exact optimum of the oracle network simplex and the LP certificate."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import certificate, costs, netsimplex
from paper_2206_11009_gb300 import synth
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _zero_some(x, frac, seed):
    x = x.copy()
    x[synth.uniform01(seed, len(x)) < frac] = 0.0
    return x / x.sum()


def _check_solution(cost, a, b, r, sol, opt, tol=1e-6):
    I, J, P, u, v = sol
    assert r.status == 0, r
    assert abs(r.obj - opt) <= tol * opt
    assert certificate.marginal_residual_l1(cost.m, cost.n, I, J, P, a, b * (a.sum() / b.sum())) <= 1e-8 * (1 + 1e-6)
    assert abs(cost.pairs(I, J) @ P - r.obj) <= 1e-12 * max(1.0, r.obj)
    # returned duals (including the completed ones of removed points): lower bound within the gap
    lb = certificate.c_transform_lower_bound(cost, a, b, v)
    assert lb <= opt * (1 + 1e-12) and (opt - lb) <= 2 * tol * opt
    assert certificate.min_reduced_cost(cost, u, v) >= -tol * (1 + cost.max_cost())


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("k,frac,kind", [(12, 0.2, "sqeuclid"), (16, 0.3, "sqeuclid"), (16, 0.15, "l1"),
                                         (32, 0.1, "sqeuclid")])
def test_zero_masses_presolved(precision, k, frac, kind):
    """Images with zero pixels (the DOTmark images have them): the presolve removes them, the
    solve reaches the exact optimum, and the coupling and duals come back in the caller's indices
    (no flow on zero-mass points, completed duals dual feasible)."""
    from paper_2206_11009_gb300 import Solver
    inst = synth.image_pair(k, 7)
    a, b = _zero_some(inst.a, frac, 100 + k), _zero_some(inst.b, frac, 200 + k)
    assert (a == 0).sum() > 0 and (b == 0).sum() > 0
    cost = costs.square_grid(k, kind)
    opt = netsimplex.solve(cost, a, b).obj
    with Solver(a, b, grid=(k, k), cost=kind, tol=1e-8, precision=precision) as s:
        r = s.solve(raise_on_error=False)
        sol = s.solution()
        I, J, P, S, u, v = s.state()
    _check_solution(cost, a, b, r, sol, opt, tol=1e-6)
    assert np.all(a[sol[0]] > 0) and np.all(b[sol[1]] > 0)
    assert len(u) == k * k and np.all(u[a == 0] == 0.0)   # state: removed points read 0


def test_zero_masses_state_round_trip():
    """get_state / set_state speak in the caller's indices under the presolve; a pair on a
    zero-mass point is rejected."""
    from paper_2206_11009_gb300 import Solver, _lib
    k = 10
    inst = synth.image_pair(k, 2)
    a, b = _zero_some(inst.a, 0.25, 5), _zero_some(inst.b, 0.25, 6)
    with Solver(a, b, grid=(k, k), tol=1e-8) as s:
        s.step()
        I, J, P, S, u, v = s.state()
        s.set_state(I, J, P, S, u, v)
        I2, J2, P2, S2, *_ = s.state()
        assert np.array_equal(I, I2) and np.array_equal(J, J2) and np.array_equal(P, P2)
        zi = int(np.nonzero(a == 0)[0][0])
        bad_I = np.concatenate([I, [zi]])
        bad_J = np.concatenate([J, [0]])
        o = np.lexsort((bad_J, bad_I))
        with pytest.raises(_lib.OTError):
            s.set_state(bad_I[o], bad_J[o], np.ones(len(o)), np.ones(len(o)), u, v)
        r = s.solve(raise_on_error=False)
        assert r.status == 0


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("src,dst", [((12, 16), (16, 10)), ((20, 7), (9, 9)), ((1, 30), (5, 9))])
def test_non_square_and_different_grids(precision, src, dst):
    """m != n: a w1 x h1 source image against a w2 x h2 target image (Section 2's general m, n)."""
    from paper_2206_11009_gb300 import Solver
    (w1, h1), (w2, h2) = src, dst
    m, n = w1 * h1, w2 * h2
    a = synth.random_masses(m, 40 + m)
    b = synth.random_masses(n, 50 + n)
    sx, sy = U.rect_coords(w1, h1)
    tx, ty = U.rect_coords(w2, h2, 3, -1)
    cost = costs.Cost.points(sx, sy, tx, ty)
    opt = netsimplex.solve(cost, a, b).obj
    with Solver(a, b, coords=(sx, sy, tx, ty), tol=1e-8, precision=precision) as s:
        r = s.solve(raise_on_error=False)
        sol = s.solution()
    _check_solution(cost, a, b, r, sol, opt)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kind", ["sqeuclid", "euclid"])
def test_point_clouds(precision, kind):
    """General point sets with explicit integer coordinates (repeated points included)."""
    from paper_2206_11009_gb300 import Solver
    m, n = 150, 220
    r0 = synth.uniform01(808, 2 * (m + n))
    sx = np.floor(r0[:m] * 40).astype(np.int32) - 20
    sy = np.floor(r0[m:2 * m] * 25).astype(np.int32)
    tx = np.floor(r0[2 * m:2 * m + n] * 35).astype(np.int32) - 10
    ty = np.floor(r0[2 * m + n:] * 30).astype(np.int32) - 5
    a = synth.random_masses(m, 9)
    b = synth.random_masses(n, 10)
    cost = costs.Cost.points(sx, sy, tx, ty, kind)
    opt = netsimplex.solve(cost, a, b).obj
    with Solver(a, b, coords=(sx, sy, tx, ty), cost=kind, tol=1e-8, precision=precision, init_cost=8.0) as s:
        r = s.solve(raise_on_error=False)
        sol = s.solution()
    _check_solution(cost, a, b, r, sol, opt)


@pytest.mark.parametrize("with_zeros", [False, True])
def test_inputs_on_device(with_zeros):
    """ot_problem.inputs_on_device: masses and coordinates given as device pointers give the same
    solve as host inputs."""
    import torch
    from paper_2206_11009_gb300 import Solver
    k = 16
    inst = synth.image_pair(k, 3)
    a, b = inst.a, inst.b
    if with_zeros:
        a, b = _zero_some(a, 0.2, 1), _zero_some(b, 0.2, 2)
    sx, sy = U.rect_coords(k, k)
    with Solver(a, b, coords=(sx, sy, sx, sy), tol=1e-8) as s:
        rh = s.solve()
        Ih, Jh, Ph, uh, vh = s.solution()
    dev = torch.device("cuda:0")
    D = lambda x: torch.as_tensor(np.ascontiguousarray(x), device=dev)
    with Solver(D(a), D(b), coords=(D(sx), D(sy), D(sx), D(sy)), tol=1e-8) as s:
        rd = s.solve()
        Id, Jd, Pd, ud, vd = s.solution()
    cost = costs.Cost.points(sx, sy, sx, sy)
    opt = netsimplex.solve(cost, a, b).obj
    assert rh.status == 0 and rd.status == 0
    assert abs(rd.obj - opt) <= 1e-6 * opt and abs(rh.obj - opt) <= 1e-6 * opt
    assert abs(rd.obj - rh.obj) <= 1e-9 * opt
    _check_solution(cost, a, b, rd, (Id, Jd, Pd, ud, vd), opt)


def test_dense_cost_on_device_with_zero_masses():
    import torch
    from paper_2206_11009_gb300 import Solver
    m, n = 30, 44
    C = synth.random_int_costs(m, n, 61, hi=25).astype(np.float64)
    a = _zero_some(synth.random_masses(m, 62), 0.2, 63)
    b = _zero_some(synth.random_masses(n, 64), 0.2, 65)
    cost = costs.Cost.dense(C)
    opt = netsimplex.solve(cost, a, b).obj
    dev = torch.device("cuda:0")
    D = lambda x: torch.as_tensor(np.ascontiguousarray(x), device=dev)
    with Solver(D(a), D(b), C=D(C), tol=1e-8, init_cost=4.0) as s:
        r = s.solve(raise_on_error=False)
        sol = s.solution()
    _check_solution(cost, a, b, r, sol, opt)


def test_invalid_dense_cost_rejected():
    from paper_2206_11009_gb300 import Solver, _lib
    C = np.ones((4, 5))
    C[2, 3] = -1.0
    with pytest.raises(_lib.OTError) as e:
        Solver(np.full(4, 0.25), np.full(5, 0.2), C=C)
    assert e.value.code == _lib.OT_ERR_ARG
