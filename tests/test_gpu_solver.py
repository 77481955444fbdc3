"""End-to-end parity of the CUDA solver with the oracle: optimal value against the exact optimum
(oracle network simplex), marginal residual, certificate, and one outer iteration from an
identical state against the oracle's plain rendition of the iteration."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import costs, ipm, netsimplex
from paper_2206_11009_gb300 import synth
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _solve(inst, k, **opts):
    from paper_2206_11009_gb300 import Solver
    with Solver(inst.a, inst.b, grid=(k, k), **opts) as s:
        r = s.solve(raise_on_error=False)
        I, J, P, u, v = s.solution()
    return r, (I, J, P, u, v)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("k,seed,spike", [(8, 0, 0.0), (8, 2, 0.0), (16, 0, 0.0), (16, 3, 0.0), (16, 0, 0.05),
                                          (32, 1, 0.0), (32, 0, 0.05)])
def test_solve_reaches_exact_optimum(precision, k, seed, spike):
    """Config 1 style (tol 1e-8): |obj - OPT| / OPT <= 1e-6 and ||f - A p||_1 <= 1e-8."""
    inst = synth.image_pair(k, seed, spike_frac=spike)
    opt = U.opt_value(k, seed, spike)
    r, (I, J, P, u, v) = _solve(inst, k, tol=1e-8, precision=precision)
    assert r.status == 0, r
    assert abs(r.obj - opt) <= 1e-6 * opt
    assert r.r1_l1 <= 1e-8
    # certified lower bound is a true lower bound, and the gap closes
    assert r.lower_bound <= opt * (1 + 1e-12) and r.rel_gap <= 1e-8
    # returned coupling: nonnegative, marginals within the residual, cost consistent
    c = costs.square_grid(k)
    assert P.min() > 0
    assert abs(c.pairs(I, J) @ P - r.obj) <= 1e-12 * max(1.0, r.obj)
    ra = inst.a - np.bincount(I, weights=P, minlength=k * k)
    rb = inst.b * (inst.a.sum() / inst.b.sum()) - np.bincount(J, weights=P, minlength=k * k)
    assert np.abs(ra).sum() + np.abs(rb).sum() <= 1e-8 * (1 + 1e-6)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("k,seed", [(16, 0), (16, 3), (32, 1)])
def test_papers_new_pair_rule_reaches_exact_optimum(precision, k, seed):
    """Section 3.2's rule for new pairs (p = s = sqrt(mu), new_col_rule 0) end to end."""
    inst = synth.image_pair(k, seed)
    opt = U.opt_value(k, seed)
    r, _ = _solve(inst, k, tol=1e-8, precision=precision, new_col_rule=0)
    assert r.status == 0, r
    assert abs(r.obj - opt) <= 1e-6 * opt
    assert r.r1_l1 <= 1e-8 and r.rel_gap <= 1e-8


@pytest.mark.parametrize("precision", [0, 1])
def test_config2_64x64(precision):
    """64x64 image pair (16.8M variables) at tol 1e-6, both precisions, against the exact optimum."""
    k = 64
    inst = synth.image_pair(k, 0)
    opt = U.opt_value(k, 0)
    r, _ = _solve(inst, k, tol=1e-6, precision=precision)
    assert r.status == 0, r
    assert abs(r.obj - opt) <= 1e-6 * opt
    assert r.r1_l1 <= 1e-8
    if precision == 1:
        # the FP32 dense factor preconditions every solve well enough that no iteration needs the
        # FP64 factorisation and the refinement CG stays short (a few iterations per solve)
        assert r.direct_iters == 0
        assert r.cg_iters <= 60 * r.iters


@pytest.mark.parametrize("rule", [1, 0])
def test_one_iteration_matches_oracle(rule):
    """From the oracle's iterate after a few iterations, one GPU iteration (tight CG tolerance)
    reproduces mu, the stopping measure, the step lengths, sigma, the new duals and the new support.
    rule 0 is Section 3.2's p = s = sqrt(mu) for new pairs, rule 1 the capped variant."""
    from paper_2206_11009_gb300 import Solver
    k = 10
    inst = synth.image_pair(k, 1)
    c = costs.square_grid(k)
    opt = ipm.Options(tol=1e-8, new_col_rule=rule)
    prob = ipm.Problem(c, inst.a, inst.b)
    I, J = ipm.initial_support(prob, opt)
    st = ipm.initial_point(prob, I, J)
    tr = ipm.Tracker()
    for it in range(4):
        _, res, _ = ipm.stop_test(prob, st, opt, tr)
        st, _, _, _, _ = ipm.one_iteration(prob, st, res, opt, tr, it)
    _, res, crit = ipm.stop_test(prob, st, opt, tr)
    new, lg, stepped, (aI, aJ, aD), rem = ipm.one_iteration(prob, st, res, opt, tr, 4)

    with Solver(inst.a, inst.b, grid=(k, k), tol=1e-8, precision=0, cg_tol_pred=1e-13, cg_tol_corr=1e-13,
                max_cg=20000, new_col_rule=rule) as s:
        assert abs(s.mass_scale - prob.sigma_f) <= 1e-15 * prob.sigma_f
        s.set_state(st.I, st.J, st.p, st.s, st.u, st.v, reset_mu0=True)
        info = s.step()
        gI, gJ, gP, gS, gu, gv = s.state()
    assert abs(info["mu"] - res.mu) <= 1e-12 * res.mu
    assert abs(info["crit"] - crit) <= 1e-10 * crit
    assert abs(info["alpha_p"] - lg.alpha_p) <= 1e-7 and abs(info["alpha_s"] - lg.alpha_s) <= 1e-7
    assert abs(info["sigma"] - lg.sigma) <= 1e-7 * max(lg.sigma, 1e-3)
    assert info["ncorr"] == lg.ncorr and info["added"] == lg.added and info["removed"] == lg.removed
    scale = max(1.0, np.abs(new.u).max())
    assert np.abs(gu - new.u).max() <= 1e-7 * scale and np.abs(gv - new.v).max() <= 1e-7 * scale
    assert np.array_equal(gI, new.I) and np.array_equal(gJ, new.J)
    assert np.allclose(gP, new.p, rtol=1e-7, atol=1e-12) and np.allclose(gS, new.s, rtol=1e-7, atol=1e-12)


def test_solution_buffer_and_state_errors():
    from paper_2206_11009_gb300 import Solver, _lib
    k = 6
    inst = synth.image_pair(k, 0)
    with Solver(inst.a, inst.b, grid=(k, k)) as s:
        import ctypes
        nnz = ctypes.c_int64(0)
        code = s._lib.ot_ipm_get_solution(s.h, None, None, None, 0, ctypes.byref(nnz), None, None)
        assert code == _lib.OT_ERR_BUF_TOO_SMALL and nnz.value > 0
        I, J, P, S, u, v = s.state()
        with pytest.raises(_lib.OTError):
            s.set_state(I[::-1], J[::-1], P, S, u, v)        # not sorted
        with pytest.raises(_lib.OTError):
            s.set_state(I, J, -P, S, u, v)                   # nonpositive p
        s.set_state(I, J, P, S, u, v)                        # the state itself is accepted


def test_unbalanced_marginals_rejected():
    from paper_2206_11009_gb300 import Solver, _lib
    a = np.full(16, 1 / 16)
    b = np.full(16, 1 / 15)
    with pytest.raises(_lib.OTError) as e:
        Solver(a, b, grid=(4, 4))
    assert e.value.code == _lib.OT_ERR_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("k,seed,spike,prec", [(128, 0, 0.05, 1), (93, 14, 0.0, 1), (93, 14, 0.0, 0)])
def test_large_grids_certified_by_oracle(k, seed, spike, prec):
    """Grids above the FP64 dense size (n > 8192): the late iterations precondition with the FP32
    dense factor.  Pinned by the oracle's certificate: the c-transform bound LB = a.u~ + b.v
    (computed on the CPU from the returned v) <= OPT <= c.p, with the gap within 1e-6 and the
    marginal residual within 1e-8 (caller units)."""
    from oracle.certificate import c_transform_lower_bound, marginal_residual_l1
    from oracle.costs import square_grid
    from paper_2206_11009_gb300 import Solver, synth
    inst = synth.image_pair(k, seed, spike)
    with Solver(inst.a, inst.b, grid=(k, k), precision=prec) as s:
        r = s.solve()
        I, J, P, u, v = s.solution()
    cost = square_grid(k)
    lb = c_transform_lower_bound(cost, inst.a, inst.b, v)
    ctp = float(cost.pairs(I, J) @ P)
    assert r.status == 0
    assert marginal_residual_l1(k * k, k * k, I, J, P, inst.a, inst.b) <= 1e-8
    assert lb <= ctp * (1 + 1e-12)
    assert (ctp - lb) / ctp <= 1e-6
    assert abs(r.obj - ctp) <= 1e-9 * ctp


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("k,seed", [(16, 0), (32, 1)])
def test_incomplete_cholesky_preconditioner_reaches_exact_optimum(precision, k, seed):
    """The paper's iterative phase: CG preconditioned by the incomplete Cholesky factor with a
    drop tolerance (Section 4.2), then the direct branch near optimality (Section 4.3)."""
    inst = synth.image_pair(k, seed)
    opt = U.opt_value(k, seed)
    r, _ = _solve(inst, k, tol=1e-8, precision=precision, precond=1)
    assert r.status == 0, r
    assert abs(r.obj - opt) <= 1e-6 * opt and r.r1_l1 <= 1e-8 and r.rel_gap <= 1e-8


def test_tensor_core_factor_update_solve_93x93():
    """A full solve whose late iterations factor S_M (n = 8649) with the tensor-core bulk update:
    certified by the oracle's c-transform bound like the SIMT path."""
    from oracle.certificate import c_transform_lower_bound
    from oracle.costs import square_grid
    from paper_2206_11009_gb300 import Solver
    k = 93
    inst = synth.image_pair(k, 14)
    with Solver(inst.a, inst.b, grid=(k, k), precision=1, tc_update=1) as s:
        r = s.solve()
        I, J, P, u, v = s.solution()
    cost = square_grid(k)
    lb = c_transform_lower_bound(cost, inst.a, inst.b, v)
    ctp = float(cost.pairs(I, J) @ P)
    assert r.status == 0 and r.direct_iters > 0
    assert lb <= ctp * (1 + 1e-12) and (ctp - lb) / ctp <= 1e-6
