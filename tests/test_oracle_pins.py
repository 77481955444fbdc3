"""Pins of the CPU oracle against facts fixed by the paper and by LP theory (no GPU).

Each test checks an oracle function against something other than itself: brute force,
closed forms, duality certificates, hand-computed fixtures, or invariants the paper states.
"""
from __future__ import annotations

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import brute, certificate, costs, ipm, netsimplex, pricing
from paper_2206_11009_gb300 import synth
from tests import goldens


# ----------------------------------------------------------------------------- generator

def test_splitmix64_known_answer():
    # first two outputs of SplitMix64 seeded with 0 (published reference values)
    z = synth.splitmix64(0, 2)
    assert int(z[0]) == 0xE220A8397B1DCDAF
    assert int(z[1]) == 0x6E789E6AA1B965F4


def test_grf_marginals_shape_and_mass():
    inst = synth.image_pair(16, 3)
    for x in (inst.a, inst.b):
        assert x.shape == (256,) and x.min() > 0 and abs(x.sum() - 1.0) < 1e-14
    assert np.array_equal(inst.a, synth.image_pair(16, 3).a)
    spiky = synth.grf_image(32, 7, spike_frac=0.05)
    assert abs(spiky.sum() - 1) < 1e-14 and spiky.max() > 5 * np.median(spiky)


# ----------------------------------------------------------------------------- O1 vs O3

@pytest.mark.parametrize("m,n,seed", [(2, 3, 0), (3, 3, 1), (3, 4, 2), (4, 3, 3), (4, 4, 4), (4, 4, 5)])
def test_netsimplex_matches_vertex_enumeration(m, n, seed):
    C = synth.random_int_costs(m, n, seed)
    a = synth.random_masses(m, 100 + seed)
    b = synth.random_masses(n, 200 + seed)
    r = netsimplex.solve(costs.Cost.dense(C), a, b)
    ve, P = brute.vertex_enumeration(C, a, b)
    assert abs(r.obj - ve) <= 1e-12 * max(1.0, abs(ve))


@pytest.mark.parametrize("n,seed", [(5, 0), (6, 1), (7, 2)])
def test_netsimplex_matches_assignment(n, seed):
    C = synth.random_int_costs(n, n, 50 + seed, hi=50)
    a = np.full(n, 1.0 / n)
    r = netsimplex.solve(costs.Cost.dense(C), a, a)
    assert abs(r.obj - brute.assignment(C)) <= 1e-12


@pytest.mark.parametrize("kind", ["sqeuclid", "l1", "euclid"])
def test_netsimplex_matches_monotone_coupling_1d(kind):
    k = 60
    c = costs.line_grid(k, kind)
    a = synth.random_masses(k, 11)
    b = synth.random_masses(k, 12)
    f = {"sqeuclid": lambda d: d * d, "l1": abs, "euclid": abs}[kind]
    r = netsimplex.solve(c, a, b)
    assert abs(r.obj - brute.monotone_1d(c.sx, a, c.tx, b, f)) <= 1e-12


@pytest.mark.parametrize("k,seed", [(8, 0), (12, 1), (16, 2)])
def test_netsimplex_lp_certificate(k, seed):
    inst = synth.image_pair(k, seed)
    c = costs.square_grid(k)
    r = netsimplex.solve(c, inst.a, inst.b)
    # dual feasibility over all m*n pairs (exact integers for this cost)
    assert certificate.min_reduced_cost(c, r.u, r.v) >= 0.0
    # zero duality gap
    assert abs(inst.a @ r.u + inst.b @ r.v - r.obj) <= 1e-12 * r.obj
    # primal feasibility, at most m+n-1 nonzeros on an acyclic support (Section 2.2)
    assert certificate.marginal_residual_l1(k * k, k * k, r.I, r.J, r.P, inst.a, inst.b) <= 1e-13
    assert r.P.min() >= 0.0 and len(r.I) <= 2 * k * k - 1
    assert certificate.is_forest(k * k, k * k, r.I, r.J)
    # complementary slackness on the tree
    d = c.pairs(r.I, r.J) - r.u[r.I] - r.v[r.J]
    assert np.all(d == 0.0)


def test_netsimplex_symmetries():
    k = 10
    inst = synth.image_pair(k, 4)
    c = costs.square_grid(k)
    base = netsimplex.solve(c, inst.a, inst.b).obj
    # a = b: the identity coupling costs 0
    assert netsimplex.solve(c, inst.a, inst.a).obj == 0.0
    # swapping source and target
    assert abs(netsimplex.solve(c, inst.b, inst.a).obj - base) <= 1e-12 * base
    # flipping both images left-right / transposing both
    fl = lambda x: x.reshape(k, k)[:, ::-1].reshape(-1)
    tr = lambda x: x.reshape(k, k).T.reshape(-1)
    assert abs(netsimplex.solve(c, fl(inst.a), fl(inst.b)).obj - base) <= 1e-12 * base
    assert abs(netsimplex.solve(c, tr(inst.a), tr(inst.b)).obj - base) <= 1e-12 * base
    # scaling the cost by lambda scales OPT by lambda
    C = c.full()
    assert abs(netsimplex.solve(costs.Cost.dense(3.0 * C), inst.a, inst.b).obj - 3.0 * base) <= 1e-11 * base


# ----------------------------------------------------------------------------- pricing rule

@pytest.mark.parametrize("case", goldens.pricing_cases())
def test_pricing_golden(case):
    C = case["C"]
    sup = case["support"]
    I = np.array([p[0] for p in sup], dtype=np.int64)
    J = np.array([p[1] for p in sup], dtype=np.int64)
    sI, sJ, _ = pricing.select(costs.Cost.dense(C), case["u"], case["v"], I, J, case["kmax"])
    assert list(zip(sI.tolist(), sJ.tolist())) == case["expect"]
    assert pricing.select_bruteforce(C, case["u"], case["v"], set(sup), case["kmax"]) == case["expect"]


@pytest.mark.parametrize("seed", range(6))
def test_pricing_matches_bruteforce(seed):
    m, n = 7, 9
    C = synth.random_int_costs(m, n, seed, hi=6)
    rng = synth.uniform01(1000 + seed, m + n + m * n)
    u = np.round(rng[:m] * 4, 1)          # coarse duals: many exact ties
    v = np.round(rng[m:m + n] * 4, 1)
    sup_mask = rng[m + n:].reshape(m, n) < 0.3
    I, J = np.nonzero(sup_mask)
    for kmax in (1, 3, m, m * n):
        sI, sJ, sD = pricing.select(costs.Cost.dense(C), u, v, I, J, kmax)
        ref = pricing.select_bruteforce(C, u, v, set(zip(I.tolist(), J.tolist())), kmax)
        assert list(zip(sI.tolist(), sJ.tolist())) == ref
        assert np.all(sD < 0)


# ----------------------------------------------------------------------------- Newton step

def _small_state(k=5, seed=0):
    inst = synth.image_pair(k, seed)
    c = costs.square_grid(k)
    prob = ipm.Problem(c, inst.a, inst.b)
    I, J = ipm.initial_support(prob, ipm.Options())
    st = ipm.initial_point(prob, I, J)
    rng = synth.uniform01(77 + seed, 2 * len(I))
    st = ipm.State(I, J, st.p * (0.5 + rng[:len(I)]), st.s * (0.5 + rng[len(I):]), st.u + 0.1, st.v - 0.3)
    return prob, st


def test_schur_complement_invariants():
    prob, st = _small_state()
    m, n = prob.m, prob.n
    theta = st.p / st.s
    S, V, M, N, Minv = ipm.schur_matrix(m, n, st.I, st.J, theta)
    Vd = V.toarray()
    # eq. matrix_relations: V e = M e, V^T e = N e
    assert np.allclose(Vd.sum(1), M, rtol=1e-14) and np.allclose(Vd.sum(0), N, rtol=1e-14)
    # Schur complement against the dense block formula
    Sd = np.diag(N) - Vd.T @ np.diag(1.0 / M) @ Vd
    assert np.allclose(S.toarray(), Sd, rtol=1e-12, atol=1e-12 * np.abs(Sd).max())
    # eq. diagdom: S_M e = 0 and weak diagonal dominance
    Sd = S.toarray()
    assert np.abs(Sd.sum(1)).max() <= 1e-12 * np.abs(Sd).max()
    off = Sd - np.diag(np.diag(Sd))
    assert off.max() <= 0.0
    assert np.all(np.diag(Sd) - np.abs(off).sum(1) >= -1e-12 * np.abs(Sd).max())


def test_newton_direction_solves_reduced_system():
    """The Schur elimination must reproduce eq. redsystem's 3x3 block system exactly."""
    prob, st = _small_state()
    m, n = prob.m, prob.n
    res = ipm.residuals(prob, st)
    rng = synth.normal(5, len(st.p))
    r3 = 0.3 * res.mu - st.p * st.s + 0.01 * rng
    d = ipm.newton_direction(prob, st, res.r1a, res.r1b, res.r2, r3)
    A = brute.constraint_matrix(m, n)[:, st.I + st.J * m]        # A_red (column-major vec)
    r1 = np.concatenate([res.r1a, res.r1b])
    dy = np.concatenate([d.du, d.dv])
    scale = max(1.0, np.abs(r1).max(), np.abs(res.r2).max(), np.abs(r3).max())
    assert np.abs(A @ d.dp - r1).max() <= 1e-10 * scale
    assert np.abs(A.T @ dy + d.ds - res.r2).max() <= 1e-10 * scale
    assert np.abs(st.s * d.dp + st.p * d.ds - r3).max() <= 1e-10 * scale
    # same dp, ds as a dense least-squares solve of the full block system
    psi = len(st.p)
    K = np.zeros((m + n + 2 * psi, psi + m + n + psi))
    K[:m + n, :psi] = A
    K[m + n:m + n + psi, psi:psi + m + n] = A.T
    K[m + n:m + n + psi, psi + m + n:] = np.eye(psi)
    K[m + n + psi:, :psi] = np.diag(st.s)
    K[m + n + psi:, psi + m + n:] = np.diag(st.p)
    x, *_ = np.linalg.lstsq(K, np.concatenate([r1, res.r2, r3]), rcond=None)
    assert np.allclose(x[:psi], d.dp, rtol=1e-8, atol=1e-9 * np.abs(d.dp).max())
    assert np.allclose(x[psi + m + n:], d.ds, rtol=1e-8, atol=1e-9 * np.abs(d.ds).max())


def test_mehrotra_start_is_least_squares_feasible():
    inst = synth.image_pair(6, 2)
    prob = ipm.Problem(costs.square_grid(6), inst.a, inst.b)
    I, J = ipm.initial_support(prob, ipm.Options())
    st = ipm.initial_point(prob, I, J)
    assert st.p.min() > 0 and st.s.min() > 0
    # p~ = A^T y solves A p~ = f; the shift adds a constant to every entry, so
    # A p - f = shift * (row/col degrees): check through the degrees
    m = n = 36
    A = brute.constraint_matrix(m, n)[:, I + J * m]
    f = np.concatenate([prob.as_, prob.bs])
    resid = A @ st.p - f
    deg = A @ np.ones(len(I))
    shift = resid / deg
    assert np.allclose(shift, shift[0], rtol=1e-9, atol=1e-12)


def test_step_to_boundary_closed_form():
    x = np.array([1.0, 2.0, 4.0])
    dx = np.array([-2.0, 1.0, -1.0])
    assert ipm.step_to_boundary(x, dx, 0.995) == pytest.approx(0.995 * 0.5)
    assert ipm.step_to_boundary(x, np.abs(dx), 0.995) == 1.0


def test_removal_keeps_last_entry_of_each_row_and_column():
    inst = synth.image_pair(3, 0)
    prob = ipm.Problem(costs.square_grid(3), inst.a, inst.b)
    I = np.array([0, 0, 1, 2, 2], dtype=np.int64)
    J = np.array([0, 1, 1, 2, 0], dtype=np.int64)
    o = np.argsort(I * 9 + J)
    I, J = I[o], J[o]
    p = np.full(5, 1e-9)
    p[0] = 2e-9
    st = ipm.State(I, J, p, np.ones(5), np.zeros(9), np.zeros(9))
    rem = ipm.removal_select(prob, st, ipm.Options(), kmax=9)
    keep = np.ones(5, bool)
    keep[rem] = False
    for lab in (I, J):
        present = set(lab.tolist())
        assert present == set(lab[keep].tolist())


# ----------------------------------------------------------------------------- O2 vs O1

@pytest.mark.parametrize("rule", [1, 0])
@pytest.mark.parametrize("k,seed,spike", [(6, 0, 0.0), (8, 1, 0.0), (8, 2, 0.05), (12, 3, 0.0), (16, 0, 0.0)])
def test_ipm_oracle_reaches_exact_optimum(k, seed, spike, rule):
    """Both new-pair rules: rule 0 is Section 3.2's p = s = sqrt(mu); rule 1 caps the flow."""
    inst = synth.image_pair(k, seed, spike_frac=spike)
    c = costs.square_grid(k)
    ref = netsimplex.solve(c, inst.a, inst.b)
    r = ipm.solve(c, inst.a, inst.b, ipm.Options(tol=1e-8, new_col_rule=rule))
    assert r.status == "optimal"
    assert abs(r.obj - ref.obj) <= 1e-7 * ref.obj
    assert r.r1_l1 <= 1e-8
    assert r.lb <= ref.obj * (1 + 1e-12) and r.gap <= 1e-8


def test_new_pairs_enter_at_sqrt_mu_under_the_papers_rule():
    """Section 3.2: a pair added by pricing starts at p = s = sqrt(mu); rule 1 keeps p s = mu
    with p capped at min(a_i, b_j)."""
    k = 8
    inst = synth.image_pair(k, 1)
    c = costs.square_grid(k)
    prob = ipm.Problem(c, inst.a, inst.b)
    I, J = ipm.initial_support(prob, ipm.Options())
    st0 = ipm.initial_point(prob, I, J)
    for rule in (0, 1):
        opt = ipm.Options(new_col_rule=rule)
        tr = ipm.Tracker()
        _, res, _ = ipm.stop_test(prob, st0, opt, tr)
        st1, lg, stepped, (aI, aJ, _), rem = ipm.one_iteration(prob, st0, res, opt, tr)
        assert len(aI) > 0 and len(rem) == 0
        mu_new = float(stepped.p @ stepped.s) / len(stepped.p)
        key = st1.I * (k * k) + st1.J
        pos = np.searchsorted(key, aI * (k * k) + aJ)
        p_new, s_new = st1.p[pos], st1.s[pos]
        r = np.sqrt(mu_new)
        if rule == 0:
            assert np.all(p_new == r) and np.all(s_new == r)
        else:
            cap = np.minimum(prob.as_[aI], prob.bs[aJ])
            assert np.allclose(p_new, np.minimum(r, cap), rtol=0, atol=0)
            assert np.allclose(p_new * s_new, mu_new, rtol=1e-14)


# ----------------------------------------------------------------------------- certificate

def test_min_reduced_cost_hand_fixture():
    """min over all pairs of (c_ij - u_i) - v_j, worked out by hand:
       C = [[4, 1, 3], [2, 5, 0]], u = (1, -2), v = (0, 3, -1)
       d = [[3, -3, 3], [4, 4, 3]]  ->  -3 at (0, 1)."""
    C = np.array([[4.0, 1.0, 3.0], [2.0, 5.0, 0.0]])
    u = np.array([1.0, -2.0])
    v = np.array([0.0, 3.0, -1.0])
    assert certificate.min_reduced_cost(costs.Cost.dense(C), u, v) == -3.0
    # dual feasible after the c-transform of v: u_i = min_j (c_ij - v_j) makes the minimum 0
    ubar = np.array([min(C[i, j] - v[j] for j in range(3)) for i in range(2)])
    assert certificate.min_reduced_cost(costs.Cost.dense(C), ubar, v) == 0.0


def test_c_transform_lower_bound_hand_fixture():
    """a^T u + b^T v with u the c-transform of v, worked out by hand:
       C = [[4, 1, 3], [2, 5, 0]], a = (0.4, 0.6), b = (0.2, 0.3, 0.5), v = (0, 3, -1)
       u = (min(4, -2, 4), min(2, 2, 1)) = (-2, 1); a^T u = -0.2, b^T v = 0.4  ->  0.2,
       below the optimum 0.9 (row 1: 0.5 to column 2 at 0 and 0.1 to column 0 at 2; row 0: 0.3 to
       column 1 at 1 and 0.1 to column 0 at 4)."""
    C = np.array([[4.0, 1.0, 3.0], [2.0, 5.0, 0.0]])
    a, b = np.array([0.4, 0.6]), np.array([0.2, 0.3, 0.5])
    v = np.array([0.0, 3.0, -1.0])
    lb = certificate.c_transform_lower_bound(costs.Cost.dense(C), a, b, v)
    assert abs(lb - 0.2) <= 1e-15
    r = netsimplex.solve(costs.Cost.dense(C), a, b)
    assert abs(r.obj - 0.9) <= 1e-15 and lb <= r.obj


def test_forest_test_and_marginal_residual_hand_fixtures():
    """The bipartite graph rows {0, 1} x columns {0, 1}: the path 0-0', 0-1', 1-1' is a tree, adding
    1-0' closes the 4-cycle; a repeated edge is a 2-cycle.  Residual by hand: a = (0.5, 0.5),
    b = (0.25, 0.75), P on (0,0), (0,1), (1,1) = (0.25, 0.2, 0.5) -> row sums (0.45, 0.5), column
    sums (0.25, 0.7) -> |0.05| + 0 + 0 + |0.05| = 0.1."""
    assert certificate.is_forest(2, 2, [0, 0, 1], [0, 1, 1])
    assert not certificate.is_forest(2, 2, [0, 0, 1, 1], [0, 1, 1, 0])
    assert not certificate.is_forest(2, 2, [0, 0], [1, 1])
    assert certificate.is_forest(3, 2, [], [])
    res = certificate.marginal_residual_l1(2, 2, np.array([0, 0, 1]), np.array([0, 1, 1]),
                                           np.array([0.25, 0.2, 0.5]), np.array([0.5, 0.5]),
                                           np.array([0.25, 0.75]))
    assert abs(res - 0.1) <= 1e-15


@pytest.mark.parametrize("k,seed", [(6, 0), (9, 1)])
def test_c_transform_lower_bound_weak_duality_and_tightness(k, seed):
    """Weak duality: for any v the bound is at most OPT; at an optimal v it equals OPT (the
    c-transform of v* is at least u* entrywise, so the bound is at least a^T u* + b^T v* = OPT)."""
    inst = synth.image_pair(k, seed)
    c = costs.square_grid(k)
    r = netsimplex.solve(c, inst.a, inst.b)
    assert abs(certificate.c_transform_lower_bound(c, inst.a, inst.b, r.v) - r.obj) <= 1e-12 * r.obj
    rng = synth.uniform01(seed + 77, 5 * k * k)
    for t in range(5):
        v = r.v + (rng[t * k * k:(t + 1) * k * k] - 0.5) * (1.0 + t)
        assert certificate.c_transform_lower_bound(c, inst.a, inst.b, v) <= r.obj * (1 + 1e-12)


@pytest.mark.parametrize("kind", ["sqeuclid", "euclid", "l1", "linf"])
def test_min_reduced_cost_matches_python_loops(kind):
    """Against pure-Python loops over every pair, on point sets with a row count that spans
    several of the function's row chunks."""
    m, n = 37, 29
    rng = synth.uniform01(4242, 2 * m + 2 * n + m + n)
    sx, sy = np.floor(rng[:m] * 9), np.floor(rng[m:2 * m] * 9)
    tx, ty = np.floor(rng[2 * m:2 * m + n] * 9), np.floor(rng[2 * m + n:2 * m + 2 * n] * 9)
    u = rng[2 * m + 2 * n:2 * m + 2 * n + m] * 20 - 5
    v = rng[2 * m + 2 * n + m:] * 20 - 5
    c = costs.Cost.points(sx, sy, tx, ty, kind)
    f = {"sqeuclid": lambda dx, dy: dx * dx + dy * dy,
         "euclid": lambda dx, dy: float(np.sqrt(dx * dx + dy * dy)),
         "l1": lambda dx, dy: abs(dx) + abs(dy),
         "linf": lambda dx, dy: max(abs(dx), abs(dy))}[kind]
    best = min((f(float(sx[i] - tx[j]), float(sy[i] - ty[j])) - float(u[i])) - float(v[j])
               for i in range(m) for j in range(n))
    assert certificate.min_reduced_cost(c, u, v) == best


# ----------------------------------------------------------------------------- removal guard

def _n_components(m, n, I, J):
    parent = list(range(m + n))

    def find(x):
        while parent[x] != x:
            x = parent[x]
        return x

    for i, j in zip(I.tolist(), J.tolist()):
        a, b = find(i), find(m + j)
        if a != b:
            parent[a] = b
    # vertices that carry at least one edge, counted by their roots
    used = set(I.tolist()) | {m + j for j in J.tolist()}
    return len({find(x) for x in used})


def test_removal_guard_breaks_a_cycle_at_its_lightest_edge():
    """Hand-built case: sources {0, 1}, targets {0, 1}, all four pairs in the support (one
    4-cycle), every pair a removal candidate.  The maximum-weight spanning forest (Kruskal by
    decreasing p) keeps the three heaviest edges, so exactly the lightest one may leave and the
    support stays one connected component."""
    m = n = 2
    prob = ipm.Problem(costs.Cost.dense(np.array([[0.0, 1.0], [1.0, 0.0]])), np.array([0.5, 0.5]),
                       np.array([0.5, 0.5]))
    I = np.array([0, 0, 1, 1], dtype=np.int64)
    J = np.array([0, 1, 0, 1], dtype=np.int64)
    p = np.array([4e-9, 3e-9, 1e-9, 2e-9])        # lightest: (1, 0)
    st = ipm.State(I, J, p, np.ones(4), np.zeros(m), np.zeros(n))
    rem = ipm.removal_select(prob, st, ipm.Options(), kmax=4)
    assert rem.tolist() == [2]
    keep = np.ones(4, bool)
    keep[rem] = False
    assert _n_components(m, n, I[keep], J[keep]) == 1


@pytest.mark.parametrize("seed", range(4))
def test_removal_guard_keeps_the_component_count(seed):
    """Random supports with many cycles, every pair a candidate: the number of connected
    components of the support graph is the same before and after removal."""
    k = 5
    m = n = k * k
    inst = synth.image_pair(k, seed)
    prob = ipm.Problem(costs.square_grid(k), inst.a, inst.b)
    rng = synth.uniform01(900 + seed, m * n + m * n)
    mask = rng[:m * n].reshape(m, n) < 0.15
    I, J = np.nonzero(mask)
    I, J = I.astype(np.int64), J.astype(np.int64)
    p = 1e-12 * (1.0 + rng[m * n:m * n + len(I)])
    st = ipm.State(I, J, p, np.ones(len(I)), np.zeros(m), np.zeros(n))
    before = _n_components(m, n, I, J)
    rem = ipm.removal_select(prob, st, ipm.Options(), kmax=m * n)
    keep = np.ones(len(I), bool)
    keep[rem] = False
    assert len(rem) > 0
    assert _n_components(m, n, I[keep], J[keep]) == before
    # what is left is a forest exactly when nothing else held the removal back (kmax large)
    assert certificate.is_forest(m, n, I[keep], J[keep])


# ----------------------------------------------------------------------------- other costs, J set

@pytest.mark.parametrize("seed", range(4))
def test_pricing_jset_matches_bruteforce(seed):
    """Section 3.4's heuristic set J: only pairs with c_ij < C_max are candidates."""
    m, n = 8, 7
    C = synth.random_int_costs(m, n, 300 + seed, hi=9).astype(np.float64)
    rng = synth.uniform01(2000 + seed, m + n + m * n)
    u = np.round(rng[:m] * 6, 1)
    v = np.round(rng[m:m + n] * 6, 1)
    I, J = np.nonzero(rng[m + n:].reshape(m, n) < 0.2)
    sup = set(zip(I.tolist(), J.tolist()))
    for cmax in (0.5, 3.0, 4.5, 100.0):
        for kmax in (2, m, m * n):
            sI, sJ, sD = pricing.select(costs.Cost.dense(C), u, v, I, J, kmax, cmax=cmax)
            ref = pricing.select_bruteforce(C, u, v, sup, kmax, cmax=cmax)
            assert list(zip(sI.tolist(), sJ.tolist())) == ref
            assert np.all(C[sI, sJ] < cmax) and np.all(sD < 0)
    # C_max above every cost: the full rule
    full = pricing.select(costs.Cost.dense(C), u, v, I, J, m * n)
    capped = pricing.select(costs.Cost.dense(C), u, v, I, J, m * n, cmax=C.max() + 1)
    assert all(np.array_equal(x, y) for x, y in zip(full, capped))


@pytest.mark.parametrize("kind", ["euclid", "l1", "linf"])
@pytest.mark.parametrize("k,seed", [(8, 1), (12, 3)])
def test_ipm_oracle_other_costs_reach_exact_optimum(kind, k, seed):
    """Section 5.1's L1, Euclidean and L-infinity distances through the oracle IPM."""
    inst = synth.image_pair(k, seed)
    c = costs.square_grid(k, kind)
    ref = netsimplex.solve(c, inst.a, inst.b)
    r = ipm.solve(c, inst.a, inst.b, ipm.Options(tol=1e-8))
    assert r.status == "optimal"
    assert abs(r.obj - ref.obj) <= 1e-7 * ref.obj and r.r1_l1 <= 1e-8


@pytest.mark.parametrize("kind,cmax", [("sqeuclid", 9.0), ("l1", 4.0), ("euclid", 3.0), ("linf", 3.0)])
def test_ipm_oracle_with_jset_reaches_exact_optimum(kind, cmax):
    """Pricing on J between full refreshes (Section 3.4) changes the trajectory, not the optimum."""
    k = 12
    inst = synth.image_pair(k, 0)
    c = costs.square_grid(k, kind)
    ref = netsimplex.solve(c, inst.a, inst.b)
    r = ipm.solve(c, inst.a, inst.b, ipm.Options(tol=1e-8, jset_cmax=cmax))
    assert r.status == "optimal"
    assert abs(r.obj - ref.obj) <= 1e-7 * ref.obj and r.r1_l1 <= 1e-8


def test_zero_masses_carry_no_flow():
    """Input handling of zero masses (presolve): a point with zero mass carries no flow, so the
    optimum equals that of the problem without those points, and the network simplex's duals
    stay feasible over all pairs."""
    k = 10
    inst = synth.image_pair(k, 5)
    rng = synth.uniform01(77, 2 * k * k)
    a, b = inst.a.copy(), inst.b.copy()
    a[rng[:k * k] < 0.2] = 0.0
    b[rng[k * k:] < 0.2] = 0.0
    a /= a.sum()
    b /= b.sum()
    c = costs.square_grid(k)
    full = netsimplex.solve(c, a, b)
    ki, kj = np.nonzero(a > 0)[0], np.nonzero(b > 0)[0]
    red = netsimplex.solve(costs.Cost.points(c.sx[ki], c.sy[ki], c.tx[kj], c.ty[kj]), a[ki], b[kj])
    assert abs(full.obj - red.obj) <= 1e-12 * red.obj
    assert certificate.min_reduced_cost(c, full.u, full.v) >= 0.0
    assert np.all(full.P[(a[full.I] == 0) | (b[full.J] == 0)] == 0.0)


def test_north_west_corner_is_a_feasible_staircase():
    """The north-west-corner rule (textbook transportation start): worked by hand for
    a = (0.5, 0.3, 0.2), b = (0.2, 0.4, 0.4): pairs (0,0) (0,1) (1,1) (1,2) (2,2); in general a
    staircase of at most m + n - 1 pairs that carries a feasible plan."""
    I, J = ipm.north_west_corner(np.array([0.5, 0.3, 0.2]), np.array([0.2, 0.4, 0.4]))
    assert list(zip(I.tolist(), J.tolist())) == [(0, 0), (0, 1), (1, 1), (1, 2), (2, 2)]
    a, b = synth.random_masses(30, 1), synth.random_masses(45, 2)
    I, J = ipm.north_west_corner(a * 30, b * 30)
    assert len(I) <= 74 and np.all(np.diff(I) >= 0) and np.all(np.diff(J) >= 0)
    # the restricted problem on these pairs is feasible: the network simplex on costs that are
    # 0 on the staircase and huge elsewhere finds a zero-cost plan
    C = np.full((30, 45), 1e6)
    C[I, J] = 0.0
    assert netsimplex.solve(costs.Cost.dense(C), a, b).obj == 0.0


def test_ipm_oracle_on_point_sets_that_do_not_overlap():
    """A vertical line of 30 sources against a 5 x 9 target grid to its right: the initial
    support {c <= 2} is empty apart from the cheapest pairs and splits; with the north-west-corner
    completion the oracle IPM reaches the exact optimum."""
    sx = np.zeros(30)
    sy = np.arange(30.0)
    t = np.arange(45)
    tx, ty = (t % 5 + 3).astype(float), (t // 5 - 1).astype(float)
    c = costs.Cost.points(sx, sy, tx, ty)
    a, b = synth.random_masses(30, 70), synth.random_masses(45, 95)
    ref = netsimplex.solve(c, a, b)
    r = ipm.solve(c, a, b, ipm.Options(tol=1e-8))
    assert r.status == "optimal" and abs(r.obj - ref.obj) <= 1e-7 * ref.obj


@pytest.mark.parametrize("workers", [1, 2])
def test_streaming_selection_equals_the_plain_rule(workers):
    """The blockwise top-k selection (for 4.29e9 pairs) against the plain rule: exact same pairs,
    order and values, ties included, with and without J."""
    k = 24
    c = costs.square_grid(k)
    rng = synth.uniform01(66, 2 * k * k)
    u = np.round(rng[:k * k] * 30, 1)
    v = np.round(rng[k * k:] * 30, 1) - 20
    I, J = np.nonzero(synth.uniform01(67, (k * k) ** 2).reshape(k * k, k * k) < 0.01)
    for kmax in (1, 37, 576, 10 ** 6):
        for cmax in (None, 20.0):
            a = pricing.select(c, u, v, I, J, kmax, cmax=cmax)
            b = pricing.select_streaming(c, u, v, I, J, kmax, cmax=cmax, rows_per_chunk=50, workers=workers)
            assert all(np.array_equal(x, y) for x, y in zip(a, b))


# ----------------------------------------------------------------------------- incomplete Cholesky

def _schur_of_random_support(k=7, seed=3, frac=0.12):
    m = n = k * k
    rng = synth.uniform01(500 + seed, m * n + m * n)
    mask = rng[:m * n].reshape(m, n) < frac
    I, J = np.nonzero(mask)
    theta = 0.1 + rng[m * n:m * n + len(I)] * 10.0
    S, V, M, N, Minv = ipm.schur_matrix(m, n, I, J, theta)
    return S


def test_ic_greedy_colouring_is_proper():
    from oracle import ic
    S = _schur_of_random_support()
    color = ic.greedy_coloring(S)
    C = S.tocoo()
    off = C.row != C.col
    assert np.all(color[C.row[off]] != color[C.col[off]])
    perm = ic.multicolor_order(color)
    assert sorted(perm.tolist()) == list(range(S.shape[0])) and np.all(np.diff(color[perm]) >= 0)


def test_ic0_reproduces_the_matrix_on_its_pattern():
    """The defining property of incomplete Cholesky without dropping: L D L^T equals S on every
    position of S's pattern (the error lives only where fill was discarded).  S: a Schur complement
    of a random support, shifted to be nonsingular."""
    from oracle import ic
    S = _schur_of_random_support()
    n = S.shape[0]
    diag = S.diagonal() + 0.05
    off = S - sp.diags(S.diagonal())
    perm, rows, D = ic.factor(off, diag, tau=0.0)
    L = np.eye(n)
    for r, row in enumerate(rows):
        for s, l in row.items():
            L[r, s] = l
    assert np.all(np.isfinite(D)) and np.all(D > 0)
    M = L @ np.diag(D) @ L.T
    A = (off + sp.diags(diag)).toarray()[np.ix_(perm, perm)]
    pat = A != 0
    assert np.abs((M - A)[pat]).max() <= 1e-12 * np.abs(A).max()
    # and the preconditioner applies M^-1 (in the original order)
    b = synth.normal(4, n)
    x = ic.apply(perm, rows, D, b)
    Mo = np.empty_like(M)
    Mo[np.ix_(perm, perm)] = M
    assert np.abs(Mo @ x - b).max() <= 1e-10 * np.abs(b).max()


def test_ic_with_a_large_drop_tolerance_is_jacobi():
    """Weak diagonal dominance gives |S_rs| <= sqrt(S_rr S_ss), so tau = 1.01 drops every entry
    (the first one of each row is S_rs itself) and the factor is the diagonal."""
    from oracle import ic
    S = _schur_of_random_support(seed=5)
    diag = S.diagonal()
    off = S - sp.diags(diag)
    perm, rows, D = ic.factor(off, diag, tau=1.01)
    assert all(all(l == 0.0 for l in row.values()) for row in rows)
    b = synth.normal(9, S.shape[0])
    assert np.allclose(ic.apply(perm, rows, D, b), b / diag, rtol=1e-15, atol=0)
