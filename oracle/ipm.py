"""O2: plain float64 rendition of the paper's sparse IPM / column-generation iteration.

Test infrastructure only (see ``oracle/__init__.py``).

Follows Sections 3-4 step by step, in the paper's order (the commented SparseIPM listing of
Section 3.4 gives the order: residuals, mu, sigma and r3, Newton direction, step lengths,
update, pricing, support update).  The Newton direction is computed exactly (a direct
solve of the Schur complement, its pseudo-inverse on each connected component) because
this is the definition the GPU's iterative and direct solvers approximate.

Readings where the paper is silent:
  * data scale: masses are scaled internally to mean 1 (sigma_f = m / sum a); the LP
    solution scales exactly with it and results are reported in the caller's units;
  * initial support: pairs with c_ij <= init_cost (2 on pixel grids: the 3x3 neighbourhood),
    plus every row's and column's cheapest pair (ties: smaller index)  (Section 3.2 end); when
    that support graph is not connected, plus the north-west-corner coupling's pairs (a feasible
    plan), so that the restricted problem is feasible;
  * initial point: Mehrotra's heuristic (Mehrotra 1992, SIAM J. Optim. 2:575) on the
    restricted problem: least-squares p and y from A A^T (Theta = I), shifted to positivity;
  * stop: max(|r1|/(1+|f|), |r2|/(1+|c_red|), psi*mu/(1+|c^T p|)) < tol (2-norms; the last
    term is the relative complementarity gap, the "optimality tolerance" of Section 5.2),
    plus ||r1||_1 <= feas_l1 in the caller's units, plus no pricing candidate below
    -tol*(1+max c_red), plus the c-transform certificate (c^T p - LB)/(1+|c^T p|) <= tol;
  * sigma: Mehrotra predictor-corrector, sigma = (mu_aff/mu)^3;
  * centrality correctors (Section 3.3): up to max_corr, symmetric neighbourhood
    [beta_min*sigma*mu, beta_max*sigma*mu], trial step alpha + 0.1, kept while the smaller
    step length grows by at least 1%;
  * step: 0.995 x step to the boundary, separate alpha_p and alpha_s, each capped at 1;
  * Schur complement S_M = N - V^T M^-1 V (Section 4), singular: right-hand side projected
    to mean zero on each connected component of the support graph, minimum-norm dv;
  * support enlargement: at most m new pairs (the most negative reduced costs, exact rule
    of ``oracle.pricing``; with ``jset_cmax`` > 0 only pairs of Section 3.4's set
    J = {c_ij < jset_cmax} are priced, except on every ``jset_refresh``-th iteration).  Section 3.2 starts them at p = s = sqrt(mu) (``new_col_rule`` 0);
    the default (``new_col_rule`` 1) keeps the product p s = mu but caps the flow at the pair's
    smaller scaled mass, p = min(sqrt(mu), a_i, b_j), s = mu / p: with masses scaled to sum m,
    sqrt(mu) can exceed a pixel's whole mass many times over while mu is still large, and m such
    pairs per iteration then dominate the primal residual;
  * support reduction, active once mu <= rm_mu_frac * mu_0: a pair leaves when
    p < rm_p_frac * min(a_i, b_j) and theta < 1; at most m leave (smallest p first, ties by
    jlin); the edges of a maximum-weight spanning forest (weights p) never leave, so the support
    graph stays connected (and no row or column loses its last pair).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csgraph
import scipy.sparse.linalg as spla

from . import pricing
from .costs import Cost


@dataclass
class Options:
    tol: float = 1e-6
    feas_l1: float = 1e-8
    max_iter: int = 200
    max_corr: int = 3
    step_scale: float = 0.995
    beta_min: float = 0.1
    beta_max: float = 10.0
    alpha_boost: float = 0.1
    accept_gain: float = 1.01
    rm_mu_frac: float = 1e-3
    rm_p_frac: float = 1e-3
    init_cost: float = 2.0
    add_max: int | None = None      # default m
    new_col_rule: int = 1           # 0: p = s = sqrt(mu) as Section 3.2; 1: flow capped at min(a_i, b_j)
    jset_cmax: float = 0.0          # > 0: Section 3.4's heuristic set J = {c_ij < jset_cmax} ...
    jset_refresh: int = 3           # ... between full pricings on iterations refresh-1, 2 refresh-1, ...


@dataclass
class State:
    I: np.ndarray       # int64, support rows, sorted by (I, J)
    J: np.ndarray
    p: np.ndarray       # scaled units
    s: np.ndarray
    u: np.ndarray
    v: np.ndarray


@dataclass
class Problem:
    cost: Cost
    a: np.ndarray        # caller's masses
    b: np.ndarray
    sigma_f: float = 0.0
    as_: np.ndarray = None   # scaled masses
    bs: np.ndarray = None

    def __post_init__(self):
        a = np.asarray(self.a, np.float64)
        b = np.asarray(self.b, np.float64)
        if a.min() < 0 or b.min() < 0:
            raise ValueError("negative mass")
        sa, sb = a.sum(), b.sum()
        if abs(sa - sb) > 1e-12 * sa:
            raise ValueError("unbalanced marginals")
        b = b * (sa / sb)
        self.sigma_f = self.cost.m / sa
        self.as_ = a * self.sigma_f
        self.bs = b * self.sigma_f

    @property
    def m(self):
        return self.cost.m

    @property
    def n(self):
        return self.cost.n


@dataclass
class Residuals:
    r1a: np.ndarray
    r1b: np.ndarray
    r2: np.ndarray
    mu: float
    ctp: float
    c_red: np.ndarray


@dataclass
class Direction:
    dp: np.ndarray
    du: np.ndarray
    dv: np.ndarray
    ds: np.ndarray


@dataclass
class IterLog:
    it: int
    psi: int
    mu: float
    crit: float
    alpha_p: float
    alpha_s: float
    sigma: float
    ncorr: int
    added: int
    removed: int


@dataclass
class Result:
    status: str
    obj: float               # c^T p in caller units
    lb: float                # certified lower bound (caller units)
    gap: float
    r1_l1: float             # ||f - A p||_1 in caller units
    iters: int
    state: State
    log: list = field(default_factory=list)


# ---------------------------------------------------------------------------------------
# building blocks (each is one step of the iteration)
# ---------------------------------------------------------------------------------------

def initial_support(prob: Problem, opt: Options):
    """Section 3.2 end: low-cost pairs, plus each row's and column's cheapest pair."""
    cost, m, n = prob.cost, prob.m, prob.n
    keys = []
    step = max(1, (1 << 22) // max(n, 1))
    colbest = np.full(n, np.inf)
    colarg = np.zeros(n, dtype=np.int64)
    for i0 in range(0, m, step):
        i1 = min(m, i0 + step)
        c = cost.block(i0, i1)
        ii, jj = np.nonzero(c <= opt.init_cost)
        keys.append((ii + i0).astype(np.int64) * n + jj)
        rarg = np.argmin(c, axis=1)                       # first minimum = smaller index
        keys.append(np.arange(i0, i1, dtype=np.int64) * n + rarg)
        cmin = c.min(axis=0)
        carg = np.argmin(c, axis=0) + i0
        better = cmin < colbest                           # strict: keep the smaller index
        colbest[better] = cmin[better]
        colarg[better] = carg[better]
    keys.append(colarg * n + np.arange(n))
    key = np.unique(np.concatenate(keys))
    I, J = key // n, key % n
    ncomp, _ = components(m, n, I, J)
    if ncomp > 1:
        # point sets that do not overlap: the support splits and the restricted problem would be
        # infeasible; the north-west-corner coupling's pairs make it feasible
        nI, nJ = north_west_corner(prob.as_, prob.bs)
        key = np.unique(np.concatenate([key, nI * n + nJ]))
        I, J = key // n, key % n
    return I, J


def north_west_corner(a, b):
    """Support of the north-west-corner coupling (sources and targets in index order): a feasible
    plan on at most m + n - 1 pairs; equal partial sums advance both sides."""
    m, n = len(a), len(b)
    I, J = [], []
    i = j = 0
    A, B = float(a[0]), float(b[0])
    while i < m and j < n:
        I.append(i)
        J.append(j)
        if A < B:
            i += 1
            A = A + float(a[i]) if i < m else A
        elif B < A:
            j += 1
            B = B + float(b[j]) if j < n else B
        else:
            i += 1
            j += 1
            A = A + float(a[i]) if i < m else A
            B = B + float(b[j]) if j < n else B
    return np.array(I, dtype=np.int64), np.array(J, dtype=np.int64)


def initial_point(prob: Problem, I, J) -> State:
    """Mehrotra's starting heuristic on the restricted problem (the paper gives none):
    p~ = A^T (A A^T)^+ f, y~ = (A A^T)^+ A c, s~ = c - A^T y~, shifted to positivity."""
    m, n = prob.m, prob.n
    c = prob.cost.pairs(I, J)
    ones = np.ones(len(I))
    comp = components(m, n, I, J)
    yu, yv = normal_solve(m, n, I, J, ones, prob.as_, prob.bs, comp)
    pt = yu[I] + yv[J]
    cu = np.bincount(I, weights=c, minlength=m)
    cv = np.bincount(J, weights=c, minlength=n)
    u, v = normal_solve(m, n, I, J, ones, cu, cv, comp)
    stl = c - u[I] - v[J]
    ph = pt + max(-1.5 * float(pt.min()), 0.0)
    sh = stl + max(-1.5 * float(stl.min()), 0.0)
    ps = float(ph @ sh)
    p = ph + 0.5 * ps / float(sh.sum())
    s = sh + 0.5 * ps / float(ph.sum())
    return State(I, J, p, s, u, v)


def residuals(prob: Problem, st: State) -> Residuals:
    """r1 = f - A_red p, r2 = c_red - A_red^T y - s, mu = p^T s / psi  (eq. redsystem)."""
    m, n = prob.m, prob.n
    c = prob.cost.pairs(st.I, st.J)
    r1a = prob.as_ - np.bincount(st.I, weights=st.p, minlength=m)
    r1b = prob.bs - np.bincount(st.J, weights=st.p, minlength=n)
    r2 = c - st.u[st.I] - st.v[st.J] - st.s
    mu = float(st.p @ st.s) / len(st.p)
    return Residuals(r1a, r1b, r2, mu, float(c @ st.p), c)


def components(m: int, n: int, I, J):
    """Connected components of the bipartite support graph; labels of the n columns."""
    g = sp.coo_matrix((np.ones(len(I)), (I, m + J)), shape=(m + n, m + n))
    ncomp, lab = csgraph.connected_components(g, directed=False)
    return ncomp, lab[m:]


def schur_matrix(m: int, n: int, I, J, theta):
    """S_M = N - V^T M^-1 V with vec(V) = theta (Section 3.5 / Section 4)."""
    V = sp.csr_matrix((theta, (I, J)), shape=(m, n))
    M = np.asarray(V.sum(axis=1)).ravel()
    N = np.asarray(V.sum(axis=0)).ravel()
    Minv = np.where(M > 0, 1.0 / np.where(M > 0, M, 1.0), 0.0)
    S = sp.diags(N) - V.T @ sp.diags(Minv) @ V
    return S.tocsr(), V, M, N, Minv


def solve_schur(S, rhs, col_label, ncomp):
    """Minimum-norm least-squares solution of S x = rhs, S singular per component."""
    n = S.shape[0]
    cnt = np.bincount(col_label, minlength=ncomp).astype(np.float64)
    rhs = rhs - (np.bincount(col_label, weights=rhs, minlength=ncomp) / cnt)[col_label]
    x = np.zeros(n)
    # ground the first column of every component, solve the rest exactly
    first = np.full(ncomp, -1)
    for j in range(n - 1, -1, -1):
        first[col_label[j]] = j
    keep = np.ones(n, dtype=bool)
    keep[first] = False
    idx = np.nonzero(keep)[0]
    if idx.size:
        Sr = S[idx][:, idx].tocsc()
        # columns whose every row is private to them have an all-zero row: leave x = 0
        diag = Sr.diagonal()
        live = diag > 0
        if live.any():
            li = idx[live]
            Sl = S[li][:, li].tocsc()
            x[li] = spla.spsolve(Sl, rhs[li])
    x = x - (np.bincount(col_label, weights=x, minlength=ncomp) / cnt)[col_label]
    return x


def normal_solve(m, n, I, J, theta, beta1, beta2, comp):
    """Solve [M V; V^T N] [du; dv] = [beta1; beta2] (eq. normaleq) through the Schur
    complement S_M (Section 4): dv = S_M^+ (beta2 - V^T M^-1 beta1), du = M^-1 (beta1 - V dv)."""
    S, V, M, N, Minv = schur_matrix(m, n, I, J, theta)
    ncomp, lab = comp
    rhs = beta2 - V.T @ (Minv * beta1)
    dv = solve_schur(S, rhs, lab, ncomp)
    du = Minv * (beta1 - V @ dv)
    return du, dv


def newton_direction(prob: Problem, st: State, r1a, r1b, r2, r3, comp=None) -> Direction:
    """Eq. normalequationsipm through the Schur complement S_M (Section 4):
    g = Theta (r2 - P^-1 r3), beta = r1 + A g, (du, dv) from ``normal_solve``,
    ds = r2 - A^T dy, dp = S^-1 (r3 - P ds)."""
    m, n = prob.m, prob.n
    theta = st.p / st.s
    if comp is None:
        comp = components(m, n, st.I, st.J)
    g = theta * (r2 - r3 / st.p)
    beta1 = r1a + np.bincount(st.I, weights=g, minlength=m)
    beta2 = r1b + np.bincount(st.J, weights=g, minlength=n)
    du, dv = normal_solve(m, n, st.I, st.J, theta, beta1, beta2, comp)
    ds = r2 - du[st.I] - dv[st.J]
    dp = (r3 - st.p * ds) / st.s
    return Direction(dp, du, dv, ds)


def step_to_boundary(x, dx, scale):
    neg = dx < 0
    if not neg.any():
        return 1.0
    return min(1.0, scale * float((-x[neg] / dx[neg]).min()))


def steps(st: State, d: Direction, opt: Options):
    return step_to_boundary(st.p, d.dp, opt.step_scale), step_to_boundary(st.s, d.ds, opt.step_scale)


def combine(d1: Direction, d2: Direction) -> Direction:
    return Direction(d1.dp + d2.dp, d1.du + d2.du, d1.dv + d2.dv, d1.ds + d2.ds)


def predictor_corrector(prob: Problem, st: State, res: Residuals, opt: Options):
    """Mehrotra predictor, corrector, then centrality correctors (Section 3.3)."""
    psi = len(st.p)
    comp = components(prob.m, prob.n, st.I, st.J)
    r3 = -st.p * st.s
    daff = newton_direction(prob, st, res.r1a, res.r1b, res.r2, r3, comp)
    ap, as_ = steps(st, daff, opt)
    mu_aff = float((st.p + ap * daff.dp) @ (st.s + as_ * daff.ds)) / psi
    sigma = min(1.0, max(0.0, (mu_aff / res.mu) ** 3))
    r3 = sigma * res.mu - st.p * st.s - daff.dp * daff.ds
    d = newton_direction(prob, st, res.r1a, res.r1b, res.r2, r3, comp)
    ap, as_ = steps(st, d, opt)
    ncorr = 0
    zm, zn = np.zeros(prob.m), np.zeros(prob.n)
    zpsi = np.zeros(psi)
    for _ in range(opt.max_corr):
        if min(ap, as_) >= 1.0:
            break
        tp, ts = min(1.0, ap + opt.alpha_boost), min(1.0, as_ + opt.alpha_boost)
        vv = (st.p + tp * d.dp) * (st.s + ts * d.ds)
        lo, hi = opt.beta_min * sigma * res.mu, opt.beta_max * sigma * res.mu
        corr = np.clip(vv, lo, hi) - vv
        corr = np.maximum(corr, -hi)
        dc = newton_direction(prob, st, zm, zn, zpsi, corr, comp)
        dn = combine(d, dc)
        ap2, as2 = steps(st, dn, opt)
        if min(ap2, as2) >= opt.accept_gain * min(ap, as_):
            d, ap, as_ = dn, ap2, as2
            ncorr += 1
        else:
            break
    return d, ap, as_, sigma, ncorr


def removal_select(prob: Problem, st: State, opt: Options, kmax: int):
    """Indices (into the support) of the pairs that leave (reading in the module doc)."""
    m, n = prob.m, prob.n
    theta = st.p / st.s
    thr = opt.rm_p_frac * np.minimum(prob.as_[st.I], prob.bs[st.J])
    cand = (st.p < thr) & (theta < 1.0)
    if not cand.any():
        return np.zeros(0, dtype=np.int64)
    jlin = st.I + st.J * m
    # never remove an edge of the maximum-weight spanning forest of the support graph (weights p,
    # ties: smaller jlin first, Kruskal): the support stays connected, so the restricted problem
    # cannot split into components whose masses do not balance
    parent = np.arange(m + n)

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for e in np.lexsort((jlin, -st.p)):
        ra, rb = find(int(st.I[e])), find(m + int(st.J[e]))
        if ra != rb:
            parent[ra] = rb
            cand[e] = False
    idx = np.nonzero(cand)[0]
    o = np.lexsort((jlin[idx], st.p[idx]))
    return idx[o[:kmax]]


def update_support(st: State, remove_idx, addI, addJ, p_new, n, cap_a=None, cap_b=None) -> State:
    """New pairs at p = s = p_new, or with masses cap_a, cap_b given at p = min(p_new, a_i, b_j)
    and s = p_new^2 / p."""
    keep = np.ones(len(st.p), dtype=bool)
    keep[remove_idx] = False
    I = np.concatenate([st.I[keep], addI])
    J = np.concatenate([st.J[keep], addJ])
    if cap_a is None:
        pa = np.full(len(addI), p_new)
        sa = np.full(len(addI), p_new)
    else:
        pa = np.minimum(p_new, np.minimum(cap_a[addI], cap_b[addJ]))
        sa = p_new * p_new / pa
    p = np.concatenate([st.p[keep], pa])
    s = np.concatenate([st.s[keep], sa])
    o = np.argsort(I * n + J, kind="stable")
    return State(I[o], J[o], p[o], s[o], st.u, st.v)


def stop_measure(prob: Problem, res: Residuals, psi: int) -> float:
    f = np.concatenate([prob.as_, prob.bs])
    r1 = np.concatenate([res.r1a, res.r1b])
    return max(np.linalg.norm(r1) / (1.0 + np.linalg.norm(f)),
               np.linalg.norm(res.r2) / (1.0 + np.linalg.norm(res.c_red)),
               psi * res.mu / (1.0 + abs(res.ctp)))


# ---------------------------------------------------------------------------------------
# the whole iteration
# ---------------------------------------------------------------------------------------

@dataclass
class Tracker:
    """Cross-iteration quantities of the outer loop."""
    mu0: float | None = None
    strong: int = 1          # pricing candidates below -tol(1 + max c_red) at the last pricing
    lb: float = -np.inf


def stop_test(prob: Problem, st: State, opt: Options, tr: Tracker):
    """Stopping test of Section 3.2 (with this project's readings); returns (stop, res, crit)."""
    from .certificate import c_transform_lower_bound
    res = residuals(prob, st)
    psi = len(st.p)
    if tr.mu0 is None:
        tr.mu0 = res.mu
    crit = stop_measure(prob, res, psi)
    r1_l1 = (np.abs(res.r1a).sum() + np.abs(res.r1b).sum()) / prob.sigma_f
    if crit < opt.tol and r1_l1 <= opt.feas_l1 and tr.strong == 0:
        tr.lb = c_transform_lower_bound(prob.cost, prob.as_, prob.bs, st.v)
        if (res.ctp - tr.lb) / (1.0 + abs(res.ctp)) <= opt.tol:
            return True, res, crit
    return False, res, crit


def one_iteration(prob: Problem, st: State, res: Residuals, opt: Options, tr: Tracker, it: int = 0):
    """Newton step, pricing and support update (the body of Section 3.4's listing)."""
    m, n = prob.m, prob.n
    psi = len(st.p)
    kadd = opt.add_max or m
    d, ap, as_, sigma, ncorr = predictor_corrector(prob, st, res, opt)
    st = State(st.I, st.J, st.p + ap * d.dp, st.s + as_ * d.ds, st.u + as_ * d.du, st.v + as_ * d.dv)
    mu_new = float(st.p @ st.s) / psi
    use_j = opt.jset_cmax > 0 and it % opt.jset_refresh != opt.jset_refresh - 1
    aI, aJ, aD = pricing.select(prob.cost, st.u, st.v, st.I, st.J, kadd, cmax=opt.jset_cmax if use_j else None)
    c_red_max = float(np.abs(res.c_red).max()) if psi else 0.0
    tr.strong = int((aD < -opt.tol * (1.0 + c_red_max)).sum())
    if mu_new <= opt.rm_mu_frac * tr.mu0:
        rem = removal_select(prob, st, opt, m)
    else:
        rem = np.zeros(0, dtype=np.int64)
    stepped = st
    capped = opt.new_col_rule == 1
    st = update_support(st, rem, aI, aJ, math.sqrt(mu_new), n, prob.as_ if capped else None,
                        prob.bs if capped else None)
    log = IterLog(it, psi, res.mu, stop_measure(prob, res, psi), ap, as_, sigma, ncorr, len(aI), len(rem))
    return st, log, stepped, (aI, aJ, aD), rem


def solve(cost: Cost, a, b, opt: Options | None = None, state: State | None = None,
          verbose: bool = False) -> Result:
    from .certificate import c_transform_lower_bound
    opt = opt or Options()
    prob = Problem(cost, a, b)
    if state is None:
        I, J = initial_support(prob, opt)
        st = initial_point(prob, I, J)
    else:
        st = state
    tr = Tracker()
    log = []
    status = "maxiter"
    it = 0
    while True:
        stop, res, crit = stop_test(prob, st, opt, tr)
        if stop:
            status = "optimal"
            break
        if it >= opt.max_iter:
            break
        st, lg, _, _, _ = one_iteration(prob, st, res, opt, tr, it)
        log.append(lg)
        if verbose:
            print(f"it {it:3d} psi {lg.psi:7d} mu {lg.mu:.3e} crit {lg.crit:.3e} ap {lg.alpha_p:.3f} "
                  f"as {lg.alpha_s:.3f} sig {lg.sigma:.2e} corr {lg.ncorr} +{lg.added} -{lg.removed}")
        it += 1
    res = residuals(prob, st)
    r1_l1 = (np.abs(res.r1a).sum() + np.abs(res.r1b).sum()) / prob.sigma_f
    lb = tr.lb if np.isfinite(tr.lb) else c_transform_lower_bound(cost, prob.as_, prob.bs, st.v)
    gap = (res.ctp - lb) / (1.0 + abs(res.ctp))
    return Result(status, res.ctp / prob.sigma_f, lb / prob.sigma_f, gap, r1_l1, it, st, log)
