"""Python front end of the GB300 OT solver: marshals arguments to the C ABI, nothing more.

Every step of the method runs in the CUDA library; this module only converts arrays to the
pointers and structs of ``include/ot_ipm.h``.  Device buffers (for ``price_topk``) are torch
CUDA tensors; the solver handle takes host arrays and owns its device state.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import OtIterInfo, OtOptions, OtProblem, OtResult, check


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def default_options(**overrides) -> OtOptions:
    lib = _lib.load()
    o = OtOptions()
    lib.ot_options_default(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(f"unknown option {k}")
        setattr(o, k, v)
    return o


@dataclass
class Result:
    status: int
    obj: float
    lower_bound: float
    rel_gap: float
    r1_l1: float
    mu: float
    iters: int
    cg_iters: int
    direct_iters: int
    psi: int
    max_fill: float
    seconds: float
    warm_added: int = 0
    warm_restarts: int = 0
    create_seconds: float = 0.0
    ms_levels: int = 0


def _is_cuda_tensor(x) -> bool:
    return type(x).__module__.startswith("torch") and getattr(x, "is_cuda", False)


class Solver:
    """One OT instance on the GPU (``ot_ipm_create`` ... ``ot_ipm_destroy``).

    a, b: masses (host arrays, or CUDA tensors: then every input is passed as a device pointer,
    ``inputs_on_device``).  Points: either ``grid=(src_w, dst_w)`` (pixel grids, pixel i at
    (i mod w, i div w)) or ``coords=(sx, sy, tx, ty)`` integer arrays; or an explicit cost
    matrix ``C`` (m x n, row-major).  ``cost``: "sqeuclid" (default), "euclid", "l1", "linf".
    """

    def __init__(self, a, b, grid=None, coords=None, stream=None, warm=None, warm_pairs=None, C=None, **options):
        """warm: optional predicted duals (u, v) in cost units; the initial support then also takes
        the pairs of least predicted reduced cost.  warm_pairs: optional (I, J) pairs that join the
        initial support (e.g. from ``WarmStart.pairs``)."""
        self._lib = _lib.load()
        self._keep = []
        prob = OtProblem()
        on_dev = _is_cuda_tensor(a)
        if on_dev:
            import torch
            conv = lambda x, dt: x.to(dtype=dt).contiguous()
            da, db = conv(a, torch.float64), conv(b, torch.float64)
            self._keep += [da, db]
            self.m, self.n = da.numel(), db.numel()
            prob.a, prob.b = da.data_ptr(), db.data_ptr()
            prob.inputs_on_device = 1
        else:
            self.a = np.ascontiguousarray(a, dtype=np.float64)
            self.b = np.ascontiguousarray(b, dtype=np.float64)
            self.m, self.n = len(self.a), len(self.b)
            prob.a, prob.b = _ptr(self.a), _ptr(self.b)
        prob.m, prob.n = self.m, self.n
        prob.cost = _lib.COST[options.pop("cost", "sqeuclid" if C is None else "dense")]
        if C is not None:
            if on_dev:
                import torch
                dC = C.to(dtype=torch.float64).contiguous()
                self._keep.append(dC)
                prob.C = dC.data_ptr()
            else:
                hC = np.ascontiguousarray(C, dtype=np.float64)
                if hC.shape != (self.m, self.n):
                    raise ValueError("C must have shape (m, n)")
                self._keep.append(hC)
                prob.C = _ptr(hC)
        elif coords is not None:
            if on_dev:
                import torch
                cs = [c.to(dtype=torch.int32).contiguous() for c in coords]
                self._keep += cs
                prob.src_x, prob.src_y, prob.dst_x, prob.dst_y = [c.data_ptr() for c in cs]
            else:
                cs = [np.ascontiguousarray(c, dtype=np.int32) for c in coords]
                self._keep += cs
                prob.src_x, prob.src_y, prob.dst_x, prob.dst_y = [_ptr(c) for c in cs]
        else:
            if grid is None:
                k = int(round(np.sqrt(self.m)))
                grid = (k, int(round(np.sqrt(self.n))))
            prob.src_w, prob.dst_w = grid
        if stream is not None:
            options["stream"] = stream
        if warm is not None:
            wu = np.ascontiguousarray(warm[0], dtype=np.float64)
            wv = np.ascontiguousarray(warm[1], dtype=np.float64)
            if wu.shape != (self.m,) or wv.shape != (self.n,):
                raise ValueError("warm duals must have shapes (m,) and (n,)")
            self._keep += [wu, wv]
            options["warm_u"], options["warm_v"] = _ptr(wu), _ptr(wv)
        if warm_pairs is not None:
            wi = np.ascontiguousarray(warm_pairs[0], dtype=np.int32)
            wj = np.ascontiguousarray(warm_pairs[1], dtype=np.int32)
            if wi.shape != wj.shape:
                raise ValueError("warm_pairs: I and J differ in length")
            self._keep += [wi, wj]
            options["warm_i"], options["warm_j"], options["warm_npairs"] = _ptr(wi), _ptr(wj), len(wi)
        self.options = default_options(**options)
        h = ctypes.c_void_p()
        check(self._lib.ot_ipm_create(ctypes.byref(prob), ctypes.byref(self.options), ctypes.byref(h)))
        self.h = h

    # -- iteration -----------------------------------------------------------------
    def step(self) -> dict:
        info = OtIterInfo()
        check(self._lib.ot_ipm_step(self.h, ctypes.byref(info)), self.h)
        return {f: getattr(info, f) for f, _ in OtIterInfo._fields_}

    def solve(self, raise_on_error: bool = True) -> Result:
        r = OtResult()
        code = self._lib.ot_ipm_solve(self.h, ctypes.byref(r))
        if raise_on_error and code not in (_lib.OT_OK,):
            check(code, self.h)
        return Result(*[getattr(r, f) for f, _ in OtResult._fields_])

    # -- results -------------------------------------------------------------------
    def solution(self):
        nnz = ctypes.c_int64(0)
        self._lib.ot_ipm_get_solution(self.h, None, None, None, 0, ctypes.byref(nnz), None, None)
        k = nnz.value
        I = np.zeros(k, np.int32)
        J = np.zeros(k, np.int32)
        P = np.zeros(k)
        u = np.zeros(self.m)
        v = np.zeros(self.n)
        check(self._lib.ot_ipm_get_solution(self.h, _ptr(I), _ptr(J), _ptr(P), k, ctypes.byref(nnz),
                                            _ptr(u), _ptr(v)), self.h)
        return I, J, P, u, v

    def state(self):
        psi = ctypes.c_int64(0)
        self._lib.ot_ipm_get_state(self.h, None, None, None, None, 0, ctypes.byref(psi), None, None)
        k = psi.value
        I = np.zeros(k, np.int32)
        J = np.zeros(k, np.int32)
        P = np.zeros(k)
        S = np.zeros(k)
        u = np.zeros(self.m)
        v = np.zeros(self.n)
        check(self._lib.ot_ipm_get_state(self.h, _ptr(I), _ptr(J), _ptr(P), _ptr(S), k, ctypes.byref(psi),
                                         _ptr(u), _ptr(v)), self.h)
        return I, J, P, S, u, v

    def set_state(self, I, J, P, S, u, v, reset_mu0: bool = False):
        arrs = [np.ascontiguousarray(I, np.int32), np.ascontiguousarray(J, np.int32),
                np.ascontiguousarray(P, np.float64), np.ascontiguousarray(S, np.float64),
                np.ascontiguousarray(u, np.float64), np.ascontiguousarray(v, np.float64)]
        check(self._lib.ot_ipm_set_state(self.h, _ptr(arrs[0]), _ptr(arrs[1]), _ptr(arrs[2]), _ptr(arrs[3]),
                                         len(arrs[0]), _ptr(arrs[4]), _ptr(arrs[5]), int(reset_mu0)), self.h)

    LINEAR_SOLVERS = {"pcg64": 0, "mixed": 1, "dense32": 2, "dense64": 3, "sparse": 4, "ic": 5, "tree": 6}

    def newton_direction(self, solver: str = "pcg64", cg_tol: float = 1e-12, max_cg: int = 20000):
        """Predictor direction (du, dv, dp, ds) at the current iterate by one linear solver
        (ot_ipm_newton_direction); returns the four arrays and the CG iteration count."""
        psi = ctypes.c_int64(0)
        self._lib.ot_ipm_get_state(self.h, None, None, None, None, 0, ctypes.byref(psi), None, None)
        k = psi.value
        du, dv, dp, ds = np.zeros(self.m), np.zeros(self.n), np.zeros(k), np.zeros(k)
        its = ctypes.c_int32(0)
        check(self._lib.ot_ipm_newton_direction(self.h, self.LINEAR_SOLVERS[solver], cg_tol, max_cg, _ptr(du),
                                                _ptr(dv), _ptr(dp), _ptr(ds), k, ctypes.byref(its)), self.h)
        return du, dv, dp, ds, its.value

    def ic_apply(self, b, tau: float = 1e-2):
        """The incomplete Cholesky preconditioner of the current iterate applied to b
        (ot_ipm_ic_apply)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.n)
        check(self._lib.ot_ipm_ic_apply(self.h, tau, _ptr(b), _ptr(x)), self.h)
        return x

    @property
    def mass_scale(self) -> float:
        return self._lib.ot_ipm_mass_scale(self.h)

    def close(self):
        if getattr(self, "h", None):
            self._lib.ot_ipm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def price_topk(sx, sy, tx, ty, u, v, sup_i, sup_j, kmax: int, precision: int = 1, stream=None,
               cost: str = "sqeuclid", scan_rows: int = 0, jset_cmax: float = 0.0, C=None):
    """Pricing + selection on device tensors (torch, cuda, contiguous): int32 coordinates,
    float64 duals, int32 support pairs sorted by (i, j).  Returns (I, J, D) device tensors.
    cost, scan_rows, jset_cmax, C (dense float64 m x n device tensor, cost "dense"): the options
    of ``ot_price_topk_ex``; with the defaults the call is ``ot_price_topk``."""
    import torch
    lib = _lib.load()
    if C is not None:
        cost = "dense"
        m, n = int(C.shape[0]), int(C.shape[1])
    else:
        m, n = int(sx.numel()), int(tx.numel())
    dev = u.device
    out_i = torch.empty(max(kmax, 1), dtype=torch.int32, device=dev)
    out_j = torch.empty(max(kmax, 1), dtype=torch.int32, device=dev)
    out_d = torch.empty(max(kmax, 1), dtype=torch.float64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    checks = [(u, torch.float64), (v, torch.float64), (sup_i, torch.int32), (sup_j, torch.int32)]
    if C is None:
        checks += [(sx, torch.int32), (sy, torch.int32), (tx, torch.int32), (ty, torch.int32)]
    else:
        checks.append((C, torch.float64))
    for t, dt in checks:
        if t.dtype != dt or not t.is_contiguous() or not t.is_cuda:
            raise TypeError("price_topk: expected contiguous CUDA tensors of the documented dtypes")
    s = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
    psi = int(sup_i.numel())
    ptr = lambda t: None if t is None else t.data_ptr()
    if cost == "sqeuclid" and scan_rows == 0 and jset_cmax <= 0 and C is None:
        check(lib.ot_price_topk(m, n, sx.data_ptr(), sy.data_ptr(), tx.data_ptr(), ty.data_ptr(), u.data_ptr(),
                                v.data_ptr(), sup_i.data_ptr() if psi else None, sup_j.data_ptr() if psi else None,
                                psi, kmax, precision, out_i.data_ptr(), out_j.data_ptr(), out_d.data_ptr(),
                                cnt.data_ptr(), ctypes.c_void_p(s)))
    else:
        po = _lib.OtPriceOpts()
        po.cost = _lib.COST[cost]
        po.scan_rows = scan_rows
        po.jset_cmax = jset_cmax
        po.C = ptr(C)
        check(lib.ot_price_topk_ex(m, n, ptr(sx), ptr(sy), ptr(tx), ptr(ty), u.data_ptr(), v.data_ptr(),
                                   sup_i.data_ptr() if psi else None, sup_j.data_ptr() if psi else None, psi, kmax,
                                   precision, out_i.data_ptr(), out_j.data_ptr(), out_d.data_ptr(), cnt.data_ptr(),
                                   ctypes.byref(po), ctypes.c_void_p(s)))
    k = int(cnt.item())
    return out_i[:k], out_j[:k], out_d[:k]


def kernel_timing(enable: bool | None = None) -> dict:
    """Enable/disable (and clear) per-kernel event timing, or read {name: (ms, launches, work)}."""
    lib = _lib.load()
    if enable is not None:
        lib.ot_kernel_timing_enable(int(enable))
        return {}
    ms = np.zeros(len(_lib.KERNEL_IDS))
    cnt = np.zeros(len(_lib.KERNEL_IDS), np.int64)
    work = np.zeros(len(_lib.KERNEL_IDS))
    lib.ot_kernel_timing_read(_ptr(ms), _ptr(cnt), _ptr(work), len(ms))
    return {k: (float(a), int(b), float(c)) for k, a, b, c in zip(_lib.KERNEL_IDS, ms, cnt, work)}


def kernel_launches() -> int:
    return int(_lib.load().ot_kernel_launches())


def solve_batch(pairs, workers: int = 2, tuning=None, create_threads: int = 8, errors: list | None = None, **options):
    """Solve independent instances concurrently (``ot_ipm_solve_batch``).

    pairs: sequence of (a, b, side) for k x k pixel grids (side = k).  tuning: optional callable
    (m, n) -> dict of launch options (e.g. ``autotune.lookup``).  Handles are created by
    `create_threads` host threads (each on its own stream), solved by the library's queue of
    `workers` threads, and destroyed afterwards.  Returns a list of Result (status per instance);
    `errors`, when given, receives (index, message) for every failed instance.
    """
    from concurrent.futures import ThreadPoolExecutor
    lib = _lib.load()

    def make(pair):
        a, b, k = pair
        opts = dict(options)
        if tuning is not None:
            opts.update(tuning(k * k, k * k))
        return Solver(a, b, grid=(k, k), **opts)

    with ThreadPoolExecutor(max_workers=max(1, create_threads)) as ex:
        solvers = list(ex.map(make, pairs))
    try:
        n = len(solvers)
        hs = (ctypes.c_void_p * n)(*[s.h.value for s in solvers])
        rs = (OtResult * n)()
        lib.ot_ipm_solve_batch(hs, n, rs, workers)
        if errors is not None:
            for i, r in enumerate(rs):
                if r.status != 0:
                    msg = lib.ot_ipm_last_error(solvers[i].h)
                    errors.append((i, (msg or b"").decode(errors="replace")))
        return [Result(*[getattr(r, f) for f, _ in OtResult._fields_]) for r in rs]
    finally:
        for s in solvers:
            s.close()
