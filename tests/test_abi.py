"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every entry point
declared in include/*.h with struct layouts matching the Python binding (no compute calls)."""
from __future__ import annotations

import ctypes
import glob
import os
import re

import numpy as np

from paper_2206_11009_gb300 import _lib, build


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(build.INCLUDE, "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for mt in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_ \*]*?)\b(ot_[a-z0-9_]+)\s*\(", txt):
            names.append(mt.group(2))
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
        assert name in _lib.SIGNATURES, f"{name} has no binding"


def test_struct_layouts_match_binding():
    build.build()
    lib = _lib.load()
    out = np.zeros(4, np.int64)
    assert lib.ot_abi_struct_sizes(out.ctypes.data_as(ctypes.c_void_p), 4) == 4
    want = [ctypes.sizeof(c) for c in (_lib.OtProblem, _lib.OtOptions, _lib.OtIterInfo, _lib.OtResult)]
    assert out.tolist() == want


def test_options_defaults_are_the_papers():
    build.build()
    from paper_2206_11009_gb300 import default_options
    o = default_options()
    # Section 5.2: tolerance 1e-6, CG 1e-6 / 1e-3, 200 IPM iterations, 1000 CG, 3 correctors
    assert (o.tol, o.cg_tol_pred, o.cg_tol_corr, o.max_iter, o.max_cg, o.max_corr) == (1e-6, 1e-6, 1e-3, 200, 1000, 3)
    assert o.step_scale == 0.995


def test_invalid_arguments_fail_without_touching_the_gpu():
    build.build()
    lib = _lib.load()
    h = ctypes.c_void_p()
    prob = _lib.OtProblem()
    prob.m = 0
    assert lib.ot_ipm_create(ctypes.byref(prob), None, ctypes.byref(h)) == _lib.OT_ERR_ARG
    assert b"sizes" in lib.ot_last_error()
    a = np.array([0.5, 0.5])
    b = np.array([0.7, 0.4])          # unbalanced
    prob.m, prob.n = 2, 2
    prob.a = a.ctypes.data_as(ctypes.c_void_p)
    prob.b = b.ctypes.data_as(ctypes.c_void_p)
    prob.src_w = prob.dst_w = 2
    assert lib.ot_ipm_create(ctypes.byref(prob), None, ctypes.byref(h)) == _lib.OT_ERR_ARG
    assert lib.ot_price_topk(0, 0, *([None] * 8), 0, 0, 1, None, None, None, None, None) == _lib.OT_ERR_ARG
