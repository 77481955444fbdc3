"""ot_price_topk_noalloc -- the pricing selection for callers that cannot allocate device
memory while they run (e.g. a serving process that reserved its whole memory budget at start-up),
with all scratch in a fixed device array of the library -- must return exactly what the
allocating entry point ot_price_topk returns.  Two calls in a row with different inputs check
that nothing left in the shared array by the previous call leaks into the next one.

This file is named so that pytest collects it last."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def _call(fn, sx, sy, tx, ty, u, v, si, sj, kmax, precision):
    import torch
    T = U.cuda_tensors(sx, sy, tx, ty, u, v, si, sj)
    dev = T[0].device
    oi = torch.full((max(kmax, 1),), -7, dtype=torch.int32, device=dev)
    oj = torch.full((max(kmax, 1),), -7, dtype=torch.int32, device=dev)
    od = torch.full((max(kmax, 1),), np.nan, dtype=torch.float64, device=dev)
    cnt = torch.full((1,), -1, dtype=torch.int32, device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    psi = len(si)
    rc = fn(len(sx), len(tx), *[t.data_ptr() for t in T[:6]], T[6].data_ptr() if psi else None,
            T[7].data_ptr() if psi else None, psi, kmax, precision, oi.data_ptr(), oj.data_ptr(), od.data_ptr(),
            cnt.data_ptr(), stream)
    torch.cuda.synchronize()
    k = int(cnt.item())
    return rc, oi[:k].cpu().numpy(), oj[:k].cpu().numpy(), od[:k].cpu().numpy()


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2206_11009_gb300 import _lib
    lib = _lib.load()
    cases = [(64, 64, 6.0, 1), (48, 40, 3.0, 0)]     # (width, height, dual slope, precision)
    for w, h, amp, precision in cases:
        sx, sy = U.rect_coords(w, h)
        u, v = U.banded_duals(sx, sy, sx, sy, seed=w + h, amp=amp, noise=2.0)
        si, sj = U.neighbourhood_support(sx, sy, sx, sy)
        kmax = len(sx)
        rc_a, ai, aj, ad = _call(lib.ot_price_topk, sx, sy, sx, sy, u, v, si, sj, kmax, precision)
        rc_b, bi, bj, bd = _call(lib.ot_price_topk_noalloc, sx, sy, sx, sy, u, v, si, sj, kmax, precision)
        assert rc_a == 0 and rc_b == 0, lib.ot_last_error()
        assert len(ai) > 0
        assert np.array_equal(ai, bi) and np.array_equal(aj, bj)
        assert np.array_equal(ad, bd)          # the pricing path is bit-exact


def _cudart():
    """The CUDA runtime the process already loaded (torch's), for reading the device's default
    memory pool -- the pool the allocating entry point draws its scratch from."""
    import torch
    torch.cuda.init()
    path = None
    with open("/proc/self/maps") as f:
        for line in f:
            if "libcudart.so" in line:
                path = line.split()[-1]
                break
    if path is None:
        import glob
        found = sorted(glob.glob("/usr/local/cuda/lib64/libcudart.so*"))
        path = found[0] if found else "libcudart.so"
    return ctypes.CDLL(path)


def _pool_used_high(rt, reset: bool) -> int:
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), 0) == 0
    attr_used_high = 0x8      # cudaMemPoolAttrUsedMemHigh
    val = ctypes.c_uint64(0)
    if reset:
        assert rt.cudaMemPoolSetAttribute(pool, attr_used_high, ctypes.byref(val)) == 0
    assert rt.cudaMemPoolGetAttribute(pool, attr_used_high, ctypes.byref(val)) == 0
    return val.value


def test_noalloc_takes_nothing_from_the_memory_pool():
    """The defining property: the call draws no device memory.  The high-water mark of the device's
    default pool stays where it was across the call, while the allocating entry point (the
    control) raises it."""
    import __graft_entry__
    import torch
    __graft_entry__.build()
    from paper_2206_11009_gb300 import _lib
    lib = _lib.load()
    rt = _cudart()
    sx, sy = U.rect_coords(64, 64)
    u, v = U.banded_duals(sx, sy, sx, sy, seed=3, amp=6.0, noise=2.0)
    si, sj = U.neighbourhood_support(sx, sy, sx, sy)
    _call(lib.ot_price_topk_noalloc, sx, sy, sx, sy, u, v, si, sj, len(sx), 1)   # module loaded, warm
    torch.cuda.synchronize()
    before = _pool_used_high(rt, reset=True)
    rc, *_ = _call(lib.ot_price_topk_noalloc, sx, sy, sx, sy, u, v, si, sj, len(sx), 1)
    assert rc == 0
    assert _pool_used_high(rt, reset=False) == before
    before = _pool_used_high(rt, reset=True)
    rc, *_ = _call(lib.ot_price_topk, sx, sy, sx, sy, u, v, si, sj, len(sx), 1)
    assert rc == 0
    assert _pool_used_high(rt, reset=False) > before


def test_noalloc_candidate_overflow_changes_no_output():
    """A candidate set beyond the fixed array (steep duals, kmax above the number of negative
    reduced costs: every one is rechecked) returns OT_ERR_BUF_TOO_SMALL, names the allocating
    entry point, and leaves every output buffer as it was."""
    import __graft_entry__
    import torch
    __graft_entry__.build()
    from paper_2206_11009_gb300 import _lib
    lib = _lib.load()
    sx, sy = U.rect_coords(64, 64)
    u, v = U.banded_duals(sx, sy, sx, sy, seed=9, amp=20.0, noise=2.0)
    si = np.zeros(0, np.int32)
    kmax = 2_000_000
    T = U.cuda_tensors(sx, sy, sx, sy, u, v)
    dev = T[0].device
    oi = torch.full((kmax,), -7, dtype=torch.int32, device=dev)
    oj = torch.full((kmax,), -7, dtype=torch.int32, device=dev)
    od = torch.full((kmax,), np.nan, dtype=torch.float64, device=dev)
    cnt = torch.full((1,), -1, dtype=torch.int32, device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    rc = lib.ot_price_topk_noalloc(len(sx), len(sx), *[t.data_ptr() for t in T], None, None, 0, kmax, 1,
                                   oi.data_ptr(), oj.data_ptr(), od.data_ptr(), cnt.data_ptr(), stream)
    torch.cuda.synchronize()
    assert rc == _lib.OT_ERR_BUF_TOO_SMALL
    assert b"ot_price_topk" in lib.ot_last_error()
    assert int(cnt.item()) == -1
    assert bool((oi == -7).all()) and bool((oj == -7).all()) and bool(torch.isnan(od).all())
    # the allocating entry point handles the same call
    rc2, ai, aj, ad = _call(lib.ot_price_topk, sx, sy, sx, sy, u, v, si, si, kmax, 1)
    assert rc2 == 0 and len(ai) > 400_000


def test_noalloc_rejects_sizes_beyond_its_limit():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2206_11009_gb300 import _lib
    lib = _lib.load()
    sx, sy = U.rect_coords(130, 130)          # m = 16900 > 16384
    u = np.zeros(len(sx))
    si = np.zeros(0, np.int32)
    rc, *_ = _call(lib.ot_price_topk_noalloc, sx, sy, sx, sy, u, u, si, si, 8, 1)
    assert rc == _lib.OT_ERR_ARG
    assert b"16384" in lib.ot_last_error()
