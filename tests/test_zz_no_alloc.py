"""GPU test of hfmm_leaf_order_noalloc, the entry point that allocates no
device memory (for callers whose device memory belongs to their own pool or
who must not trigger cudaMalloc's device synchronisation).

It is compared, through the C ABI, with the leaf order the existing entry
points produce (hfmm_plan_create + hfmm_plan_get_tree at the same leaf
level), on two calls in a row with different inputs, so that state left in
its shared static scratch by the first call cannot leak into the second.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1703_09136_gb300 import Plan, _native  # noqa: E402
from paper_1703_09136_gb300 import build as _build  # noqa: E402


def _morton(ix, iy):
    out = np.zeros(ix.shape, dtype=np.int64)
    for b in range(16):
        out |= ((ix.astype(np.int64) >> b) & 1) << (2 * b)
        out |= ((iy.astype(np.int64) >> b) & 1) << (2 * b + 1)
    return out


def _reference(xy, medium, levels):
    plan = Plan(xy, medium, levels=levels)
    perm, ix, iy = plan.tree()
    plan.close()
    counts = np.bincount(_morton(ix, iy), minlength=4 ** levels)
    begin = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    return perm, begin


def _noalloc(lib, xy, levels):
    n = xy.shape[0]
    d_xy = torch.from_numpy(xy).cuda()
    d_perm = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    d_begin = torch.full((4 ** levels + 1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.hfmm_leaf_order_noalloc(ctypes.c_int64(n), ctypes.c_void_p(d_xy.data_ptr()), levels,
                                     ctypes.c_void_p(d_perm.data_ptr()), ctypes.c_void_p(d_begin.data_ptr()),
                                     ctypes.c_void_p(stream))
    _native.check(st)
    torch.cuda.synchronize()
    return d_perm.cpu().numpy(), d_begin.cpu().numpy()


def test_noalloc_leaf_order_matches_plan_tree_on_two_calls():
    _build.build()
    lib = _native.lib()
    cases = [
        (W.points(3, 50000), W.WORKLOADS[3].medium, 6),     # two-layer cloud, 4096 leaves
        (W.points(1), W.WORKLOADS[1].medium, 3),            # smaller second call: old scratch must not leak
    ]
    for xy, med, levels in cases:
        perm_ref, begin_ref = _reference(xy, med, levels)
        perm, begin = _noalloc(lib, xy, levels)
        assert np.array_equal(perm, perm_ref)
        assert np.array_equal(begin, begin_ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    # rejected on the host before any device work (the pointers are never read)
    lib = _native.lib()
    st = lib.hfmm_leaf_order_noalloc(ctypes.c_int64((1 << 18) + 1), ctypes.c_void_p(1), 4,
                                     ctypes.c_void_p(1), ctypes.c_void_p(1), None)
    assert st == 1 and b"scratch" in lib.hfmm_last_error()
    st = lib.hfmm_leaf_order_noalloc(ctypes.c_int64(100), ctypes.c_void_p(1), 10,
                                     ctypes.c_void_p(1), ctypes.c_void_p(1), None)
    assert st == 1
