"""The allocation-free simplex projection (cqk_project_simplex_noalloc).

It exists for callers that cannot allocate device memory at call time (for example a plugin
whose host application owns the device allocator, or a fixed-memory real-time loop), so it
keeps its scratch in a static device array instead of a caller workspace.  This test calls
it through the C ABI twice in a row -- the second time with different data, so stale
contents of the shared array would show -- and compares each result with the oracle's
sort-based projection and with the regular cqk_project_simplex on the same input, within the
tolerances of the other tests (FP64 and FP32 storage), the free mask included.  The file is
named to be collected last."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2603_15910_b300 import api, workloads as W
from helpers import TOL_FEAS, TOL_X, assert_x_close, mask_bits, np64

pytestmark = pytest.mark.gpu


def _fn():
    f = api.library().cqk_project_simplex_noalloc
    f.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(api._Options), ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def _noalloc(y, r, init, want_mask):
    x = torch.empty_like(y)
    mask = torch.zeros((y.numel() + 31) // 32, dtype=torch.int32, device=y.device) if want_mask else None
    info = torch.zeros(api.INFO_BYTES, dtype=torch.uint8, device=y.device)
    opt = api.make_options(init=init)
    rc = _fn()(y.numel(), api.dtype_code(y.dtype), api.ptr(y), r, api.ptr(x), api.ptr(mask), api.ptr(info),
               ctypes.byref(opt), api.stream_handle())
    assert rc == 0, api.library().cqk_status_string(rc)
    return x, api.Info.from_bytes(info.cpu().numpy().tobytes()), mask


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_matches_oracle_and_regular_projection_twice(dtype):
    for call, (n, seed, r, init, want_mask) in enumerate([(1_000_003, 1, 1.0, api.Init.CONDAT, True),
                                                          (250_001, 2, 3.5, api.Init.FORMULA, False)]):
        y = W.simplex_normal(n, seed=seed, device="cuda", dtype=dtype)
        x_ref, info_ref, _ = api.project_simplex(y, r, init=init)
        x, info, mask = _noalloc(y, r, init, want_mask)
        assert info.status == api.Status.OK and info_ref.status == api.Status.OK, (call, info)
        xs = np64(x)
        # the oracle's exact projection of the same (stored) values
        lam_star, xstar = oracle.project_simplex_sort(np64(y), r)
        assert_x_close(xs, xstar, dtype, f"call {call} vs oracle")
        assert_x_close(xs, np64(x_ref), dtype, f"call {call} vs cqk_project_simplex")
        res = abs(float(np.sum(xs, dtype=np.longdouble)) - r)
        assert res <= TOL_FEAS[dtype] * r, (call, res)
        if want_mask:
            assert np.array_equal(mask_bits(mask, n), xs > 0), call
            assert info.nfree == int((xs > 0).sum())
        # the same multiplier as the workspace path: the same kernel, the same grid partition
        assert abs(info.lam - info_ref.lam) <= TOL_X[dtype] * (1 + abs(info_ref.lam)), (info.lam, info_ref.lam)


def test_noalloc_rejects_a_grid_beyond_its_scratch():
    y = torch.randn(1000, dtype=torch.float64, device="cuda")
    x = torch.empty_like(y)
    info = torch.zeros(api.INFO_BYTES, dtype=torch.uint8, device="cuda")
    opt = api.make_options(max_blocks=100000)
    rc = _fn()(1000, 0, api.ptr(y), 1.0, api.ptr(x), None, api.ptr(info), ctypes.byref(opt), api.stream_handle())
    assert rc == api.Status.BAD_ARG
