"""The allocation-free simplex projection (cqk_project_simplex_noalloc).

It exists for callers that cannot allocate device memory at call time (for example a plugin
whose host application owns the device allocator, or a fixed-memory real-time loop), so it
keeps its scratch in a static device array instead of a caller workspace.  This test calls
it through the C ABI twice in a row -- the second time with different data, so stale
contents of the shared array would show -- and compares each result with the regular
cqk_project_simplex on the same input, within the FP64 tolerance of the other tests.  The
file is named to be collected last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2603_15910_b300 import api, workloads as W
from helpers import TOL_X, np64

pytestmark = pytest.mark.gpu


def _noalloc(y, r, init):
    lib = api.library()
    f = lib.cqk_project_simplex_noalloc
    f.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(api._Options), ctypes.c_void_p]
    f.restype = ctypes.c_int
    x = torch.empty_like(y)
    info = torch.zeros(api.INFO_BYTES, dtype=torch.uint8, device=y.device)
    opt = api.make_options(init=init)
    rc = f(y.numel(), api.dtype_code(y.dtype), api.ptr(y), r, api.ptr(x), None, api.ptr(info), ctypes.byref(opt),
           api.stream_handle())
    assert rc == 0, lib.cqk_status_string(rc)
    return x, api.Info.from_bytes(info.cpu().numpy().tobytes())


def test_noalloc_matches_regular_projection_twice():
    for call, (n, seed, r, init) in enumerate([(1_000_003, 1, 1.0, api.Init.CONDAT),
                                               (250_001, 2, 3.5, api.Init.FORMULA)]):
        y = W.simplex_normal(n, seed=seed, device="cuda")
        x_ref, info_ref, _ = api.project_simplex(y, r, init=init)
        x, info = _noalloc(y, r, init)
        assert info.status == api.Status.OK and info_ref.status == api.Status.OK, (call, info)
        err = float(np.max(np.abs(np64(x) - np64(x_ref))))
        assert err <= TOL_X[torch.float64] * (1 + float(np.max(np.abs(np64(x_ref))))), (call, err)
        assert abs(float(x.sum()) - r) <= 1e-12 * r


def test_noalloc_rejects_a_grid_beyond_its_scratch():
    lib = api.library()
    y = torch.randn(1000, dtype=torch.float64, device="cuda")
    x = torch.empty_like(y)
    info = torch.zeros(api.INFO_BYTES, dtype=torch.uint8, device="cuda")
    opt = api.make_options(max_blocks=100000)
    f = lib.cqk_project_simplex_noalloc
    f.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(api._Options), ctypes.c_void_p]
    assert f(1000, 0, api.ptr(y), 1.0, api.ptr(x), None, api.ptr(info), ctypes.byref(opt), api.stream_handle()) == 7
