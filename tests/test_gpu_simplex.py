"""GPU parity of the simplex and l1-ball projections (cqk_project_simplex,
cqk_project_l1) against the FP64 oracle, through the C ABI."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2603_15910_b300 import api, workloads as W
from helpers import assert_x_close, mask_bits, np64

pytestmark = pytest.mark.gpu
DEV = "cuda"
INITS = [api.Init.FORMULA, api.Init.CONDAT]


def _sum_abs_tol(x, r, dtype):
    res = abs(float(np.sum(np.abs(x), dtype=np.longdouble)) - r)
    assert res <= (1e-12 if dtype == torch.float64 else 1e-5) * r, res


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("init", INITS)
@pytest.mark.parametrize("n", [1, 2, 3, 31, 257, 1000, 10003, 200001])
def test_simplex_matches_oracle(n, init, dtype):
    for sparse in (False, True):
        y = W.simplex_normal(n, seed=n + 7, sparse=sparse, dtype=dtype)
        y64 = np64(y)
        x, info, mask = api.project_simplex(y.to(DEV), 1.0, init=init, want_mask=True)
        assert info.status == api.Status.OK, info
        lam_star, xstar = oracle.project_simplex_sort(y64, 1.0)
        xs = np64(x)
        assert_x_close(xs, xstar, dtype, f"n={n} init={init}")
        _sum_abs_tol(xs, 1.0, dtype)
        assert np.array_equal(mask_bits(mask, n), xs > 0)
        assert info.nfree == int((xs > 0).sum())
        if dtype == torch.float64:
            if init == api.Init.CONDAT:
                lam0, S, C = oracle.condat_chunks(y64, 1.0, info.tile, info.nchunks)
                assert math.isclose(info.lambda0, lam0, rel_tol=1e-13, abs_tol=1e-15), (info, lam0)
                nw = oracle.newton_simplex(y64, 1.0, lam0=info.lambda0)
            else:
                nw = oracle.newton_simplex(y64, 1.0)
                assert math.isclose(info.lambda0, max(nw["lam0"], -y64.max()), rel_tol=1e-12, abs_tol=1e-14)
            assert abs(info.iters - nw["evals"]) <= 1, (info.iters, nw["evals"])


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("init", INITS)
@pytest.mark.parametrize("n", [1, 5, 64, 999, 10001, 150000])
def test_l1_matches_oracle(n, init, dtype):
    for scale in (1.0, 1e-4):
        y = W.simplex_normal(n, seed=3 * n + 1, dtype=dtype) * scale
        y64 = np64(y)
        x, info, mask = api.project_l1(y.to(DEV), 1.0, init=init, want_mask=True)
        assert info.status == api.Status.OK, info
        lam, xstar, inside = oracle.project_l1(y64, 1.0)
        xs = np64(x)
        assert_x_close(xs, xstar, dtype, f"n={n} scale={scale}")
        if inside:
            assert info.stop == "inside" and np.array_equal(xs, y64)
        else:
            _sum_abs_tol(xs, 1.0, dtype)
            assert np.array_equal(np.sign(xs[xs != 0]), np.sign(y64[xs != 0]))
            if dtype == torch.float64 and init == api.Init.CONDAT:
                lam0, S, C = oracle.condat_chunks(y64, 1.0, info.tile, info.nchunks, l1=True)
                assert math.isclose(info.lambda0, lam0, rel_tol=1e-13, abs_tol=1e-15)
        assert np.array_equal(mask_bits(mask, n), xs != 0)


def test_simplex_special_cases():
    cases = [np.full(9, 0.25), np.array([0.1, 5.0, -0.3, 0.2]), np.array([-3.0]), np.array([0.2, 0.3, 0.5]),
             np.array([3.0, 1.0, 0.0, 2.0]), np.zeros(100), np.arange(1000, dtype=np.float64)]
    for y in cases:
        for init in INITS:
            x, info, _ = api.project_simplex(torch.tensor(y, device=DEV), 1.0, init=init)
            assert info.status == api.Status.OK
            assert_x_close(np64(x), oracle.project_simplex_sort(y, 1.0)[1], torch.float64, str(y[:4]))


def test_given_start_and_radius():
    y = W.simplex_normal(20000, seed=5)
    for r in (0.01, 1.0, 37.5):
        lam_star = oracle.project_simplex_sort(y.numpy(), r)[0]
        for lam0 in (lam_star + 1.0, lam_star - 1.0, 0.0):
            x, info, _ = api.project_simplex(y.to(DEV), r, init=api.Init.GIVEN, lambda0=lam0)
            assert info.status == api.Status.OK
            assert_x_close(np64(x), oracle.project_simplex_sort(y.numpy(), r)[1], torch.float64)
            nw = oracle.newton_simplex(y.numpy(), r, lam0=lam0)
            assert abs(info.iters - nw["evals"]) <= 1


def test_theorem_3_1_monotone_from_condat_start():
    y = W.simplex_normal(300000, seed=11)
    x, info, _ = api.project_simplex(y.to(DEV), 1.0, init=api.Init.CONDAT)
    lam_star = oracle.project_simplex_sort(y.numpy(), 1.0)[0]
    assert info.lambda0 >= lam_star - 1e-12 and info.lam >= lam_star - 1e-12


def test_nan_is_bad_input():
    for init in INITS:
        y = W.simplex_normal(5000, seed=2)
        y[123] = float("nan")
        _, info, _ = api.project_simplex(y.to(DEV), 1.0, init=init)
        assert info.status == api.Status.BAD_INPUT


def test_timeout_status():
    y = W.simplex_normal(100000, seed=2).to(DEV)
    _, info, _ = api.project_simplex(y, 1.0, fault_inject=True, spin_limit_us=100000)
    assert info.status == api.Status.TIMEOUT
    x, info, _ = api.project_simplex(y, 1.0)
    assert info.status == api.Status.OK


@pytest.mark.parametrize("l1", [False, True])
def test_timeout_status_scan_queue(l1):
    # a block chunk of 64 tiles or more: the walking warp queues nothing (fault_inject = 2), the
    # scanning warp's bounded wait for the queue runs out, the call reports CQK_TIMEOUT and the
    # context stays usable
    y = W.simplex_normal(400_000, seed=4).to(DEV)
    f = api.project_l1 if l1 else api.project_simplex
    _, info, _ = f(y, 1.0, fault_inject=2, spin_limit_us=100000, max_blocks=1)
    assert info.status == api.Status.TIMEOUT
    x, info, _ = f(y, 1.0, max_blocks=1)
    assert info.status == api.Status.OK
    _, info, _ = f(y, 1.0, fault_inject=2, spin_limit_us=100000)  # chunks too short to split
    assert info.status == api.Status.OK
