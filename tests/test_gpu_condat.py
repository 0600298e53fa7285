"""GPU parity of the parallel Alg. 2 start (CQK_INIT_CONDAT) on inputs that put the scan's
tests on a knife edge: integer-valued y (y_j + lambda = 0 and lambda_{J u {j}} = r - y_j hold
exactly, so the double-float shortcut must defer to FP64), magnitudes outside the
double-float range, and a large r.  lambda_0 must equal the oracle's chunked Alg. 2."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2603_15910_b300 import api
from helpers import assert_x_close, np64

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _check(y, r, l1, dtype=torch.float64, **kw):
    yt = torch.from_numpy(y).to(dtype)
    y64 = np64(yt)
    fn = api.project_l1 if l1 else api.project_simplex
    x, info, _ = fn(yt.to(DEV), r, init=api.Init.CONDAT, **kw)
    assert info.status == api.Status.OK, info
    if l1:
        lam, xstar, inside = oracle.project_l1(y64, r)
        if inside:
            return
    else:
        lam, xstar = oracle.project_simplex_sort(y64, r)
    assert_x_close(np64(x), xstar, dtype)
    l0, S, C = oracle.condat_chunks(y64, r, info.tile, info.nchunks, l1=l1)
    assert math.isclose(info.lambda0, l0, rel_tol=1e-13, abs_tol=1e-300), (info.lambda0, l0, info)


@pytest.mark.parametrize("l1", [False, True])
@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_condat_integer_ties(seed, l1, dtype):
    rng = np.random.default_rng(seed)
    n = [1000, 70000, 1_000_000, 3][seed]
    y = rng.integers(-3, 4, size=n).astype(np.float64)
    _check(y, float(rng.integers(1, 6)), l1, dtype)


@pytest.mark.parametrize("l1", [False, True])
def test_condat_outside_the_double_float_range(l1):
    rng = np.random.default_rng(5)
    y = rng.normal(size=200_000)
    y[::7] *= 1e-70
    y[3::11] *= 1e70
    _check(y, 1.0, l1)
    _check(rng.normal(size=50_000) * 1e-80, 1e-79, l1)


@pytest.mark.parametrize("l1", [False, True])
def test_condat_large_radius_and_scale(l1):
    rng = np.random.default_rng(6)
    y = rng.normal(size=300_000) * 1e30
    _check(y, 3e31, l1)
    _check(rng.uniform(size=300_000), 50.0, l1)


@pytest.mark.parametrize("l1", [False, True])
@pytest.mark.parametrize("scan_warps", [1, 2, 4])
@pytest.mark.parametrize("n,blocks", [(100, 1), (3000, 1), (9000, 1), (70001, 1), (300000, 3), (2_000_003, 0)])
def test_condat_scan_warps_partition(n, blocks, scan_warps, l1):
    # each block deals its tiles to scan_warps chunks: the partition has blocks * scan_warps
    # chunks of round-robin tiles, which the oracle reproduces from info.nchunks
    rng = np.random.default_rng(n + scan_warps)
    y = rng.normal(size=n) * 2.0
    for dtype in (torch.float64, torch.float32):
        _check(y, 1.0, l1, dtype, scan_warps=scan_warps, max_blocks=blocks)


def test_condat_scan_warps_batched():
    lens = [9000, 1, 40000, 0, 70001, 517, 200000]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    n = int(off[-1])
    y = np.random.default_rng(3).normal(size=n)
    r = torch.ones(len(lens), dtype=torch.float64)
    for l1 in (False, True):
        fn = api.project_l1_batched if l1 else api.project_simplex_batched
        for sw in (0, 1, 2, 4):
            x, infos, _ = fn(torch.from_numpy(y).to(DEV), torch.from_numpy(off), r, init=api.Init.CONDAT,
                             scan_warps=sw, warp_elems=-1)
            xs = np64(x)
            for k, m in enumerate(lens):
                if m == 0:
                    continue
                lo, hi = int(off[k]), int(off[k + 1])
                assert infos[k].status == api.Status.OK, (k, sw, infos[k])
                if l1:
                    lam, xstar, inside = oracle.project_l1(y[lo:hi], 1.0)
                else:
                    (lam, xstar), inside = oracle.project_simplex_sort(y[lo:hi], 1.0), False
                assert_x_close(xs[lo:hi], xstar, torch.float64, f"instance {k} scan_warps {sw}")
                if not inside:
                    l0, S, C = oracle.condat_chunks(y[lo:hi], 1.0, infos[k].tile, infos[k].nchunks, l1=l1,
                                                    shift=lo % infos[k].tile)
                    assert math.isclose(infos[k].lambda0, l0, rel_tol=1e-13, abs_tol=1e-300), (k, sw)


@pytest.mark.parametrize("scan_warps", [2, 4])
def test_condat_scan_warps_warm_start(scan_warps):
    # the warm start's support filter with several chunks per block
    n = 150001
    y = np.random.default_rng(21).normal(size=n)
    lam, xs = oracle.project_simplex_sort(y + 0.05 * np.random.default_rng(3).normal(size=n), 1.0)
    xbar = torch.from_numpy(xs).to(DEV)
    x, info, _ = api.project_simplex(torch.from_numpy(y).to(DEV), 1.0, init=api.Init.WARM, xbar=xbar,
                                     scan_warps=scan_warps, max_blocks=1)
    assert info.status == api.Status.OK
    assert_x_close(np64(x), oracle.project_simplex_sort(y, 1.0)[1], torch.float64)
    l0, S, C = oracle.condat_chunks_warm(y, xs, 1.0, info.tile, info.nchunks)
    assert math.isclose(info.lambda0, l0, rel_tol=1e-13, abs_tol=1e-15), (info.lambda0, l0, info.nchunks)


@pytest.mark.parametrize("l1", [False, True])
@pytest.mark.parametrize("n,blocks", [(300_000, 1), (2_000_003, 4), (1_048_576 + 17, 2)])
def test_condat_split_scan(n, blocks, l1):
    # chunks of 64 tiles or more: one warp walks the tiles and queues the survivors, another
    # takes them; lambda_0 must still be the oracle's chunked Alg. 2, in FP64 and FP32 storage
    rng = np.random.default_rng(n + blocks)
    y = rng.normal(size=n) * 3.0
    for dtype in (torch.float64, torch.float32):
        _check(y, 1.0, l1, dtype, max_blocks=blocks)


@pytest.mark.parametrize("l1", [False, True])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_condat_split_scan_survivor_flood(l1, dtype):
    # integer ties and an ascending run: tiles with far more survivors than the queue holds,
    # so the walking warp waits for room; exact-tie decisions go to the FP64 quotient
    rng = np.random.default_rng(11)
    y = rng.integers(-3, 4, size=600_000).astype(np.float64)
    _check(y, 2.0, l1, dtype, max_blocks=1)
    z = np.linspace(-5.0, 5.0, 400_000)
    _check(z, 1.0, l1, dtype, max_blocks=1)


def test_condat_split_scan_warm_start():
    # the warm start's support filter on split chunks
    n = 400_001
    y = np.random.default_rng(23).normal(size=n)
    lam, xs = oracle.project_simplex_sort(y + 0.05 * np.random.default_rng(4).normal(size=n), 1.0)
    xbar = torch.from_numpy(xs).to(DEV)
    x, info, _ = api.project_simplex(torch.from_numpy(y).to(DEV), 1.0, init=api.Init.WARM, xbar=xbar, max_blocks=2)
    assert info.status == api.Status.OK
    assert_x_close(np64(x), oracle.project_simplex_sort(y, 1.0)[1], torch.float64)
    l0, S, C = oracle.condat_chunks_warm(y, xs, 1.0, info.tile, info.nchunks)
    assert math.isclose(info.lambda0, l0, rel_tol=1e-13, abs_tol=1e-15), (info.lambda0, l0, info.nchunks)
