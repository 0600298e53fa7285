"""GPU parity of the warm starts (CQK_INIT_WARM): eq. (CQKlambda0) over the free set of a
primal estimate for cqk_solve (Sec. 2), Alg. 2 per chunk on the estimate's support for the
projections (Sec. 3.3), single and batched, against the oracle's warm starts."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2603_15910_b300 import api, workloads as W
from helpers import assert_feasible, assert_x_close, np64

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _estimate(x, l, u, seed, frac=0.1):
    """x* with a fraction of its entries moved (some onto their bounds, some inside)."""
    rng = np.random.default_rng(seed)
    xb = x.copy()
    k = rng.uniform(size=x.size) < frac
    xb[k] = np.where(rng.uniform(size=int(k.sum())) < 0.5, l[k], (l[k] + u[k]) / 2)
    return xb


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n", [5, 1000, 10003, 300001])
def test_general_warm_start_matches_oracle(n, dtype):
    p = W.uncorrelated_box(n, seed=n, dtype=dtype)
    a, b, d, l, u = (np64(p[k]) for k in "abdlu")
    ref = oracle.newton_cqk(a, b, d, l, u, p["r"])
    xb = _estimate(ref["x"], l, u, seed=n)
    xbar = torch.from_numpy(xb).to(dtype).to(DEV)
    dev = [p[k].to(DEV) for k in "abdlu"]
    x, info, _ = api.solve(*dev, p["r"], init=api.Init.WARM, xbar=xbar)
    assert info.status == api.Status.OK
    l0 = oracle.lambda0_warm(a, b, d, l, u, np64(xbar), p["r"])
    # FP32 storage forms the weights b/d in float (the start only needs to be close)
    rel = 1e-10 if dtype == torch.float64 else 1e-6
    assert math.isclose(info.lambda0, l0, rel_tol=rel, abs_tol=rel), (info.lambda0, l0)
    xstar = ref["x"] if n > 4096 else oracle.solve_sort(a, b, d, l, u, p["r"])[2]
    assert_x_close(np64(x), xstar, dtype)
    assert_feasible(np64(x), b, p["r"], dtype)
    if dtype == torch.float64:
        nw = oracle.newton_cqk(a, b, d, l, u, p["r"], lam0=info.lambda0)
        assert abs(info.iters - nw["evals"]) <= 1, (info.iters, nw["evals"])
        # (the paper's warm formula drops the active bounds' share of r, so on this family it
        # need not beat the cold start; only the agreement with the oracle is asserted)


def test_general_warm_start_empty_free_set_is_the_cold_start():
    p = W.uncorrelated_box(5000, seed=3)
    xbar = p["l"].clone().to(DEV)  # every variable at its lower bound: J empty
    dev = [p[k].to(DEV) for k in "abdlu"]
    _, warm, _ = api.solve(*dev, p["r"], init=api.Init.WARM, xbar=xbar)
    _, cold, _ = api.solve(*dev, p["r"])
    # the same formula over all variables; the two passes sum in different orders (plain loads
    # vs the staged tiles of the cold start), so lambda_0 agrees to rounding
    assert math.isclose(warm.lambda0, cold.lambda0, rel_tol=1e-13) and warm.iters == cold.iters


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("l1", [False, True])
@pytest.mark.parametrize("n", [1, 77, 20000, 1000003])
def test_projection_warm_start_matches_oracle(n, dtype, l1):
    y = W.simplex_normal(n, seed=n + 1, dtype=dtype)
    y64 = np64(y)
    # the estimate: the projection of a perturbed y
    yp = y64 + 0.05 * np.random.default_rng(n).normal(size=n)
    if l1:
        _, xb, _ = oracle.project_l1(yp, 1.0)
    else:
        _, xb = oracle.project_simplex_sort(yp, 1.0)
    xbar = torch.from_numpy(xb).to(dtype).to(DEV)
    fn = api.project_l1 if l1 else api.project_simplex
    x, info, _ = fn(y.to(DEV), 1.0, init=api.Init.WARM, xbar=xbar)
    assert info.status == api.Status.OK
    if l1:
        lam, xstar, inside = oracle.project_l1(y64, 1.0)
    else:
        lam, xstar = oracle.project_simplex_sort(y64, 1.0)
        inside = False
    assert_x_close(np64(x), xstar, dtype)
    if not inside:
        xbq = np64(xbar)
        l0, S, C = oracle.condat_chunks_warm(y64, xbq, 1.0, info.tile, info.nchunks, l1=l1)
        if dtype == torch.float64:
            assert math.isclose(info.lambda0, l0, rel_tol=1e-13, abs_tol=1e-15), (info.lambda0, l0)
        else:
            assert math.isclose(info.lambda0, l0, rel_tol=1e-6, abs_tol=1e-7), (info.lambda0, l0)


def test_projection_warm_start_empty_support_fallback():
    y = W.simplex_normal(5000, seed=2)
    y64 = np64(y)
    for l1 in (False, True):
        fn = api.project_l1 if l1 else api.project_simplex
        x, info, _ = fn(y.to(DEV), 1.0, init=api.Init.WARM, xbar=torch.zeros(5000, dtype=torch.float64, device=DEV))
        y1 = abs(y64[0]) if l1 else y64[0]
        assert info.lambda0 == max(1.0 / 5000, -y1)
        assert info.status == api.Status.OK
        ref = oracle.project_l1(y64, 1.0)[1] if l1 else oracle.project_simplex_sort(y64, 1.0)[1]
        assert_x_close(np64(x), ref, torch.float64)


def test_warm_start_from_the_solution_needs_few_iterations():
    y = W.simplex_normal(2_000_000, seed=5).to(DEV)
    x0, cold, _ = api.project_simplex(y, 1.0)
    x1, warm, _ = api.project_simplex(y, 1.0, init=api.Init.WARM, xbar=x0)
    assert warm.iters <= 2 and cold.iters > warm.iters
    assert math.isclose(warm.lambda0, cold.lam, rel_tol=1e-13, abs_tol=1e-15)
    assert torch.equal(x0, x1) or float((x0 - x1).abs().max()) <= 1e-12


@pytest.mark.parametrize("l1", [False, True])
def test_batched_warm_start_matches_oracle(l1):
    lens = [3000, 1, 0, 517, 20000, 64, 9999]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    n = int(off[-1])
    y = W.simplex_normal(n, seed=9)
    y64 = np64(y)
    xb = np.zeros(n)
    rng = np.random.default_rng(1)
    for k, m in enumerate(lens):
        lo, hi = int(off[k]), int(off[k + 1])
        if m == 0:
            continue
        yp = y64[lo:hi] + 0.05 * rng.normal(size=m)
        xb[lo:hi] = oracle.project_l1(yp, 1.0)[1] if l1 else oracle.project_simplex_sort(yp, 1.0)[1]
    r = torch.ones(len(lens), dtype=torch.float64)
    fn = api.project_l1_batched if l1 else api.project_simplex_batched
    xbar = torch.from_numpy(xb).to(DEV)
    x, infos, _ = fn(y.to(DEV), torch.from_numpy(off), r, init=api.Init.WARM, xbar=xbar)
    xs = np64(x)
    for k, m in enumerate(lens):
        if m == 0:
            continue
        lo, hi = int(off[k]), int(off[k + 1])
        if l1:
            lam, xstar, inside = oracle.project_l1(y64[lo:hi], 1.0)
        else:
            (lam, xstar), inside = oracle.project_simplex_sort(y64[lo:hi], 1.0), False
        assert infos[k].status == api.Status.OK
        assert_x_close(xs[lo:hi], xstar, torch.float64, f"instance {k}")
        if not inside:
            l0, S, C = oracle.condat_chunks_warm(y64[lo:hi], xb[lo:hi], 1.0, infos[k].tile, infos[k].nchunks, l1=l1,
                                                 shift=lo % infos[k].tile)
            assert math.isclose(infos[k].lambda0, l0, rel_tol=1e-13, abs_tol=1e-15), (k, infos[k].lambda0, l0)


def test_batched_general_warm_start():
    lens = [2000, 0, 31, 40000, 777]
    parts = [W.uncorrelated_box(m, seed=20 + k) for k, m in enumerate(lens)]
    cat = {k: torch.cat([p[k] for p in parts]) for k in "abdlu"}
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    r = torch.tensor([p["r"] for p in parts], dtype=torch.float64)
    xb = np.zeros(int(off[-1]))
    for k, m in enumerate(lens):
        lo, hi = int(off[k]), int(off[k + 1])
        if m:
            ref = oracle.newton_cqk(*(np64(parts[k][q]) for q in "abdlu"), parts[k]["r"])
            xb[lo:hi] = _estimate(ref["x"], np64(parts[k]["l"]), np64(parts[k]["u"]), seed=k)
    xbar = torch.from_numpy(xb).to(DEV)
    x, infos, _ = api.solve_batched(*(cat[k].to(DEV) for k in "abdlu"), torch.from_numpy(off), r,
                                    init=api.Init.WARM, xbar=xbar)
    xs = np64(x)
    for k, m in enumerate(lens):
        lo, hi = int(off[k]), int(off[k + 1])
        if m == 0:
            continue
        a, b, d, l, u = (np64(parts[k][q]) for q in "abdlu")
        l0 = oracle.lambda0_warm(a, b, d, l, u, xb[lo:hi], parts[k]["r"])
        assert math.isclose(infos[k].lambda0, l0, rel_tol=1e-10, abs_tol=1e-12)
        xstar = oracle.newton_cqk(a, b, d, l, u, parts[k]["r"])["x"]
        assert_x_close(xs[lo:hi], xstar, torch.float64, f"instance {k}")


def test_warm_start_requires_an_estimate():
    y = W.simplex_normal(100, seed=1).to(DEV)
    with pytest.raises(RuntimeError):
        api.project_simplex(y, 1.0, init=api.Init.WARM)
