"""GPU parity of the general CQK solve (cqk_solve) and of one map-reduce pass (cqk_phi)
against the FP64 oracle, through the C ABI."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2603_15910_b300 import api, workloads as W
from helpers import assert_feasible, assert_x_close, mask_bits, np64

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _dev(p, dtype):
    return {k: (v.to(DEV, dtype) if torch.is_tensor(v) else v) for k, v in p.items()}


def _np(p):
    return [np64(p[k]) for k in "abdlu"]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n", [1, 2, 3, 7, 1000, 4097, 10000, 65537])
def test_phi_pass_matches_oracle(n, dtype):
    p = _dev(W.uncorrelated_box(n, seed=n, dtype=dtype), dtype)
    a, b, d, l, u = _np(p)
    tol = 1e-13 if dtype == torch.float64 else 1e-6
    for lam in (-0.7, -0.05, 0.0, 0.13, 1.9):
        got = api.phi(p["a"], p["b"], p["d"], p["l"], p["u"], lam)
        want = oracle.phi(lam, a, b, d, l, u)
        scale = want[3]
        assert abs(got[0] - want[0]) <= tol * scale + 1e-300, (lam, got, want)
        assert abs(got[3] - want[3]) <= tol * scale
        q = np.sum(b * b / d)
        assert abs(got[1] - want[1]) <= max(tol, 1e-12) * q
        assert abs(got[2] - want[2]) <= max(tol, 1e-12) * q


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n", [1, 2, 5, 12, 33, 1000, 4099, 10000])
def test_solve_matches_oracle_box_family(n, dtype):
    for seed in range(3):
        p = _dev(W.uncorrelated_box(n, seed=100 + seed, dtype=dtype), dtype)
        a, b, d, l, u = _np(p)
        r = p["r"]
        x, info, mask = api.solve(p["a"], p["b"], p["d"], p["l"], p["u"], r, want_mask=True)
        assert info.status == api.Status.OK, info
        st, lam_star, xstar = oracle.solve_sort(a, b, d, l, u, r)
        assert st == "ok"
        xs = np64(x)
        assert_x_close(xs, xstar, dtype, f"n={n} seed={seed}")
        assert_feasible(xs, b, r, dtype, f"n={n} seed={seed}")
        if dtype == torch.float64:
            nw = oracle.newton_cqk(a, b, d, l, u, r)
            assert abs(info.iters - nw["evals"]) <= 1, (info.iters, nw["evals"])
            assert math.isclose(info.lambda0, nw["lam0"], rel_tol=1e-12, abs_tol=1e-15)
            fr = mask_bits(mask, n)
            assert np.array_equal(fr, (xs > l) & (xs < u))
            assert info.nfree == int(fr.sum())
        assert abs(info.residual) <= (1e-12 if dtype == torch.float64 else 1e-5) * info.abs_bx


@pytest.mark.parametrize("kind", ["uncorrelated", "weak", "correlated"])
def test_solve_paper_families_fp64(kind):
    for seed in range(3):
        p = _dev(W.paper_family(kind, 20000, seed=seed), torch.float64)
        a, b, d, l, u = _np(p)
        x, info, _ = api.solve(p["a"], p["b"], p["d"], p["l"], p["u"], p["r"])
        st, lam_star, xstar = oracle.solve_sort(a, b, d, l, u, p["r"])
        assert info.status == api.Status.OK
        assert_x_close(np64(x), xstar, torch.float64)
        assert_feasible(np64(x), b, p["r"], torch.float64)
        nw = oracle.newton_cqk(a, b, d, l, u, p["r"])
        assert abs(info.iters - nw["evals"]) <= 1


def test_correlated_family_fp64_and_fp32():
    for dtype in (torch.float64, torch.float32):
        p = _dev(W.correlated(50000, seed=3, dtype=dtype), dtype)
        a, b, d, l, u = _np(p)
        x, info, _ = api.solve(p["a"], p["b"], p["d"], p["l"], p["u"], p["r"])
        assert info.status == api.Status.OK
        st, lam_star, xstar = oracle.solve_sort(a, b, d, l, u, p["r"])
        assert_x_close(np64(x), xstar, dtype)
        assert_feasible(np64(x), b, p["r"], dtype)


def test_brute_force_small_instances():
    rng = np.random.default_rng(5)
    for trial in range(60):
        n = int(rng.integers(1, 13))
        d = rng.uniform(1, 100, n); b = rng.uniform(10, 25, n); a = rng.uniform(-10, 10, n)
        l = rng.uniform(-5, 0, n); u = l + rng.uniform(0.5, 5, n)
        if trial % 4 == 1:
            l[rng.uniform(size=n) < 0.3] = -np.inf
            u[rng.uniform(size=n) < 0.3] = np.inf
        lf, uf = np.where(np.isinf(l), -5, l), np.where(np.isinf(u), 5, u)
        r = float(b @ (lf + rng.uniform(0, 1, n) * (uf - lf)))
        if n > 10:
            lam, xstar = oracle.solve_sort(a, b, d, l, u, r)[1:]
        else:
            lam, xstar = oracle.brute_force_cqk(a, b, d, l, u, r)
        t = [torch.tensor(v, device=DEV) for v in (a, b, d, l, u)]
        x, info, _ = api.solve(*t, r)
        assert info.status == api.Status.OK, (trial, info)
        assert_x_close(np64(x), xstar, torch.float64, f"trial {trial}")


def test_breakpoint_search_and_secant_paths():
    # start far left: phi'_+ = 0 -> closest-breakpoint steps (Alg. 1)
    p = _dev(W.uncorrelated_box(3000, seed=9), torch.float64)
    a, b, d, l, u = _np(p)
    lam0 = float(np.min((d * l - a) / b)) - 10.0
    x, info, _ = api.solve(p["a"], p["b"], p["d"], p["l"], p["u"], p["r"], init=api.Init.GIVEN, lambda0=lam0)
    nw = oracle.newton_cqk(a, b, d, l, u, p["r"], lam0=lam0)
    assert nw["bpsearch"] >= 1 and info.status == api.Status.OK
    assert info.passes >= info.iters + nw["bpsearch"]
    assert_x_close(np64(x), oracle.solve_sort(a, b, d, l, u, p["r"])[2], torch.float64)
    assert abs(info.iters - nw["evals"]) <= 1, (info, nw["evals"])
    # steep variables make Newton steps leave the bracket (secant steps)
    rng = np.random.default_rng(1)
    hits = 0
    for s in range(40):
        n = 40
        d = rng.uniform(1, 100, n) * np.where(rng.uniform(size=n) < 0.2, 1e-3, 1.0)
        b, a = rng.uniform(10, 25, n), rng.uniform(-10, 10, n)
        l = rng.uniform(-5, 0, n); u = l + rng.uniform(0.5, 5, n)
        r = float(b @ (l + rng.uniform(0, 1, n) * (u - l)))
        lam0 = float(rng.uniform(-50, 50))
        nw = oracle.newton_cqk(a, b, d, l, u, r, lam0=lam0)
        t = [torch.tensor(v, device=DEV) for v in (a, b, d, l, u)]
        x, info, _ = api.solve(*t, r, init=api.Init.GIVEN, lambda0=lam0)
        assert info.status == api.Status.OK
        assert_x_close(np64(x), oracle.solve_sort(a, b, d, l, u, r)[2], torch.float64)
        hits += nw["secant"] > 0
    assert hits >= 1


def test_infeasible_and_bad_input():
    p = _dev(W.uncorrelated_box(1000, seed=4), torch.float64)
    bu = float((p["b"] * p["u"]).sum())
    _, info, _ = api.solve(p["a"], p["b"], p["d"], p["l"], p["u"], bu + 10.0)
    assert info.status == api.Status.INFEASIBLE
    for key, val in (("d", 0.0), ("b", -1.0), ("a", float("nan"))):
        q = {k: v.clone() if torch.is_tensor(v) else v for k, v in p.items()}
        q[key][17] = val
        _, info, _ = api.solve(q["a"], q["b"], q["d"], q["l"], q["u"], q["r"])
        assert info.status == api.Status.BAD_INPUT, key
    q = {k: v.clone() if torch.is_tensor(v) else v for k, v in p.items()}
    q["l"][5] = q["u"][5] + 1.0
    _, info, _ = api.solve(q["a"], q["b"], q["d"], q["l"], q["u"], q["r"])
    assert info.status == api.Status.BAD_INPUT


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("init", ["formula", "given"])
def test_bad_input_in_every_array(dtype, init):
    # the sanity checks of Sec. 5.1.1 reject a NaN in any array, d <= 0, b <= 0 and l > u,
    # whichever pass makes them (the lambda_0 pass, or the first Newton pass for l and u of FP32
    # data and for a given start); elements past the first tiles exercise every block's checks
    base = W.uncorrelated_box(20011, seed=31)
    cases = [("a", 17, float("nan")), ("b", 4001, float("nan")), ("d", 9000, float("nan")),
             ("l", 12345, float("nan")), ("u", 20010, float("nan")), ("d", 3, 0.0), ("d", 777, -2.0),
             ("b", 15000, -1.0), ("b", 6, 0.0)]
    for key, i, val in cases:
        h = {k: v.clone() if torch.is_tensor(v) else v for k, v in base.items()}
        h[key][i] = val
        p = _dev(h, dtype)
        kw = {} if init == "formula" else dict(init=api.Init.GIVEN, lambda0=0.1)
        _, info, _ = api.solve(p["a"], p["b"], p["d"], p["l"], p["u"], p["r"], **kw)
        assert info.status == api.Status.BAD_INPUT, (key, i, val, info)
    h = {k: v.clone() if torch.is_tensor(v) else v for k, v in base.items()}
    h["l"][11111] = h["u"][11111] + 0.5
    p = _dev(h, dtype)
    _, info, _ = api.solve(p["a"], p["b"], p["d"], p["l"], p["u"], p["r"])
    assert info.status == api.Status.BAD_INPUT, info


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("init", ["formula", "given"])
def test_signed_zero_bounds_are_valid(dtype, init):
    # l = +0, u = -0 satisfies l <= u (IEEE: the two zeros are equal), so the sanity check of
    # Sec. 5.1.1 passes and x_i = 0; also with an element outside the double-float range,
    # which takes the exact checks
    h = W.uncorrelated_box(3000, seed=21)
    h["l"][::97] = 0.0
    h["u"][::97] = -0.0
    if dtype == torch.float64:
        h["a"][5] *= 1e-25
    h["r"] = float((h["b"] * (h["l"] + h["u"]) / 2).sum())
    p = _dev(h, dtype)
    a, b, d, l, u = _np(p)
    assert np.all(l <= u)
    st, lam_star, xstar = oracle.solve_sort(a, b, d, l, u, p["r"])
    assert st == "ok"
    kw = {} if init == "formula" else dict(init=api.Init.GIVEN, lambda0=lam_star * 0.9)
    x, info, _ = api.solve(p["a"], p["b"], p["d"], p["l"], p["u"], p["r"], **kw)
    assert info.status == api.Status.OK, info
    xs = np64(x)
    assert np.all(xs[::97] == 0.0)
    assert_x_close(xs, xstar, dtype, init)


def test_values_outside_the_double_float_range_are_exact():
    p = W.uncorrelated_box(5000, seed=12)
    p["a"][::7] *= 1e-25
    p["d"][::11] *= 1e22
    u = p["u"]
    u[::13] = torch.where(u[::13] > 0, u[::13] * 1e21, u[::13])  # keeps l <= u
    q = _dev(p, torch.float64)
    a, b, d, l, u = _np(q)
    x, info, _ = api.solve(q["a"], q["b"], q["d"], q["l"], q["u"], q["r"])
    st, lam, xstar = oracle.solve_sort(a, b, d, l, u, q["r"])
    assert info.status == api.Status.OK, info
    assert_x_close(np64(x), xstar, torch.float64)


def test_unaligned_arrays_and_host_tensors():
    p = W.uncorrelated_box(2001, seed=2)
    big = {k: torch.zeros(2002, dtype=torch.float64, device=DEV) for k in "abdlu"}
    views = {}
    for k in "abdlu":
        big[k][1:] = p[k].to(DEV)
        views[k] = big[k][1:]  # 8-byte aligned only
    x, info, _ = api.solve(views["a"], views["b"], views["d"], views["l"], views["u"], p["r"])
    st, lam, xstar = oracle.solve_sort(*[p[k].numpy() for k in "abdlu"], p["r"])
    assert_x_close(np64(x), xstar, torch.float64)
    xh, info, _ = api.solve(p["a"], p["b"], p["d"], p["l"], p["u"], p["r"])  # CPU tensors in, CPU out
    assert xh.device.type == "cpu"
    assert_x_close(xh.numpy(), xstar, torch.float64)


def test_bounded_wait_reports_timeout_and_context_survives():
    p = _dev(W.uncorrelated_box(100000, seed=1), torch.float64)
    _, info, _ = api.solve(p["a"], p["b"], p["d"], p["l"], p["u"], p["r"], fault_inject=True, spin_limit_us=200000)
    assert info.status == api.Status.TIMEOUT
    torch.cuda.synchronize()
    x, info, _ = api.solve(p["a"], p["b"], p["d"], p["l"], p["u"], p["r"])
    assert info.status == api.Status.OK


def test_runs_are_deterministic():
    p = _dev(W.correlated(300000, seed=8), torch.float64)
    x1, i1, _ = api.solve(p["a"], p["b"], p["d"], p["l"], p["u"], p["r"])
    x2, i2, _ = api.solve(p["a"], p["b"], p["d"], p["l"], p["u"], p["r"])
    assert torch.equal(x1, x2) and i1.lam == i2.lam and i1.iters == i2.iters
