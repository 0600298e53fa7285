"""Pins of the FP64 oracle for the general CQK problem (CPU only).

The oracle (oracle/) is checked against things other than itself: brute-force
active-set enumeration, the KKT conditions, the no-active-bound closed form
(eq. (CQKlambda0)), a numerical derivative of phi, a direct breakpoint scan,
infeasibility of r outside [b'l, b'u], and the iteration counts printed in the
paper's Table 3."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_15910_b300 import workloads as W


def box(n, seed, inf_frac=0.0):
    rng = np.random.default_rng(seed)
    d = rng.uniform(1, 100, n)
    b = rng.uniform(10, 25, n)
    a = rng.uniform(-10, 10, n)
    l = rng.uniform(-5, 0, n)
    u = l + rng.uniform(0.5, 5, n)
    if inf_frac:
        l = np.where(rng.uniform(size=n) < inf_frac, -np.inf, l)
        u = np.where(rng.uniform(size=n) < inf_frac, np.inf, u)
    lf = np.where(np.isinf(l), -5.0, l)
    uf = np.where(np.isinf(u), 5.0, u)
    r = float(b @ (lf + uf) / 2)
    return a, b, d, l, u, r


@pytest.mark.parametrize("n", list(range(1, 13)))
def test_sort_solver_matches_brute_force(n):
    seeds = range(12) if n <= 8 else range(2)
    for s in seeds:
        a, b, d, l, u, r = box(n, 100 * n + s, inf_frac=0.2 if s % 3 == 1 else 0.0)
        bf = oracle.brute_force_cqk(a, b, d, l, u, r)
        st, lam, x = oracle.solve_sort(a, b, d, l, u, r)
        assert bf is not None and st == "ok"
        np.testing.assert_allclose(x, bf[1], rtol=0, atol=1e-11 * (1 + np.max(np.abs(bf[1]))))
        nw = oracle.newton_cqk(a, b, d, l, u, r)
        assert nw["status"] == "ok"
        np.testing.assert_allclose(nw["x"], bf[1], rtol=0, atol=1e-10 * (1 + np.max(np.abs(bf[1]))))


def test_kkt_of_sort_and_newton_on_box_family():
    for s in range(5):
        p = W.uncorrelated_box(10000, seed=s)
        a, b, d, l, u = (p[k].numpy() for k in "abdlu")
        st, lam, x = oracle.solve_sort(a, b, d, l, u, p["r"])
        assert st == "ok"
        dx, feas = oracle.kkt_residuals(x, lam, a, b, d, l, u, p["r"])
        assert dx == 0.0 and feas < 1e-13
        nw = oracle.newton_cqk(a, b, d, l, u, p["r"])
        assert nw["status"] == "ok"
        assert np.max(np.abs(nw["x"] - x)) <= 1e-10 * (1 + np.max(np.abs(x)))
        dx, feas = oracle.kkt_residuals(nw["x"], nw["lam"], a, b, d, l, u, p["r"])
        assert feas < 1e-12


def test_no_active_bound_closed_form():
    # wide bounds: the unconstrained multiplier of eq. (CQKlambda0) is optimal
    rng = np.random.default_rng(3)
    n = 500
    d, b, a = rng.uniform(1, 100, n), rng.uniform(10, 25, n), rng.uniform(-10, 10, n)
    l, u = np.full(n, -1e6), np.full(n, 1e6)
    r = 7.5
    lam0 = oracle.lambda0_formula(a, b, d, r)
    s = np.sum(b * a / d)
    q = np.sum(b * b / d)
    assert math.isclose(lam0, (r - s) / q, rel_tol=1e-13)
    st, lam, x = oracle.solve_sort(a, b, d, l, u, r)
    assert math.isclose(lam, lam0, rel_tol=1e-12, abs_tol=1e-14)
    np.testing.assert_allclose(x, (a + lam0 * b) / d, rtol=1e-12, atol=1e-14)
    nw = oracle.newton_cqk(a, b, d, l, u, r)
    assert nw["evals"] == 1 and nw["stop"] in ("exact", "residual")


def test_phi_slopes_are_one_sided_derivatives():
    # eq. (phideriv) against difference quotients of eq. (opt): phi is piecewise
    # linear, so a step smaller than the distance to the next breakpoint is exact
    a, b, d, l, u, r = box(200, 11)
    bl = (d * l - a) / b
    bu = (d * u - a) / b
    brk = np.sort(np.concatenate([bl, bu]))
    for lam in (-1.3, -0.2, 0.05, 0.4, 2.0):
        gap = np.min(np.abs(brk - lam))
        h = gap / 4
        f0, dp, dm, _ = oracle.phi(lam, a, b, d, l, u)
        fp = oracle.phi(lam + h, a, b, d, l, u)[0]
        fm = oracle.phi(lam - h, a, b, d, l, u)[0]
        assert math.isclose((fp - f0) / h, dp, rel_tol=1e-6, abs_tol=1e-9)
        assert math.isclose((f0 - fm) / h, dm, rel_tol=1e-6, abs_tol=1e-9)
        assert math.isclose(f0, float(np.sum(b * np.clip((a + lam * b) / d, l, u))), rel_tol=1e-13)
    # at a breakpoint the lateral slopes differ by that variable's b^2/d
    i = 17
    lam = bl[i]
    _, dp, dm, _ = oracle.phi(lam, a, b, d, l, u)
    assert math.isclose(dp - dm, b[i] ** 2 / d[i], rel_tol=1e-9)


def test_phi_is_monotone():
    a, b, d, l, u, r = box(300, 5)
    lams = np.linspace(-3, 3, 601)
    vals = [oracle.phi(t, a, b, d, l, u)[0] for t in lams]
    assert np.all(np.diff(vals) >= -1e-12)


def test_breakpoint_search_is_the_nearest_breakpoint():
    a, b, d, l, u, r = box(100, 21)
    allb = np.concatenate([(d * l - a) / b, (d * u - a) / b])
    for lam in (-0.7, 0.0, 0.3):
        right = oracle.breakpoint_search(lam, +1, a, b, d, l, u)
        left = oracle.breakpoint_search(lam, -1, a, b, d, l, u)
        assert right == np.min(allb[allb > lam])
        assert left == np.max(allb[allb < lam])
    assert oracle.breakpoint_search(np.max(allb) + 1, +1, a, b, d, l, u) is None


def test_zero_slope_start_uses_breakpoints():
    # start far to the left: every variable sits at its lower bound, phi'_+ = 0,
    # so Alg. 1 must move to the closest breakpoint (and still converge)
    a, b, d, l, u, r = box(50, 8)
    lam0 = np.min((d * l - a) / b) - 10.0
    f = oracle.phi(lam0, a, b, d, l, u)
    assert f[1] == 0.0 and f[0] < r
    nw = oracle.newton_cqk(a, b, d, l, u, r, lam0=lam0)
    assert nw["status"] == "ok" and nw["bpsearch"] >= 1
    st, lam, x = oracle.solve_sort(a, b, d, l, u, r)
    np.testing.assert_allclose(nw["x"], x, atol=1e-10)
    lam0 = np.max((d * u - a) / b) + 10.0
    nw = oracle.newton_cqk(a, b, d, l, u, r, lam0=lam0)
    assert nw["status"] == "ok" and nw["bpsearch"] >= 1
    np.testing.assert_allclose(nw["x"], x, atol=1e-10)


def test_secant_steps_happen_and_converge():
    # a few variables with tiny d make phi very steep in narrow ranges, which
    # pushes Newton steps outside the bracket
    found = 0
    for s in range(200):
        rng = np.random.default_rng(s)
        n = 30
        d = rng.uniform(1, 100, n) * np.where(rng.uniform(size=n) < 0.2, 1e-3, 1.0)
        b, a = rng.uniform(10, 25, n), rng.uniform(-10, 10, n)
        l = rng.uniform(-5, 0, n)
        u = l + rng.uniform(0.5, 5, n)
        r = float(b @ (l + rng.uniform(0, 1, n) * (u - l)))
        lam0 = rng.uniform(-50, 50)
        nw = oracle.newton_cqk(a, b, d, l, u, r, lam0=lam0)
        bf_st, lam, x = oracle.solve_sort(a, b, d, l, u, r)
        assert nw["status"] == "ok"
        np.testing.assert_allclose(nw["x"], x, atol=1e-9 * (1 + np.max(np.abs(x))))
        found += nw["secant"] > 0
    assert found >= 3


def test_infeasible_right_hand_side():
    a, b, d, l, u, r = box(40, 2)
    for rr in (float(b @ u) + 1.0, float(b @ l) - 1.0):
        assert oracle.solve_sort(a, b, d, l, u, rr)[0] == "infeasible"
        assert oracle.newton_cqk(a, b, d, l, u, rr)["status"] == "infeasible"
        assert oracle.brute_force_cqk(a[:6], b[:6], d[:6], l[:6], u[:6],
                                      float(b[:6] @ u[:6]) + 1.0) is None
    # just inside the feasibility boundary the solution is x ~ u (resp. l)
    bu = float(b @ u)
    st, lam, x = oracle.solve_sort(a, b, d, l, u, bu * (1 - 1e-12))
    assert st == "ok"
    np.testing.assert_allclose(x, u, atol=1e-8)
    bl = float(b @ l)
    st, lam, x = oracle.solve_sort(a, b, d, l, u, bl + abs(bl) * 1e-12)
    assert st == "ok"
    np.testing.assert_allclose(x, l, atol=1e-8)


def test_infinite_bounds_both_sides():
    a, b, d, l, u, r = box(400, 9, inf_frac=0.5)
    st, lam, x = oracle.solve_sort(a, b, d, l, u, r)
    assert st == "ok"
    dx, feas = oracle.kkt_residuals(x, lam, a, b, d, l, u, r)
    assert dx == 0.0 and feas < 1e-13
    nw = oracle.newton_cqk(a, b, d, l, u, r)
    np.testing.assert_allclose(nw["x"], x, atol=1e-10 * (1 + np.max(np.abs(x))))


def _golden(name):
    rows = []
    with open(__file__.replace("test_oracle_general.py", f"golden/{name}")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(v) for v in line.split()])
    return rows


def test_table3_iteration_counts():
    # The paper's GPU counts include the eq. (CQKlambda0) MapReduce pass, so
    # they equal the number of phi evaluations + 1.
    for row in _golden("table3_gpu_iterations.txt"):
        n = int(row[0])
        if n > 100000:
            continue
        for kind, want in zip(("uncorrelated", "weak", "correlated"), row[1:]):
            ev = []
            for s in range(20):
                p = W.paper_family(kind, n, seed=s)
                a, b, d, l, u = (p[k].numpy() for k in "abdlu")
                nw = oracle.newton_cqk(a, b, d, l, u, p["r"])
                assert nw["status"] == "ok"
                ev.append(nw["evals"] + 1)
            assert abs(np.mean(ev) - want) <= 0.8, (kind, n, np.mean(ev), want)
