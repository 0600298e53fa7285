"""Pins of the oracle's implicit-function gradients against FP64 central finite
differences of the exact solution map (CPU only).  The paper has no backward
pass; the formulas are derived in oracle/exact.py."""
import numpy as np

import oracle


def _solve(a, b, d, l, u, r):
    st, lam, x = oracle.solve_sort(a, b, d, l, u, r)
    assert st == "ok"
    return lam, x


def _instance(seed, n=25):
    rng = np.random.default_rng(seed)
    d = rng.uniform(1, 100, n)
    b = rng.uniform(10, 25, n)
    a = rng.uniform(-10, 10, n)
    l = rng.uniform(-5, 0, n)
    u = l + rng.uniform(0.5, 5, n)
    r = float(b @ (l + u) / 2)
    g = rng.normal(size=n)
    return a, b, d, l, u, r, g


def _far_from_kinks(x, lam, a, b, d, l, u, margin=1e-4):
    t = (a + lam * b) / d
    return np.all(np.minimum(np.abs(t - l), np.abs(t - u)) > margin)


def test_general_gradient_vs_finite_differences():
    checked = 0
    for seed in range(40):
        a, b, d, l, u, r, g = _instance(seed)
        lam, x = _solve(a, b, d, l, u, r)
        if not _far_from_kinks(x, lam, a, b, d, l, u):
            continue
        gr = oracle.grad_cqk(x, lam, a, b, d, l, u, g)
        assert not gr["nondiff"]
        args = dict(a=a, b=b, d=d, l=l, u=u)
        for name in "abdlu":
            for i in range(len(a)):
                h = 1e-6 * max(1.0, abs(args[name][i]))
                vp = {k: v.copy() for k, v in args.items()}
                vm = {k: v.copy() for k, v in args.items()}
                vp[name][i] += h
                vm[name][i] -= h
                fp = g @ _solve(vp["a"], vp["b"], vp["d"], vp["l"], vp["u"], r)[1]
                fm = g @ _solve(vm["a"], vm["b"], vm["d"], vm["l"], vm["u"], r)[1]
                fd = (fp - fm) / (2 * h)
                assert abs(fd - gr[name][i]) <= 1e-6 * (1 + abs(fd)), (name, i, fd, gr[name][i])
        h = 1e-6 * max(1.0, abs(r))
        fd = (g @ _solve(a, b, d, l, u, r + h)[1] - g @ _solve(a, b, d, l, u, r - h)[1]) / (2 * h)
        assert abs(fd - gr["r"]) <= 1e-6 * (1 + abs(fd))
        checked += 1
    assert checked >= 5


def test_simplex_gradient_is_the_sparsemax_jacobian_and_matches_fd():
    rng = np.random.default_rng(5)
    for s in range(10):
        y = rng.normal(size=30)
        g = rng.normal(size=30)
        lam, x = oracle.project_simplex_sort(y, 1.0)
        if np.min(np.abs(y + lam)) < 1e-4:
            continue
        gr = oracle.grad_simplex(x, g)
        # general formula with b = d = 1, l = 0, u = inf
        ones = np.ones(30)
        gg = oracle.grad_cqk(x, lam, y, ones, ones, np.zeros(30), np.full(30, np.inf), g)
        np.testing.assert_allclose(gr["y"], gg["a"], atol=1e-14)
        assert abs(gr["r"] - gg["r"]) < 1e-14
        for i in range(30):
            h = 1e-6
            yp, ym = y.copy(), y.copy()
            yp[i] += h
            ym[i] -= h
            fd = (g @ oracle.project_simplex_sort(yp, 1.0)[1] - g @ oracle.project_simplex_sort(ym, 1.0)[1]) / (2 * h)
            assert abs(fd - gr["y"][i]) < 1e-6
        fd = (g @ oracle.project_simplex_sort(y, 1.0 + 1e-6)[1] - g @ oracle.project_simplex_sort(y, 1.0 - 1e-6)[1]) / 2e-6
        assert abs(fd - gr["r"]) < 1e-6


def test_l1_gradient_vs_finite_differences():
    rng = np.random.default_rng(6)
    for scale in (1.0, 0.01):
        y = rng.normal(size=20) * scale
        g = rng.normal(size=20)
        lam, x, inside = oracle.project_l1(y, 1.0)
        gr = oracle.grad_l1(y, x, g, inside)
        for i in range(20):
            h = 1e-7
            yp, ym = y.copy(), y.copy()
            yp[i] += h
            ym[i] -= h
            fd = (g @ oracle.project_l1(yp, 1.0)[1] - g @ oracle.project_l1(ym, 1.0)[1]) / (2 * h)
            assert abs(fd - gr["y"][i]) < 1e-6
        fd = (g @ oracle.project_l1(y, 1.0 + 1e-7)[1] - g @ oracle.project_l1(y, 1.0 - 1e-7)[1]) / 2e-7
        assert abs(fd - gr["r"]) < 1e-6
