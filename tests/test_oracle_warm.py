"""Pins of the oracle's warm starts (Sec. 2: eq. (CQKlambda0) over the variables a primal
estimate leaves free; Sec. 3.3: Alg. 2 on the support of a primal estimate) against the
exact solvers and the cold starts (CPU only)."""
import math

import numpy as np
import pytest

import oracle


def _box(seed, n):
    rng = np.random.default_rng(seed)
    d = rng.uniform(1, 100, n)
    b = rng.uniform(10, 25, n)
    a = rng.uniform(-10, 10, n)
    l = rng.uniform(-5, 0, n)
    u = l + rng.uniform(0.5, 5, n)
    return a, b, d, l, u, float(b @ (l + u) / 2)


def test_warm_lambda0_all_free_is_the_cold_formula():
    a, b, d, l, u, r = _box(1, 500)
    xbar = (l + u) / 2  # strictly inside every box
    assert oracle.lambda0_warm(a, b, d, l, u, xbar, r) == oracle.lambda0_formula(a, b, d, r)


def test_warm_lambda0_empty_free_set_falls_back_to_all_variables():
    a, b, d, l, u, r = _box(2, 300)
    xbar = np.where(np.arange(300) % 2 == 0, l, u)  # every variable at a bound
    assert oracle.lambda0_warm(a, b, d, l, u, xbar, r) == oracle.lambda0_formula(a, b, d, r)
    xbar = l - 1.0  # violating every bound: no free variable either
    assert oracle.lambda0_warm(a, b, d, l, u, xbar, r) == oracle.lambda0_formula(a, b, d, r)


@pytest.mark.parametrize("seed", range(6))
def test_warm_lambda0_from_the_solution_is_exact_when_active_bounds_are_zero(seed):
    # with every active bound equal to 0, b'x = r reduces to the free variables, so
    # eq. (CQKlambda0) over J = the free set of x* gives lambda* itself
    rng = np.random.default_rng(100 + seed)
    n = 400
    d = rng.uniform(1, 10, n)
    b = rng.uniform(1, 3, n)
    a = rng.normal(size=n) * 5
    l = np.zeros(n)
    u = np.full(n, np.inf)
    r = float(rng.uniform(5, 20))
    st, lam, x = oracle.solve_sort(a, b, d, l, u, r)
    assert st == "ok"
    free = (x > l) & (x < u)
    assert 0 < free.sum() < n
    l0 = oracle.lambda0_warm(a, b, d, l, u, x, r)
    assert math.isclose(l0, lam, rel_tol=1e-12, abs_tol=1e-12)
    # the cold start is not exact on the same instance
    assert abs(oracle.lambda0_formula(a, b, d, r) - lam) > 1e-6


@pytest.mark.parametrize("l1", [False, True])
@pytest.mark.parametrize("tile,chunks", [(3000, 1), (64, 5), (512, 8), (16, 300)])
def test_warm_condat_from_the_exact_support_gives_lambda_star(l1, tile, chunks):
    rng = np.random.default_rng(7)
    for s in range(5):
        y = rng.normal(size=3000) * (1 + s)
        if l1:
            lam, x, inside = oracle.project_l1(y, 1.0)
            assert not inside
        else:
            lam, x = oracle.project_simplex_sort(y, 1.0)
        l0, S, C = oracle.condat_chunks_warm(y, x, 1.0, tile, chunks, l1=l1)
        assert C == int(np.count_nonzero(x))
        assert math.isclose(l0, lam, rel_tol=1e-13, abs_tol=1e-14)


def test_warm_condat_with_full_support_is_the_cold_partition():
    rng = np.random.default_rng(3)
    y = rng.normal(size=5000)
    for l1 in (False, True):
        for tile, chunks, shift in ((512, 8, 0), (64, 7, 13)):
            cold = oracle.condat_chunks(y, 1.0, tile, chunks, l1=l1, shift=shift)
            warm = oracle.condat_chunks_warm(y, np.ones(5000), 1.0, tile, chunks, l1=l1, shift=shift)
            assert cold == warm


def test_warm_condat_is_an_upper_bound_and_handles_an_empty_support():
    rng = np.random.default_rng(4)
    y = rng.normal(size=2000)
    lam, x = oracle.project_simplex_sort(y, 1.0)
    for s in range(20):
        xbar = np.where(rng.uniform(size=2000) < 0.05, 1.0, 0.0)
        xbar[rng.integers(0, 2000)] = 1.0
        l0, S, C = oracle.condat_chunks_warm(y, xbar, 1.0, 64, 6)
        assert l0 >= lam - 1e-12  # eq. (lambdaJ) for any J
    # no candidate at all: lambda = max{r/n, -y_1}, which is >= -max y
    l0, S, C = oracle.condat_chunks_warm(y, np.zeros(2000), 1.0, 64, 6)
    assert C == 0 and l0 == max(1.0 / 2000, -y[0]) and l0 >= -y.max()
    l0, S, C = oracle.condat_chunks_warm(y, np.zeros(2000), 1.0, 64, 6, l1=True)
    assert C == 0 and l0 == max(1.0 / 2000, -abs(y[0]))
