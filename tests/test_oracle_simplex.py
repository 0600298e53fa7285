"""Pins of the FP64 oracle for the simplex and l1-ball projections (CPU only).

Checked against: the general CQK oracle with D = I, b = 1, l = 0, u = +inf
(Sec. 1); brute force; Condat's Alg. 3; closed-form special cases; the
invariants of Theorem 3.1; the bound lambda_J >= lambda* of eq. (lambdaJ);
the subgradient optimality conditions of the l1-ball projection; and the
iteration counts printed in Table 4."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_15910_b300 import workloads as W


def _sum(v):
    return float(np.sum(v, dtype=np.longdouble))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11])
def test_simplex_routes_agree_with_brute_force(n):
    for s in range(10):
        y = np.random.default_rng(1000 * n + s).normal(size=n) * (3 if s % 2 else 1)
        r = [1.0, 0.3, 4.0][s % 3]
        ones, zeros, inf = np.ones(n), np.zeros(n), np.full(n, np.inf)
        bf = oracle.brute_force_cqk(y, ones, ones, zeros, inf, r)
        lam_s, x_s = oracle.project_simplex_sort(y, r)
        lam_c, x_c = oracle.condat_project(y, r)
        nw = oracle.newton_simplex(y, r)
        lam_c0 = oracle.condat_init(y, r)[0]
        nw2 = oracle.newton_simplex(y, r, lam0=lam_c0)
        st, lam_g, x_g = oracle.solve_sort(y, ones, ones, zeros, inf, r)
        for x in (x_c, nw["x"], nw2["x"], x_g):
            np.testing.assert_allclose(x, bf[1], atol=1e-12)
        np.testing.assert_allclose(x_s, bf[1], atol=1e-12)
        assert math.isclose(lam_s, lam_c, abs_tol=1e-12) and math.isclose(lam_s, lam_g, abs_tol=1e-12)


def test_simplex_special_cases():
    # all equal: x = r/n
    lam, x = oracle.project_simplex_sort(np.full(7, 0.4), 1.0)
    np.testing.assert_allclose(x, np.full(7, 1 / 7), atol=1e-15)
    # one dominant entry: x = r e_k
    y = np.array([0.1, 5.0, -0.3, 0.2])
    for f in (oracle.project_simplex_sort, oracle.condat_project):
        lam, x = f(y, 1.0)
        np.testing.assert_allclose(x, [0, 1, 0, 0], atol=1e-15)
    nw = oracle.newton_simplex(y, 1.0)
    np.testing.assert_allclose(nw["x"], [0, 1, 0, 0], atol=1e-15)
    # n = 1: x = r
    assert oracle.newton_simplex(np.array([-3.0]), 2.5)["x"][0] == 2.5
    # already on the simplex: x = y
    y = np.array([0.2, 0.3, 0.5])
    np.testing.assert_allclose(oracle.project_simplex_sort(y, 1.0)[1], y, atol=1e-15)


def test_theorem_3_1_invariants():
    for s in range(20):
        y = W.paper_simplex(["uniform", "normal", "narrow"][s % 3], 20000, seed=s).numpy()
        nw = oracle.newton_simplex(y, 1.0)
        tr = nw["trace"]
        assert tr[0] >= -np.max(y)                   # line 1 of Alg. 4
        lam_star = oracle.project_simplex_sort(y, 1.0)[0]
        # items 3 and 4: for k >= 1, lambda_k >= lambda_{k+1} >= lambda*, phi(lambda_k) > r
        assert np.all(np.diff(tr[1:]) <= 0)
        assert np.all(tr[1:] >= lam_star - 1e-12)
        for lam in tr[1:-1]:
            assert _sum(np.maximum(0, y + lam)) > 1.0


def test_lambda_J_is_an_upper_bound():
    # eq. (lambdaJ): lambda_J >= lambda* for every nonempty J
    rng = np.random.default_rng(4)
    y = rng.normal(size=5000)
    lam_star = oracle.project_simplex_sort(y, 1.0)[0]
    for _ in range(50):
        J = rng.choice(5000, size=rng.integers(1, 5000), replace=False)
        assert (1.0 - _sum(y[J])) / J.size >= lam_star - 1e-12
    lam2, S, C = oracle.condat_init(y, 1.0)
    assert math.isclose(lam2, (1.0 - S) / C, rel_tol=1e-12) and lam2 >= lam_star - 1e-12
    for tile, chunks in ((1, 7), (64, 5), (256, 3), (2, 1000)):
        lam0, S, C = oracle.condat_chunks(y, 1.0, tile, chunks)
        assert lam0 >= lam_star - 1e-12
        assert math.isclose(lam0, (1.0 - S) / C, rel_tol=1e-12)
    # one chunk covering everything is Alg. 2 itself
    lam0, S, C = oracle.condat_chunks(y, 1.0, 5000, 1)
    assert (lam0, C) == (lam2, oracle.condat_init(y, 1.0)[2])


def test_alg2_multiplier_never_increases_in_the_scan():
    # both branches of the first loop of Alg. 2 lower lambda; a parallel scan
    # may therefore discard an element as soon as it fails the test
    for s in range(10):
        y = np.random.default_rng(s).normal(size=3000) * (1 + 4 * (s % 2))
        for l1 in (False, True):
            lam, S, C, tr = oracle.condat_init(y, 1.0, l1=l1, return_trace=True)
            assert np.all(np.diff(tr) <= 0)


@pytest.mark.parametrize("shift", [0, 1, 7, 15])
def test_alg2_chunk_union_matches_manual_partition(shift):
    # a problem that starts inside a tile (a batch member) sees its first tile cut short
    y = np.random.default_rng(8).normal(size=1000)
    tile, chunks = 16, 6
    S, C = 0.0, 0
    for c in range(chunks):
        idx = np.array([i for i in range(1000) if ((i + shift) // tile) % chunks == c])
        _, s, k = oracle.condat_init(y, 1.0, idx=idx)
        S += s
        C += k
    lam0, S2, C2 = oracle.condat_chunks(y, 1.0, tile, chunks, shift=shift)
    assert C == C2 and math.isclose(S, S2, rel_tol=1e-13)


def test_l1_ball_projection_optimality():
    rng = np.random.default_rng(12)
    for s in range(20):
        n = int(rng.integers(1, 400))
        y = rng.normal(size=n) * (0.01 if s % 4 == 0 else 1.0)
        if s % 5 == 0:
            y[rng.integers(0, n)] = 0.0
        r = 1.0
        lam, x, inside = oracle.project_l1(y, r)
        if _sum(np.abs(y)) <= r:
            assert inside and np.array_equal(x, y)
            continue
        assert lam <= 0.0 and not inside
        theta = -lam
        # subgradient conditions of min 1/2|x-y|^2 s.t. |x|_1 <= r (active):
        nz = x != 0
        np.testing.assert_allclose((y - x)[nz], theta * np.sign(x[nz]), atol=1e-12)
        assert np.all(np.abs(y[~nz]) <= theta + 1e-12)
        assert math.isclose(_sum(np.abs(x)), r, rel_tol=1e-12)
        assert np.all(np.sign(x[nz]) == np.sign(y[nz])) and np.all(x[y == 0] == 0)
        # Newton on |y| with the strengthened Alg. 2 test reaches the same point
        lam0 = oracle.condat_init(y, r, l1=True)[0]
        nw = oracle.newton_simplex(y, r, lam0=lam0, l1=True)
        np.testing.assert_allclose(np.sign(y) * nw["x"], x, atol=1e-12)


def test_l1_strengthened_test_skips_zeros():
    # Lemma 3.2: a zero entry stays zero; with min{|y|, |y|+lam} > 0 it never enters J
    y = np.array([0.0, 2.0, 0.0, 3.0, -0.5])
    lam, S, C = oracle.condat_init(y, 1.0, l1=True)
    assert C >= 1 and S == pytest.approx(3.0)


def _golden(name):
    rows = []
    with open(__file__.replace("test_oracle_simplex.py", f"golden/{name}")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(v) for v in line.split()])
    return rows


def test_table4_iteration_counts():
    # GPU counts (formula start) = phi evaluations + 1 (the eq. (CQKlambda0)
    # pass); CPU counts (Alg. 2 start) = phi evaluations.
    kinds = ("uniform", "normal", "narrow")
    for row in _golden("table4_simplex_iterations.txt"):
        n = int(row[0])
        for j, kind in enumerate(kinds):
            gpu, cpu = [], []
            for s in range(20):
                y = W.paper_simplex(kind, n, seed=s).numpy()
                gpu.append(oracle.newton_simplex(y, 1.0)["evals"] + 1)
                lam0 = oracle.condat_init(y, 1.0)[0]
                cpu.append(oracle.newton_simplex(y, 1.0, lam0=lam0)["evals"])
            assert abs(np.mean(gpu) - row[1 + j]) <= 0.8, (kind, n, np.mean(gpu), row[1 + j])
            assert abs(np.mean(cpu) - row[4 + j]) <= 1.1, (kind, n, np.mean(cpu), row[4 + j])


def test_alg4_hand_worked_examples():
    # y = (3, 1, 0), r = 1, formula start lambda_0 = (1 - 4)/3 = -1 (>= -max y = -3).
    # phi(-1) = 2 > r, phi'_-(-1) = #{y_i > 1} = 1  ->  lambda_1 = -1 - (2 - 1)/1 = -2.
    # phi(-2) = 1 = r: Alg. 4 stops at k = 1 (phi(lambda_k) <= r); x = (1, 0, 0).
    nw = oracle.newton_simplex(np.array([3.0, 1.0, 0.0]), 1.0)
    assert list(nw["trace"]) == [-1.0, -2.0] and nw["evals"] == 2 and nw["stop"] == "below"
    np.testing.assert_array_equal(nw["x"], [1.0, 0.0, 0.0])
    # Start on a breakpoint: y = (3, 1, 0, 2), lambda_0 = -1 = -y_2.  phi(-1) = 3 > r,
    # phi'_-(-1) = #{y_i > 1} = 2 (phi'_+ would count y_2 too), so lambda_1 = -1 - 2/2 = -2,
    # phi(-2) = 1 = r and the method stops with x = (1, 0, 0, 0).
    nw = oracle.newton_simplex(np.array([3.0, 1.0, 0.0, 2.0]), 1.0, lam0=-1.0)
    assert list(nw["trace"]) == [-1.0, -2.0] and nw["evals"] == 2 and nw["stop"] == "below"
    # From below: y = (0.5, 0.2), r = 1, lambda_0 = -0.5 (clamped to -max y = -0.5).
    # phi(-0.5) = 0 < r, phi'_+(-0.5) = #{y_i >= 0.5} = 1 -> lambda_1 = 0.5;
    # phi(0.5) = 1 + 0.7 = 1.7 > r, phi'_-(0.5) = 2 -> lambda_2 = 0.5 - 0.7/2 = 0.15;
    # phi(0.15) = 0.65 + 0.35 = 1.0 -> stop; x = (0.65, 0.35).
    nw = oracle.newton_simplex(np.array([0.5, 0.2]), 1.0, lam0=-2.0)
    np.testing.assert_allclose(nw["trace"], [-0.5, 0.5, 0.15], atol=1e-15)
    assert nw["evals"] == 3 and nw["stop"] == "below"
    np.testing.assert_allclose(nw["x"], [0.65, 0.35], atol=1e-15)
