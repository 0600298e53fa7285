"""The oracle's multi-threaded form (the paper's CPU Jacobi variant, used only to time the
all-core CPU baseline) computes what the sequential oracle computes: the same phi, slopes and
breakpoints up to the rounding order of the sums, the same Alg. 1 / Alg. 4 solutions, and the
same per-chunk Alg. 2 start (every chunk is still scanned sequentially, in index order)."""
import math

import numpy as np
import pytest

import oracle
from oracle import reference as R
from paper_2603_15910_b300 import workloads as W


@pytest.fixture
def threads():
    prev = R.set_threads(1)
    yield lambda t: R.set_threads(t)
    R.set_threads(prev)


def _box(n, seed):
    p = W.uncorrelated_box(n, seed=seed)
    return [p[k].numpy() for k in "abdlu"], p["r"]


def test_phi_and_breakpoints_match_the_sequential_oracle(threads):
    (a, b, d, l, u), r = _box(200_001, 3)
    lams = (-3.0, -0.4, 0.0, 0.7)
    seq = [oracle.phi(lam, a, b, d, l, u) for lam in lams]
    bps = [oracle.breakpoint_search(lam, s, a, b, d, l, u) for lam in lams for s in (1, -1)]
    threads(4)
    par = [oracle.phi(lam, a, b, d, l, u) for lam in lams]
    bpp = [oracle.breakpoint_search(lam, s, a, b, d, l, u) for lam in lams for s in (1, -1)]
    for s, p in zip(seq, par):
        for x, y in zip(s, p):
            assert math.isclose(x, y, rel_tol=1e-14, abs_tol=1e-9), (s, p)
    assert bps == bpp  # a minimum is exact whatever the order


def test_newton_solutions_match_the_sequential_oracle(threads):
    (a, b, d, l, u), r = _box(100_003, 5)
    y = W.simplex_normal(300_007, seed=2).numpy()
    s1 = oracle.newton_cqk(a, b, d, l, u, r)
    p1 = oracle.newton_simplex(y, 1.0)
    c1 = oracle.condat_chunks(y, 1.0, 4096, 8)
    threads(4)
    s4 = oracle.newton_cqk(a, b, d, l, u, r)
    p4 = oracle.newton_simplex(y, 1.0)
    c4 = oracle.condat_chunks(y, 1.0, 4096, 8)
    assert s4["status"] == s1["status"] == "ok"
    assert np.max(np.abs(s4["x"] - s1["x"])) <= 1e-12 * (1 + np.max(np.abs(s1["x"])))
    assert abs(s4["evals"] - s1["evals"]) <= 1
    assert np.max(np.abs(p4["x"] - p1["x"])) <= 1e-12
    assert abs(p4["evals"] - p1["evals"]) <= 1
    # the per-chunk scans are sequential in either form; only the union's sums are reordered
    assert c4[2] == c1[2] and math.isclose(c4[0], c1[0], rel_tol=1e-13)


def test_default_is_one_thread():
    assert R.set_threads(1) == 1
