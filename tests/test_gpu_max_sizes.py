"""Maximum sizes: single problems of 2^31 + 3 elements (FP32 storage, 8.6 GB per array), past
32-bit element, vector and mask-word indices, in the default launch configuration.

At this size the oracle's sort-based solvers are too slow, so each result is checked by the
conditions that make it the solution (they hold at any size), evaluated on the host chunk by
chunk in FP64:
  * simplex (eq. (proj_Delta)): x = max{0, y + lambda} for the reported lambda, and sum x = r;
    and lambda itself against the oracle's sort-based projection of the candidates y_i >
    -lambda - 1 (every other element is zero at that lambda, which the test checks), so the
    exact multiplier is pinned as well;
  * l1 ball (Lemma 3.2): the same on |y|, with sgn(x) = sgn(y);
  * general CQK (eq. (xopt), eq. (opt)): x = clip((a + lambda b)/d, l, u) and b'x = r within
    the FP32-storage tolerance."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_15910_b300 import api, workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"
N = (1 << 31) + 3
CHUNK = 1 << 27


def _chunks(n):
    for lo in range(0, n, CHUNK):
        yield lo, min(n, lo + CHUNK)


@pytest.mark.parametrize("l1", [False, True])
def test_projection_past_2_31_elements(l1):
    y = W.simplex_normal(N, seed=7, device=DEV, dtype=torch.float32)
    torch.cuda.empty_cache()
    fn = api.project_l1 if l1 else api.project_simplex
    x, info, mask = fn(y, 1.0, want_mask=True)
    assert info.status == api.Status.OK, info
    lam = info.lam
    total = 0.0
    nonzero = 0
    cand = []
    for lo, hi in _chunks(N):
        yc = y[lo:hi].double().cpu().numpy()
        xc = x[lo:hi].double().cpu().numpy()
        yy = np.abs(yc) if l1 else yc
        want = np.maximum(0.0, yy + lam)
        got = np.abs(xc) if l1 else xc
        assert np.max(np.abs(got - want)) <= 1e-6 * (1.0 + np.max(want)), (lo, np.max(np.abs(got - want)))
        if l1:
            nz = xc != 0
            assert np.array_equal(np.sign(xc[nz]), np.sign(yc[nz])), lo
        total += float(np.sum(got, dtype=np.longdouble))
        nonzero += int(np.count_nonzero(got))
        sel = yy > -lam - 1.0
        cand.append(yy[sel])
    assert abs(total - 1.0) <= 1e-5, total
    assert info.nfree == nonzero
    # the exact multiplier from the oracle's sort-based projection of the candidates
    c = np.concatenate(cand)
    lam_star, _ = oracle.project_simplex_sort(c, 1.0)
    assert -lam - 1.0 <= -lam_star, "a non-candidate element would be positive at lambda*"
    assert abs(lam - lam_star) <= 1e-5 * (1.0 + abs(lam_star)), (lam, lam_star)
    # the mask covers the whole vector: its popcount is the number of nonzero x
    m = mask.cpu().numpy().view(np.uint32)
    assert int(np.unpackbits(m.view(np.uint8)).sum()) == nonzero


def test_general_past_2_31_elements():
    p = W.correlated(N, seed=1, device=DEV, dtype=torch.float32)
    torch.cuda.empty_cache()
    x, info, mask = api.solve(p["a"], p["b"], p["d"], p["l"], p["u"], p["r"], want_mask=True)
    assert info.status == api.Status.OK, info
    lam = info.lam
    bx = 0.0
    absbx = 0.0
    nfree = 0
    for lo, hi in _chunks(N):
        a, b, d, l, u, xc = [t[lo:hi].double().cpu().numpy() for t in (p["a"], p["b"], p["d"], p["l"], p["u"], x)]
        want = np.clip((a + lam * b) / d, l, u)
        assert np.max(np.abs(xc - want)) <= 1e-5 * (1.0 + np.max(np.abs(want))), lo
        prod = b * xc
        bx += float(np.sum(prod, dtype=np.longdouble))
        absbx += float(np.sum(np.abs(prod)))
        nfree += int(np.count_nonzero((xc > l) & (xc < u)))
    assert abs(bx - p["r"]) <= 1e-5 * absbx, (bx, p["r"], absbx)
    assert info.nfree == nfree
