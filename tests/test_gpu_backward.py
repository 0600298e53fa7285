"""GPU parity of the adjoint kernels (cqk_backward, cqk_backward_simplex, cqk_backward_l1)
and of the autograd wrappers, against the oracle's implicit-function gradients (which the
CPU suite pins to finite differences of the exact solution map), and a finite-difference
check of the whole differentiable GPU solve.

The reference gradient is always evaluated at the oracle's own solution (x*, lambda*) of the
stored data -- never at the GPU's x or lambda -- so a forward that put an element on the
wrong side of a bound fails here.  The GPU free mask must equal the oracle's free set except
within a narrow band around the bounds (elements whose status two correct solutions may
round differently); gradients are compared element by element outside that band."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_15910_b300 import api, autograd as AD, workloads as W
from helpers import mask_bits, np64

pytestmark = pytest.mark.gpu
DEV = "cuda"
TOL = {torch.float64: 1e-10, torch.float32: 1e-5}
TIE = {torch.float64: 1e-9, torch.float32: 4e-6}


def _close(got, want, dtype, what="", keep=None):
    got, want = np.asarray(got, dtype=np.float64), np.asarray(want, dtype=np.float64)
    if keep is not None:
        got, want = got[keep], want[keep]
    err = float(np.max(np.abs(got - want))) if got.size else 0.0
    bound = TOL[dtype] * (1.0 + (float(np.max(np.abs(want))) if want.size else 0.0))
    assert err <= bound, f"{what}: max err {err:.3e} > {bound:.3e}"


def _oracle_general(a, b, d, l, u, r):
    st, lam, xstar = oracle.solve_sort(a, b, d, l, u, r)
    assert st == "ok"
    return lam, xstar


def _general_ties(a, b, d, l, u, lam, dtype):
    # relative to the terms of v = a + lambda b against d l, d u (the kernel's tie rule)
    with np.errstate(invalid="ignore"):
        v = a + lam * b
        sc = np.abs(a) + np.abs(lam * b)
        dl, du = d * l, d * u
        tl = np.abs(v - dl) <= TIE[dtype] * (sc + np.abs(dl))
        tu = np.abs(v - du) <= TIE[dtype] * (sc + np.abs(du))
    return tl | tu


def _check_general_grads(out, ref, sl, dtype, mask_bits_, a, b, d, l, u, lam_star, xstar, what, gr=None):
    """GPU gradients of one instance (slice sl of out) against the oracle's, outside the tie band;
    the GPU mask against the oracle's free set there."""
    keep = ~_general_ties(a, b, d, l, u, lam_star, dtype)
    assert keep.sum() >= keep.size - 3, (what, int((~keep).sum()))
    free_star = (xstar > l) & (xstar < u)
    if mask_bits_ is not None:
        assert np.array_equal(mask_bits_[keep], free_star[keep]), what
    for k in "abdlu":
        _close(np64(out[k][sl]), ref[k], dtype, f"{what} d{k}", keep)
    g_r = float(out["r"][0]) if gr is None else gr
    assert abs(g_r - ref["r"]) <= TOL[dtype] * (1 + abs(ref["r"])), (what, g_r, ref["r"])


def _oracle_projection(y64, r, l1):
    """(lam*, x*, inside) of the oracle's exact projection of the stored y."""
    if l1:
        return oracle.project_l1(y64, r)
    lam, xstar = oracle.project_simplex_sort(y64, r)
    return lam, xstar, False


def _projection_ref(y64, g64, r, l1):
    lam, xstar, inside = _oracle_projection(y64, r, l1)
    ref = oracle.grad_l1(y64, xstar, g64, inside) if l1 else oracle.grad_simplex(xstar, g64)
    yy = np.abs(y64) if l1 else y64
    ties = np.zeros(y64.shape, dtype=bool) if inside else np.abs(yy + lam) <= 1e-9 * (np.abs(yy) + abs(lam))
    return ref, xstar, ties


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n", [1, 7, 2000, 10003, 200001])
@pytest.mark.parametrize("use_mask", [True, False])
def test_general_backward_matches_oracle(n, dtype, use_mask):
    p = W.uncorrelated_box(n, seed=n + 3, dtype=dtype)
    dev = {k: p[k].to(DEV) for k in ("a", "b", "d", "l", "u")}
    ws = api.Workspace(n, 1, dtype)
    x, info, mask = api.solve(*(dev[k] for k in ("a", "b", "d", "l", "u")), p["r"], want_mask=True, ws=ws)
    assert info.status == api.Status.OK
    g = torch.randn(n, generator=torch.Generator().manual_seed(n), dtype=torch.float64).to(dtype)
    out = api.backward("general", g.to(DEV), x, ws.info, a=dev["a"], b=dev["b"], d=dev["d"], l=dev["l"], u=dev["u"],
                       mask=mask if use_mask else None)
    host = [np64(p[k]) for k in ("a", "b", "d", "l", "u")]
    lam_star, xstar = _oracle_general(*host, p["r"])
    ref = oracle.grad_cqk(xstar, lam_star, *host, np64(g))
    assert int(out["status"][0]) == (api.Status.NONDIFF if ref["nondiff"] else api.Status.OK)
    _check_general_grads(out, ref, slice(None), dtype, mask_bits(mask, n), *host, lam_star, xstar, f"n={n}")


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("l1", [False, True])
@pytest.mark.parametrize("n", [1, 33, 4096, 150001])
def test_projection_backward_matches_oracle(n, dtype, l1):
    for scale in ((1.0, 1e-5) if l1 else (1.0,)):
        y = (W.simplex_normal(n, seed=2 * n + 1, dtype=dtype) * scale).to(dtype)
        ws = api.Workspace(n, 1, dtype)
        fn = api.project_l1 if l1 else api.project_simplex
        x, info, mask = fn(y.to(DEV), 1.0, want_mask=True, ws=ws)
        g = torch.randn(n, generator=torch.Generator().manual_seed(n + 5), dtype=torch.float64).to(dtype)
        out = api.backward("l1" if l1 else "simplex", g.to(DEV), x, ws.info, mask=mask)
        ref, xstar, ties = _projection_ref(np64(y), np64(g), 1.0, l1)
        assert not ties.any()
        assert np.array_equal(mask_bits(mask, n), xstar != 0) or (l1 and info.stop == "inside")
        _close(np64(out["y"]), ref["y"], dtype, f"dy n={n} scale={scale}")
        assert abs(float(out["r"][0]) - ref["r"]) <= TOL[dtype] * (1 + abs(ref["r"]))
        assert int(out["status"][0]) == api.Status.OK


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_backward_matches_oracle(dtype):
    lens = [300, 0, 1, 5, 4099, 77, 20000, 2, 65536]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    parts = [W.uncorrelated_box(m, seed=40 + k, dtype=dtype) for k, m in enumerate(lens)]
    cat = {k: torch.cat([p[k] for p in parts]).to(DEV) for k in ("a", "b", "d", "l", "u")}
    r = torch.tensor([p["r"] for p in parts], dtype=torch.float64)
    offd = torch.from_numpy(off).to(DEV)
    n = int(off[-1])
    ws = api.Workspace(n, len(lens), dtype)
    x, infos, mask = api.solve_batched(*(cat[k] for k in ("a", "b", "d", "l", "u")), offd, r, want_mask=True, ws=ws)
    g = torch.randn(n, generator=torch.Generator().manual_seed(9), dtype=torch.float64).to(dtype).to(DEV)
    out = api.backward("general", g, x, ws.info, offsets=offd, mask=mask, **{k: cat[k] for k in "abdlu"})
    gr, st = out["r"].cpu().numpy(), out["status"].cpu().numpy()
    bits = mask_bits(mask, n)
    for k, m in enumerate(lens):
        lo, hi = int(off[k]), int(off[k + 1])
        if m == 0:
            assert st[k] == api.Status.NONDIFF and gr[k] == 0.0
            continue
        host = [np64(cat[key][lo:hi]) for key in "abdlu"]
        lam_star, xstar = _oracle_general(*host, float(r[k]))
        ref = oracle.grad_cqk(xstar, lam_star, *host, np64(g[lo:hi]))
        _check_general_grads(out, ref, slice(lo, hi), dtype, bits[lo:hi], *host, lam_star, xstar, f"instance {k}",
                             gr=float(gr[k]))
    # simplex / l1 batches
    y = W.simplex_normal(n, seed=3, dtype=dtype).to(DEV)
    rr = torch.full((len(lens),), 1.0, dtype=torch.float64)
    rr[3] = 1e6  # l1: inside the ball
    for l1 in (False, True):
        fn = api.project_l1_batched if l1 else api.project_simplex_batched
        ws = api.Workspace(n, len(lens), dtype)
        x, infos, mask = fn(y, offd, rr, want_mask=True, ws=ws)
        out = api.backward("l1" if l1 else "simplex", g, x, ws.info, offsets=offd, mask=mask)
        gr = out["r"].cpu().numpy()
        for k, m in enumerate(lens):
            lo, hi = int(off[k]), int(off[k + 1])
            if m == 0 or (not l1 and rr[k] != 1.0):
                continue
            ref, xstar, ties = _projection_ref(np64(y[lo:hi]), np64(g[lo:hi]), float(rr[k]), l1)
            assert not ties.any()
            _close(np64(out["y"][lo:hi]), ref["y"], dtype, f"l1={l1} instance {k}")
            assert abs(gr[k] - ref["r"]) <= TOL[dtype] * (1 + abs(ref["r"]))


def test_backward_fixed_variables_and_nondiff():
    # every variable fixed (l = u): F is empty, the map is not differentiable in r
    n = 50
    p = W.uncorrelated_box(n, seed=1)
    l = p["l"]
    r = float(torch.sum(p["b"] * l))
    dev = {k: v.to(DEV) for k, v in dict(a=p["a"], b=p["b"], d=p["d"], l=l, u=l.clone()).items()}
    ws = api.Workspace(n, 1, torch.float64)
    x, info, mask = api.solve(*(dev[k] for k in "abdlu"), r, want_mask=True, ws=ws)
    assert info.status == api.Status.OK
    g = torch.randn(n, dtype=torch.float64)
    out = api.backward("general", g.to(DEV), x, ws.info, mask=mask, **dev)
    host = [np64(p["a"]), np64(p["b"]), np64(p["d"]), np64(l), np64(l)]
    # l = u: the only feasible point is x* = l (r = b'l up to the rounding of the sum, which
    # the exact solver's feasibility test may see either way); with F empty the gradients in
    # a, b, d and r do not depend on lambda
    xstar = host[3].copy()
    ref = oracle.grad_cqk(xstar, 0.0, *host, np64(g))
    assert ref["nondiff"] and int(out["status"][0]) == api.Status.NONDIFF
    for k in "abd":
        _close(np64(out[k]), ref[k], torch.float64, f"d{k}")
    assert float(out["r"][0]) == 0.0 and ref["r"] == 0.0
    # lambda* is not unique here (phi is flat at r), and which bound a fixed variable counts as
    # active depends on it; whatever lambda, each g_i goes to exactly one of dl_i, du_i
    gl, gu, gg = np64(out["l"]), np64(out["u"]), np64(g)
    assert not np.any((gl != 0) & (gu != 0))
    _close(gl + gu, gg, torch.float64, "dl + du")  # (double-float arithmetic: equal to 2^-44)


def test_autograd_general_vs_oracle_and_fd():
    n = 40
    p = W.uncorrelated_box(n, seed=11)
    leaves = {k: p[k].to(DEV).requires_grad_(True) for k in "abdlu"}
    r = torch.tensor(p["r"], dtype=torch.float64, requires_grad=True)
    g = torch.randn(n, generator=torch.Generator().manual_seed(2), dtype=torch.float64).to(DEV)
    x = AD.cqk_solve(leaves["a"], leaves["b"], leaves["d"], leaves["l"], leaves["u"], r)
    (x * g).sum().backward()
    lam, xstar = _oracle_general(*(np64(p[k]) for k in "abdlu"), p["r"])
    ref = oracle.grad_cqk(xstar, lam, *(np64(p[k]) for k in "abdlu"), np64(g))
    for k in "abdlu":
        _close(np64(leaves[k].grad), ref[k], torch.float64, f"autograd d{k}")
    assert abs(float(r.grad) - ref["r"]) <= 1e-10 * (1 + abs(ref["r"]))
    # central finite differences of g'x through the GPU solve (instance away from kinks)
    t = (np64(p["a"]) + lam * np64(p["b"])) / np64(p["d"])
    assert np.min(np.minimum(np.abs(t - np64(p["l"])), np.abs(t - np64(p["u"])))) > 1e-4
    base = {k: p[k].clone().to(DEV) for k in "abdlu"}

    def f(vals, rv):
        xx, info, _ = api.solve(*(vals[k] for k in "abdlu"), rv)
        return float(torch.dot(xx, g))

    rng = np.random.default_rng(0)
    for k in "abdlu":
        for i in rng.choice(n, size=6, replace=False):
            h = 1e-6 * max(1.0, abs(float(base[k][i])))
            vp = {q: v.clone() for q, v in base.items()}
            vm = {q: v.clone() for q, v in base.items()}
            vp[k][i] += h
            vm[k][i] -= h
            fd = (f(vp, p["r"]) - f(vm, p["r"])) / (2 * h)
            got = float(leaves[k].grad[i])
            assert abs(fd - got) <= 1e-6 * (1 + abs(fd)), (k, i, fd, got)
    h = 1e-6 * abs(p["r"])
    fd = (f(base, p["r"] + h) - f(base, p["r"] - h)) / (2 * h)
    assert abs(fd - float(r.grad)) <= 1e-6 * (1 + abs(fd))


@pytest.mark.parametrize("l1", [False, True])
def test_autograd_batched_projection(l1):
    d = W.batched_simplex(batch=64, lo=16, hi=4096, seed=7, dtype=torch.float32)
    y = d["y"].to(DEV).requires_grad_(True)
    r = d["r"].clone().requires_grad_(True)
    off = d["offsets"].to(DEV)
    fn = AD.l1_projection if l1 else AD.simplex_projection
    x = fn(y, r, offsets=off)
    g = d["g"].to(DEV)
    (x * g).sum().backward()
    offs = d["offsets"].numpy()
    for k in range(0, 64, 7):
        lo, hi = int(offs[k]), int(offs[k + 1])
        gs, ys = np64(g[lo:hi]), np64(y[lo:hi])
        ref, xstar, ties = _projection_ref(ys, gs, 1.0, l1)
        assert not ties.any()
        _close(np64(x[lo:hi]), xstar, torch.float32, f"instance {k} x")
        _close(np64(y.grad[lo:hi]), ref["y"], torch.float32, f"instance {k}")
        assert abs(float(r.grad[k]) - ref["r"]) <= 1e-5 * (1 + abs(ref["r"]))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_projection_backward_unaligned_and_batched_staging(dtype):
    # the simplex adjoint with the forward mask streams g through shared-memory stages when
    # every array is 16-byte aligned and reads it directly otherwise: both must agree with
    # the oracle, single and batched, including instances that start inside a tile
    n = 70001
    y = W.simplex_normal(n, seed=13, dtype=dtype).to(DEV)
    g = torch.randn(n, generator=torch.Generator().manual_seed(4), dtype=torch.float64).to(dtype).to(DEV)
    ws = api.Workspace(n, 1, dtype)
    x, info, mask = api.project_simplex(y, 1.0, want_mask=True, ws=ws)
    ref, xstar, ties = _projection_ref(np64(y), np64(g), 1.0, False)
    assert not ties.any() and np.array_equal(mask_bits(mask, n), xstar > 0)
    out = api.backward("simplex", g, x, ws.info, mask=mask)
    _close(np64(out["y"]), ref["y"], dtype, "aligned")
    gbig = torch.zeros(n + 1, dtype=dtype, device=DEV)
    gbig[1:] = g
    out_u = api.backward("simplex", gbig[1:], x, ws.info, mask=mask)  # g only 4/8-byte aligned
    _close(np64(out_u["y"]), ref["y"], dtype, "unaligned")
    assert abs(float(out_u["r"][0]) - ref["r"]) <= TOL[dtype] * (1 + abs(ref["r"]))
    lens = [5000, 0, 3, 40000, 1, 24997]  # the whole array of n = 70001
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    offd = torch.from_numpy(off).to(DEV)
    yb = y[: int(off[-1])].contiguous()
    gb = g[: int(off[-1])].contiguous()
    wsb = api.Workspace(int(off[-1]), len(lens), dtype)
    xb, infos, mb = api.project_simplex_batched(yb, offd, torch.ones(len(lens), dtype=torch.float64), want_mask=True,
                                                ws=wsb, warp_elems=-1)
    outb = api.backward("simplex", gb, xb, wsb.info, offsets=offd, mask=mb)
    st = outb["status"].cpu().numpy()
    for k, m in enumerate(lens):
        lo, hi = int(off[k]), int(off[k + 1])
        if m == 0:
            assert st[k] == api.Status.NONDIFF
            continue
        refk, xstar, ties = _projection_ref(np64(yb[lo:hi]), np64(gb[lo:hi]), 1.0, False)
        assert not ties.any()
        _close(np64(outb["y"][lo:hi]), refk["y"], dtype, f"instance {k}")
        assert abs(float(outb["r"][k]) - refk["r"]) <= TOL[dtype] * (1 + abs(refk["r"]))


def test_autograd_reports_a_failed_forward():
    # r beyond b'u: the forward's status is CQK_INFEASIBLE and the autograd wrapper raises
    p = W.uncorrelated_box(100, seed=6)
    leaves = {k: p[k].to(DEV).requires_grad_(True) for k in "abdlu"}
    bu = float(torch.sum(p["b"] * p["u"]))
    with pytest.raises(AD.CQKSolveError, match="INFEASIBLE"):
        AD.cqk_solve(*(leaves[k] for k in "abdlu"), bu + 1.0)
    y = torch.randn(50, dtype=torch.float64, device=DEV, requires_grad=True)
    off = torch.tensor([0, 20, 20, 50], dtype=torch.int64, device=DEV)  # instance 1 is empty
    with pytest.raises(AD.CQKSolveError, match="instance 1"):
        AD.simplex_projection(y, torch.ones(3, dtype=torch.float64), offsets=off)
    x = AD.simplex_projection(y, torch.ones(3, dtype=torch.float64), offsets=off, check=False)
    assert x.shape == y.shape


@pytest.mark.parametrize("t", [0.25, 0.5, 1.0, 2.0, 1024.0])
def test_adjoint_results_just_inside_a_power_of_two(t):
    # gy_i = g_i - mean_F(g) with every element free.  With g = (4c, 0, 0, 0) the mean is c
    # and gy = (3c, -c, -c, -c); c just below t makes -c a double-float pair whose high part
    # is exactly -t and whose low part points toward zero: the FP64 result then lies in the
    # binade below t, where one ulp is half as large as above it.
    for c in (t - 3e-9 * t, t - 1e-13 * t, t + 3e-9 * t):
        y = torch.ones(4, dtype=torch.float64, device=DEV)
        g = torch.tensor([4 * c, 0.0, 0.0, 0.0], dtype=torch.float64, device=DEV)
        ws = api.Workspace(4, 1, torch.float64)
        x, info, mask = api.project_simplex(y, 1.0, want_mask=True, ws=ws)
        out = api.backward("simplex", g, x, ws.info, mask=mask)
        ref, xstar, ties = _projection_ref(np64(y), np64(g), 1.0, False)
        got = np64(out["y"])
        # the map is double-float (~2^-44 relative); the binade slip was lo/2, ~1.5e-9 t here
        assert np.max(np.abs(got - ref["y"])) <= 2.0 ** -40 * (1 + np.max(np.abs(ref["y"]))), (c, got, ref["y"])
