"""GPU parity of the adjoint kernels (cqk_backward, cqk_backward_simplex, cqk_backward_l1)
and of the autograd wrappers, against the oracle's implicit-function gradients (which the
CPU suite pins to finite differences of the exact solution map), and a finite-difference
check of the whole differentiable GPU solve."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_15910_b300 import api, autograd as AD, workloads as W
from helpers import np64

pytestmark = pytest.mark.gpu
DEV = "cuda"
TOL = {torch.float64: 1e-10, torch.float32: 1e-5}


def _close(got, want, dtype, what=""):
    got, want = np.asarray(got, dtype=np.float64), np.asarray(want, dtype=np.float64)
    err = float(np.max(np.abs(got - want))) if got.size else 0.0
    bound = TOL[dtype] * (1.0 + (float(np.max(np.abs(want))) if want.size else 0.0))
    assert err <= bound, f"{what}: max err {err:.3e} > {bound:.3e}"


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
    ref = oracle.grad_cqk(np64(x), info.lam, *(np64(p[k]) for k in ("a", "b", "d", "l", "u")), np64(g))
    assert int(out["status"][0]) == (api.Status.NONDIFF if ref["nondiff"] else api.Status.OK)
    for k in "abdlu":
        _close(np64(out[k]), ref[k], dtype, f"d{k} n={n}")
    assert abs(float(out["r"][0]) - ref["r"]) <= TOL[dtype] * (1 + abs(ref["r"]))


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
        if l1:
            ref = oracle.grad_l1(np64(y), np64(x), np64(g), info.stop == "inside")
        else:
            ref = oracle.grad_simplex(np64(x), np64(g))
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
    for k, m in enumerate(lens):
        lo, hi = int(off[k]), int(off[k + 1])
        if m == 0:
            assert st[k] == api.Status.NONDIFF and gr[k] == 0.0
            continue
        ref = oracle.grad_cqk(np64(x[lo:hi]), infos[k].lam, *(np64(cat[key][lo:hi]) for key in "abdlu"),
                              np64(g[lo:hi]))
        for key in "abdlu":
            _close(np64(out[key][lo:hi]), ref[key], dtype, f"instance {k} d{key}")
        assert abs(gr[k] - ref["r"]) <= TOL[dtype] * (1 + abs(ref["r"]))
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
            if m == 0:
                continue
            if l1:
                ref = oracle.grad_l1(np64(y[lo:hi]), np64(x[lo:hi]), np64(g[lo:hi]), infos[k].stop == "inside")
            else:
                ref = oracle.grad_simplex(np64(x[lo:hi]), np64(g[lo:hi]))
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
    ref = oracle.grad_cqk(np64(x), info.lam, np64(p["a"]), np64(p["b"]), np64(p["d"]), np64(l), np64(l), np64(g))
    assert ref["nondiff"] and int(out["status"][0]) == api.Status.NONDIFF
    for k in "abdlu":
        _close(np64(out[k]), ref[k], torch.float64, f"d{k}")


def test_autograd_general_vs_oracle_and_fd():
    n = 40
    p = W.uncorrelated_box(n, seed=11)
    leaves = {k: p[k].to(DEV).requires_grad_(True) for k in "abdlu"}
    r = torch.tensor(p["r"], dtype=torch.float64, requires_grad=True)
    g = torch.randn(n, generator=torch.Generator().manual_seed(2), dtype=torch.float64).to(DEV)
    x = AD.cqk_solve(leaves["a"], leaves["b"], leaves["d"], leaves["l"], leaves["u"], r)
    (x * g).sum().backward()
    lam = float(oracle.solve_sort(*(np64(p[k]) for k in "abdlu"), p["r"])[1])
    ref = oracle.grad_cqk(np64(x), lam, *(np64(p[k]) for k in "abdlu"), np64(g))
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
        xs, gs, ys = np64(x[lo:hi]), np64(g[lo:hi]), np64(y[lo:hi])
        if l1:
            inside = float(np.sum(np.abs(ys))) <= 1.0
            ref = oracle.grad_l1(ys, xs, gs, inside)
        else:
            ref = oracle.grad_simplex(xs, gs)
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
    ref = oracle.grad_simplex(np64(x), np64(g))
    out = api.backward("simplex", g, x, ws.info, mask=mask)
    _close(np64(out["y"]), ref["y"], dtype, "aligned")
    gbig = torch.zeros(n + 1, dtype=dtype, device=DEV)
    gbig[1:] = g
    out_u = api.backward("simplex", gbig[1:], x, ws.info, mask=mask)  # g only 4/8-byte aligned
    _close(np64(out_u["y"]), ref["y"], dtype, "unaligned")
    assert abs(float(out_u["r"][0]) - ref["r"]) <= TOL[dtype] * (1 + abs(ref["r"]))
    lens = [5000, 0, 3, 40000, 1, 25000]
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
        refk = oracle.grad_simplex(np64(xb[lo:hi]), np64(gb[lo:hi]))
        _close(np64(outb["y"][lo:hi]), refk["y"], dtype, f"instance {k}")
        assert abs(float(outb["r"][k]) - refk["r"]) <= TOL[dtype] * (1 + abs(refk["r"]))
