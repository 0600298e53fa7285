"""GPU parity of the batched entry points (cqk_solve_batched, cqk_project_simplex_batched,
cqk_project_l1_batched) against the FP64 oracle, instance by instance, through the C ABI.

Ragged batches cover empty instances, single elements, instance boundaries that cut 16-byte
vectors, and instances solved by groups of several blocks (small group_elems)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2603_15910_b300 import api, workloads as W
from helpers import assert_feasible, assert_x_close, mask_bits, np64

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _lengths(seed, count, hi):
    rng = np.random.default_rng(seed)
    lens = [int(v) for v in np.exp(rng.uniform(0.0, math.log(hi), size=count)).round()]
    # edge cases: empty instances, singletons, odd lengths that misalign the next instance
    lens[1] = 0
    lens[2] = 1
    lens[3] = 3
    lens[-1] = 0
    return lens


def _offsets(lens):
    return np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)


def _check_simplex_instance(y64, x, info, r, dtype, l1, off0, what):
    m = y64.size
    if l1:
        lam, xstar, inside = oracle.project_l1(y64, r)
    else:
        lam, xstar = oracle.project_simplex_sort(y64, r)
    assert info.status == api.Status.OK, (what, info)
    assert_x_close(x, xstar, dtype, what)
    res = abs(float(np.sum(np.abs(x), dtype=np.longdouble)) - r)
    if not (l1 and info.stop == "inside"):
        assert res <= (1e-12 if dtype == torch.float64 else 1e-5) * r, (what, res)
    assert info.nfree == int((x != 0).sum()), (what, info)
    if dtype == torch.float64 and info.stop != "inside":
        lam0, S, C = oracle.condat_chunks(y64, r, info.tile, info.nchunks, l1=l1, shift=off0 % info.tile)
        assert math.isclose(info.lambda0, lam0, rel_tol=1e-13, abs_tol=1e-15), (what, info, lam0)
        nw = oracle.newton_simplex(y64, r, lam0=info.lambda0, l1=l1)
        assert abs(info.iters - nw["evals"]) <= 1, (what, info.iters, nw["evals"])


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("l1", [False, True])
@pytest.mark.parametrize("group_elems", [0, 2048])
def test_batched_projection_matches_oracle(dtype, l1, group_elems):
    lens = _lengths(11 + l1, 48, 60000)
    off = _offsets(lens)
    n = int(off[-1])
    g = torch.Generator().manual_seed(5)
    y = torch.randn(n, generator=g, dtype=torch.float64)
    y[: n // 3] *= 3.0
    y = y.to(dtype)
    rng = np.random.default_rng(1)
    r = rng.uniform(0.5, 4.0, size=len(lens))
    if l1:
        r[5] = 1e9  # y inside the ball: x = y
    fn = api.project_l1_batched if l1 else api.project_simplex_batched
    x, infos, mask = fn(y.to(DEV), torch.from_numpy(off), torch.from_numpy(r), want_mask=True,
                        group_elems=group_elems)
    xs = np64(x)
    ys = np64(y)
    bits = mask_bits(mask, n)
    for k, m in enumerate(lens):
        lo, hi = int(off[k]), int(off[k + 1])
        what = f"instance {k} (m={m}, lo={lo})"
        if m == 0:
            if l1:
                assert infos[k].status == api.Status.OK and infos[k].stop == "inside", infos[k]
            else:
                assert infos[k].status == api.Status.INFEASIBLE, infos[k]
            continue
        _check_simplex_instance(ys[lo:hi], xs[lo:hi], infos[k], float(r[k]), dtype, l1, lo, what)
        assert np.array_equal(bits[lo:hi], xs[lo:hi] != 0), what


@pytest.mark.parametrize("init", [api.Init.FORMULA, api.Init.CONDAT])
def test_batched_simplex_formula_and_condat(init):
    lens = _lengths(3, 20, 200000)
    off = _offsets(lens)
    y = W.simplex_normal(int(off[-1]), seed=9, sparse=True)
    r = np.ones(len(lens))
    x, infos, _ = api.project_simplex_batched(y.to(DEV), torch.from_numpy(off), torch.from_numpy(r), init=init)
    xs, ys = np64(x), np64(y)
    for k, m in enumerate(lens):
        if m == 0:
            continue
        lo, hi = int(off[k]), int(off[k + 1])
        lam, xstar = oracle.project_simplex_sort(ys[lo:hi], 1.0)
        assert infos[k].status == api.Status.OK
        assert_x_close(xs[lo:hi], xstar, torch.float64, f"instance {k}")
        if init == api.Init.FORMULA:
            nw = oracle.newton_simplex(ys[lo:hi], 1.0)
            assert math.isclose(infos[k].lambda0, max(nw["lam0"], -ys[lo:hi].max()), rel_tol=1e-12, abs_tol=1e-14)
            assert abs(infos[k].iters - nw["evals"]) <= 1


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("group_elems", [0, 1024])
def test_batched_general_matches_oracle(dtype, group_elems):
    lens = _lengths(21, 36, 40000)
    parts = [W.uncorrelated_box(m, seed=100 + k, dtype=dtype) for k, m in enumerate(lens)]
    cat = {key: torch.cat([p[key] for p in parts]) for key in ("a", "b", "d", "l", "u")}
    r = np.array([p["r"] for p in parts], dtype=np.float64)
    r[1] = 0.0  # empty instance with r = 0: feasible
    off = _offsets(lens)
    x, infos, mask = api.solve_batched(*(cat[k].to(DEV) for k in ("a", "b", "d", "l", "u")), torch.from_numpy(off),
                                       torch.from_numpy(r), want_mask=True, group_elems=group_elems)
    xs = np64(x)
    bits = mask_bits(mask, xs.size)
    for k, m in enumerate(lens):
        lo, hi = int(off[k]), int(off[k + 1])
        what = f"instance {k} (m={m}, lo={lo})"
        if m == 0:
            want = api.Status.OK if r[k] == 0.0 else api.Status.INFEASIBLE
            assert infos[k].status == want, (what, infos[k])
            continue
        a, b, d, l, u = (np64(cat[key][lo:hi]) for key in ("a", "b", "d", "l", "u"))
        ref = oracle.newton_cqk(a, b, d, l, u, float(r[k]))
        assert infos[k].status == api.Status.OK, (what, infos[k])
        xstar = oracle.solve_sort(a, b, d, l, u, float(r[k]))[2] if m <= 4096 else ref["x"]
        assert_x_close(xs[lo:hi], xstar, dtype, what)
        assert_feasible(xs[lo:hi], b, float(r[k]), dtype, what)
        free = (xs[lo:hi] > l) & (xs[lo:hi] < u)
        assert np.array_equal(bits[lo:hi], free), what
        if dtype == torch.float64:
            assert abs(infos[k].iters - ref["evals"]) <= 1, (what, infos[k].iters, ref["evals"])


@pytest.mark.parametrize("init", [api.Init.FORMULA, api.Init.CONDAT])
def test_batched_matches_single_calls(init):
    # every instance of a batch gets the same answer as its own single call (to tolerance:
    # the partition of the sums differs, and with the Alg. 2 start so does the chunking)
    lens = [5000, 1, 77, 12345, 0, 640, 99999]
    off = _offsets(lens)
    y = W.simplex_normal(int(off[-1]), seed=4)
    r = np.full(len(lens), 2.0)
    xb, infos, _ = api.project_simplex_batched(y.to(DEV), torch.from_numpy(off), torch.from_numpy(r), init=init)
    for k, m in enumerate(lens):
        if m == 0:
            continue
        lo, hi = int(off[k]), int(off[k + 1])
        xs, info, _ = api.project_simplex(y[lo:hi].to(DEV), 2.0, init=init)
        assert_x_close(np64(xb[lo:hi]), np64(xs), torch.float64, f"instance {k}")
        if init == api.Init.FORMULA:  # the same start: the same Newton sequence up to rounding
            assert abs(infos[k].iters - info.iters) <= 1


def test_batched_is_deterministic():
    d = W.batched_simplex(batch=64, lo=16, hi=1 << 16, seed=3, dtype=torch.float32)
    y = d["y"].to(DEV)
    x1, i1, m1 = api.project_simplex_batched(y, d["offsets"], d["r"], want_mask=True)
    x2, i2, m2 = api.project_simplex_batched(y, d["offsets"], d["r"], want_mask=True)
    assert torch.equal(x1, x2) and torch.equal(m1, m2)
    assert [(a.lam, a.iters) for a in i1] == [(b.lam, b.iters) for b in i2]


def test_batched_bad_instances_are_reported():
    # a decreasing offsets pair and a NaN r are reported in the instance's info; the others solve
    y = W.simplex_normal(40, seed=2)
    off = torch.tensor([0, 10, 5, 5, 40], dtype=torch.int64)
    r = torch.tensor([1.0, 1.0, 1.0, float("nan")], dtype=torch.float64)
    x, infos, _ = api.project_simplex_batched(y.to(DEV), off, r)
    assert infos[0].status == api.Status.OK
    assert infos[1].status == api.Status.BAD_ARG
    assert infos[2].status == api.Status.INFEASIBLE  # empty
    assert infos[3].status == api.Status.BAD_ARG
    lam, xstar = oracle.project_simplex_sort(np64(y[:10]), 1.0)
    assert_x_close(np64(x[:10]), xstar, torch.float64)
    a = W.uncorrelated_box(30, seed=1)
    off = torch.tensor([0, 30, 30], dtype=torch.int64)
    r = torch.tensor([a["r"], float("nan")], dtype=torch.float64)
    x, infos, _ = api.solve_batched(*(a[k].to(DEV) for k in ("a", "b", "d", "l", "u")), off, r)
    assert infos[0].status == api.Status.OK and infos[1].status == api.Status.BAD_ARG


def test_batched_bad_input_flagged_per_instance():
    a = W.uncorrelated_box(3000, seed=8)
    off = torch.tensor([0, 1000, 2000, 3000], dtype=torch.int64)
    r = torch.tensor([float(torch.sum(a["b"][o:o + 1000] * (a["l"][o:o + 1000] + a["u"][o:o + 1000]) / 2))
                      for o in (0, 1000, 2000)], dtype=torch.float64)
    d = a["d"].clone()
    d[1500] = -1.0  # instance 1 invalid
    x, infos, _ = api.solve_batched(a["a"].to(DEV), a["b"].to(DEV), d.to(DEV), a["l"].to(DEV), a["u"].to(DEV), off, r)
    assert infos[1].status == api.Status.BAD_INPUT
    assert infos[0].status == api.Status.OK and infos[2].status == api.Status.OK


def test_batched_config_shape_simplex_f32():
    # the ragged simplex batch recipe (log-uniform lengths, FP32 y ~ N(0,1), r = 1), sampled
    d = W.batched_simplex(batch=512, lo=16, hi=1 << 18, seed=0, dtype=torch.float32)
    x, infos, _ = api.project_simplex_batched(d["y"].to(DEV), d["offsets"], d["r"])
    off = d["offsets"].numpy()
    xs, ys = np64(x), np64(d["y"])
    assert all(i.status == api.Status.OK for i in infos)
    for k in range(0, 512, 37):
        lo, hi = int(off[k]), int(off[k + 1])
        lam, xstar = oracle.project_simplex_sort(ys[lo:hi], 1.0)
        assert_x_close(xs[lo:hi], xstar, torch.float32, f"instance {k}")


BUILDS = [(256, 0), (128, 0), (512, 0), (256, 1)]


@pytest.mark.parametrize("block_threads,unroll", BUILDS)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_general_builds_match_oracle(block_threads, unroll, dtype):
    # every build of the batched general kernel and its adjoint (block size, per-lane unroll),
    # with multi-block groups (small group_elems) and one-block instances
    lens = _lengths(31, 24, 30000)
    parts = [W.uncorrelated_box(m, seed=300 + k, dtype=dtype) for k, m in enumerate(lens)]
    cat = {key: torch.cat([p[key] for p in parts]).to(DEV) for key in ("a", "b", "d", "l", "u")}
    r = np.array([p["r"] for p in parts], dtype=np.float64)
    r[1] = 0.0
    off = torch.from_numpy(_offsets(lens)).to(DEV)
    n = int(off[-1])
    g = torch.randn(n, generator=torch.Generator().manual_seed(3), dtype=torch.float64).to(dtype).to(DEV)
    for ge in (0, 2048):
        opts = dict(block_threads=block_threads, unroll=unroll, group_elems=ge)
        ws = api.Workspace(n, len(lens), dtype)
        x, infos, mask = api.solve_batched(*(cat[k] for k in "abdlu"), off, torch.from_numpy(r), want_mask=True, ws=ws,
                                           **opts)
        out = api.backward("general", g, x, ws.info, offsets=off, mask=mask, **{k: cat[k] for k in "abdlu"}, **opts)
        xs, gr = np64(x), out["r"].cpu().numpy()
        bits = mask_bits(mask, n)
        for k, m in enumerate(lens):
            lo, hi = int(off[k]), int(off[k + 1])
            what = f"build {block_threads}/{unroll} ge={ge} instance {k} (m={m})"
            if m == 0:
                assert infos[k].status == api.Status.OK, what
                continue
            host = [np64(cat[q][lo:hi]) for q in "abdlu"]
            st, lam, xstar = oracle.solve_sort(*host, float(r[k]))
            assert infos[k].status == api.Status.OK, (what, infos[k])
            assert_x_close(xs[lo:hi], xstar, dtype, what)
            assert_feasible(xs[lo:hi], host[1], float(r[k]), dtype, what)
            assert np.array_equal(bits[lo:hi], (xs[lo:hi] > host[3]) & (xs[lo:hi] < host[4])), what
            ref = oracle.grad_cqk(xstar, lam, *host, np64(g[lo:hi]))
            tol = 1e-10 if dtype == torch.float64 else 1e-5
            for q in "abdlu":
                err = float(np.max(np.abs(np64(out[q][lo:hi]) - ref[q])))
                assert err <= tol * (1 + float(np.max(np.abs(ref[q])))), (what, q, err)
            assert abs(gr[k] - ref["r"]) <= tol * (1 + abs(ref["r"])), what


@pytest.mark.parametrize("block_threads,unroll", BUILDS)
@pytest.mark.parametrize("l1", [False, True])
def test_batched_projection_builds_match_oracle(block_threads, unroll, l1):
    # the projection forward has the default and the half-unroll build; its adjoint every build
    dtype = torch.float32
    lens = _lengths(41 + l1, 40, 100000)
    off = torch.from_numpy(_offsets(lens)).to(DEV)
    n = int(off[-1])
    y = W.simplex_normal(n, seed=17, dtype=dtype).to(DEV)
    g = torch.randn(n, generator=torch.Generator().manual_seed(5), dtype=torch.float64).to(dtype).to(DEV)
    r = torch.ones(len(lens), dtype=torch.float64)
    fwd_unroll = unroll if block_threads == 256 else 0
    fn = api.project_l1_batched if l1 else api.project_simplex_batched
    ws = api.Workspace(n, len(lens), dtype)
    x, infos, mask = fn(y, off, r, want_mask=True, ws=ws, unroll=fwd_unroll)
    out = api.backward("l1" if l1 else "simplex", g, x, ws.info, offsets=off, mask=mask, block_threads=block_threads,
                       unroll=unroll)
    xs, ys, gs, gy, gr = np64(x), np64(y), np64(g), np64(out["y"]), out["r"].cpu().numpy()
    for k, m in enumerate(lens):
        lo, hi = int(off[k]), int(off[k + 1])
        if m == 0:
            continue
        what = f"build {block_threads}/{unroll} l1={l1} instance {k} (m={m})"
        if l1:
            lam, xstar, inside = oracle.project_l1(ys[lo:hi], 1.0)
            ref = oracle.grad_l1(ys[lo:hi], xstar, gs[lo:hi], inside)
        else:
            lam, xstar = oracle.project_simplex_sort(ys[lo:hi], 1.0)
            ref = oracle.grad_simplex(xstar, gs[lo:hi])
        assert infos[k].status == api.Status.OK, (what, infos[k])
        assert_x_close(xs[lo:hi], xstar, dtype, what)
        err = float(np.max(np.abs(gy[lo:hi] - ref["y"])))
        assert err <= 1e-5 * (1 + float(np.max(np.abs(ref["y"])))), (what, err)
        assert abs(gr[k] - ref["r"]) <= 1e-5 * (1 + abs(ref["r"])), what


def test_unsupported_builds_are_rejected():
    # the projection forward has no 128/512-thread build; single-instance calls have one build
    y = W.simplex_normal(1000, seed=1).to(DEV)
    off = torch.tensor([0, 500, 1000], dtype=torch.int64, device=DEV)
    r = torch.ones(2, dtype=torch.float64)
    for bt in (128, 512, 64):
        with pytest.raises(RuntimeError, match="bad_arg"):
            api.project_simplex_batched(y, off, r, block_threads=bt)
    with pytest.raises(RuntimeError, match="bad_arg"):
        api.project_simplex(y, 1.0, unroll=1)
    with pytest.raises(RuntimeError, match="bad_arg"):
        api.project_simplex_batched(y, off, r, block_threads=512, unroll=1)
