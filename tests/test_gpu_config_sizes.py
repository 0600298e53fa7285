"""GPU parity at the benchmarked sizes, in the launch configuration the benchmark times.

Every call uses the library's default options and automatic persistent grid, as bench.py
does:
  * general CQK, uncorrelated box family, n = 4e6, and correlated family, n = 2e7 and 1e8,
    FP64 and FP32 storage: the whole grid runs, each block streaming many bulk-copy tiles of
    the five arrays and flushing its sums many times;
  * simplex and l1-ball projections, n = 1e8, FP64, y ~ N(0,1) and the 1%-sparse variant,
    Condat start (the benchmark's projections);
  * the ragged simplex batch: 4096 instances, lengths log-uniform in [16, 2^20], FP32,
    forward and adjoint;
  * the ragged general batch: 256 instances, lengths log-uniform in [1e3, 1e6], FP64 (the box
    family, instance i drawn with seed 1000 + i), forward, adjoint and central finite
    differences in a, b, d and r.
Every solution is compared element by element with the oracle's exact solver (breakpoint
sort and search; sort-based simplex projection) run on the stored input values, every free
mask with the oracle's free set away from ties, and every gradient with the oracle's
implicit-function gradient evaluated at the oracle's own solution.  The oracle solves
independent instances on all host cores."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2603_15910_b300 import api, workloads as W
from helpers import TOL_FEAS, assert_feasible, assert_x_close, mask_bits, np64, oracle_map

pytestmark = pytest.mark.gpu
DEV = "cuda"
TOL_G = {torch.float64: 1e-10, torch.float32: 1e-5}
# half-width of the band around a bound (relative) inside which the free status of an element
# may differ between two correct solutions (rounding of lambda and of x)
# Half-width of the band around a bound inside which the free status of an element may differ
# between two correct solutions, relative to the terms of v = a + lambda b against d l, d u (the
# kernel's own tie rule has 2^-42 for FP64 data and 2^-20 for FP32 data), and for the
# projections relative to |y| + |lambda|.
TIE = {torch.float64: 1e-9, torch.float32: 4e-6}
TIE_PROJ = 1e-9


def _ties_general(a, b, d, l, u, lam, dtype):
    with np.errstate(invalid="ignore"):
        v = a + lam * b
        sc = np.abs(a) + np.abs(lam * b)
        dl, du = d * l, d * u
        tl = np.abs(v - dl) <= TIE[dtype] * (sc + np.abs(dl))
        tu = np.abs(v - du) <= TIE[dtype] * (sc + np.abs(du))
    return tl | tu


def _ties_proj(y, lam):
    return np.abs(y + lam) <= TIE_PROJ * (np.abs(y) + abs(lam))


def _solve_general(p):
    """GPU solve of p (device arrays); returns the host copies of data and results."""
    a, b, d, l, u = (p[k] for k in "abdlu")
    x, info, mask = api.solve(a, b, d, l, u, p["r"], want_mask=True)
    out = dict(host=[np64(v) for v in (a, b, d, l, u)], r=p["r"], x=np64(x), info=info,
               bits=mask_bits(mask, x.numel()), dtype=a.dtype)
    del x, mask
    return out


def _check_general(sol, exact, newton, what):
    """Compare one GPU solve with the oracle's exact solution (and Alg. 1's iteration count)."""
    dtype, info, xs, bits = sol["dtype"], sol["info"], sol["x"], sol["bits"]
    ha, hb, hd, hl, hu = sol["host"]
    assert info.status == api.Status.OK, (what, info)
    st, lam_star, xstar = exact
    assert st == "ok", what
    assert_x_close(xs, xstar, dtype, what)
    assert_feasible(xs, hb, sol["r"], dtype, what)
    assert abs(info.residual) <= TOL_FEAS[dtype] * info.abs_bx, (what, info)
    free_gpu = (xs > hl) & (xs < hu)
    assert np.array_equal(bits, free_gpu), what
    assert info.nfree == int(free_gpu.sum()), what
    free_star = (xstar > hl) & (xstar < hu)
    ties = _ties_general(ha, hb, hd, hl, hu, lam_star, dtype)
    assert np.array_equal(bits[~ties], free_star[~ties]), what
    if newton is not None:
        assert abs(info.iters - newton["evals"]) <= 1, (what, info.iters, newton["evals"])


def _general_case(make, what, newton_dtypes):
    """GPU solves in FP64 and FP32 storage, then the oracle on both at once (host threads)."""
    sols = {}
    for dtype in (torch.float64, torch.float32):
        sols[dtype] = _solve_general(make(dtype))
        torch.cuda.empty_cache()
    jobs = [(dt, "exact") for dt in sols] + [(dt, "newton") for dt in sols if dt in newton_dtypes]

    def run(job):
        dt, kind = job
        sol = sols[dt]
        if kind == "exact":
            return oracle.solve_sort(*sol["host"], sol["r"])
        return oracle.newton_cqk(*sol["host"], sol["r"])

    res = dict(zip(jobs, oracle_map(run, jobs)))
    for dt, sol in sols.items():
        _check_general(sol, res[(dt, "exact")], res.get((dt, "newton")), f"{what} {dt}")


def test_general_full_grid_box_family():
    _general_case(lambda dt: W.uncorrelated_box(4_000_000, seed=21, device=DEV, dtype=dt), "box n=4e6",
                  (torch.float64,))


@pytest.mark.parametrize("n", [20_000_000, 100_000_000])
def test_general_correlated_family_at_size(n):
    _general_case(lambda dt: W.correlated(n, seed=0, device=DEV, dtype=dt), f"correlated n={n}",
                  (torch.float64,) if n <= 20_000_000 else ())


def test_projections_at_size():
    """The benchmark's projections (n = 1e8, FP64, Condat start) and the 1%-sparse variant,
    every element against the sort-based oracle."""
    n = 100_000_000
    results = {}
    for sparse in (False, True):
        y = W.simplex_normal(n, seed=0, sparse=sparse, device=DEV)
        for l1 in (False, True):
            fn = api.project_l1 if l1 else api.project_simplex
            x, info, mask = fn(y, 1.0, init=api.Init.CONDAT, want_mask=True)
            assert info.status == api.Status.OK, (sparse, l1, info)
            results[(sparse, l1)] = (np64(x), info, mask_bits(mask, n))
        ys = np64(y)
        del y, x, mask
        torch.cuda.empty_cache()

        def exact(l1):
            if l1:
                lam, xstar, inside = oracle.project_l1(ys, 1.0)
                assert not inside
                return lam, xstar
            return oracle.project_simplex_sort(ys, 1.0)

        for l1, (lam_star, xstar) in zip((False, True), oracle_map(exact, (False, True))):
            xs, info, bits = results.pop((sparse, l1))
            what = f"sparse={sparse} l1={l1}"
            assert_x_close(xs, xstar, torch.float64, what)
            res = abs(float(np.sum(np.abs(xs), dtype=np.longdouble)) - 1.0)
            assert res <= 1e-12, (what, res)
            assert np.array_equal(bits, xs != 0), what
            yy = np.abs(ys) if l1 else ys
            ties = _ties_proj(yy, lam_star)
            assert np.array_equal(bits[~ties], (xstar != 0)[~ties]), what
            # the Alg. 2 start over the block-chunk partition the kernel reports
            lam0, _, _ = oracle.condat_chunks(ys, 1.0, info.tile, info.nchunks, l1=l1)
            assert math.isclose(info.lambda0, lam0, rel_tol=1e-13, abs_tol=1e-15), (what, info.lambda0, lam0)


def _ragged_simplex_batch():
    return W.batched_simplex(batch=4096, lo=16, hi=1 << 20, seed=0, device=DEV, dtype=torch.float32)


def test_ragged_simplex_batch_forward_and_adjoint():
    """Every instance of the 4096-instance FP32 batch, forward and adjoint, in the benchmark's
    launch configuration (default options, the forward's mask passed to the adjoint)."""
    d = _ragged_simplex_batch()
    y, off, r, g = d["y"], d["offsets"], d["r"], d["g"]
    B = off.numel() - 1
    n = y.numel()
    ws = api.Workspace(n, B, y.dtype)
    x, infos, mask = api.project_simplex_batched(y, off, r, want_mask=True, ws=ws)
    out = api.backward("simplex", g, x, ws.info, offsets=off, mask=mask, ws=api.Workspace(n, B, y.dtype))
    ys, xs, gs, gys = np64(y), np64(x), np64(g), np64(out["y"])
    bits = mask_bits(mask, n)
    grs, sts = out["r"].cpu().numpy(), out["status"].cpu().numpy()
    offs = off.cpu().numpy()
    assert all(i.status == api.Status.OK for i in infos)
    assert np.array_equal(bits, xs > 0)

    def exact(k):
        lo, hi = int(offs[k]), int(offs[k + 1])
        return oracle.project_simplex_sort(ys[lo:hi], 1.0)

    sols = oracle_map(exact, range(B))
    skipped = 0
    for k, (lam_star, xstar) in enumerate(sols):
        lo, hi = int(offs[k]), int(offs[k + 1])
        what = f"instance {k} (m={hi - lo})"
        assert_x_close(xs[lo:hi], xstar, torch.float32, what)
        assert abs(float(np.sum(xs[lo:hi], dtype=np.longdouble)) - 1.0) <= 1e-5, what
        ties = _ties_proj(ys[lo:hi], lam_star)
        free_star = xstar > 0
        assert np.array_equal(bits[lo:hi][~ties], free_star[~ties]), what
        assert sts[k] == api.Status.OK, what
        if ties.any():  # the gradient depends on F as a whole: compare where F is unambiguous
            skipped += 1
            continue
        ref = oracle.grad_simplex(xstar, gs[lo:hi])
        err = float(np.max(np.abs(gys[lo:hi] - ref["y"])))
        assert err <= TOL_G[torch.float32] * (1 + float(np.max(np.abs(ref["y"])))), (what, err)
        assert abs(grs[k] - ref["r"]) <= TOL_G[torch.float32] * (1 + abs(ref["r"])), what
    assert skipped <= B // 100, skipped


def _fd_general(host, r, g, i, which, xstar_base, lam_base):
    """Central finite difference of g'x* of one instance in coordinate i of `which` (or r), by
    the oracle's exact solver.  Returns None when an element other than i changes status
    between the two perturbed solutions (a kink inside the step)."""
    a, b, d, l, u = host
    vals = {"a": a, "b": b, "d": d}
    if which == "r":
        h = 1e-3
    elif which == "a":
        h = 1e-4 * (1.0 + abs(a[i]))
    else:
        h = 1e-5 * abs(vals[which][i])
    fs, stats = [], []
    for sgn in (1.0, -1.0):
        arrs = dict(a=a, b=b, d=d)
        rr = r
        if which == "r":
            rr = r + sgn * h
        else:
            v = vals[which].copy()
            v[i] += sgn * h
            arrs[which] = v
        st, lam, xx = oracle.solve_sort(arrs["a"], arrs["b"], arrs["d"], l, u, rr)
        assert st == "ok"
        fs.append(np.sum(g.astype(np.longdouble) * xx.astype(np.longdouble)))
        stats.append(np.where(xx <= l, 1, np.where(xx >= u, 2, 0)))
    same = stats[0] == stats[1]
    if which != "r":
        same[i] = True
    if not same.all():
        return None
    return float((fs[0] - fs[1]) / (2.0 * h))


def test_ragged_general_batch_forward_adjoint_and_fd():
    """Every instance of the 256-instance FP64 batch: x against the exact oracle, the free mask,
    the adjoint against the oracle gradient at the oracle's own (x*, lambda*), and central
    finite differences of g'x* in a, b, d (one free coordinate per instance) and r on every
    eighth instance, rel err <= 1e-6."""
    dt = torch.float64
    p = W.batched_general(batch=256, lo=1000, hi=1000000, seed=0, device=DEV, dtype=dt)
    off, r, g = p["offsets"], p["r"], p["g"]
    B = off.numel() - 1
    n = p["a"].numel()
    ws = api.Workspace(n, B, dt)
    x, infos, mask = api.solve_batched(*(p[k] for k in "abdlu"), off, r, want_mask=True, ws=ws)
    out = api.backward("general", g, x, ws.info, offsets=off, mask=mask, ws=api.Workspace(n, B, dt),
                       **{k: p[k] for k in "abdlu"})
    host = {k: np64(p[k]) for k in "abdlu"}
    xs, gs = np64(x), np64(g)
    grads = {k: np64(out[k]) for k in "abdlu"}
    grs, sts = out["r"].cpu().numpy(), out["status"].cpu().numpy()
    rs = r.cpu().numpy()
    bits = mask_bits(mask, n)
    offs = off.cpu().numpy()

    def sl(k):
        return slice(int(offs[k]), int(offs[k + 1]))

    def exact(k):
        return oracle.solve_sort(*(host[q][sl(k)] for q in "abdlu"), float(rs[k]))

    sols = oracle_map(exact, range(B))
    skipped = 0
    for k, (st, lam_star, xstar) in enumerate(sols):
        s = sl(k)
        what = f"instance {k} (m={s.stop - s.start})"
        assert st == "ok" and infos[k].status == api.Status.OK and sts[k] == api.Status.OK, what
        a, b, d, l, u = (host[q][s] for q in "abdlu")
        assert_x_close(xs[s], xstar, dt, what)
        assert_feasible(xs[s], b, float(rs[k]), dt, what)
        assert np.array_equal(bits[s], (xs[s] > l) & (xs[s] < u)), what
        ties = _ties_general(a, b, d, l, u, lam_star, dt)
        assert np.array_equal(bits[s][~ties], ((xstar > l) & (xstar < u))[~ties]), what
        if ties.any():
            skipped += 1
            continue
        ref = oracle.grad_cqk(xstar, lam_star, a, b, d, l, u, gs[s])
        for q in "abdlu":
            err = float(np.max(np.abs(grads[q][s] - ref[q])))
            assert err <= TOL_G[dt] * (1 + float(np.max(np.abs(ref[q])))), (what, q, err)
        assert abs(grs[k] - ref["r"]) <= TOL_G[dt] * (1 + abs(ref["r"])), what
    assert skipped <= B // 50, skipped

    # finite differences of the exact solution map against the GPU gradient
    rng = np.random.default_rng(0)
    jobs = []
    for k in range(0, B, 8):
        s = sl(k)
        a, b, d, l, u = (host[q][s] for q in "abdlu")
        lam_star, xstar = sols[k][1], sols[k][2]
        t = (a + lam_star * b) / d
        margin = np.minimum(np.abs(t - l), np.abs(t - u))
        cand = np.nonzero(margin > 1e-2)[0]
        for which in ("a", "b", "d", "r"):
            i = int(rng.choice(cand)) if which != "r" else -1
            jobs.append((k, which, i))

    def run(job):
        k, which, i = job
        s = sl(k)
        hk = [host[q][s] for q in "abdlu"]
        return _fd_general(hk, float(rs[k]), gs[s], i, which, sols[k][2], sols[k][1])

    fds = oracle_map(run, jobs)
    done = 0
    for (k, which, i), fd in zip(jobs, fds):
        if fd is None:
            continue
        got = float(grs[k]) if which == "r" else float(grads[which][sl(k)][i])
        assert abs(fd - got) <= 1e-6 * (1 + abs(fd)), (k, which, i, fd, got)
        done += 1
    assert done >= 0.9 * len(jobs), (done, len(jobs))
