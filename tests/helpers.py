"""Shared helpers of the GPU parity tests (tolerances and comparisons)."""
import numpy as np
import torch

# Tolerances: FP64 form |x - x*|_inf <= 1e-10 (1 + |x*|_inf) and |b'x - r| <= 1e-12 sum |b_i x_i|;
# FP32-storage form: 1e-5 relative for both.
TOL_X = {torch.float64: 1e-10, torch.float32: 1e-5}
TOL_FEAS = {torch.float64: 1e-12, torch.float32: 1e-5}


def np64(t):
    return t.detach().double().cpu().numpy()


def assert_x_close(x, xstar, dtype, what=""):
    x, xstar = np.asarray(x, dtype=np.float64), np.asarray(xstar, dtype=np.float64)
    err = np.max(np.abs(x - xstar)) if x.size else 0.0
    bound = TOL_X[dtype] * (1 + (np.max(np.abs(xstar)) if xstar.size else 0.0))
    assert err <= bound, f"{what} |x - x*|_inf = {err:.3e} > {bound:.3e}"
    return err


def assert_feasible(x, b, r, dtype, what=""):
    x, b = np.asarray(x, dtype=np.float64), np.asarray(b, dtype=np.float64)
    bx = b * x
    res = abs(float(np.sum(bx, dtype=np.longdouble)) - r)
    scale = float(np.sum(np.abs(bx)))
    assert res <= TOL_FEAS[dtype] * max(scale, 1e-300), f"{what} |b'x - r| = {res:.3e} > {TOL_FEAS[dtype]:.0e} * {scale:.3e}"
    return res / max(scale, 1e-300)


def mask_bits(mask, n):
    m = mask.cpu().numpy().view(np.uint32)
    bits = np.unpackbits(m.view(np.uint8), bitorder="little")[:n]
    return bits.astype(bool)


def oracle_map(fn, items, workers=None):
    """[fn(item) for item in items], run on a thread pool: the C oracle's calls release the
    GIL (ctypes), so independent instances solve on all host cores."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    items = list(items)
    workers = workers or max(1, min(len(items), len(os.sched_getaffinity(0))))
    if workers == 1 or len(items) <= 1:
        return [fn(it) for it in items]
    with ThreadPoolExecutor(max_workers=workers) as pool:
        return list(pool.map(fn, items))


def rel_err_x(x, xstar):
    """max |x - x*| / (1 + max |x*|) (the norm of the x tolerance)."""
    x, xstar = np.asarray(x, dtype=np.float64), np.asarray(xstar, dtype=np.float64)
    if x.size == 0:
        return 0.0
    return float(np.max(np.abs(x - xstar))) / (1.0 + float(np.max(np.abs(xstar))))
