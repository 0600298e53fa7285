"""The autotuner: workload signatures and the cache (CPU), and a tuning run on the GPU whose
chosen options still solve the batch exactly."""
import os
import tempfile

import numpy as np
import pytest
import torch

from paper_2603_15910_b300 import tune


def _off(lens):
    return torch.tensor(np.concatenate([[0], np.cumsum(lens)]), dtype=torch.int64)


def test_signature_groups_batches_of_the_same_shape():
    a = tune.signature("simplex", torch.float32, _off([10, 300, 5000, 70000]))
    b = tune.signature("simplex", torch.float32, _off([12, 290, 5100, 69000]))
    c = tune.signature("simplex", torch.float64, _off([10, 300, 5000, 70000]))
    d = tune.signature("simplex", torch.float32, _off([70000] * 4))
    assert a == b and a != c and a != d
    assert a[2] == 4


def test_cache_round_trip():
    sig_off = _off([100, 200])
    with tune._lock:
        tune._cache[tune.signature("l1", torch.float64, sig_off)] = {"group_elems": 4096}
    with tempfile.TemporaryDirectory() as td:
        p = os.path.join(td, "tune.json")
        tune.save(p)
        with tune._lock:
            tune._cache.clear()
        assert tune.tuned_options("l1", torch.float64, sig_off) is None
        assert tune.load(p) >= 1
    assert tune.tuned_options("l1", torch.float64, sig_off) == {"group_elems": 4096}


def test_batched_calls_apply_a_remembered_tuning():
    from paper_2603_15910_b300 import api
    off = _off([100, 2000, 30])
    tune.clear()
    assert api._with_tuning("simplex", torch.float32, off, {}, True) == {}
    with tune._lock:
        tune._cache[tune.signature("simplex", torch.float32, off)] = {"group_elems": 4096, "unroll": 1}
    try:
        assert api._with_tuning("simplex", torch.float32, off, {}, True) == {"group_elems": 4096, "unroll": 1}
        # options the caller sets win; use_tuning=False and another shape look nothing up
        assert api._with_tuning("simplex", torch.float32, off, {"warp_elems": 64}, True) == {"warp_elems": 64}
        assert api._with_tuning("simplex", torch.float32, off, {}, False) == {}
        assert api._with_tuning("simplex_bwd", torch.float32, off, {}, True) == {}
    finally:
        tune.clear()


def test_candidates_cover_block_size_and_unroll():
    for cands in (tune.GENERAL_CANDIDATES, tune.SIMPLEX_BWD_CANDIDATES, tune.GENERAL_BWD_CANDIDATES):
        builds = {(c["block_threads"], c["unroll"]) for c in cands}
        assert builds == {(256, 0), (128, 0), (512, 0), (256, 1)}
    assert {(c["block_threads"], c["unroll"]) for c in tune.SIMPLEX_CANDIDATES} == {(256, 0), (256, 1)}
    assert {c["warp_elems"] for c in tune.SIMPLEX_CANDIDATES} == {4096, 16384, 1 << 17}


@pytest.mark.gpu
def test_tuning_run_picks_valid_options():
    """Tune a ragged batch (forward and adjoint), then solve it with the chosen options through
    the ordinary batched calls (which pick up the remembered tuning) and check every instance
    against the oracle."""
    import oracle
    from paper_2603_15910_b300 import api, workloads as W
    tune.clear()
    try:
        d = W.batched_simplex(batch=96, lo=16, hi=1 << 17, seed=4, device="cuda", dtype=torch.float64)
        fwd, bwd, t_f, t_b = tune.tune_fwd_bwd("simplex", d["y"], offsets=d["offsets"], r=d["r"], g=d["g"], reps=1)
        assert len(t_f) == len(tune.SIMPLEX_CANDIDATES) and fwd == t_f[0][1]
        assert len(t_b) == len(tune.SIMPLEX_BWD_CANDIDATES) and bwd == t_b[0][1]
        assert tune.tuned_options("simplex", torch.float64, d["offsets"]) == fwd
        assert tune.tuned_options("simplex_bwd", torch.float64, d["offsets"]) == bwd
        ws = api.Workspace(d["y"].numel(), 96, torch.float64)
        x, infos, mask = api.project_simplex_batched(d["y"], d["offsets"], d["r"], want_mask=True, ws=ws)
        out = api.backward("simplex", d["g"], x, ws.info, offsets=d["offsets"], mask=mask)
        off = d["offsets"].cpu().numpy()
        ys, xs, gs, gy = d["y"].cpu().numpy(), x.cpu().numpy(), d["g"].cpu().numpy(), out["y"].cpu().numpy()
        for k in range(96):
            lo, hi = int(off[k]), int(off[k + 1])
            lam, xstar = oracle.project_simplex_sort(ys[lo:hi], 1.0)
            assert np.max(np.abs(xs[lo:hi] - xstar)) <= 1e-10 * (1 + np.max(np.abs(xstar)))
            ref = oracle.grad_simplex(xstar, gs[lo:hi])
            assert np.max(np.abs(gy[lo:hi] - ref["y"])) <= 1e-10 * (1 + np.max(np.abs(ref["y"])))
        g = W.batched_general(batch=12, lo=1000, hi=50000, seed=1, device="cuda")
        arrays = tuple(g[k] for k in "abdlu")
        fwd, bwd, _, _ = tune.tune_fwd_bwd("general", *arrays, offsets=g["offsets"], r=g["r"], g=g["g"], reps=1)
        assert fwd in tune.GENERAL_CANDIDATES and bwd in tune.GENERAL_BWD_CANDIDATES
        x, infos, _ = api.solve_batched(*arrays, g["offsets"], g["r"])
        off = g["offsets"].cpu().numpy()
        for k in range(12):
            lo, hi = int(off[k]), int(off[k + 1])
            host = [g[q][lo:hi].cpu().numpy() for q in "abdlu"]
            st, lam, xstar = oracle.solve_sort(*host, float(g["r"][k]))
            assert np.max(np.abs(x[lo:hi].cpu().numpy() - xstar)) <= 1e-10 * (1 + np.max(np.abs(xstar)))
    finally:
        tune.clear()
