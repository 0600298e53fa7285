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


@pytest.mark.gpu
def test_tuning_run_picks_valid_options():
    import oracle
    from paper_2603_15910_b300 import api, workloads as W
    d = W.batched_simplex(batch=96, lo=16, hi=1 << 17, seed=4, device="cuda", dtype=torch.float64)
    best, timings = tune.tune_batched("simplex", d["y"], offsets=d["offsets"], r=d["r"], reps=1)
    assert len(timings) == len(tune.SIMPLEX_CANDIDATES) and best == timings[0][1]
    assert tune.tuned_options("simplex", torch.float64, d["offsets"]) == best
    x, infos, _ = api.project_simplex_batched(d["y"], d["offsets"], d["r"], **best)
    off = d["offsets"].cpu().numpy()
    ys, xs = d["y"].cpu().numpy(), x.cpu().numpy()
    for k in range(0, 96, 11):
        lo, hi = int(off[k]), int(off[k + 1])
        lam, xstar = oracle.project_simplex_sort(ys[lo:hi], 1.0)
        assert np.max(np.abs(xs[lo:hi] - xstar)) <= 1e-10 * (1 + np.max(np.abs(xstar)))
    g = W.batched_general(batch=12, lo=1000, hi=50000, seed=1, device="cuda")
    best, timings = tune.tune_batched("general", g["a"], g["b"], g["d"], g["l"], g["u"], offsets=g["offsets"],
                                      r=g["r"], reps=1)
    assert best in tune.GENERAL_CANDIDATES
