"""Autotuner for the batched entry points: times the library's batched launch for candidate
launch options on the caller's own batch and remembers the fastest per workload signature.

Tunables (all options of ``cqk_options``; the kernels are the same, only the work split
changes):
  group_elems   elements per block of an instance's group (how many blocks solve one instance)
  condat_chunk  minimum elements per chunk of the parallel Alg. 2 start (projections)
  warp_elems    instances shorter than this are solved by one warp each (projections)
  max_blocks    an upper bound on the persistent grid

The signature of a batch is (entry point, dtype, number of instances, log2 of the total
length, and the histogram of log2 instance lengths in four coarse bands), so batches with
the same shape reuse a tuning.  Timing uses CUDA events on the current stream after one
warm-up call per candidate; results of every candidate are valid solves.
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

from . import api

_cache: dict = {}
_lock = threading.Lock()

SIMPLEX_CANDIDATES = [
    dict(group_elems=ge, condat_chunk=cc, warp_elems=we)
    for ge in (1 << 16, 1 << 18, 1 << 20, (1 << 31) - 1)
    for cc in (512, 1 << 14)
    for we in (4096, 16384, 1 << 17)
]
GENERAL_CANDIDATES = [dict(group_elems=ge) for ge in (1 << 14, 1 << 15, 1 << 16, 1 << 17, 1 << 18)]


def signature(kind: str, dtype, offsets) -> tuple:
    """Workload signature of a batch (host-side; reads the offsets once)."""
    off = offsets.detach().to("cpu", torch.int64)
    lens = (off[1:] - off[:-1]).clamp(min=0).tolist()
    n = int(off[-1]) if off.numel() else 0
    bands = [0, 0, 0, 0]  # < 2^8, < 2^12, < 2^16, larger
    for m in lens:
        b = 0 if m < (1 << 8) else 1 if m < (1 << 12) else 2 if m < (1 << 16) else 3
        bands[b] += 1
    total = max(1, len(lens))
    shape = tuple(round(4 * c / total) for c in bands)  # quarters of the batch per band
    return (kind, str(dtype).replace("torch.", ""), len(lens), int(math.log2(max(n, 1))), shape)


def _time(fn, reps):
    fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def tune_batched(kind: str, *arrays, offsets, r, candidates=None, reps: int = 3, ws=None, **fixed):
    """Time `candidates` (option dicts) for one batched call and return (best_options, timings).

    kind: "simplex", "l1" or "general"; arrays: (y,) or (a, b, d, l, u) on the device."""
    if kind == "general":
        cands = candidates or GENERAL_CANDIDATES
        call = api.solve_batched
    else:
        cands = candidates or SIMPLEX_CANDIDATES
        call = api.project_simplex_batched if kind == "simplex" else api.project_l1_batched
    x = torch.empty_like(arrays[0])
    n = arrays[0].numel()
    B = offsets.numel() - 1
    ws = ws or api.Workspace(n, max(B, 1), arrays[0].dtype, arrays[0].device)
    timings = []
    for opt in cands:
        kw = dict(fixed)
        kw.update(opt)
        ms = _time(lambda: call(*arrays, offsets, r, out=x, ws=ws, sync=False, **kw), reps)
        timings.append((ms, opt))
    timings.sort(key=lambda t: t[0])
    best = dict(timings[0][1])
    with _lock:
        _cache[signature(kind, arrays[0].dtype, offsets)] = best
    return best, timings


def tuned_options(kind: str, dtype, offsets) -> dict | None:
    """The remembered best options for a batch of this signature, if any."""
    with _lock:
        return _cache.get(signature(kind, dtype, offsets))


def save(path: str) -> None:
    """Write the tuning cache as JSON (signature -> options)."""
    with _lock:
        items = [{"signature": list(k), "options": v} for k, v in _cache.items()]
    with open(path, "w") as f:
        json.dump(items, f, indent=1)


def load(path: str) -> int:
    """Merge a cache written by save(); returns the number of entries read."""
    if not os.path.exists(path):
        return 0
    with open(path) as f:
        items = json.load(f)
    with _lock:
        for it in items:
            sig = it["signature"]
            sig[4] = tuple(sig[4])
            _cache[tuple(sig)] = it["options"]
    return len(items)
