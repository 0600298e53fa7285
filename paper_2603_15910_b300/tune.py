"""Autotuner for the batched entry points: times the library's batched launches for candidate
launch options on the caller's own batch and remembers the fastest per workload signature.

Tunables (all fields of ``cqk_options``; every candidate solves the same problems, only the
work split and the kernel build change):
  group_elems    elements per block of an instance's group: how many blocks solve one instance
                 (the split between one block and a multi-block group per instance)
  warp_elems     instances shorter than this are solved by one warp each (projections; the
                 split between segment-per-warp and segment-per-block)
  condat_chunk   minimum elements per chunk of the parallel Alg. 2 start (projections)
  scan_warps     chunks (scan warps) per block of the Alg. 2 start (projections)
  block_threads  threads per block of the persistent kernel: 128, 256 or 512 (general batches
                 and the adjoints; the projection forward runs 256)
  unroll         elements per thread: 0 = the full per-lane unroll of the streaming loops, 1 =
                 half of it (256 threads)

The forward and the adjoint are tuned separately (kinds "simplex", "l1", "general" and
"simplex_bwd", "l1_bwd", "general_bwd"); ``tune_fwd_bwd`` does both.  The signature of a batch
is (kind, dtype, number of instances, log2 of the total length, and the histogram of log2
instance lengths in four coarse bands), so batches of the same shape reuse a tuning, and the
batched calls of ``api`` apply a remembered tuning automatically (see ``api.solve_batched``).
Timing uses CUDA events on the current stream after one warm-up call per candidate.
"""
from __future__ import annotations

import itertools
import json
import math
import os
import threading

import torch

from . import api

_cache: dict = {}
_lock = threading.Lock()

# (block_threads, unroll) builds of the batched kernels
BUILDS_ALL = [dict(block_threads=256, unroll=0), dict(block_threads=128, unroll=0),
              dict(block_threads=512, unroll=0), dict(block_threads=256, unroll=1)]
BUILDS_PROJECTION_FORWARD = [dict(block_threads=256, unroll=0), dict(block_threads=256, unroll=1)]


def _grid(**axes):
    keys = list(axes)
    out = []
    for vals in itertools.product(*(axes[k] for k in keys)):
        d = {}
        for k, v in zip(keys, vals):
            if isinstance(v, dict):
                d.update(v)
            else:
                d[k] = v
        out.append(d)
    return out


SIMPLEX_CANDIDATES = _grid(group_elems=(1 << 16, 1 << 18, 1 << 20, (1 << 31) - 1), condat_chunk=(512, 1 << 14),
                           warp_elems=(4096, 16384, 1 << 17), scan_warps=(1, 4), build=BUILDS_PROJECTION_FORWARD)
GENERAL_CANDIDATES = _grid(group_elems=(1 << 14, 1 << 15, 1 << 16, 1 << 17, 1 << 18), build=BUILDS_ALL)
SIMPLEX_BWD_CANDIDATES = _grid(group_elems=(1 << 16, 1 << 18, 1 << 20), warp_elems=(4096, 16384, 1 << 17),
                               build=BUILDS_ALL)
GENERAL_BWD_CANDIDATES = _grid(group_elems=(1 << 13, 1 << 14, 1 << 15, 1 << 16, 1 << 17), build=BUILDS_ALL)

TUNABLE_KEYS = ("group_elems", "warp_elems", "condat_chunk", "scan_warps", "block_threads", "unroll", "max_blocks")


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


def _remember(kind, dtype, offsets, best):
    with _lock:
        _cache[signature(kind, dtype, offsets)] = dict(best)


def tune_batched(kind: str, *arrays, offsets, r, candidates=None, reps: int = 3, ws=None, **fixed):
    """Time `candidates` (option dicts) for one batched forward call and return
    (best_options, timings sorted fastest first).

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
        ms = _time(lambda: call(*arrays, offsets, r, out=x, ws=ws, sync=False, use_tuning=False, **kw), reps)
        timings.append((ms, opt))
    timings.sort(key=lambda t: t[0])
    best = dict(timings[0][1])
    _remember(kind, arrays[0].dtype, offsets, best)
    return best, timings


def tune_backward(kind: str, g, x, info, *, offsets, arrays=(), mask=None, candidates=None, reps: int = 3, ws=None,
                  **fixed):
    """Time `candidates` for the batched adjoint (cqk_backward*, after the forward whose x, mask
    and info buffer are given) and return (best_options, timings).  kind: "simplex", "l1" or
    "general" (arrays = (a, b, d, l, u) for "general")."""
    cands = candidates or (GENERAL_BWD_CANDIDATES if kind == "general" else SIMPLEX_BWD_CANDIDATES)
    B = offsets.numel() - 1
    ws = ws or api.Workspace(x.numel(), max(B, 1), x.dtype, x.device)
    extra = dict(zip("abdlu", arrays)) if kind == "general" else {}
    timings = []
    for opt in cands:
        kw = dict(fixed)
        kw.update(opt)
        ms = _time(lambda: api.backward(kind, g, x, info, offsets=offsets, mask=mask, ws=ws, use_tuning=False,
                                        **extra, **kw), reps)
        timings.append((ms, opt))
    timings.sort(key=lambda t: t[0])
    best = dict(timings[0][1])
    _remember(kind + "_bwd", x.dtype, offsets, best)
    return best, timings


def tune_fwd_bwd(kind: str, *arrays, offsets, r, g, reps: int = 3):
    """Tune the forward, run it once with the chosen options (keeping x, the mask and the info
    buffer), then tune the adjoint on that forward.  Returns (forward options, adjoint options,
    forward timings, adjoint timings)."""
    fwd, t_fwd = tune_batched(kind, *arrays, offsets=offsets, r=r, reps=reps)
    n = arrays[0].numel()
    B = offsets.numel() - 1
    ws = api.Workspace(n, max(B, 1), arrays[0].dtype, arrays[0].device)
    if kind == "general":
        x, _, mask = api.solve_batched(*arrays, offsets, r, want_mask=True, ws=ws, sync=False, use_tuning=False,
                                       **fwd)
    else:
        call = api.project_simplex_batched if kind == "simplex" else api.project_l1_batched
        x, _, mask = call(*arrays, offsets, r, want_mask=True, ws=ws, sync=False, use_tuning=False, **fwd)
    bwd, t_bwd = tune_backward(kind, g, x, ws.info, offsets=offsets, arrays=arrays, mask=mask, reps=reps)
    return fwd, bwd, t_fwd, t_bwd


def tuned_options(kind: str, dtype, offsets) -> dict | None:
    """The remembered best options for a batch of this signature, if any."""
    with _lock:
        if not _cache:
            return None
        return _cache.get(signature(kind, dtype, offsets))


def has_tunings() -> bool:
    with _lock:
        return bool(_cache)


def clear() -> None:
    with _lock:
        _cache.clear()


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
