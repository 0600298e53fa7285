"""Seeded synthetic inputs for the CQK solver (no solver arithmetic here).

This module only draws random arrays.  It is the one module that both the CUDA
path's tests/benchmarks and the FP64 oracle consume; neither the oracle nor the
CUDA library imports the other.

Recipes (problem shapes of the paper's test families, Sec. 5.1.1 and 5.2.1):

* ``uncorrelated_box``  d~U[1,100], b~U[10,25], a~U[-10,10], l~U[-5,0],
  u = l + U[0.5,5], r = b'(l+u)/2 (always feasible, strictly inside).
* ``correlated``        b~U[10,25], d = b*U[0.5,1.5], a = b + U[-5,5],
  l~U[1,15], u~U[l, l+15], r = b'(l+u)/2.
* ``simplex_normal``    y~N(0,1); sparse variant y~N(0,1) + 10*Bernoulli(0.01).
* ``paper_family``      the paper's general families: uncorrelated d,a,b~U[10,25];
  weakly correlated b~U[10,25], d,a~U[b-5,b+5]; correlated b~U[10,25],
  d = a = b+5; l,u = min/max of two U[10,25] draws; r~U[b'l, b'u].
* ``paper_simplex``     y~U(0,1), N(0,1) or N(0, sigma=1e-3).
* ``ragged_lengths``    lengths round(exp(U[ln lo, ln hi])) for batches.

All draws use a torch.Generator seeded with ``seed`` on ``device``; the same
(seed, device) always gives the same arrays.  Arrays are drawn in float64 and
cast to ``dtype`` afterwards; r is computed in float64 from the stored (cast)
arrays so that it is exact data for the FP32-storage form too.
"""
from __future__ import annotations

import math

import torch


def _gen(seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _u(g, n, lo, hi, device):
    return torch.rand(n, generator=g, device=device, dtype=torch.float64) * (hi - lo) + lo


def _bdot(b, v):
    # in pieces of 2^30 (the library dot product takes at most 2^31 - 1 elements); one piece,
    # the same value as a single dot, for every smaller array
    step = 1 << 30
    return float(sum(torch.dot(b[i:i + step].double(), v[i:i + step].double()).item()
                     for i in range(0, max(b.numel(), 1), step)))


def uncorrelated_box(n, seed=0, device="cpu", dtype=torch.float64):
    """General CQK, uncorrelated box family.  Returns dict(a, b, d, l, u, r)."""
    g = _gen(seed, device)
    d = _u(g, n, 1.0, 100.0, device)
    b = _u(g, n, 10.0, 25.0, device)
    a = _u(g, n, -10.0, 10.0, device)
    l = _u(g, n, -5.0, 0.0, device)
    u = l + _u(g, n, 0.5, 5.0, device)
    a, b, d, l, u = (v.to(dtype) for v in (a, b, d, l, u))
    r = _bdot(b, l.double() + u.double()) / 2.0
    return dict(a=a, b=b, d=d, l=l, u=u, r=r)


def correlated(n, seed=0, device="cpu", dtype=torch.float64):
    """General CQK, correlated family.  Returns dict(a, b, d, l, u, r)."""
    g = _gen(seed, device)
    b = _u(g, n, 10.0, 25.0, device)
    d = b * _u(g, n, 0.5, 1.5, device)
    a = b + _u(g, n, -5.0, 5.0, device)
    l = _u(g, n, 1.0, 15.0, device)
    u = l + _u(g, n, 0.0, 15.0, device)
    a, b, d, l, u = (v.to(dtype) for v in (a, b, d, l, u))
    r = _bdot(b, l.double() + u.double()) / 2.0
    return dict(a=a, b=b, d=d, l=l, u=u, r=r)


def simplex_normal(n, seed=0, sparse=False, device="cpu", dtype=torch.float64):
    """y~N(0,1), or N(0,1) + 10*Bernoulli(0.01) when sparse."""
    g = _gen(seed, device)
    y = torch.randn(n, generator=g, device=device, dtype=torch.float64)
    if sparse:
        y = y + 10.0 * (torch.rand(n, generator=g, device=device, dtype=torch.float64) < 0.01).double()
    return y.to(dtype)


def paper_family(kind, n, seed=0, device="cpu", dtype=torch.float64):
    """The paper's general families ('uncorrelated', 'weak', 'correlated')."""
    g = _gen(seed, device)
    b = _u(g, n, 10.0, 25.0, device)
    if kind == "uncorrelated":
        d = _u(g, n, 10.0, 25.0, device)
        a = _u(g, n, 10.0, 25.0, device)
    elif kind == "weak":
        d = b + _u(g, n, -5.0, 5.0, device)
        a = b + _u(g, n, -5.0, 5.0, device)
    elif kind == "correlated":
        d = b + 5.0
        a = b + 5.0
    else:
        raise ValueError(kind)
    p = _u(g, n, 10.0, 25.0, device)
    q = _u(g, n, 10.0, 25.0, device)
    l, u = torch.minimum(p, q), torch.maximum(p, q)
    a, b, d, l, u = (v.to(dtype) for v in (a, b, d, l, u))
    lo, hi = _bdot(b, l), _bdot(b, u)
    t = float(torch.rand(1, generator=g, device=device, dtype=torch.float64).item())
    r = lo + t * (hi - lo)
    return dict(a=a, b=b, d=d, l=l, u=u, r=r)


def paper_simplex(kind, n, seed=0, device="cpu", dtype=torch.float64):
    """The paper's simplex families: 'uniform' U(0,1), 'normal' N(0,1), 'narrow' N(0, 1e-3)."""
    g = _gen(seed, device)
    if kind == "uniform":
        y = torch.rand(n, generator=g, device=device, dtype=torch.float64)
    elif kind == "normal":
        y = torch.randn(n, generator=g, device=device, dtype=torch.float64)
    elif kind == "narrow":
        y = 1e-3 * torch.randn(n, generator=g, device=device, dtype=torch.float64)
    else:
        raise ValueError(kind)
    return y.to(dtype)


def ragged_lengths(batch, lo, hi, seed=0):
    """Lengths round(exp(U[ln lo, ln hi])) (log-uniform), on the CPU, as a list of ints."""
    g = _gen(seed, "cpu")
    t = torch.rand(batch, generator=g, dtype=torch.float64)
    v = torch.exp(t * (math.log(hi) - math.log(lo)) + math.log(lo))
    return [int(max(lo, min(hi, round(float(x))))) for x in v]


def offsets_of(lengths):
    """CSR offsets [0, len0, len0+len1, ...] as a CPU int64 tensor."""
    off = torch.zeros(len(lengths) + 1, dtype=torch.int64)
    off[1:] = torch.cumsum(torch.tensor(lengths, dtype=torch.int64), 0)
    return off


def batched_simplex(batch=4096, lo=16, hi=1 << 20, seed=0, device="cpu", dtype=torch.float32):
    """Ragged batch of simplex projections: lengths log-uniform in [lo, hi], y~N(0,1),
    r = 1 for every instance, upstream gradient g~N(0,1).  Returns dict(y, offsets, r, g)."""
    lengths = ragged_lengths(batch, lo, hi, seed)
    off = offsets_of(lengths)
    n = int(off[-1])
    gen = _gen(seed + 1, device)
    y = torch.randn(n, generator=gen, device=device, dtype=torch.float64).to(dtype)
    g = torch.randn(n, generator=gen, device=device, dtype=torch.float64).to(dtype)
    r = torch.ones(batch, dtype=torch.float64, device=device)
    return dict(y=y, offsets=off.to(device), r=r, g=g, lengths=lengths)


def batched_general(batch=256, lo=1000, hi=1000000, seed=0, device="cpu", dtype=torch.float64):
    """Ragged batch of general CQK instances (uncorrelated box recipe), instance i
    drawn with seed 1000+i; lengths log-uniform in [lo, hi].  Returns dict of
    concatenated a, b, d, l, u, offsets, per-instance r, and g~N(0,1)."""
    lengths = ragged_lengths(batch, lo, hi, seed)
    parts = [uncorrelated_box(m, seed=1000 + i, device=device, dtype=dtype) for i, m in enumerate(lengths)]
    cat = {k: torch.cat([p[k] for p in parts]) for k in ("a", "b", "d", "l", "u")}
    cat["r"] = torch.tensor([p["r"] for p in parts], dtype=torch.float64, device=device)
    cat["offsets"] = offsets_of(lengths).to(device)
    gen = _gen(seed + 7, device)
    cat["g"] = torch.randn(int(sum(lengths)), generator=gen, device=device, dtype=torch.float64).to(dtype)
    cat["lengths"] = lengths
    return cat
