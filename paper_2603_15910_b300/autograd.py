"""Differentiable solves: ``torch.autograd.Function`` wrappers whose forward is the library's
solve (single or batched) and whose backward is the library's adjoint kernel
(cqk_backward*), reusing the forward's x, free mask and multiplier (the info buffer).

    x = cqk_solve(a, b, d, l, u, r)                       # gradients in a, b, d, l, u, r
    x = simplex_projection(y, r)                          # gradients in y, r
    x = l1_projection(y, r)
    x = simplex_projection(y, r, offsets=off)             # ragged batch; r has one entry per instance

Nothing runs on the CPU: the forward and backward are kernels of libcqk.

Failures: with check=True (the default) the forward synchronises once to read the status of
every instance and raises ``CQKSolveError`` unless all are CQK_OK, and the backward does the
same for the adjoint's status (CQK_NONDIFF is accepted: its gradients are the documented
mu = 0 values).  check=False issues no host synchronisation and reports nothing; the status
words are then only in the library's info buffers.
"""
from __future__ import annotations

import torch

from . import api

# byte offset of cqk_info.status (int32) in one 72-byte cqk_info
_STATUS_OFF = 52


class CQKSolveError(RuntimeError):
    pass


def _check_forward(info, B, what):
    st = info[: B * api.INFO_BYTES].view(B, api.INFO_BYTES)[:, _STATUS_OFF:_STATUS_OFF + 4].contiguous()
    st = st.view(torch.int32).flatten().cpu()
    bad = torch.nonzero(st != api.Status.OK).flatten().tolist()
    if bad:
        k = bad[0]
        raise CQKSolveError(f"{what}: instance {k} ended with status {api.Status(int(st[k])).name} "
                            f"({len(bad)} of {B} instances not OK)")


def _check_backward(status, what):
    st = status.cpu()
    bad = torch.nonzero((st != api.Status.OK) & (st != api.Status.NONDIFF)).flatten().tolist()
    if bad:
        k = bad[0]
        raise CQKSolveError(f"{what} adjoint: instance {k} ended with status {api.Status(int(st[k])).name}")


def _r_tensor(r, B, device):
    if torch.is_tensor(r):
        return r
    return torch.full((B,), float(r), dtype=torch.float64, device=device) if B > 1 else torch.tensor(float(r),
                                                                                                      dtype=torch.float64)


def _r_grad(gr, r):
    """Per-instance dr (float64, device) shaped and typed like r."""
    if r.dim() == 0:
        g = gr[0].reshape(())
    else:
        g = gr[: r.numel()].reshape(r.shape)
    return g.to(device=r.device, dtype=r.dtype)


def _forward_info(n, B, dtype, device):
    ws = api.Workspace(n, max(B, 1), dtype, device)
    return ws


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a, b, d, l, u, r, offsets, check, opts):
        B = 1 if offsets is None else offsets.numel() - 1
        ws = _forward_info(a.numel(), B, a.dtype, a.device)
        if offsets is None:
            x, _, mask = api.solve(a, b, d, l, u, float(r), want_mask=True, ws=ws, sync=False, **opts)
        else:
            x, _, mask = api.solve_batched(a, b, d, l, u, offsets, r.to(a.device), want_mask=True, ws=ws,
                                           sync=False, **opts)
        if check:
            _check_forward(ws.info, max(B, 1), "cqk_solve")
        ctx.ws = ws
        ctx.check = check
        ctx.save_for_backward(a, b, d, l, u, r, x, mask, ws.info, offsets if offsets is not None else a.new_empty(0))
        ctx.batched = offsets is not None
        return x

    @staticmethod
    def backward(ctx, gx):
        a, b, d, l, u, r, x, mask, info, offsets = ctx.saved_tensors
        want = tuple(k for k, need in zip("abdlu", ctx.needs_input_grad[:5]) if need)
        out = api.backward("general", gx.contiguous(), x, info, a=a, b=b, d=d, l=l, u=u, mask=mask,
                           offsets=offsets if ctx.batched else None, want=want, ws=ctx.ws)
        if ctx.check:
            _check_backward(out["status"], "cqk_solve")
        gr = _r_grad(out["r"], r) if ctx.needs_input_grad[5] else None
        return out.get("a"), out.get("b"), out.get("d"), out.get("l"), out.get("u"), gr, None, None, None


class _Project(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, r, offsets, l1, check, opts):
        B = 1 if offsets is None else offsets.numel() - 1
        ws = _forward_info(y.numel(), B, y.dtype, y.device)
        if offsets is None:
            fn = api.project_l1 if l1 else api.project_simplex
            x, _, mask = fn(y, float(r), want_mask=True, ws=ws, sync=False, **opts)
        else:
            fn = api.project_l1_batched if l1 else api.project_simplex_batched
            x, _, mask = fn(y, offsets, r.to(y.device), want_mask=True, ws=ws, sync=False, **opts)
        if check:
            _check_forward(ws.info, max(B, 1), "l1 projection" if l1 else "simplex projection")
        ctx.ws = ws
        ctx.check = check
        ctx.l1 = l1
        ctx.batched = offsets is not None
        ctx.save_for_backward(r, x, mask, ws.info, offsets if offsets is not None else y.new_empty(0))
        return x

    @staticmethod
    def backward(ctx, gx):
        r, x, mask, info, offsets = ctx.saved_tensors
        out = api.backward("l1" if ctx.l1 else "simplex", gx.contiguous(), x, info, mask=mask,
                           offsets=offsets if ctx.batched else None, ws=ctx.ws)
        if ctx.check:
            _check_backward(out["status"], "l1 projection" if ctx.l1 else "simplex projection")
        gr = _r_grad(out["r"], r) if ctx.needs_input_grad[1] else None
        return out["y"], gr, None, None, None, None


def cqk_solve(a, b, d, l, u, r, offsets=None, check=True, **opts):
    """x*(a, b, d, l, u, r) of (CQK), differentiable in every argument.  With offsets (device
    int64, B + 1 entries) the arrays hold B instances and r has B entries."""
    B = 1 if offsets is None else offsets.numel() - 1
    return _Solve.apply(a, b, d, l, u, _r_tensor(r, B, a.device), offsets, check, opts)


def simplex_projection(y, r=1.0, offsets=None, check=True, **opts):
    """Projection onto {x >= 0, sum x = r}, differentiable in y and r."""
    B = 1 if offsets is None else offsets.numel() - 1
    return _Project.apply(y, _r_tensor(r, B, y.device), offsets, False, check, opts)


def l1_projection(y, r=1.0, offsets=None, check=True, **opts):
    """Projection onto {sum |x_i| <= r}, differentiable in y and r."""
    B = 1 if offsets is None else offsets.numel() - 1
    return _Project.apply(y, _r_tensor(r, B, y.device), offsets, True, check, opts)
