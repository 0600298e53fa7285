"""ctypes binding of libcqk (include/cqk.h).  Argument marshalling only: every step of the
solve runs in the library's CUDA kernels; torch provides device memory and streams.

There is no CPU fallback: if libcqk.so is missing or no CUDA device is present, the calls
raise ``CQKLibraryError``.
"""
from __future__ import annotations

import ctypes
import enum
import os
import threading
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libcqk.so")
_lock = threading.Lock()
_lib = None


class CQKLibraryError(RuntimeError):
    pass


class Status(enum.IntEnum):
    OK = 0
    INFEASIBLE = 1
    MAXITER = 2
    BAD_INPUT = 3
    NONDIFF = 4
    TIMEOUT = 5
    CUDA_ERROR = 6
    BAD_ARG = 7


class Init(enum.IntEnum):
    FORMULA = 0
    CONDAT = 1
    WARM = 2
    GIVEN = 3


STOP_NAMES = {0: "none", 1: "exact", 2: "residual", 3: "step", 4: "same", 5: "bracket", 6: "below", 7: "inside"}


class _Options(ctypes.Structure):
    _fields_ = [
        ("max_iter", ctypes.c_int32),
        ("init", ctypes.c_int32),
        ("lambda0", ctypes.c_double),
        ("validate", ctypes.c_int32),
        ("final_step", ctypes.c_int32),
        ("spin_limit_us", ctypes.c_int64),
        ("max_blocks", ctypes.c_int32),
        ("fault_inject", ctypes.c_int32),
        ("group_elems", ctypes.c_int32),
        ("condat_chunk", ctypes.c_int32),
        ("xbar", ctypes.c_void_p),
        ("warp_elems", ctypes.c_int32),
        ("scan_warps", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
        ("unroll", ctypes.c_int32),
    ]


class _Info(ctypes.Structure):
    _fields_ = [
        ("lambda_", ctypes.c_double),
        ("residual", ctypes.c_double),
        ("abs_bx", ctypes.c_double),
        ("slope", ctypes.c_double),
        ("lambda0", ctypes.c_double),
        ("nfree", ctypes.c_int64),
        ("iters", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("passes", ctypes.c_int32),
        ("stop", ctypes.c_int32),
        ("nchunks", ctypes.c_int32),
        ("tile", ctypes.c_int32),
    ]


INFO_BYTES = ctypes.sizeof(_Info)


@dataclass
class Info:
    """Outcome of one solve (cqk_info)."""
    lam: float
    residual: float
    abs_bx: float
    slope: float
    lambda0: float
    nfree: int
    iters: int
    status: Status
    passes: int
    stop: str
    nchunks: int
    tile: int

    @staticmethod
    def from_bytes(buf: bytes) -> "Info":
        s = _Info.from_buffer_copy(buf)
        st = Status(s.status) if s.status in Status._value2member_map_ else s.status
        return Info(s.lambda_, s.residual, s.abs_bx, s.slope, s.lambda0, s.nfree, s.iters, st, s.passes,
                    STOP_NAMES.get(s.stop, str(s.stop)), s.nchunks, s.tile)


def lib_path() -> str:
    return _LIB_PATH


def library():
    """Load libcqk.so (once).  Raises CQKLibraryError if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise CQKLibraryError(f"libcqk.so not built ({_LIB_PATH}); run python -m paper_2603_15910_b300.build_lib")
        lib = ctypes.CDLL(_LIB_PATH)
        vp, i64, i32, dbl, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_size_t
        lib.cqk_default_options.argtypes = [ctypes.POINTER(_Options)]
        lib.cqk_default_options.restype = None
        lib.cqk_workspace_bytes.argtypes = [i64, i32, i32]
        lib.cqk_workspace_bytes.restype = sz
        lib.cqk_solve.argtypes = [i64, i32, vp, vp, vp, vp, vp, dbl, vp, vp, vp, ctypes.POINTER(_Options), vp, sz, vp]
        lib.cqk_solve.restype = ctypes.c_int
        lib.cqk_phi.argtypes = [i64, i32, vp, vp, vp, vp, vp, dbl, vp, vp, vp, sz, vp]
        lib.cqk_phi.restype = ctypes.c_int
        for name in ("cqk_project_simplex", "cqk_project_l1"):
            f = getattr(lib, name)
            f.argtypes = [i64, i32, vp, dbl, vp, vp, vp, ctypes.POINTER(_Options), vp, sz, vp]
            f.restype = ctypes.c_int
        lib.cqk_solve_batched.argtypes = [i32, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.POINTER(_Options),
                                          vp, sz, vp]
        lib.cqk_solve_batched.restype = ctypes.c_int
        for name in ("cqk_project_simplex_batched", "cqk_project_l1_batched"):
            f = getattr(lib, name)
            f.argtypes = [i32, vp, i32, vp, vp, vp, vp, vp, ctypes.POINTER(_Options), vp, sz, vp]
            f.restype = ctypes.c_int
        lib.cqk_backward.argtypes = [i32, vp, i64, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                     ctypes.POINTER(_Options), vp, sz, vp]
        lib.cqk_backward.restype = ctypes.c_int
        for name in ("cqk_backward_simplex", "cqk_backward_l1"):
            f = getattr(lib, name)
            f.argtypes = [i32, vp, i64, i32, vp, vp, vp, vp, vp, vp, vp, ctypes.POINTER(_Options), vp, sz, vp]
            f.restype = ctypes.c_int
        lib.cqk_status_string.argtypes = [ctypes.c_int]
        lib.cqk_status_string.restype = ctypes.c_char_p
        lib.cqk_last_cuda_error.argtypes = []
        lib.cqk_last_cuda_error.restype = ctypes.c_int
        lib.cqk_version.argtypes = []
        lib.cqk_version.restype = ctypes.c_int
        _lib = lib
        return lib


def dtype_code(dtype) -> int:
    if dtype == torch.float64:
        return 0
    if dtype == torch.float32:
        return 1
    raise TypeError(f"unsupported dtype {dtype}; use float64 or float32")


def _check_device(*ts):
    if not torch.cuda.is_available():
        raise CQKLibraryError("no CUDA device: libcqk has no CPU path")
    dev = ts[0].device
    for t in ts:
        if t.device.type != "cuda" or t.device != dev:
            raise ValueError("all arrays must be on the same CUDA device")
        if not t.is_contiguous():
            raise ValueError("arrays must be contiguous")


def ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def stream_handle(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_options(init=None, max_iter=100, lambda0=0.0, validate=True, final_step=None, spin_limit_us=2_000_000,
                 max_blocks=0, fault_inject=False, group_elems=0, condat_chunk=0, xbar=None,
                 warp_elems=0, scan_warps=0, block_threads=0, unroll=0) -> _Options:
    o = _Options()
    library().cqk_default_options(ctypes.byref(o))
    o.max_iter = int(max_iter)
    o.init = -1 if init is None else int(init)
    o.lambda0 = float(lambda0)
    o.validate = 1 if validate else 0
    if final_step is not None:
        o.final_step = 1 if final_step else 0
    o.spin_limit_us = int(spin_limit_us)
    o.max_blocks = int(max_blocks)
    o.fault_inject = int(fault_inject)  # testing only: True / 1 device-wide waits, 2 the Alg. 2 scan queue
    o.group_elems = int(group_elems)
    o.condat_chunk = int(condat_chunk)
    o.xbar = xbar.data_ptr() if xbar is not None else None
    o.warp_elems = int(warp_elems)
    o.scan_warps = int(scan_warps)
    o.block_threads = int(block_threads)
    o.unroll = int(unroll)
    return o


_TUNABLE = ("group_elems", "warp_elems", "condat_chunk", "scan_warps", "block_threads", "unroll", "max_blocks")


def _with_tuning(kind, dtype, offsets, kw, use_tuning):
    """The launch options of a batched call: the caller's, or -- when the caller sets none of the
    work-split options and the autotuner (tune.py) has a tuning for a batch of this signature --
    the tuned ones.  Looking a tuning up reads the offsets on the host (one synchronisation);
    nothing is looked up while no tuning exists."""
    if not use_tuning or any(k in kw for k in _TUNABLE):
        return kw
    from . import tune
    if not tune.has_tunings():
        return kw
    best = tune.tuned_options(kind, dtype, offsets)
    if best:
        kw = dict(kw)
        kw.update(best)
    return kw


class Workspace:
    """A reusable device workspace and info buffer for repeated calls on one stream."""

    def __init__(self, n_total: int, batch: int = 1, dtype=torch.float64, device=None):
        lib = library()
        self.nbytes = int(lib.cqk_workspace_bytes(int(n_total), int(batch), dtype_code(dtype)))
        if self.nbytes == 0:
            raise ValueError("invalid workspace request")
        device = device or torch.device("cuda", torch.cuda.current_device())
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        self.info = torch.zeros(INFO_BYTES * max(1, batch), dtype=torch.uint8, device=device)

    def read_info(self, i: int = 0) -> Info:
        raw = self.info[i * INFO_BYTES:(i + 1) * INFO_BYTES].cpu().numpy().tobytes()
        return Info.from_bytes(raw)

    def read_infos(self, count: int) -> list:
        """The first `count` infos, in one device-to-host copy."""
        raw = self.info[:count * INFO_BYTES].cpu().numpy().tobytes()
        return [Info.from_bytes(raw[i * INFO_BYTES:(i + 1) * INFO_BYTES]) for i in range(count)]


def check_rc(rc, what):
    if rc != 0:
        lib = library()
        msg = lib.cqk_status_string(rc).decode()
        if rc == Status.CUDA_ERROR:
            msg += f" (cudaError {lib.cqk_last_cuda_error()})"
        raise RuntimeError(f"{what}: {msg}")


def _on_device(ts):
    host = ts[0].device.type != "cuda"
    dev = torch.device("cuda", torch.cuda.current_device()) if host else ts[0].device
    return host, dev, [t.to(dev, non_blocking=True) if t.device != dev else t for t in ts]


def solve(a, b, d, l, u, r, *, init=Init.FORMULA, max_iter=100, lambda0=0.0, validate=True, final_step=None,
          out=None, want_mask=False, ws: Workspace | None = None, stream=None, sync=True, **kw):
    """Solve min 1/2 x'Dx - a'x s.t. b'x = r, l <= x <= u (cqk_solve).

    a, b, d, l, u: 1-D float64 or float32 tensors of one dtype on one CUDA device (CPU
    tensors are copied to the current device and x is copied back).  Returns
    (x, info, mask); with sync=False no host synchronisation happens and info is None."""
    host, dev, (a, b, d, l, u) = _on_device([a, b, d, l, u])
    _check_device(a, b, d, l, u)
    n = a.numel()
    for t in (b, d, l, u):
        if t.dtype != a.dtype or t.numel() != n:
            raise ValueError("a, b, d, l, u must share dtype and length")
    x = out if out is not None else torch.empty_like(a)
    mask = torch.zeros((n + 31) // 32, dtype=torch.int32, device=dev) if want_mask else None
    ws = ws or Workspace(n, 1, a.dtype, dev)
    opt = make_options(init=init, max_iter=max_iter, lambda0=lambda0, validate=validate, final_step=final_step, **kw)
    rc = library().cqk_solve(n, dtype_code(a.dtype), ptr(a), ptr(b), ptr(d), ptr(l), ptr(u), float(r), ptr(x),
                             ptr(mask), ptr(ws.info), ctypes.byref(opt), ptr(ws.buf), ws.nbytes,
                             stream_handle(stream))
    check_rc(rc, "cqk_solve")
    info = ws.read_info() if sync else None
    if host:
        x = x.cpu()
        mask = mask.cpu() if mask is not None else None
    return x, info, mask


def phi(a, b, d, l, u, lam, *, want_x=False, ws: Workspace | None = None, stream=None):
    """(phi(lam), phi'_+(lam), phi'_-(lam), sum |b_i x_i(lam)|) by one map-reduce pass (cqk_phi)."""
    _check_device(a, b, d, l, u)
    n = a.numel()
    ws = ws or Workspace(n, 1, a.dtype, a.device)
    out = torch.zeros(4, dtype=torch.float64, device=a.device)
    x = torch.empty_like(a) if want_x else None
    rc = library().cqk_phi(n, dtype_code(a.dtype), ptr(a), ptr(b), ptr(d), ptr(l), ptr(u), float(lam), ptr(x),
                           ptr(out), ptr(ws.buf), ws.nbytes, stream_handle(stream))
    check_rc(rc, "cqk_phi")
    vals = tuple(float(v) for v in out.cpu())
    return (vals, x) if want_x else vals


def _project(name, y, r, init, max_iter, lambda0, validate, out, want_mask, ws, stream, sync, kw):
    host, dev, (y,) = _on_device([y])
    _check_device(y)
    n = y.numel()
    x = out if out is not None else torch.empty_like(y)
    mask = torch.zeros((n + 31) // 32, dtype=torch.int32, device=dev) if want_mask else None
    ws = ws or Workspace(n, 1, y.dtype, dev)
    opt = make_options(init=init, max_iter=max_iter, lambda0=lambda0, validate=validate, **kw)
    fn = getattr(library(), name)
    rc = fn(n, dtype_code(y.dtype), ptr(y), float(r), ptr(x), ptr(mask), ptr(ws.info), ctypes.byref(opt), ptr(ws.buf),
            ws.nbytes, stream_handle(stream))
    check_rc(rc, name)
    info = ws.read_info() if sync else None
    if host:
        x = x.cpu()
        mask = mask.cpu() if mask is not None else None
    return x, info, mask


def project_simplex(y, r=1.0, *, init=Init.CONDAT, max_iter=100, lambda0=0.0, validate=True, out=None,
                    want_mask=False, ws: Workspace | None = None, stream=None, sync=True, **kw):
    """Projection of y onto {x >= 0, sum x = r} (cqk_project_simplex).  Returns (x, info, mask)."""
    return _project("cqk_project_simplex", y, r, init, max_iter, lambda0, validate, out, want_mask, ws, stream, sync,
                    kw)


def project_l1(y, r=1.0, *, init=Init.CONDAT, max_iter=100, lambda0=0.0, validate=True, out=None,
               want_mask=False, ws: Workspace | None = None, stream=None, sync=True, **kw):
    """Projection of y onto {sum |x_i| <= r} (cqk_project_l1).  Returns (x, info, mask)."""
    return _project("cqk_project_l1", y, r, init, max_iter, lambda0, validate, out, want_mask, ws, stream, sync, kw)


def _batch_args(arrays, offsets, r):
    host, dev, arrays = _on_device(list(arrays))
    if not (torch.is_tensor(offsets) and offsets.device.type == "cuda"):
        # offsets given on the host: the instances must lie inside the arrays (device offsets
        # are read by the kernels only; a decreasing pair is reported per instance there)
        off_h = torch.as_tensor(offsets, dtype=torch.int64)
        if off_h.numel() and (int(off_h[0]) < 0 or int(off_h[-1]) > arrays[0].numel()):
            raise ValueError(f"offsets span [{int(off_h[0])}, {int(off_h[-1])}) outside the {arrays[0].numel()} "
                             "elements of the arrays")
    offsets = torch.as_tensor(offsets, dtype=torch.int64).to(dev).contiguous()
    r = torch.as_tensor(r, dtype=torch.float64).to(dev).contiguous()
    _check_device(*arrays, offsets, r)
    B = offsets.numel() - 1
    if B < 0 or r.numel() != B:
        raise ValueError("offsets must hold B + 1 entries and r B entries")
    n = arrays[0].numel()
    for t in arrays[1:]:
        if t.dtype != arrays[0].dtype or t.numel() != n:
            raise ValueError("the arrays must share dtype and length")
    return host, dev, arrays, offsets, r, B, n


def _batch_finish(host, x, mask, ws, B, sync):
    infos = ws.read_infos(B) if sync else None
    if host:
        x = x.cpu()
        mask = mask.cpu() if mask is not None else None
    return x, infos, mask


def solve_batched(a, b, d, l, u, offsets, r, *, init=Init.FORMULA, max_iter=100, lambda0=0.0, validate=True,
                  final_step=None, out=None, want_mask=False, ws: Workspace | None = None, stream=None, sync=True,
                  use_tuning=True, **kw):
    """B general CQK instances in one launch (cqk_solve_batched): instance k is the element
    range offsets[k]:offsets[k+1] of the concatenated a, b, d, l, u, with right-hand side
    r[k].  Returns (x, infos, mask); infos is a list of B Info (None with sync=False).
    With use_tuning (default) and none of the work-split options given, a tuning of this
    batch shape remembered by tune.py is applied."""
    host, dev, (a, b, d, l, u), offsets, r, B, n = _batch_args([a, b, d, l, u], offsets, r)
    kw = _with_tuning("general", a.dtype, offsets, kw, use_tuning)
    x = out if out is not None else torch.empty_like(a)
    mask = torch.zeros((n + 31) // 32, dtype=torch.int32, device=dev) if want_mask else None
    ws = ws or Workspace(n, max(B, 1), a.dtype, dev)
    opt = make_options(init=init, max_iter=max_iter, lambda0=lambda0, validate=validate, final_step=final_step, **kw)
    rc = library().cqk_solve_batched(B, ptr(offsets), dtype_code(a.dtype), ptr(a), ptr(b), ptr(d), ptr(l), ptr(u),
                                     ptr(r), ptr(x), ptr(mask), ptr(ws.info), ctypes.byref(opt), ptr(ws.buf),
                                     ws.nbytes, stream_handle(stream))
    check_rc(rc, "cqk_solve_batched")
    return _batch_finish(host, x, mask, ws, B, sync)


def _project_batched(name, y, offsets, r, init, max_iter, lambda0, validate, out, want_mask, ws, stream, sync, kw,
                     use_tuning=True):
    host, dev, (y,), offsets, r, B, n = _batch_args([y], offsets, r)
    kw = _with_tuning("l1" if "l1" in name else "simplex", y.dtype, offsets, kw, use_tuning)
    x = out if out is not None else torch.empty_like(y)
    mask = torch.zeros((n + 31) // 32, dtype=torch.int32, device=dev) if want_mask else None
    ws = ws or Workspace(n, max(B, 1), y.dtype, dev)
    opt = make_options(init=init, max_iter=max_iter, lambda0=lambda0, validate=validate, **kw)
    rc = getattr(library(), name)(B, ptr(offsets), dtype_code(y.dtype), ptr(y), ptr(r), ptr(x), ptr(mask),
                                  ptr(ws.info), ctypes.byref(opt), ptr(ws.buf), ws.nbytes, stream_handle(stream))
    check_rc(rc, name)
    return _batch_finish(host, x, mask, ws, B, sync)


def project_simplex_batched(y, offsets, r, *, init=Init.CONDAT, max_iter=100, lambda0=0.0, validate=True, out=None,
                            want_mask=False, ws: Workspace | None = None, stream=None, sync=True, use_tuning=True,
                            **kw):
    """B simplex projections in one launch (cqk_project_simplex_batched); use_tuning as for
    solve_batched."""
    return _project_batched("cqk_project_simplex_batched", y, offsets, r, init, max_iter, lambda0, validate, out,
                            want_mask, ws, stream, sync, kw, use_tuning)


def project_l1_batched(y, offsets, r, *, init=Init.CONDAT, max_iter=100, lambda0=0.0, validate=True, out=None,
                       want_mask=False, ws: Workspace | None = None, stream=None, sync=True, use_tuning=True, **kw):
    """B l1-ball projections in one launch (cqk_project_l1_batched); use_tuning as for
    solve_batched."""
    return _project_batched("cqk_project_l1_batched", y, offsets, r, init, max_iter, lambda0, validate, out,
                            want_mask, ws, stream, sync, kw, use_tuning)


def backward(kind, g, x, info, *, a=None, b=None, d=None, l=None, u=None, mask=None, offsets=None,
             want=("a", "b", "d", "l", "u"), ws: Workspace | None = None, stream=None, use_tuning=True, **kw):
    """Adjoint of a solve (cqk_backward, cqk_backward_simplex, cqk_backward_l1).

    kind: "general", "simplex" or "l1".  g, x (and a, b, d, l, u for "general") are device
    tensors of one dtype; info is the forward's info buffer (the Workspace.info tensor or a
    copy of it, one cqk_info per instance); offsets (device int64, B + 1) selects a batch.
    Returns dict with the requested gradients ("a".."u"; "y" for the projections), "r"
    (float64 tensor, one per instance) and "status" (int32 tensor).  No host synchronisation
    (except for the lookup of a remembered tuning of a batch, see solve_batched)."""
    _check_device(g, x)
    n = x.numel()
    B = 1 if offsets is None else offsets.numel() - 1
    out = {}
    gr = torch.empty(max(B, 1), dtype=torch.float64, device=x.device)
    status = torch.empty(max(B, 1), dtype=torch.int32, device=x.device)
    ws = ws or Workspace(n, max(B, 1), x.dtype, x.device)
    if offsets is not None:
        kw = _with_tuning(kind + "_bwd", x.dtype, offsets, kw, use_tuning)
    opt = make_options(**kw)
    lib = library()
    if kind == "general":
        for k in ("a", "b", "d", "l", "u"):
            out[k] = torch.empty_like(x) if k in want else None
        rc = lib.cqk_backward(B, ptr(offsets), n, dtype_code(x.dtype), ptr(g), ptr(x), ptr(a), ptr(b), ptr(d), ptr(l),
                              ptr(u), ptr(mask), ptr(info), ptr(out["a"]), ptr(out["b"]), ptr(out["d"]), ptr(out["l"]),
                              ptr(out["u"]), ptr(gr), ptr(status), ctypes.byref(opt), ptr(ws.buf), ws.nbytes,
                              stream_handle(stream))
        name = "cqk_backward"
    else:
        name = "cqk_backward_simplex" if kind == "simplex" else "cqk_backward_l1"
        out["y"] = torch.empty_like(x)
        rc = getattr(lib, name)(B, ptr(offsets), n, dtype_code(x.dtype), ptr(g), ptr(x), ptr(mask), ptr(info),
                                ptr(out["y"]), ptr(gr), ptr(status), ctypes.byref(opt), ptr(ws.buf), ws.nbytes,
                                stream_handle(stream))
    check_rc(rc, name)
    out["r"] = gr
    out["status"] = status
    return out
