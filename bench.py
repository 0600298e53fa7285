"""Benchmark of the CQK semismooth Newton hot path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-extras]

Workload (default): projection of y ~ N(0,1), n = 10^8, FP64, onto the unit simplex and onto
the unit l1 ball, Condat start (Alg. 2 per chunk, then Alg. 4); one step = both projections
of the same y.  The inputs (800 MB) exceed the 126 MB L2, so no L2 flush is needed between
steps.  Metric: elements x Newton iterations per second, summed over the step's
projections (n x phi evaluations / time); the roofline object reports the achieved HBM
bandwidth of the projection kernel from its algorithmic bytes (8 bytes per element per read
pass + 8 per element written) and its CUDA-event time.

For N > 1 (torchrun, one process per GPU) every rank projects its own vector (seed = rank):
independent replicas, weak scaling, no data-path collective; rank 0 prints one JSON line
with the max over ranks of the timed region.

--impl reference times the FP64 CPU oracle (its sequential Alg. 2 + Alg. 4, the paper's CPU
method) on the host cores on a bounded sample of the same workload, same metric.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "elements·Newton-iters/sec and achieved HBM GB/s vs ~8 TB/s; batched fwd+bwd speedup"
UNIT = "elem*iter/s"
N_DEFAULT = 100_000_000
CPU_SAMPLE = 20_000_000


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# ------------------------------------------------------------------------------ clocks
class _NvmlCtypes:
    """Read-only NVML queries through the driver's libnvidia-ml (SM clock, its maximum and
    the clock-event reason bits), for images without the pynvml module."""

    NVML_CLOCK_SM = 1

    def __init__(self, bus):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        rc = self.lib.nvmlInit_v2()
        if rc != 0:
            raise RuntimeError(f"nvmlInit_v2 -> {rc}")
        self.h = ctypes.c_void_p()
        rc = self.lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(self.h))
        if rc != 0:
            raise RuntimeError(f"nvmlDeviceGetHandleByPciBusId_v2 -> {rc}")
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def max_sm(self):
        v = self.ct.c_uint()
        rc = self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.NVML_CLOCK_SM, self.ct.byref(v))
        return v.value if rc == 0 else None

    def sample(self):
        v = self.ct.c_uint()
        r = self.ct.c_ulonglong()
        rc1 = self.lib.nvmlDeviceGetClockInfo(self.h, self.NVML_CLOCK_SM, self.ct.byref(v))
        rc2 = self.reasons_fn(self.h, self.ct.byref(r))
        if rc1 != 0 or rc2 != 0:
            raise RuntimeError(f"nvml query -> {rc1}, {rc2}")
        return v.value, r.value


class ClockSampler:
    """Samples the SM clock and the clock-event reasons of the CUDA device while running:
    NVML addressed by the device's PCI bus id, or `nvidia-smi -lms` when NVML is unusable."""

    REASONS = {0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x10: "sync_boost",
               0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
               0x100: "display_clock_setting"}

    def __init__(self, cuda_index):
        import torch
        self.samples, self.reasons, self.max_mhz = [], set(), None
        self.source, self.error = None, None
        self._stop = threading.Event()
        self._t = None
        self._proc = None
        p = torch.cuda.get_device_properties(cuda_index)
        self.bus = f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
        try:
            try:
                import pynvml
                pynvml.nvmlInit()
                self.nv = pynvml
                self.h = pynvml.nvmlDeviceGetHandleByPciBusId(self.bus.encode())
                self.max_mhz = pynvml.nvmlDeviceGetMaxClockInfo(self.h, pynvml.NVML_CLOCK_SM)
                self.source = "nvml"
            except ImportError:
                self.nv = _NvmlCtypes(self.bus)
                self.h = None
                self.max_mhz = self.nv.max_sm()
                self.source = "nvml (libnvidia-ml via ctypes)"
        except Exception as e:  # noqa: BLE001
            self.nv = None
            self.error = f"nvml: {type(e).__name__}: {e}"

    def _run(self):
        while not self._stop.is_set():
            try:
                if isinstance(self.nv, _NvmlCtypes):
                    clk, bits = self.nv.sample()
                else:
                    clk = self.nv.nvmlDeviceGetClockInfo(self.h, self.nv.NVML_CLOCK_SM)
                    bits = self.nv.nvmlDeviceGetCurrentClocksEventReasons(self.h)
                self.samples.append(clk)
                self._bits(bits)
            except Exception as e:  # noqa: BLE001
                self.error = f"nvml sample: {type(e).__name__}: {e}"
            time.sleep(0.002)

    def _bits(self, bits):
        for b, name in self.REASONS.items():
            if bits & b:
                self.reasons.add(name)

    def __enter__(self):
        if self.nv is not None:
            self._t = threading.Thread(target=self._run, daemon=True)
            self._t.start()
        else:
            import subprocess
            try:
                self._proc = subprocess.Popen(
                    ["nvidia-smi", "-i", self.bus, "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active",
                     "--format=csv,noheader,nounits", "-lms", "100"], stdout=subprocess.PIPE, text=True)
                self.source = "nvidia-smi"
            except Exception as e:  # noqa: BLE001
                self.error = (self.error or "") + f"; nvidia-smi: {e}"
        return self

    def __exit__(self, *exc):
        self._stop.set()
        if self._t is not None:
            self._t.join()
        if self._proc is not None:
            self._proc.terminate()
            out, _ = self._proc.communicate(timeout=5)
            for line in out.splitlines():
                parts = [x.strip() for x in line.split(",")]
                try:
                    self.samples.append(float(parts[0]))
                    self.max_mhz = float(parts[1])
                    self._bits(int(parts[2], 16))
                except Exception:  # noqa: BLE001
                    pass

    def summary(self):
        d = {"sm_mhz": statistics.median(self.samples) if self.samples else None, "sm_max_mhz": self.max_mhz,
             "reasons": sorted(self.reasons), "samples": len(self.samples), "source": self.source}
        if self.error and not self.samples:
            d["error"] = self.error
        return d


# ------------------------------------------------------------------------------ our arm
def kernel_sources_sha256():
    """Hash of the kernel sources with comments and blank space removed: a profile's counters
    stay valid across edits of comments only, and not across any change of code."""
    import glob
    import hashlib
    import re
    pkg = os.path.join(ROOT, "paper_2603_15910_b300", "csrc")
    files = sorted(glob.glob(os.path.join(pkg, "*.cu")) + glob.glob(os.path.join(pkg, "*.cuh")) +
                   glob.glob(os.path.join(pkg, "*.h"))) + [os.path.join(ROOT, "include", "cqk.h")]
    # comments (outside string literals) and runs of blank space
    token = re.compile(r'"(?:\\.|[^"\\])*"|//[^\n]*|/\*.*?\*/|\s+', re.S)
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, encoding="utf-8") as fh:
            src = fh.read()
        code = token.sub(lambda m: m.group(0) if m.group(0).startswith('"') else " ", src)
        h.update(re.sub(" +", " ", code).encode())
    return h.hexdigest()


def measured_traffic(n):
    """DRAM bytes of the step's two launches from the committed ncu summary, if it was taken on
    these kernel sources at this size; else None."""
    path = os.path.join(ROOT, "profiles", "simplex_kernel_f64_n1e8_dram.md")
    try:
        with open(path) as f:
            line = next(ln for ln in f if "traffic_json:" in ln)
        rec = json.loads(line.split("traffic_json:", 1)[1])
    except Exception:  # noqa: BLE001
        return None
    if n != N_DEFAULT or rec.get("sources_sha256") != kernel_sources_sha256():
        return None
    return rec["bytes_per_step"]


def algorithmic_bytes_projection(n, elem_bytes, info):
    """Bytes one projection must move: every read pass streams y once, the final pass
    also writes x (info.passes counts the start, Newton and final passes)."""
    return n * elem_bytes * info.passes + n * elem_bytes


def run_ours(args, world, rank, local):
    import torch
    import torch.distributed as dist

    from paper_2603_15910_b300 import api, workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    n = args.n
    y = W.simplex_normal(n, seed=rank, device=dev)
    x1 = torch.empty_like(y)
    x2 = torch.empty_like(y)
    ws1 = api.Workspace(n, 1, y.dtype, dev)
    ws2 = api.Workspace(n, 1, y.dtype, dev)
    stream = torch.cuda.current_stream()

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        api.project_simplex(y, 1.0, init=api.Init.CONDAT, out=x1, ws=ws1, sync=False)
        if ev is not None:
            ev[1].record(stream)
        api.project_l1(y, 1.0, init=api.Init.CONDAT, out=x2, ws=ws2, sync=False)
        if ev is not None:
            ev[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    i1, i2 = ws1.read_info(), ws2.read_info()
    for inf in (i1, i2):
        if inf.status != api.Status.OK:
            raise RuntimeError(f"projection failed: {inf}")

    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0.record(stream)
        for k in range(K):
            step(evs[k])
        t1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = t0.elapsed_time(t1)
    if world > 1:
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    t_s = sum(e[0].elapsed_time(e[1]) for e in evs) / K
    t_l = sum(e[1].elapsed_time(e[2]) for e in evs) / K
    iters = i1.iters + i2.iters
    value = world * n * iters * K / (ms * 1e-3)

    # roofline of the projection kernel (both launches of the step), live CUDA events
    bytes_s = algorithmic_bytes_projection(n, 8, i1)
    bytes_l = algorithmic_bytes_projection(n, 8, i2)
    achieved = (bytes_s + bytes_l) / ((t_s + t_l) * 1e-3) / 1e9
    peak, peak_kind = measured_peak_hbm()
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"simplex + l1-ball projection, n={n}, FP64, y~N(0,1), r=1, Condat start "
                               "(Alg. 2 per block chunk) then Alg. 4",
                   "n": n, "init": "condat", "projections_per_step": 2, "iters_simplex": i1.iters,
                   "iters_l1": i2.iters, "passes_simplex": i1.passes, "passes_l1": i2.passes,
                   "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (800 MB per vector)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": measured_traffic(n), "traffic_unit": "bytes per step (both launches), ncu",
                     "kernel": "simplex_kernel<double> (simplex + l1 launches)",
                     "peak_source": peak_kind, "ms_simplex": t_s, "ms_l1": t_l,
                     "algorithmic_bytes": bytes_s + bytes_l, "frac_of_8TBs": achieved / 8000.0},
        "gpu_launches": 2 * K,
        "clocks": clk.summary(),
    }

    # end to end through the public API with host buffers: every step copies its y from pinned
    # host memory to the device, runs both projections and copies both x back to pinned host
    # memory.  Three streams overlap step k's copies out with step k+1's copy in and compute
    # (the host link is full duplex and the copy engines run beside the kernels); inputs and
    # outputs are double-buffered on the device.
    y_host = y.cpu().pin_memory()
    xh1 = torch.empty(n, dtype=y.dtype, pin_memory=True)
    xh2 = torch.empty(n, dtype=y.dtype, pin_memory=True)
    yd = [torch.empty_like(y), torch.empty_like(y)]
    xo1 = [x1, torch.empty_like(y)]
    xo2 = [x2, torch.empty_like(y)]
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event(), torch.cuda.Event()]
    ev_x1 = [torch.cuda.Event(), torch.cuda.Event()]
    ev_x2 = [torch.cuda.Event(), torch.cuda.Event()]
    ev_done = [torch.cuda.Event(), torch.cuda.Event()]  # buffer k % 2 free again
    for b in range(2):
        ev_done[b].record(stream)

    def e2e_step(k):
        b = k % 2
        with torch.cuda.stream(s_in):
            s_in.wait_event(ev_done[b])
            yd[b].copy_(y_host, non_blocking=True)
            ev_in[b].record(s_in)
        stream.wait_event(ev_in[b])
        api.project_simplex(yd[b], 1.0, init=api.Init.CONDAT, out=xo1[b], ws=ws1, sync=False, stream=stream)
        ev_x1[b].record(stream)
        api.project_l1(yd[b], 1.0, init=api.Init.CONDAT, out=xo2[b], ws=ws2, sync=False, stream=stream)
        ev_x2[b].record(stream)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_x1[b])
            xh1.copy_(xo1[b], non_blocking=True)
            s_out.wait_event(ev_x2[b])
            xh2.copy_(xo2[b], non_blocking=True)
            ev_done[b].record(s_out)

    for k in range(2):
        e2e_step(k)
    torch.cuda.synchronize()
    Ke = max(3, K // 2)
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    for k in range(Ke):
        e2e_step(k)
    e1.record(s_out)  # after the last copy out (it follows every earlier one on its stream)
    torch.cuda.synchronize()
    ems = e0.elapsed_time(e1)
    if world > 1:
        tt = torch.tensor([ems], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ems = float(tt.item())
    out["e2e"] = {"value": world * n * iters * Ke / (ems * 1e-3), "unit": UNIT, "h2d_bytes_per_step": 8 * n,
                  "d2h_bytes_per_step": 16 * n, "ms_per_step": ems / Ke,
                  "overlap": "copy in, compute and copy out on three streams, double-buffered"}

    if args.extras and rank == 0:
        out["variants"] = extras(args, api, W, dev, stream)
        out["batched"] = batched_extras(api, W, dev, stream)
    if rank == 0 and args.cpu_baseline:
        yc = y[:CPU_SAMPLE].cpu().numpy()
        out["cpu_baseline"] = cpu_baseline(yc)
    if world > 1:
        dist.destroy_process_group()
    return out if rank == 0 else None


def _time(fn, stream, reps=5):
    import torch
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def extras(args, api, W, dev, stream):
    """Side measurements (not part of `value`): the plain (formula) start, the 1%-sparse
    variant, and the general CQK solve of the correlated family at n = 1e8 in FP64 and
    FP32 storage."""
    import torch
    n = args.n
    res = {}
    y = W.simplex_normal(n, seed=0, device=dev)
    ys = W.simplex_normal(n, seed=0, sparse=True, device=dev)
    x = torch.empty_like(y)
    ws = api.Workspace(n, 1, y.dtype, dev)
    for name, vec in (("dense", y), ("sparse", ys)):
        for init in (api.Init.CONDAT, api.Init.FORMULA):
            for proj in ("simplex", "l1"):
                f = api.project_simplex if proj == "simplex" else api.project_l1
                ms = _time(lambda: f(vec, 1.0, init=init, out=x, ws=ws, sync=False), stream)
                inf = ws.read_info()
                byt = algorithmic_bytes_projection(n, 8, inf)
                res[f"{proj}_{name}_{init.name.lower()}"] = {
                    "ms": ms, "iters": inf.iters, "passes": inf.passes, "status": int(inf.status),
                    "elem_iter_per_s": n * inf.iters / (ms * 1e-3), "GBps": byt / (ms * 1e-3) / 1e9}
    del y, ys, x
    for dt, tag in ((torch.float64, "f64"), (torch.float32, "f32")):
        p = W.correlated(n, seed=0, device=dev, dtype=dt)
        xg = torch.empty_like(p["a"])
        wsg = api.Workspace(n, 1, dt, dev)
        ms = _time(lambda: api.solve(p["a"], p["b"], p["d"], p["l"], p["u"], p["r"], out=xg, ws=wsg, sync=False),
                   stream, reps=3)
        inf = wsg.read_info()
        es = 8 if dt == torch.float64 else 4
        # pass 0 reads a, b, d; each Newton pass reads 5 arrays; the final pass reads 5, writes x
        byt = n * es * (3 + 5 * (inf.passes - 2) + 6)
        res[f"general_correlated_{tag}"] = {"ms": ms, "iters": inf.iters, "passes": inf.passes,
                                            "status": int(inf.status), "elem_iter_per_s": n * inf.iters / (ms * 1e-3),
                                            "GBps": byt / (ms * 1e-3) / 1e9}
        del p, xg
        torch.cuda.empty_cache()
    return res


def batched_extras(api, W, dev, stream):
    """The batched, differentiable workloads: forward + backward of a ragged batch in two
    launches (captured once in a CUDA graph and replayed) against the same solves issued as
    one forward and one backward launch per instance.
      simplex: 4096 instances, lengths log-uniform in [16, 2^20], FP32 y ~ N(0,1), r = 1
      general: 256 instances, lengths log-uniform in [1e3, 1e6], FP64 uncorrelated box"""
    import torch
    res = {}
    cases = (
        ("simplex_f32_b4096", lambda: W.batched_simplex(batch=4096, lo=16, hi=1 << 20, seed=0, device=dev,
                                                        dtype=torch.float32)),
        ("general_f64_b256", lambda: W.batched_general(batch=256, lo=1000, hi=1000000, seed=0, device=dev,
                                                       dtype=torch.float64)),
    )
    for name, make in cases:
        d = make()
        general = "a" in d
        vec = d["a"] if general else d["y"]
        n, B = vec.numel(), d["offsets"].numel() - 1
        off = d["offsets"]
        r = d["r"].to(dev)
        g = d["g"]
        x = torch.empty_like(vec)
        mask = torch.zeros((n + 31) // 32, dtype=torch.int32, device=dev)
        ws = api.Workspace(n, B, vec.dtype, dev)
        grads = {k: torch.empty_like(vec) for k in ("a", "b", "d", "l", "u", "y")}
        gr = torch.empty(B, dtype=torch.float64, device=dev)
        st = torch.empty(B, dtype=torch.int32, device=dev)
        lib = api.library()
        opt = api.make_options()
        P = api.ptr
        code = api.dtype_code(vec.dtype)

        def fwd_bwd(s=None):
            sh = api.stream_handle(s or stream)
            if general:
                rc = lib.cqk_solve_batched(B, P(off), code, P(d["a"]), P(d["b"]), P(d["d"]), P(d["l"]), P(d["u"]),
                                           P(r), P(x), P(mask), P(ws.info), api.ctypes.byref(opt), P(ws.buf),
                                           ws.nbytes, sh)
                api.check_rc(rc, "cqk_solve_batched")
                rc = lib.cqk_backward(B, P(off), n, code, P(g), P(x), P(d["a"]), P(d["b"]), P(d["d"]), P(d["l"]),
                                      P(d["u"]), P(mask), P(ws.info), P(grads["a"]), P(grads["b"]), P(grads["d"]),
                                      P(grads["l"]), P(grads["u"]), P(gr), P(st), api.ctypes.byref(opt),
                                      P(ws.buf), ws.nbytes, sh)
                api.check_rc(rc, "cqk_backward")
            else:
                rc = lib.cqk_project_simplex_batched(B, P(off), code, P(d["y"]), P(r), P(x), P(mask), P(ws.info),
                                                     api.ctypes.byref(opt), P(ws.buf), ws.nbytes,
                                                     sh)
                api.check_rc(rc, "cqk_project_simplex_batched")
                rc = lib.cqk_backward_simplex(B, P(off), n, code, P(g), P(x), P(mask), P(ws.info), P(grads["y"]),
                                              P(gr), P(st), api.ctypes.byref(opt), P(ws.buf), ws.nbytes,
                                              sh)
                api.check_rc(rc, "cqk_backward_simplex")

        ms_batched = _time(fwd_bwd, stream)
        infos = ws.read_infos(B)
        ok = sum(int(i.status) == 0 for i in infos)
        graph_ms = None
        try:
            gph = torch.cuda.CUDAGraph()
            cs = torch.cuda.Stream()
            cs.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(cs):
                fwd_bwd(cs)
                torch.cuda.synchronize()
                with torch.cuda.graph(gph, stream=cs):
                    fwd_bwd(cs)
            graph_ms = _time(gph.replay, torch.cuda.current_stream())
        except Exception as e:  # capture unsupported: report, do not fail the bench
            graph_ms = f"capture failed: {type(e).__name__}: {e}"
        # per-instance launches (one forward + one backward per instance), same arrays
        offs = off.cpu().tolist()
        rl = d["r"].cpu().tolist()
        ws1 = api.Workspace(max(offs[k + 1] - offs[k] for k in range(B)), 1, vec.dtype, dev)
        info1 = ws1.info

        def per_instance():
            for k in range(B):
                lo, hi = offs[k], offs[k + 1]
                m = hi - lo
                if m == 0:
                    continue
                es = vec.element_size()
                if general:
                    ap = [P(d[q][lo:hi]) for q in ("a", "b", "d", "l", "u")]
                    lib.cqk_solve(m, code, *ap, float(rl[k]), P(x[lo:hi]), None, P(info1), api.ctypes.byref(opt),
                                  P(ws1.buf), ws1.nbytes, api.stream_handle(stream))
                    lib.cqk_backward(1, None, m, code, P(g[lo:hi]), P(x[lo:hi]), *ap, None, P(info1),
                                     P(grads["a"][lo:hi]), P(grads["b"][lo:hi]), P(grads["d"][lo:hi]),
                                     P(grads["l"][lo:hi]), P(grads["u"][lo:hi]), P(gr[k:k + 1]), P(st[k:k + 1]),
                                     api.ctypes.byref(opt), P(ws1.buf), ws1.nbytes, api.stream_handle(stream))
                else:
                    lib.cqk_project_simplex(m, code, P(d["y"][lo:hi]), float(rl[k]), P(x[lo:hi]), None, P(info1),
                                            api.ctypes.byref(opt), P(ws1.buf), ws1.nbytes, api.stream_handle(stream))
                    lib.cqk_backward_simplex(1, None, m, code, P(g[lo:hi]), P(x[lo:hi]), None, P(info1),
                                             P(grads["y"][lo:hi]), P(gr[k:k + 1]), P(st[k:k + 1]),
                                             api.ctypes.byref(opt), P(ws1.buf), ws1.nbytes, api.stream_handle(stream))

        ms_loop = _time(per_instance, stream, reps=2)
        res[name] = {"instances": B, "n_total": n, "dtype": str(vec.dtype).replace("torch.", ""),
                     "ms_fwd_bwd_batched": ms_batched, "ms_fwd_bwd_graph": graph_ms,
                     "ms_fwd_bwd_per_instance_launches": ms_loop,
                     "speedup_vs_per_instance": ms_loop / (graph_ms if isinstance(graph_ms, float) else ms_batched),
                     "instances_ok": ok, "mean_iters": sum(i.iters for i in infos) / B,
                     "elements_per_s_fwd_bwd": n / ((graph_ms if isinstance(graph_ms, float) else ms_batched) * 1e-3)}
        del d, x, mask, ws, grads, ws1
        torch.cuda.empty_cache()
    return res


# ------------------------------------------------------------------------------ oracle timing
def cpu_baseline(y, max_seconds=30.0):
    """The FP64 oracle as it stands (sequential C: Alg. 2 start + Alg. 4), on the host, for
    the same two projections of a bounded sample of the workload."""
    import numpy as np

    import oracle
    n = y.shape[0]
    t = time.perf_counter()
    evals = 0
    reps = 0
    while True:
        lam0, _, _ = oracle.condat_init(y, 1.0)
        evals += oracle.newton_simplex(y, 1.0, lam0=lam0)["evals"]
        lam0, _, _ = oracle.condat_init(y, 1.0, l1=True)
        evals += oracle.newton_simplex(y, 1.0, lam0=lam0, l1=True)["evals"]
        reps += 1
        if time.perf_counter() - t > max_seconds / 3 or reps >= 3:
            break
    el = time.perf_counter() - t
    return {"value": n * evals / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {n} elements of the n=1e8 vector, {reps} step(s) (simplex + l1, Alg. 2 start + "
                      f"Alg. 4, sequential C oracle)",
            "seconds": el, "host_cores_available": len(os.sched_getaffinity(0))}


def run_reference(args, world, rank):
    if rank != 0:
        return None
    import torch

    from paper_2603_15910_b300 import workloads as W
    y = W.simplex_normal(args.n, seed=0, device="cpu")[:CPU_SAMPLE].numpy()
    import oracle
    oracle.reference.build()
    for _ in range(min(args.warmup, 1)):
        cpu_baseline(y[:1_000_000])
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(y, max_seconds=10.0))
        if time.perf_counter() - t0 > 150:
            break
    v = statistics.median([c["value"] for c in vals])
    cb = dict(vals[0])
    cb["value"] = v
    return {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": len(vals), "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.median([c["seconds"] for c in vals]), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "simplex + l1-ball projection, n=1e8, FP64, y~N(0,1), r=1, Condat start",
                       "n": args.n, "sample": CPU_SAMPLE},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--no-extras", dest="extras", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, world, rank)
    else:
        out = run_ours(args, world, rank, local)
    if out is not None and rank == 0:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
