"""Benchmark of the CQK semismooth Newton hot path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-extras]
                    [--no-cpu-baseline] [--no-oracle-check]
    python bench.py --case general|batched_simplex|batched_general [--n N] [--batch B]

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

Every result is also compared with the FP64 oracle's exact solution on the host
(err_vs_oracle: the headline projections, every variant, config 0 and every instance of the
two batches, forward and adjoint), after the GPU timing it describes.

Extra keys: variants (formula vs Condat start, the 1%-sparse input, the general correlated
family at n = 1e8 in FP64 and FP32 storage), config0 (the latency-bound n = 10,000 solve, L2
warm and cold), batched (the two ragged batches forward + adjoint: batched launch, CUDA
graph, autotuned options, per-instance launches from Python and in one CUDA graph, roofline
at the algorithmic bytes) and cpu_baseline (the oracle on all host cores and on one core).

--case runs one side workload alone and prints its CUDA-event timings (a profiling aid: the
commands of the ncu summaries): the general solve of the correlated family at --n in FP64 and
FP32 storage (one warm-up and 7 timed solves each), or a ragged batch of --batch instances
(the simplex recipe in FP32, the general recipe in FP64) forward + adjoint, twice.

--impl reference times the FP64 CPU oracle -- Alg. 2 per thread chunk and Alg. 4 with
OpenMP map-reduce passes, the paper's CPU Jacobi form -- on all host cores on the same
workload, same metric.
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


def algorithmic_bytes_general(n, elem_bytes, info):
    """Bytes of one general solve: the eq. (CQKlambda0) pass reads a, b, d; every Newton pass
    reads a, b, d, l, u; the final pass reads the five arrays and writes x."""
    return n * elem_bytes * (3 + 5 * (info.passes - 2) + 6)


def host_cores():
    return len(os.sched_getaffinity(0))


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def pool_map(fn, items):
    """[fn(i) for i in items] on a thread pool of all host cores: the C oracle's calls release
    the GIL (ctypes), so independent solves run in parallel."""
    from concurrent.futures import ThreadPoolExecutor
    items = list(items)
    if len(items) <= 1:
        return [fn(i) for i in items]
    with ThreadPoolExecutor(max_workers=max(1, min(len(items), host_cores()))) as pool:
        return list(pool.map(fn, items))


# ------------------------------------------------------------------------------ error vs oracle
TOL_X = {"f64": 1e-10, "f32": 1e-5}
TOL_FEAS = {"f64": 1e-12, "f32": 1e-5}


def _x_rel(x, xstar):
    import numpy as np
    return float(np.max(np.abs(x - xstar))) / (1.0 + float(np.max(np.abs(xstar)))) if x.size else 0.0


def exact_projection(y64, l1, r=1.0):
    """(lambda*, x*) of the oracle's sort-based projection (l1 ball: Lemma 3.2)."""
    import oracle
    if l1:
        lam, xstar, _ = oracle.project_l1(y64, r)
        return lam, xstar
    return oracle.project_simplex_sort(y64, r)


def err_projection(x64, xstar, r, dt):
    """Error of a projection against the oracle's exact one: max |x - x*| / (1 + max |x*|) and
    |sum |x_i| - r| / r, with the tolerances of the storage type."""
    import numpy as np
    xr = _x_rel(x64, xstar)
    fr = abs(float(np.sum(np.abs(x64), dtype=np.longdouble)) - r) / r
    return {"x_rel": xr, "feas_rel": fr, "tol_x": TOL_X[dt], "tol_feas": TOL_FEAS[dt],
            "within_tol": bool(xr <= TOL_X[dt] and fr <= TOL_FEAS[dt])}


def err_general(host, r, x64, exact, dt):
    """Error of a general solve against the oracle's exact solution: max |x - x*| / (1 + max |x*|)
    and |b'x - r| / sum |b_i x_i| (the problem statement's feasibility, eq. (CQK))."""
    import numpy as np
    st, lam, xstar = exact
    bx = host[1] * x64
    fr = abs(float(np.sum(bx, dtype=np.longdouble)) - r) / max(float(np.sum(np.abs(bx))), 1e-300)
    xr = _x_rel(x64, xstar) if st == "ok" else float("nan")
    return {"x_rel": xr, "feas_rel": fr, "tol_x": TOL_X[dt], "tol_feas": TOL_FEAS[dt],
            "within_tol": bool(st == "ok" and xr <= TOL_X[dt] and fr <= TOL_FEAS[dt])}


def _max_err(items):
    """Worst of per-instance error dicts."""
    keys = [k for k in items[0] if k.endswith("_rel")]
    out = {k: max(it[k] for it in items) for k in keys}
    out.update({k: items[0][k] for k in items[0] if k.startswith("tol")})
    out["within_tol"] = all(it["within_tol"] for it in items)
    out["instances"] = len(items)
    return out


def job_totals(ms, units, world, device=None):
    """Whole-job figures of a timed region run by every rank: the longest rank's time (the job
    ends when its slowest rank does) and the units of work summed over the ranks (each rank
    projects its own vector, so their Newton iteration counts may differ).  Called by every
    rank after the closing barrier; with world == 1 it returns its arguments."""
    if world <= 1:
        return ms, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ------------------------------------------------------------------------------ our arm
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
    t_s = sum(e[0].elapsed_time(e[1]) for e in evs) / K
    t_l = sum(e[1].elapsed_time(e[2]) for e in evs) / K
    iters = i1.iters + i2.iters
    ms, units = job_totals(t0.elapsed_time(t1), n * iters * K, world, dev)
    value = units / (ms * 1e-3)

    # roofline of the projection kernel (both launches of the step), live CUDA events
    bytes_s = algorithmic_bytes_projection(n, 8, i1)
    bytes_l = algorithmic_bytes_projection(n, 8, i2)
    achieved = (bytes_s + bytes_l) / ((t_s + t_l) * 1e-3) / 1e9
    peak, peak_kind = measured_peak_hbm()
    traffic = measured_traffic(n)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_unit": "bytes per step (both launches), ncu",
            "kernel": "simplex_kernel<double> (simplex + l1 launches)",
            "achieved_basis": "algorithmic bytes / CUDA-event time (effective bandwidth)",
            "peak_source": peak_kind, "ms_simplex": t_s, "ms_l1": t_l,
            "algorithmic_bytes": bytes_s + bytes_l, "frac_of_8TBs": achieved / 8000.0}
    if traffic:
        # DRAM bytes the ncu capture counted for the same launches, over the same live time
        dram = traffic / ((t_s + t_l) * 1e-3) / 1e9
        roof.update({"dram_GBps": dram, "dram_frac": dram / peak})
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"simplex + l1-ball projection, n={n}, FP64, y~N(0,1), r=1, Condat start "
                               "(Alg. 2 per block chunk) then Alg. 4",
                   "n": n, "init": "condat", "projections_per_step": 2, "iters_simplex": i1.iters,
                   "iters_l1": i2.iters, "passes_simplex": i1.passes, "passes_l1": i2.passes,
                   "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (800 MB per vector)"},
        "roofline": roof,
        "gpu_launches": 2 * K,
        "clocks": clk.summary(),
    }

    # error of the step's two projections against the oracle's exact ones (host, all cores)
    if rank == 0 and args.oracle_check:
        y64, xs1, xs2 = y.cpu().numpy(), x1.cpu().numpy(), x2.cpu().numpy()
        ex = pool_map(lambda l1: exact_projection(y64, l1), (False, True))
        out["err_vs_oracle"] = {"simplex": err_projection(xs1, ex[0][1], 1.0, "f64"),
                                "l1": err_projection(xs2, ex[1][1], 1.0, "f64"),
                                "oracle": "sort-based projection (l1: Lemma 3.2), FP64, long double sums"}
        exact_dense = {False: ex[0][1], True: ex[1][1]}
        del xs1, xs2
    else:
        y64, exact_dense = None, None

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
    ems, e_units = job_totals(e0.elapsed_time(e1), n * iters * Ke, world, dev)
    out["e2e"] = {"value": e_units / (ems * 1e-3), "unit": UNIT, "h2d_bytes_per_step": 8 * n,
                  "d2h_bytes_per_step": 16 * n, "ms_per_step": ems / Ke,
                  "overlap": "copy in, compute and copy out on three streams, double-buffered"}
    del y_host, xh1, xh2, yd, xo1, xo2
    torch.cuda.empty_cache()

    if args.extras and rank == 0:
        out["variants"] = extras(args, api, W, dev, stream, y64, exact_dense)
        out["config0"] = config0(api, W, dev, stream, args.oracle_check)
        out["batched"] = batched_extras(api, W, dev, stream, args.oracle_check)
    if rank == 0 and args.cpu_baseline:
        ycpu = y64 if y64 is not None else y.cpu().numpy()
        out["cpu_baseline"] = cpu_baseline(ycpu)
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


def extras(args, api, W, dev, stream, y64=None, exact_dense=None):
    """Side measurements (not part of `value`): the plain (formula) start, the 1%-sparse
    variant, and the general CQK solve of the correlated family at n = 1e8 in FP64 and
    FP32 storage; each with its error against the oracle's exact solution."""
    import torch
    n = args.n
    peak, _ = measured_peak_hbm()
    res = {}
    y = W.simplex_normal(n, seed=0, device=dev)
    ys = W.simplex_normal(n, seed=0, sparse=True, device=dev)
    x = torch.empty_like(y)
    ws = api.Workspace(n, 1, y.dtype, dev)
    xs_host = {}
    for name, vec in (("dense", y), ("sparse", ys)):
        for init in (api.Init.CONDAT, api.Init.FORMULA):
            for proj in ("simplex", "l1"):
                f = api.project_simplex if proj == "simplex" else api.project_l1
                ms = _time(lambda: f(vec, 1.0, init=init, out=x, ws=ws, sync=False), stream)
                inf = ws.read_info()
                byt = algorithmic_bytes_projection(n, 8, inf)
                key = f"{proj}_{name}_{init.name.lower()}"
                res[key] = {
                    "ms": ms, "iters": inf.iters, "passes": inf.passes, "status": int(inf.status),
                    "elem_iter_per_s": n * inf.iters / (ms * 1e-3), "GBps": byt / (ms * 1e-3) / 1e9,
                    "frac": byt / (ms * 1e-3) / 1e9 / peak}
                if args.oracle_check:
                    xs_host[key] = x.cpu().numpy()
    if args.oracle_check:
        vecs = {"dense": y64 if y64 is not None else y.cpu().numpy(), "sparse": ys.cpu().numpy()}
        jobs = [(nm, l1) for nm in ("dense", "sparse") for l1 in (False, True)
                if not (nm == "dense" and exact_dense is not None)]
        ex = dict(zip(jobs, pool_map(lambda j: exact_projection(vecs[j[0]], j[1])[1], jobs)))
        if exact_dense is not None:
            ex[("dense", False)], ex[("dense", True)] = exact_dense[False], exact_dense[True]
        for key, xh in xs_host.items():
            proj, nm, _ = key.split("_")
            res[key]["err_vs_oracle"] = err_projection(xh, ex[(nm, proj == "l1")], 1.0, "f64")
        del vecs, ex, xs_host
    del y, ys, x
    torch.cuda.empty_cache()
    sols = {}
    for dt, tag in ((torch.float64, "f64"), (torch.float32, "f32")):
        p = W.correlated(n, seed=0, device=dev, dtype=dt)
        xg = torch.empty_like(p["a"])
        wsg = api.Workspace(n, 1, dt, dev)
        ms = _time(lambda: api.solve(p["a"], p["b"], p["d"], p["l"], p["u"], p["r"], out=xg, ws=wsg, sync=False),
                   stream, reps=3)
        inf = wsg.read_info()
        es = 8 if dt == torch.float64 else 4
        byt = algorithmic_bytes_general(n, es, inf)
        res[f"general_correlated_{tag}"] = {
            "ms": ms, "iters": inf.iters, "passes": inf.passes, "status": int(inf.status),
            "elem_iter_per_s": n * inf.iters / (ms * 1e-3), "GBps": byt / (ms * 1e-3) / 1e9,
            "frac": byt / (ms * 1e-3) / 1e9 / peak,
            "arithmetic": "per element: double-float (hi + lo float pair, ~2^-46 relative) for FP64 data in "
                          "[2^-60, 2^60], exact FP64 outside; FP32 with a double-float multiplier for FP32 "
                          "data; lambda and the sums FP64 (double-float partial sums flushed into FP64)"}
        if args.oracle_check:
            sols[tag] = ([p[k].double().cpu().numpy() for k in "abdlu"], p["r"], xg.double().cpu().numpy())
        del p, xg
        torch.cuda.empty_cache()
    if args.oracle_check:
        import oracle
        tags = list(sols)
        exact = pool_map(lambda t: oracle.solve_sort(*sols[t][0], sols[t][1]), tags)
        for t, e in zip(tags, exact):
            host, r, xh = sols[t]
            res[f"general_correlated_{t}"]["err_vs_oracle"] = err_general(host, r, xh, e, t)
        del sols, exact
    return res


def config0(api, W, dev, stream, oracle_check=True):
    """The latency-bound single solve: general CQK, box family, n = 10,000, FP64 (400 KB per
    iteration, L2-resident).  Each solve is timed alone with CUDA events: 50 with the data
    warm in L2, 20 after a write of 256 MiB (larger than L2) that evicts it; and 20 solves
    captured in one CUDA graph (launch gaps removed)."""
    import statistics as st

    import torch
    n = 10_000
    p = W.uncorrelated_box(n, seed=0, device=dev)
    x = torch.empty_like(p["a"])
    ws = api.Workspace(n, 1, p["a"].dtype, dev)

    def solve(s=None):
        api.solve(p["a"], p["b"], p["d"], p["l"], p["u"], p["r"], out=x, ws=ws, sync=False, stream=s)

    for _ in range(5):
        solve()
    torch.cuda.synchronize()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(reps, cold):
        out = []
        for _ in range(reps):
            if cold:
                flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            solve()
            b.record(stream)
            b.synchronize()
            out.append(a.elapsed_time(b) * 1e3)
        return out

    warm = timed(50, False)
    cold = timed(20, True)
    graph_us = None
    try:
        g = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream(dev)
        cs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cs):
            solve(cs)
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=cs):
                for _ in range(20):
                    solve(cs)
        graph_us = _time(g.replay, torch.cuda.current_stream(), reps=10) * 1e3 / 20
    except Exception as e:  # noqa: BLE001
        graph_us = f"capture failed: {type(e).__name__}: {e}"
    inf = ws.read_info()
    res = {"workload": "general CQK, box family (d~U[1,100], b~U[10,25], a~U[-10,10], l~U[-5,0], "
                       "u=l+U[0.5,5], r=b'(l+u)/2), n=10000, FP64, seed 0",
           "iters": inf.iters, "passes": inf.passes, "status": int(inf.status),
           "us_warm_min": min(warm), "us_warm_median": st.median(warm),
           "us_cold_min": min(cold), "us_cold_median": st.median(cold),
           "us_per_solve_graph": graph_us,
           "elem_iter_per_s_warm": n * inf.iters / (st.median(warm) * 1e-6),
           "elem_iter_per_s_cold": n * inf.iters / (st.median(cold) * 1e-6),
           "l2": "warm: data resident in L2; cold: 256 MiB written before each solve"}
    if oracle_check:
        import oracle
        host = [p[k].cpu().numpy() for k in "abdlu"]
        res["err_vs_oracle"] = err_general(host, p["r"], x.cpu().numpy(), oracle.solve_sort(*host, p["r"]), "f64")
        # the sequential oracle (Alg. 1 from eq. (CQKlambda0)) on one core, same instance, for context
        t = []
        for _ in range(20):
            t0 = time.perf_counter()
            oracle.newton_cqk(*host, p["r"])
            t.append(time.perf_counter() - t0)
        res["cpu_oracle_us_min_1core"] = min(t) * 1e6
    del flush
    return res


def batched_extras(api, W, dev, stream, oracle_check=True):
    """The batched, differentiable workloads: forward + backward of a ragged batch in two
    launches (captured once in a CUDA graph and replayed) against the same solves issued as
    one forward and one backward launch per instance, from Python and captured in one CUDA
    graph; the options the autotuner picks for the batch against the defaults; the achieved
    bandwidth at the algorithmic bytes; and the error of every instance against the oracle.
      simplex: 4096 instances, lengths log-uniform in [16, 2^20], FP32 y ~ N(0,1), r = 1
      general: 256 instances, lengths log-uniform in [1e3, 1e6], FP64 uncorrelated box"""
    import numpy as np
    import torch

    from paper_2603_15910_b300 import tune
    peak, _ = measured_peak_hbm()
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
        grads = {k: torch.empty_like(vec) for k in (("a", "b", "d", "l", "u") if general else ("y",))}
        gr = torch.empty(B, dtype=torch.float64, device=dev)
        st = torch.empty(B, dtype=torch.int32, device=dev)
        lib = api.library()
        P = api.ptr
        code = api.dtype_code(vec.dtype)
        es = vec.element_size()

        def fwd_bwd(s=None, opt=None, opt_b=None):
            opt = opt or api.make_options()
            opt_b = opt_b or opt
            sh = api.stream_handle(s or stream)
            if general:
                rc = lib.cqk_solve_batched(B, P(off), code, P(d["a"]), P(d["b"]), P(d["d"]), P(d["l"]), P(d["u"]),
                                           P(r), P(x), P(mask), P(ws.info), api.ctypes.byref(opt), P(ws.buf),
                                           ws.nbytes, sh)
                api.check_rc(rc, "cqk_solve_batched")
                rc = lib.cqk_backward(B, P(off), n, code, P(g), P(x), P(d["a"]), P(d["b"]), P(d["d"]), P(d["l"]),
                                      P(d["u"]), P(mask), P(ws.info), P(grads["a"]), P(grads["b"]), P(grads["d"]),
                                      P(grads["l"]), P(grads["u"]), P(gr), P(st), api.ctypes.byref(opt_b),
                                      P(ws.buf), ws.nbytes, sh)
                api.check_rc(rc, "cqk_backward")
            else:
                rc = lib.cqk_project_simplex_batched(B, P(off), code, P(d["y"]), P(r), P(x), P(mask), P(ws.info),
                                                     api.ctypes.byref(opt), P(ws.buf), ws.nbytes, sh)
                api.check_rc(rc, "cqk_project_simplex_batched")
                rc = lib.cqk_backward_simplex(B, P(off), n, code, P(g), P(x), P(mask), P(ws.info), P(grads["y"]),
                                              P(gr), P(st), api.ctypes.byref(opt_b), P(ws.buf), ws.nbytes, sh)
                api.check_rc(rc, "cqk_backward_simplex")

        def graph_of(fn):
            gph = torch.cuda.CUDAGraph()
            cs = torch.cuda.Stream(dev)
            cs.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(cs):
                fn(cs)
                torch.cuda.synchronize()
                with torch.cuda.graph(gph, stream=cs):
                    fn(cs)
            torch.cuda.synchronize()
            return gph

        ms_batched = _time(fwd_bwd, stream)
        infos = ws.read_infos(B)
        ok = sum(int(i.status) == 0 for i in infos)
        try:
            graph_ms = _time(graph_of(fwd_bwd).replay, torch.cuda.current_stream())
        except Exception as e:  # capture unsupported: report, do not fail the bench
            graph_ms = f"capture failed: {type(e).__name__}: {e}"
        best_ms = graph_ms if isinstance(graph_ms, float) else ms_batched
        # algorithmic bytes of the forward (per instance: its passes) and of the adjoint
        offs = off.cpu().tolist()
        lens = [offs[k + 1] - offs[k] for k in range(B)]
        if general:
            fwd_bytes = sum(es * m * (3 + 5 * (i.passes - 2) + 6) + m / 8 for m, i in zip(lens, infos) if m)
            bwd_bytes = sum(es * m * (3 + 6 + 5) + m / 4 for m in lens)  # g,b,d | g,x,b,d,l,u -> 5 grads
        else:
            fwd_bytes = sum(es * m * (i.passes + 1) + m / 8 for m, i in zip(lens, infos) if m)
            bwd_bytes = sum(es * m * 3 + m / 4 for m in lens)  # g | g -> gy, mask read twice
        alg = fwd_bytes + bwd_bytes
        # per-instance launches (one forward + one backward per instance), same arrays
        rl = d["r"].cpu().tolist()
        ws1 = api.Workspace(max(lens), 1, vec.dtype, dev)
        info1 = ws1.info
        opt1 = api.make_options()

        def per_instance(s=None):
            sh = api.stream_handle(s or stream)
            for k in range(B):
                lo, hi = offs[k], offs[k + 1]
                m = hi - lo
                if m == 0:
                    continue
                if general:
                    ap = [P(d[q][lo:hi]) for q in ("a", "b", "d", "l", "u")]
                    lib.cqk_solve(m, code, *ap, float(rl[k]), P(x[lo:hi]), None, P(info1), api.ctypes.byref(opt1),
                                  P(ws1.buf), ws1.nbytes, sh)
                    lib.cqk_backward(1, None, m, code, P(g[lo:hi]), P(x[lo:hi]), *ap, None, P(info1),
                                     P(grads["a"][lo:hi]), P(grads["b"][lo:hi]), P(grads["d"][lo:hi]),
                                     P(grads["l"][lo:hi]), P(grads["u"][lo:hi]), P(gr[k:k + 1]), P(st[k:k + 1]),
                                     api.ctypes.byref(opt1), P(ws1.buf), ws1.nbytes, sh)
                else:
                    lib.cqk_project_simplex(m, code, P(d["y"][lo:hi]), float(rl[k]), P(x[lo:hi]), None, P(info1),
                                            api.ctypes.byref(opt1), P(ws1.buf), ws1.nbytes, sh)
                    lib.cqk_backward_simplex(1, None, m, code, P(g[lo:hi]), P(x[lo:hi]), None, P(info1),
                                             P(grads["y"][lo:hi]), P(gr[k:k + 1]), P(st[k:k + 1]),
                                             api.ctypes.byref(opt1), P(ws1.buf), ws1.nbytes, sh)

        ms_loop = _time(per_instance, stream, reps=2)
        try:
            ms_loop_graph = _time(graph_of(per_instance).replay, torch.cuda.current_stream(), reps=3)
        except Exception as e:  # noqa: BLE001
            ms_loop_graph = f"capture failed: {type(e).__name__}: {e}"
        # the autotuner on this batch: forward + backward with the options it picks
        kind = "general" if general else "simplex"
        arrays = tuple(d[q] for q in ("a", "b", "d", "l", "u")) if general else (d["y"],)
        t0 = time.perf_counter()
        best_f, best_b, t_f, t_b = tune.tune_fwd_bwd(kind, *arrays, offsets=off, r=r, g=g, reps=2)
        tune_s = time.perf_counter() - t0
        tune.clear()
        ms_tuned = _time(lambda s=None: fwd_bwd(s, api.make_options(**best_f), api.make_options(**best_b)), stream)
        entry = {"instances": B, "n_total": n, "dtype": str(vec.dtype).replace("torch.", ""),
                 "ms_fwd_bwd_batched": ms_batched, "ms_fwd_bwd_graph": graph_ms,
                 "ms_fwd_bwd_tuned": ms_tuned, "tuned_options": {"forward": best_f, "adjoint": best_b},
                 "tuned_ms": {"forward_best": t_f[0][0], "adjoint_best": t_b[0][0],
                              "forward_worst": t_f[-1][0], "adjoint_worst": t_b[-1][0]},
                 "speedup_tuned_vs_default": ms_batched / ms_tuned,
                 "tuning_seconds": tune_s, "tuning_candidates": len(t_f) + len(t_b),
                 "ms_fwd_bwd_per_instance_launches": ms_loop, "ms_fwd_bwd_per_instance_graph": ms_loop_graph,
                 "speedup_vs_per_instance_launches": ms_loop / best_ms,
                 "speedup_vs_per_instance_graph": (ms_loop_graph / best_ms if isinstance(ms_loop_graph, float)
                                                   else None),
                 "instances_ok": ok, "mean_iters": sum(i.iters for i in infos) / B,
                 "elements_per_s_fwd_bwd": n / (best_ms * 1e-3),
                 "roofline": {"bound": "hbm", "algorithmic_bytes": alg, "fwd_bytes": fwd_bytes,
                              "bwd_bytes": bwd_bytes, "achieved": alg / (best_ms * 1e-3) / 1e9, "unit": "GB/s",
                              "peak": peak, "frac": alg / (best_ms * 1e-3) / 1e9 / peak,
                              "basis": "forward: every pass streams the instance's arrays (info.passes), the final "
                                       "pass writes x and the mask; adjoint: two passes (DESIGN table)"}}
        if oracle_check:
            fwd_bwd()  # default options: the results checked below
            torch.cuda.synchronize()
            entry["err_vs_oracle"] = _batch_errors(general, d, x, grads, gr, offs, B, vec.dtype)
        res[name] = entry
        del d, x, mask, ws, grads, ws1
        torch.cuda.empty_cache()
    return res


def _batch_errors(general, d, x, grads, gr, offs, B, dtype):
    """Per-instance error of the forward and of the adjoint against the oracle (exact solution;
    implicit-function gradient at the oracle's own solution), worst over the batch."""
    import numpy as np

    import oracle
    dt = "f64" if dtype.itemsize == 8 else "f32"
    xs = x.double().cpu().numpy()
    grs = gr.cpu().numpy()
    gs = d["g"].double().cpu().numpy()
    if general:
        host = {k: d[k].double().cpu().numpy() for k in "abdlu"}
        gh = {k: grads[k].double().cpu().numpy() for k in "abdlu"}
        rs = d["r"].cpu().numpy()

        def one(k):
            s = slice(offs[k], offs[k + 1])
            hk = [host[q][s] for q in "abdlu"]
            ex = oracle.solve_sort(*hk, float(rs[k]))
            e = err_general(hk, float(rs[k]), xs[s], ex, dt)
            ref = oracle.grad_cqk(ex[2], ex[1], *hk, gs[s])
            e["grad_rel"] = max(_x_rel(gh[q][s], ref[q]) for q in "abdlu")
            e["grad_r_rel"] = abs(grs[k] - ref["r"]) / (1 + abs(ref["r"]))
            return e
    else:
        ys = d["y"].double().cpu().numpy()
        gy = grads["y"].double().cpu().numpy()

        def one(k):
            s = slice(offs[k], offs[k + 1])
            lam, xstar = oracle.project_simplex_sort(ys[s], 1.0)
            e = err_projection(xs[s], xstar, 1.0, dt)
            ref = oracle.grad_simplex(xstar, gs[s])
            e["grad_rel"] = _x_rel(gy[s], ref["y"])
            e["grad_r_rel"] = abs(grs[k] - ref["r"]) / (1 + abs(ref["r"]))
            return e

    items = [e for e in pool_map(one, [k for k in range(B) if offs[k + 1] > offs[k]])]
    out = _max_err(items)
    out["tol_grad"] = 1e-10 if dt == "f64" else 1e-5
    out["grad_basis"] = "oracle gradient at the oracle's own solution; an element whose free status is a tie " \
                        "would show here as a large grad_rel"
    return out


# ------------------------------------------------------------------------------ oracle timing
def _oracle_step(y, threads):
    """One step of the CPU method on y: simplex and l1 projection, each by Alg. 2 then Alg. 4
    (one thread: Alg. 2 over all of y; several: Alg. 2 per contiguous chunk, one chunk per
    thread, and lambda_0 from the union of the J's, Sec. 4).  Returns phi evaluations."""
    import oracle
    n = y.shape[0]
    evals = 0
    for l1 in (False, True):
        if threads == 1:
            lam0, _, _ = oracle.condat_init(y, 1.0, l1=l1)
        else:
            lam0, _, _ = oracle.condat_chunks(y, 1.0, (n + threads - 1) // threads, threads, l1=l1)
        evals += oracle.newton_simplex(y, 1.0, lam0=lam0, l1=l1)["evals"]
    return evals


def _time_oracle(y, threads, max_seconds, min_reps=3):
    """Min and median seconds per step over repetitions (the paper's protocol: the minimum over
    repeated runs), and the phi evaluations of a step."""
    import oracle
    prev = oracle.reference.set_threads(threads)
    try:
        times, evals = [], 0
        t_start = time.perf_counter()
        while True:
            t0 = time.perf_counter()
            evals = _oracle_step(y, threads)
            times.append(time.perf_counter() - t0)
            if len(times) >= min_reps and time.perf_counter() - t_start > max_seconds:
                break
            if len(times) >= 50:
                break
    finally:
        oracle.reference.set_threads(prev)
    return min(times), statistics.median(times), evals, len(times)


def cpu_baseline(y):
    """The FP64 oracle on the host cores for the same two projections: the sequential oracle
    (Alg. 2 + Alg. 4) on one core on the first 2e7 elements; the same algorithms with
    OpenMP-parallel passes and per-thread Alg. 2 chunks (the paper's CPU Jacobi form) on all
    cores on the whole vector; and the sort-based projection on one core."""
    import oracle
    oracle.reference.build()
    n = y.shape[0]
    cores = host_cores()
    t_min, t_med, evals, reps = _time_oracle(y, cores, max_seconds=10.0)
    one = y[:CPU_SAMPLE]
    o_min, o_med, o_evals, o_reps = _time_oracle(one, 1, max_seconds=8.0, min_reps=2)
    t0 = time.perf_counter()
    oracle.project_simplex_sort(one, 1.0)
    sort_s = time.perf_counter() - t0
    return {"value": n * evals / t_min, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"the whole n={n} vector, simplex + l1 per step, Alg. 2 per thread chunk ({cores} chunks) "
                      f"+ Alg. 4 with OpenMP map-reduce passes; min over {reps} steps",
            "seconds_per_step_min": t_min, "seconds_per_step_median": t_med, "phi_evaluations_per_step": evals,
            "cpu_model": cpu_model(),
            "one_core": {"value": one.shape[0] * o_evals / o_min, "unit": UNIT, "cores": 1,
                         "sample": f"first {one.shape[0]} elements, sequential Alg. 2 + Alg. 4, min over "
                                   f"{o_reps} steps", "seconds_per_step_min": o_min,
                         "seconds_per_step_median": o_med},
            "sort_oracle_one_core": {"seconds_per_projection": sort_s, "elements": one.shape[0],
                                     "elements_per_s": one.shape[0] / sort_s,
                                     "what": "textbook sort-based simplex projection (the exact checker)"}}


def run_reference(args, world, rank):
    if rank != 0:
        return None
    from paper_2603_15910_b300 import workloads as W
    import oracle
    oracle.reference.build()
    y = W.simplex_normal(args.n, seed=0, device="cpu").numpy()
    cores = host_cores()
    prev = oracle.reference.set_threads(cores)
    try:
        for _ in range(min(args.warmup, 1)):
            _oracle_step(y[:1_000_000], cores)
        times, evals = [], 0
        t_start = time.perf_counter()
        for _ in range(args.steps):
            t0 = time.perf_counter()
            evals = _oracle_step(y, cores)
            times.append(time.perf_counter() - t0)
            if time.perf_counter() - t_start > 150:
                break
    finally:
        oracle.reference.set_threads(prev)
    ms = 1e3 * sum(times) / len(times)
    v = args.n * evals * len(times) / sum(times)
    cb = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
          "sample": f"the whole n={args.n} vector (y~N(0,1) from the CPU generator), simplex + l1 per step, "
                    f"Alg. 2 per thread chunk + Alg. 4 with OpenMP map-reduce passes on {cores} cores"}
    return {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": len(times), "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "simplex + l1-ball projection, n=1e8, FP64, y~N(0,1), r=1, Condat start",
                       "n": args.n},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_case(args):
    """One side workload alone (see the module docstring), for profiling."""
    import torch

    from paper_2603_15910_b300 import api, workloads as W
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    out = {"case": args.case}

    def timed(f, reps):
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            f()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    if args.case == "general":
        n = args.n
        for dt, tag in ((torch.float64, "f64"), (torch.float32, "f32")):
            p = W.correlated(n, seed=0, device=dev, dtype=dt)
            x = torch.empty_like(p["a"])
            ws = api.Workspace(n, 1, dt, dev)

            def f():
                api.solve(p["a"], p["b"], p["d"], p["l"], p["u"], p["r"], out=x, ws=ws, sync=False)
            f()
            ms = timed(f, 7)
            inf = ws.read_info()
            out[tag] = {"ms": ms, "passes": inf.passes, "iters": inf.iters, "status": int(inf.status)}
            del p, x
            torch.cuda.empty_cache()
    else:
        B = args.batch
        if args.case == "batched_simplex":
            d = W.batched_simplex(batch=B, lo=16, hi=1 << 20, seed=0, device=dev, dtype=torch.float32)
            ws = api.Workspace(d["y"].numel(), B, torch.float32, dev)

            def f():
                x, _, m = api.project_simplex_batched(d["y"], d["offsets"], d["r"], want_mask=True, ws=ws,
                                                      sync=False, use_tuning=False)
                api.backward("simplex", d["g"], x, ws.info, offsets=d["offsets"], mask=m, ws=ws, use_tuning=False)
        else:
            d = W.batched_general(batch=B, lo=1000, hi=1000000, seed=0, device=dev)
            ws = api.Workspace(d["a"].numel(), B, torch.float64, dev)
            arr = [d[k] for k in "abdlu"]

            def f():
                x, _, m = api.solve_batched(*arr, d["offsets"], d["r"], want_mask=True, ws=ws, sync=False,
                                            use_tuning=False)
                api.backward("general", d["g"], x, ws.info, offsets=d["offsets"], mask=m, ws=ws, use_tuning=False,
                             **dict(zip("abdlu", arr)))
        out["ms_fwd_bwd"] = [timed(f, 1), timed(f, 1)]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--no-extras", dest="extras", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-oracle-check", dest="oracle_check", action="store_false")
    ap.add_argument("--case", default=None, choices=["general", "batched_simplex", "batched_general"])
    ap.add_argument("--batch", type=int, default=1024)
    args = ap.parse_args()
    if args.case:
        print(json.dumps(run_case(args)), flush=True)
        return
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
