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
            import pynvml
            pynvml.nvmlInit()
            self.nv = pynvml
            self.h = pynvml.nvmlDeviceGetHandleByPciBusId(self.bus.encode())
            self.max_mhz = pynvml.nvmlDeviceGetMaxClockInfo(self.h, pynvml.NVML_CLOCK_SM)
            self.source = "nvml"
        except Exception as e:  # noqa: BLE001
            self.nv = None
            self.error = f"nvml: {type(e).__name__}: {e}"

    def _run(self):
        while not self._stop.is_set():
            try:
                self.samples.append(self.nv.nvmlDeviceGetClockInfo(self.h, self.nv.NVML_CLOCK_SM))
                bits = self.nv.nvmlDeviceGetCurrentClocksEventReasons(self.h)
                self._bits(bits)
            except Exception as e:  # noqa: BLE001
                self.error = f"nvml sample: {type(e).__name__}: {e}"
            time.sleep(0.02)

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
        "config": {"workload": "simplex + l1-ball projection, n=1e8, FP64, y~N(0,1), r=1, Condat start "
                               "(Alg. 2 per warp chunk) then Alg. 4",
                   "n": n, "init": "condat", "projections_per_step": 2, "iters_simplex": i1.iters,
                   "iters_l1": i2.iters, "passes_simplex": i1.passes, "passes_l1": i2.passes,
                   "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (800 MB per vector)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "simplex_kernel<double> (simplex + l1 launches)",
                     "peak_source": peak_kind, "ms_simplex": t_s, "ms_l1": t_l,
                     "algorithmic_bytes": bytes_s + bytes_l, "frac_of_8TBs": achieved / 8000.0},
        "gpu_launches": 2 * K,
        "clocks": clk.summary(),
    }

    # end to end through the public API with host buffers: pinned y -> device, both
    # projections, both x -> pinned host, every step
    y_host = y.cpu().pin_memory()
    xh1 = torch.empty(n, dtype=y.dtype, pin_memory=True)
    xh2 = torch.empty(n, dtype=y.dtype, pin_memory=True)
    yd = torch.empty_like(y)

    def e2e_step():
        yd.copy_(y_host, non_blocking=True)
        api.project_simplex(yd, 1.0, init=api.Init.CONDAT, out=x1, ws=ws1, sync=False)
        api.project_l1(yd, 1.0, init=api.Init.CONDAT, out=x2, ws=ws2, sync=False)
        xh1.copy_(x1, non_blocking=True)
        xh2.copy_(x2, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    Ke = max(3, K // 2)
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(Ke):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    ems = e0.elapsed_time(e1)
    if world > 1:
        tt = torch.tensor([ems], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ems = float(tt.item())
    out["e2e"] = {"value": world * n * iters * Ke / (ems * 1e-3), "unit": UNIT, "h2d_bytes_per_step": 8 * n,
                  "d2h_bytes_per_step": 16 * n, "ms_per_step": ems / Ke}

    if args.extras and rank == 0:
        out["variants"] = extras(args, api, W, dev, stream)
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
