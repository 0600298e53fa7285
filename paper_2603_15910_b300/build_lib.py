"""Build libcqk.so (the CUDA library) in-tree with nvcc for sm_103a.

    python -m paper_2603_15910_b300.build_lib [--force]

Sources: csrc/*.cu; public header: include/cqk.h at the repository root.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libcqk.so")
BUILD = os.path.join(HERE, "_build")

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-fmad=false",  # no implicit contraction: every fused operation is an explicit fmaf
    "-Xcompiler", "-fPIC",
]


# Builds of the batched kernels besides the default one (suffix, preprocessor definitions,
# translation units): 128 and 512 threads per block for the general batch and the adjoints,
# and the half-unroll build of every batched kernel.  The autotuner chooses among them through
# cqk_options.block_threads and cqk_options.unroll.
VARIANTS = [
    ("_t128", ["-DCQK_NT=128"], ["cqk_batched.cu", "cqk_general.cu", "cqk_backward.cu"]),
    ("_t512", ["-DCQK_NT=512"], ["cqk_batched.cu", "cqk_general.cu", "cqk_backward.cu"]),
    ("_u", ["-DCQK_UNROLL_HALF"], ["cqk_batched.cu", "cqk_simplex.cu", "cqk_general.cu", "cqk_backward.cu"]),
]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def units():
    """(source, object, extra flags) of every translation unit of the library."""
    out = [(src, os.path.join(BUILD, os.path.basename(src) + ".o"), []) for src in sources()]
    for sfx, defs, files in VARIANTS:
        for f in files:
            out.append((os.path.join(CSRC, f), os.path.join(BUILD, f + sfx + ".o"),
                        [*defs, f"-DCQK_VARIANT={sfx}", "-DCQK_BATCH_ONLY"]))
    return out


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        [os.path.join(INCLUDE, "cqk.h"), __file__]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force=False, verbose=False):
    if not force and not _stale():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    os.makedirs(BUILD, exist_ok=True)
    cmds, objs = [], []
    for src, obj, extra in units():
        cmds.append([nvcc, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj])
        objs.append(obj)

    def compile_one(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)

    # translation units compile independently: one nvcc process per unit
    workers = max(1, min(len(cmds), os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as pool:
        for f in [pool.submit(compile_one, c) for c in cmds]:
            f.result()
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call([nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", *objs, "-o", tmp,
                           "-lcudart"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
