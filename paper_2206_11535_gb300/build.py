"""Build libm3e.so in-tree with nvcc for sm_103a (no torch extension machinery).

The translation units compile in parallel; the result is
``paper_2206_11535_gb300/libm3e.so``.  Flags: the approximate (non-IEEE) FP32
division and square root (CUDA's documented few-ulp forms, about 1e-7 relative,
far inside the FP32-vs-FP64 tolerances of the parity tests), no flush-to-zero,
no fast-math intrinsics for the transcendental functions.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libm3e.so")
UNITS = ["m3e_staged.cu", "m3e_fused.cu", "m3e_stream.cu", "m3e_grad.cu", "m3e_ingest.cu", "m3e_abi.cu"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
         "--prec-div=false", "--prec-sqrt=false", "-ftz=false", "--fmad=true",
         "-Xcompiler", "-fPIC", "-Xcompiler", "-pthread", "-I" + os.path.join(ROOT, "include")]


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, src_dir: str = SRC, out: str = OUT) -> str:
    """Compile the units of ``src_dir`` and link ``out`` (defaults: this package)."""
    hdrs = [os.path.join(src_dir, "m3e_internal.cuh"), os.path.join(src_dir, "m3e_device.cuh"),
            os.path.join(ROOT, "include", "m3e.h"), __file__]
    objs = []
    jobs = []
    for u in UNITS:
        src = os.path.join(src_dir, u)
        obj = os.path.join(src_dir, u.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [src] + hdrs):
            jobs.append([NVCC] + FLAGS + (["-Xptxas", "-v"] if verbose else []) + ["-c", src, "-o", obj])
    with ThreadPoolExecutor(len(jobs) or 1) as ex:
        for r in ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs):
            if r.returncode != 0:
                raise RuntimeError("nvcc failed:\n" + r.stdout + r.stderr)
            if verbose:
                sys.stderr.write(r.stderr)
    if force or jobs or _stale(out, objs):
        subprocess.check_call([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-cudart", "static",
                               "-Xcompiler", "-pthread", "-o", out] + objs)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
