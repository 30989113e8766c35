"""In-tree build of libqem.so for sm_103a (nvcc, no cmake).

Each CUDA translation unit compiles in parallel to an object under _build/,
then one link step writes paper_2503_08264_gb300/libqem.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libqem.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale(obj: str, deps: list) -> bool:
    return not os.path.exists(obj) or any(os.path.getmtime(d) > os.path.getmtime(obj) for d in deps)


def build(verbose: bool = False, extra: list | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdrs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    jobs = []
    for s in srcs:
        obj = os.path.join(BUILD, os.path.basename(s) + ".o")
        if _stale(obj, [s] + hdrs):
            cmd = [nvcc(), *ARCH, *FLAGS, *(extra or []), "-c", s, "-o", obj]
            jobs.append((s, cmd))
    def run(job):
        src, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        return r.stderr
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for log in ex.map(run, jobs):
            if verbose and log:
                print(log)
    objs = [os.path.join(BUILD, os.path.basename(s) + ".o") for s in srcs]
    if _stale(OUT, objs):
        tmp = OUT + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs])
        os.replace(tmp, OUT)
    return OUT


def build_unit_peaks() -> str:
    """Compile the unit-rate probe (probes/unit_peaks.cu, a standalone program
    that measures the per-SM rates behind the rooflines); returns its path."""
    src = os.path.join(HERE, "probes", "unit_peaks.cu")
    exe = os.path.join(BUILD, "unit_peaks")
    os.makedirs(BUILD, exist_ok=True)
    if _stale(exe, [src]):
        subprocess.check_call([nvcc(), *ARCH, "-O3", "-o", exe, src])
    return exe


if __name__ == "__main__":
    import sys
    print(build(verbose="-v" in sys.argv, extra=["-Xptxas", "-v"] if "-v" in sys.argv else None))
