"""In-tree build of the CUDA library libmpr.so for sm_103a (nvcc, no cmake).

Each translation unit is compiled in parallel, then linked into
``_build/libmpr.so`` next to this file.  Rebuilds only what changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmpr.so")
SOURCES = ["mpr_api.cu", "mpr_tiled.cu", "mpr_tiled_32x16.cu", "mpr_tiled_16x16.cu",
           "mpr_tiled_16x16_lit.cu", "mpr_tiled_16x16_gmrf.cu",
           "mpr_tiled_32x32.cu", "mpr_plain.cu", "mpr_lattice.cu", "mpr_noalloc.cu",
           "mpr_qcv.cu"]
HEADERS = ["mpr_device.cuh", "mpr_internal.h", "mpr_async.cuh", "mpr_tiled_kernel.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-ftz=true", "-Xcompiler", "-fPIC",
         "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _mtime(p):
    return os.path.getmtime(p) if os.path.exists(p) else 0.0


def build(verbose: bool = False, extra_flags=None) -> str:
    """Compile every translation unit (in parallel) and link libmpr.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    inc = os.path.join(os.path.dirname(HERE), "include")
    deps = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(inc, "mpr.h")]
    flags = FLAGS + list(extra_flags or [])
    # a change of flags rebuilds everything
    stamp = os.path.join(BUILD, "flags.txt")
    sig = " ".join(ARCH + flags)
    old = open(stamp).read() if os.path.exists(stamp) else ""
    if old != sig:
        with open(stamp, "w") as f:
            f.write(sig)
    deps.append(stamp)
    dep_time = max(_mtime(d) for d in deps)

    def compile_one(src):
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        if _mtime(o) > max(_mtime(s), dep_time) and not extra_flags:
            return o, False
        cmd = [nvcc, *ARCH, *flags, "-I", inc, "-c", s, "-o", o]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr.strip():
            print(r.stderr, file=sys.stderr)
        return o, True

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    objs = [o for o, _ in results]
    if any(changed for _, changed in results) or _mtime(LIB) < max(_mtime(o) for o in objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
