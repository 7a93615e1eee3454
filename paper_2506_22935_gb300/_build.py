"""Builds ``libgraf.so`` (the C-ABI CUDA library) in-tree for sm_103a.

Generates the twiddle tables, compiles every ``csrc/*.cu`` translation unit
in parallel with nvcc (one -gencode, arch=compute_103a, code=sm_103a) and
links them into ``paper_2506_22935_gb300/libgraf.so``.  Rebuilds only when a
source is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgraf.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fvisibility=hidden"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgraf.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.py"))
            + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)])


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in _deps())


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    if not force and not needs_build():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    subprocess.check_call([sys.executable, os.path.join(CSRC, "gen_twiddles.py"),
                           os.path.join(BUILD, "twiddles.inc")])
    srcs = _sources()
    objs = [os.path.join(BUILD, os.path.basename(s)[:-3] + ".o") for s in srcs]
    extra = ["-Xptxas", "-v"] if verbose else []

    def compile_one(src_obj):
        src, obj = src_obj
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-I", CSRC, "-I", BUILD, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
        return r.stdout + r.stderr

    # the largest translation units first, so the parallel build ends sooner
    prio = ["graf_af_m64", "graf_af_m16384", "graf_af_m8192", "graf_af_m4096", "graf_af_m2048", "graf_af_m1024",
            "graf_af_m32", "graf_af_m512", "graf_af_m256", "graf_af_m128"]

    def rank(so):
        name = os.path.basename(so[0])[:-3]
        return prio.index(name) if name in prio else len(prio)

    order = sorted(zip(srcs, objs), key=rank)
    jobs = jobs or max(1, min(len(order), os.cpu_count() or 1))
    logs = []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        for log in ex.map(compile_one, order):
            logs.append(log)
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    if verbose:
        print("\n".join(logs))
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
