"""In-tree build of the CUDA library (libipcheck.so) for sm_103a.

Every .cu file under csrc/ is compiled by its own nvcc process (in parallel) and the
objects are linked into paper_2405_04463_gb300/libipcheck.so. The device half of the
workload generator (synth/synth_gen.cu) is built the same way into synth/libsynth.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libipcheck.so")
SYNTH_SRC = os.path.join(ROOT, "synth", "synth_gen.cu")
SYNTH_LIB = os.path.join(ROOT, "synth", "libsynth.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, obj: str, extra=()):
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdrs = sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(ROOT, "include", "ipcheck.h")]
    jobs = []
    with cf.ThreadPoolExecutor(max_workers=max(2, min(len(srcs) + 1, os.cpu_count() or 4))) as ex:
        objs = []
        for s in srcs:
            o = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
            objs.append(o)
            if force or _stale(o, [s] + hdrs):
                jobs.append(ex.submit(_compile, s, o))
        synth_obj = os.path.join(BUILD, "synth_gen.o")
        if force or _stale(synth_obj, [SYNTH_SRC]):
            jobs.append(ex.submit(_compile, SYNTH_SRC, synth_obj))
        for j in jobs:
            j.result()
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    if force or _stale(SYNTH_LIB, [synth_obj]):
        tmp = SYNTH_LIB + f".tmp{os.getpid()}"
        r = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, synth_obj, "-lcudart"], capture_output=True,
                           text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, SYNTH_LIB)
    if verbose:
        print("built", LIB, SYNTH_LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
