"""Build step for libvx.so: compiles csrc/*.cu for sm_103a with nvcc and
csrc/*.cpp with g++, then links one shared library next to this file.

Incremental: an object is rebuilt when its source or any header is newer.
Usage: python -m paper_2410_14128_b300._build [--force] [-j N]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libvx.so")
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
                     "--expt-relaxed-constexpr", f"-I{INCLUDE}"]
GXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-Wall", "-fopenmp", f"-I{INCLUDE}", f"-I{CUDA_HOME}/include"]


def _headers():
    return glob.glob(os.path.join(CSRC, "*.hpp")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(src: str, obj: str, hdr_mtime: float) -> bool:
    if not os.path.exists(obj):
        return True
    m = os.path.getmtime(obj)
    return m < os.path.getmtime(src) or m < hdr_mtime


def _compile(src: str, obj: str):
    if src.endswith(".cu"):
        cmd = [NVCC, *NVCC_FLAGS, *_extra_nvcc_flags(), "-c", src, "-o", obj]
    else:
        cmd = ["g++", *GXX_FLAGS, "-c", src, "-o", obj]
    p = subprocess.run(cmd, capture_output=True, text=True)
    log = obj + ".log"
    with open(log, "w") as f:
        f.write(" ".join(cmd) + "\n" + p.stdout + p.stderr)
    if p.returncode != 0:
        raise RuntimeError(f"compile failed: {src}\n{p.stdout}\n{p.stderr}")
    return src


def _extra_nvcc_flags():
    """Extra nvcc flags from VX_NVCC_FLAGS (e.g. -DVX_CACHE_TN=0)."""
    return os.environ.get("VX_NVCC_FLAGS", "").split()


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    hdr = max((os.path.getmtime(h) for h in _headers()), default=0.0)
    objs, todo = [], []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s) + ".o")
        objs.append(o)
        if force or _stale(s, o, hdr):
            todo.append((s, o))
    if todo:
        n = jobs or min(len(todo), os.cpu_count() or 1)
        with cf.ThreadPoolExecutor(max_workers=n) as ex:
            for s in ex.map(lambda so: _compile(*so), todo):
                if verbose:
                    print("compiled", os.path.relpath(s, HERE), file=sys.stderr)
    if todo or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + ".tmp"
        cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lgomp", "-lpthread", "-ldl", "-lrt"]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"link failed\n{p.stdout}\n{p.stderr}")
        os.replace(tmp, LIB)
    return LIB


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("-j", type=int, default=None)
    a = ap.parse_args()
    print(build(force=a.force, jobs=a.j, verbose=True))


if __name__ == "__main__":
    main()
