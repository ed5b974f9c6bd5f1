"""Builds libmdn.so (all CUDA kernels + the C ABI) for sm_103a, in tree.

Each translation unit under csrc/ is compiled by nvcc in parallel, then
linked into paper_1802_06130_gb300/_build/libmdn.so with the static CUDA
runtime.  Rebuilds only what changed (object newer than its source and every
header).

build(check=True) makes the bounds-checked debug library instead
(_build_check/libmdn_check.so, -DMDN_CHECK): every checked shared- and
global-memory index is tested against its buffer, and the first violation is
recorded (site and index, read by mdn_check_status) and its access skipped.
Relocatable device code lets one device status word serve every unit.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmdn.so")
BUILD_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(BUILD_CHECK, "libmdn_check.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-warn-spills"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _newest_header() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return max(os.path.getmtime(h) for h in hs)


def build(verbose: bool = False, jobs: int | None = None, check: bool = False) -> str:
    bdir, lib = (BUILD_CHECK, LIB_CHECK) if check else (BUILD, LIB)
    extra = ["-DMDN_CHECK", "-rdc=true"] if check else []
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdr = _newest_header()
    todo = []
    objs = []
    for s in srcs:
        o = os.path.join(bdir, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr):
            todo.append((s, o))

    def one(so):
        s, o = so
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-I", INCLUDE, "-c", s, "-o", o + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(s)}:\n{r.stderr}")
        os.replace(o + ".tmp", o)
        return r.stderr

    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs or min(len(todo), os.cpu_count() or 4)) as ex:
            for log in ex.map(one, todo):
                if verbose and log.strip():
                    print(log)
    if todo or not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        tmp = lib + f".{os.getpid()}.tmp"
        link_rdc = ["-rdc=true"] if check else []
        cmd = [nvcc, *ARCH, *link_rdc, "-shared", "-cudart=static", "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True))
