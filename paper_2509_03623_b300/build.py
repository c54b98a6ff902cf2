"""Build librt_b300.so (all CUDA sources under csrc/) for sm_103a with nvcc.

Each source compiles to its own object under _build/ (in parallel; a source is recompiled when
it, a header under csrc/ or include/, or this file is newer than its object), then nvcc links
the shared library.

Usage: python -m paper_2509_03623_b300.build [--force] [-v]
"""

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OBJ = os.path.join(os.path.dirname(HERE), "_build")
LIB = os.path.join(HERE, "librt_b300.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-warn-spills"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + sorted(
        glob.glob(os.path.join(INCLUDE, "*.h"))) + [os.path.abspath(__file__)]


def deps():
    return sources() + headers()


def _obj(src):
    return os.path.join(OBJ, os.path.basename(src) + ".o")


def build(force: bool = False, verbose: bool = False) -> str:
    newest_hdr = max(os.path.getmtime(p) for p in headers())
    os.makedirs(OBJ, exist_ok=True)
    stale = [s for s in sources()
             if force or not os.path.exists(_obj(s))
             or os.path.getmtime(_obj(s)) < max(newest_hdr, os.path.getmtime(s))]
    objs = [_obj(s) for s in sources()]
    if not stale and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
            os.path.getmtime(o) for o in objs):
        return LIB

    def compile_one(src):
        tmp = _obj(src) + ".tmp%d" % os.getpid()
        cmd = [NVCC] + ARCH + FLAGS + ["-I", INCLUDE, "-c", "-o", tmp, src]
        if verbose:
            cmd += ["-Xptxas", "-v"]
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
        os.replace(tmp, _obj(src))

    with ThreadPoolExecutor(max_workers=min(len(stale), os.cpu_count() or 1) or 1) as ex:
        for f in [ex.submit(compile_one, s) for s in stale]:
            f.result()
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call([NVCC] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
