"""Build libeik.so in-tree with nvcc for sm_103a (B300).

    python -m paper_2609_14982_b300.build [--force] [--checked]

--checked builds libeik_checked.so instead: the same library compiled with -DEIK_CHECKED,
whose traversal kernels check every index they gather through and report a bad one as a
device fault (EIK_ERR_CUDA from tangent_status) instead of reading out of bounds.  Load it
by setting EIK_LIB to its path before importing the binding.

Every .cu file under csrc/ is compiled to an object and linked into one shared
library next to this file.  eik_setup.cu and eik_forward.cu are compiled without
fused multiply-adds (-fmad=false): the sign decisions of the upwind rows and the
iterates of the state solve follow a fixed sequence of IEEE operations.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libeik.so")
LIB_CHECKED = os.path.join(HERE, "libeik_checked.so")
BUILD_DIR = os.path.join(ROOT, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NO_FMAD = {"eik_setup.cu", "eik_forward.cu", "eik_points.cu"}


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _digest() -> str:
    h = hashlib.sha256()
    for f in _sources() + sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))) + \
            [os.path.join(INCLUDE, "eik.h"), __file__]:
        h.update(open(f, "rb").read())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib_out = LIB_CHECKED if checked else LIB
    build_dir = BUILD_DIR + ("_checked" if checked else "")
    stamp = lib_out + ".sha256"
    dig = _digest()
    if not force and os.path.exists(lib_out) and os.path.exists(stamp) and open(stamp).read().strip() == dig:
        return lib_out
    os.makedirs(build_dir, exist_ok=True)
    objs, cmds = [], []
    for src in _sources():
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
               *(["-DEIK_CHECKED"] if checked else []), "-c", src, "-o", obj]
        if os.path.basename(src) in NO_FMAD:
            cmd.insert(-4, "-fmad=false")
        if verbose:
            cmd.insert(-4, "-Xptxas=-v")
            print(" ".join(cmd), flush=True)
        cmds.append(cmd)
        objs.append(obj)
    # the translation units compile independently: run them side by side
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=max(1, min(len(cmds), os.cpu_count() or 1))) as pool:
        for f in [pool.submit(subprocess.check_call, c) for c in cmds]:
            f.result()
    tmp = lib_out + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
    os.replace(tmp, lib_out)
    with open(stamp, "w") as f:
        f.write(dig)
    return lib_out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("-v", "--verbose", action="store_true")
    ap.add_argument("--checked", action="store_true", help="build libeik_checked.so (-DEIK_CHECKED)")
    a = ap.parse_args()
    print(build(force=a.force, verbose=a.verbose, checked=a.checked))
    sys.exit(0)
