"""In-tree build of libmeta.so (sm_103a) with nvcc: one object per .cu, compiled
in parallel, then linked into a shared library next to this file."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from typing import List

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmeta.so")
# the bounds-checked debug build (-DMETA_CHECK_BOUNDS): the same sources, its own objects
BUILD_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(HERE, "libmeta_check.so")
SOURCES = ["meta_api.cu", "meta_blur.cu", "meta_step.cu", "meta_adjoint.cu", "meta_noalloc.cu",
           "meta_lbfgs.cu", "meta_persist.cu", "meta_tuning.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(extra: List[str]) -> List[str]:
    return ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2",
                   "-I", INCLUDE, "-I", CSRC] + extra


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "meta.h"),
                                                                 __file__]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, extra: List[str] = (),
          check: bool = False) -> str:
    """Compile every .cu for sm_103a and link libmeta.so (skipped when up to date).
    check=True: the bounds-checked debug build, libmeta_check.so (every data-dependent
    index -- feet, decoded record cells -- checked and clamped, violations latched in
    the workspace status word); load it with META_LIB=check."""
    lib, bdir = (LIB_CHECK, BUILD_CHECK) if check else (LIB, BUILD)
    if check:
        extra = list(extra) + ["-DMETA_CHECK_BOUNDS"]
    if not force and not _stale(lib):
        return lib
    nvcc = _nvcc()
    os.makedirs(bdir, exist_ok=True)
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc] + _flags(list(extra)) + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stdout.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(cmd[-3])
    if failed:
        raise RuntimeError("nvcc failed for %s" % ", ".join(failed))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-Xcompiler", "-fPIC", "-o", tmp] + objs + ["-ldl"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [])
