"""Build libpjds.so in-tree for sm_103a (GB300).

Each translation unit under csrc/ compiles in its own process (nvcc for .cu,
g++ for .cpp, both with OpenMP for the host converter), then nvcc links the
shared library with the static CUDA runtime. Objects go to csrc/_build/;
unchanged sources are not recompiled.

Run as ``python -m paper_1112_5588_gb300.build [--force] [--ptxas] [--checked]`` or call ``build()``;
``--checked`` builds libpjds_checked.so (device-side extent checks, a test build).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OBJDIR = os.path.join(CSRC, "_build")
LIB = os.path.join(HERE, "libpjds.so")
# the checked build (PJDS_CHECKED: device-side extent checks, a test build)
OBJDIR_CHECKED = os.path.join(CSRC, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libpjds_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpjds")


def _deps() -> list:
    return glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(
        os.path.join(INCLUDE, "*.h"))


def _stale(src: str, obj: str, deps: list) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src] + deps)


def _compile(src: str, verbose_ptxas: bool, objdir: str = OBJDIR, defines=()) -> str:
    obj = os.path.join(objdir, os.path.basename(src) + ".o")
    common = ["-O3", "-std=c++17", f"-I{INCLUDE}", f"-I{CSRC}", *[f"-D{d}" for d in defines]]
    if src.endswith(".cu"):
        cmd = [_nvcc(), *ARCH, "-lineinfo", *common, "-Xcompiler", "-fPIC,-fopenmp", "-c", src, "-o", obj]
        if verbose_ptxas:
            cmd.insert(1, "-Xptxas=-v")
    else:
        cmd = ["g++", *common, "-fPIC", "-fopenmp", "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if verbose_ptxas and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None, checked: bool = False) -> str:
    """Compile every csrc/ source for sm_103a and link libpjds.so (checked=True:
    libpjds_checked.so with PJDS_CHECKED, the device-side extent checks);
    returns its path."""
    objdir, lib = (OBJDIR_CHECKED, LIB_CHECKED) if checked else (OBJDIR, LIB)
    defines = ("PJDS_CHECKED",) if checked else ()
    os.makedirs(objdir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    deps = _deps()
    todo = [s for s in srcs if force or verbose_ptxas or _stale(s, os.path.join(objdir, os.path.basename(s) + ".o"), deps)]
    objs = [os.path.join(objdir, os.path.basename(s) + ".o") for s in srcs]
    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs or min(len(todo), os.cpu_count() or 4)) as ex:
            list(ex.map(lambda s: _compile(s, verbose_ptxas, objdir, defines), todo))
    if todo or not os.path.exists(lib) or any(os.path.getmtime(o) > os.path.getmtime(lib) for o in objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lgomp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="--ptxas" in sys.argv, checked="--checked" in sys.argv))
