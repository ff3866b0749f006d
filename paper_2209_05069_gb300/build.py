"""Builds libdock.so (the CUDA docking library) in-tree for sm_103a.

The translation units compile in parallel with nvcc (one -gencode, sm_103a only) and link into
``paper_2209_05069_gb300/lib/libdock.so``; the CUDA runtime is linked statically.  The kernel
instantiations are split into one unit per (grid dtype, warps per item) so they compile side by side.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ = os.path.join(PKG, "_build")
LIB_DIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIB_DIR, "libdock.so")
# The counter build: the same sources with DOCK_COUNT_WORK, whose kernels count the work they
# execute (dock_exec_counters); a separate library so the product kernels carry none of it.
OBJ_COUNT = os.path.join(PKG, "_build_count")
LIB_COUNT = os.path.join(LIB_DIR, "libdock_count.so")

# (object name, source, extra defines)
UNITS = [(f"dock_kernels_f{f}_g{g}_t{t}", "dock_kernels_inst.cu",
          [f"-DDOCK_INST_GT={f}", f"-DDOCK_INST_G={g}", f"-DDOCK_INST_T={t}"])
         for f in (0, 1, 2) for g, t in ((1, 1), (2, 1), (4, 1), (8, 1), (1, 2), (2, 2))] + [
    (f"dock_latency_f{f}", "dock_latency_inst.cu", [f"-DDOCK_INST_GT={f}"]) for f in (0, 1, 2)] + [
    ("dock_launch", "dock_launch.cu", []), ("dock_host", "dock_host.cpp", []), ("dock_noalloc", "dock_noalloc.cu", []),
    ("dock_select", "dock_select.cu", []), ("dock_gather_peak", "dock_gather_peak.cu", [])]
HEADERS = ["dock_internal.h", "dock_kernels.cuh", "dock_latency.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: libdock.so cannot be built")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, counters: bool = False) -> str:
    """Compiles what changed and links libdock.so (``counters``: libdock_count.so, the counter
    build); returns its path."""
    obj_dir, lib = (OBJ_COUNT, LIB_COUNT) if counters else (OBJ, LIB)
    os.makedirs(obj_dir, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "dock.h"), __file__]
    cc = nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    if counters:
        common.append("-DDOCK_COUNT_WORK")

    def compile_one(unit):
        name, src, defs = unit
        s = os.path.join(CSRC, src)
        o = os.path.join(obj_dir, name + ".o")
        if force or _stale(o, [s] + headers):
            cmd = [cc] + ARCH + common + defs + ["-c", s, "-o", o + ".tmp"]
            if src.endswith(".cu"):
                cmd += ["-Xptxas", "-v"] if verbose else []
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {name}:\n{r.stdout}\n{r.stderr}")
            if verbose:
                sys.stderr.write(r.stderr)
            os.replace(o + ".tmp", o)
        return o

    with ThreadPoolExecutor(max_workers=min(len(UNITS), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    if force or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        r = subprocess.run([cc] + ARCH + ["-shared", "-o", tmp] + objs, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


def build_all(force: bool = False) -> str:
    """Both libraries, compiled together (all units in one pool); returns libdock.so's path."""
    with ThreadPoolExecutor(max_workers=2) as ex:
        a = ex.submit(build, force, False, False)
        b = ex.submit(build, force, False, True)
        b.result()
        return a.result()


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, counters="--counters" in sys.argv))
