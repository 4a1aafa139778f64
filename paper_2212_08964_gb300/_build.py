"""Build liblbspmv.so in-tree with nvcc for sm_103a (GB300).

Each translation unit compiles in its own nvcc process, in parallel, then one link step
produces ``paper_2212_08964_gb300/liblbspmv.so``.  The CUDA runtime is linked shared so
the library and PyTorch use the same runtime instance.

A second, range-checked build of the same sources, ``liblbspmv_checked.so`` (LB_CHECKED,
relocatable device code so that every kernel reaches the one device error word), tests
every index a kernel reads from its inputs before using it and records LB_ERR_OUT_OF_RANGE
instead of accessing memory outside an array.  It stands in for a memory checker; the
binding loads it instead of the normal build when LBSPMV_CHECKED=1.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
VARIANTS = {
    # name: (library, object directory, extra compile flags, extra link flags)
    "release": (os.path.join(PKG, "liblbspmv.so"), BUILD, [], []),
    "checked": (os.path.join(PKG, "liblbspmv_checked.so"), os.path.join(BUILD, "checked"),
                ["-DLB_CHECKED", "-rdc=true"], ["-rdc=true"]),
}
VARIANT = "checked" if os.environ.get("LBSPMV_CHECKED") == "1" else "release"
LIB = VARIANTS[VARIANT][0]

SOURCES = [
    "lb_merge_f32.cu",
    "lb_merge_bf16.cu",
    "lb_merge_f16.cu",
    "lb_transpose.cu",
    "lb_backward.cu",
    "lb_mapped.cu",
    "lb_partition.cu",
    "lb_api.cu",
    "lb_static.cu",
    "lb_tune.cu",
    "lb_spmm.cu",
    "lb_calibrate.cu",
    "lb_graph.cu",
    "lb_nzsplit.cu",
]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build liblbspmv")
    return path


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    files.append(os.path.join(INCLUDE, "lbspmv.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date(variant: str = VARIANT) -> bool:
    lib = VARIANTS[variant][0]
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, variant: str = VARIANT) -> str:
    """Compile and link one variant of the library (by default the one the binding loads)
    unless it is up to date; returns the .so path."""
    lib, objdir, xcflags, xlflags = VARIANTS[variant]
    if not force and not ptxas_info and up_to_date(variant):
        return lib
    os.makedirs(objdir, exist_ok=True)
    cc = nvcc()

    def compile_one(src: str):
        obj = os.path.join(objdir, os.path.splitext(src)[0] + ".o")
        cmd = [cc, *ARCH, *CFLAGS, *xcflags, "-c", os.path.join(CSRC, src), "-o", obj]
        if ptxas_info:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose or ptxas_info:
        for (_, log), src in zip(results, SOURCES):
            if log.strip():
                print(f"== {src}\n{log}")
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, *xlflags, "-shared", "-cudart", "shared", "-o", tmp, *[o for o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build_all(force: bool = False) -> list[str]:
    """Both variants: the normal library and the range-checked one."""
    return [build(force=force, variant=v) for v in VARIANTS]


if __name__ == "__main__":
    import sys

    for v in VARIANTS:
        print(build(force=True, verbose=True, ptxas_info="--ptxas" in sys.argv, variant=v))
