"""Builds the CUDA library libpa_gb300.so in-tree with nvcc for sm_103a.

The translation units are compiled in parallel and linked into one shared
library next to this file.  Host code is compiled without floating-point
contraction so that the per-beta acceptance thresholds are reproducible.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libpa_gb300.so")
# the same library with the kernels' bounds tests compiled in (PA_CHECKED, pa_internal.cuh)
LIB_CHECKED = os.path.join(HERE, "libpa_gb300_checked.so")
SOURCES = ["pa_sweep.cu", "pa_resample.cu", "pa_capi.cu", "pa_reweight.cu", "pa_batch.cu", "pa_batch_hi.cu",
           "pa_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "pa.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Builds libpa_gb300.so (checked: libpa_gb300_checked.so, the kernels'
    bounds tests compiled in) unless it is newer than every source."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    nvcc = _nvcc()
    obj_dir = os.path.join(HERE, "_build_checked" if checked else "_build")
    os.makedirs(obj_dir, exist_ok=True)
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-I", INCLUDE,
                     "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math"]
    if checked:
        common += ["-DPA_CHECKED=1"]
    if verbose:
        common += ["-Xptxas", "-v"]
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(obj_dir, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + common
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stderr.write(out)
        if p.returncode != 0:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    tmp = lib + f".{os.getpid()}.tmp"
    subprocess.run([nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-ldl"], check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
