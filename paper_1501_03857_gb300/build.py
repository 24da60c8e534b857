"""Build liblbboil.so (the C-ABI library of include/lb.h) in-tree for sm_103a.

The translation units are compiled in parallel with nvcc and linked into
``paper_1501_03857_gb300/_lib/liblbboil.so`` (CUDA runtime linked
statically). The same sources are also built with -DLB_CHECKED into
``liblbboil_checked.so``, whose fused step checks every global and
shared-memory address it touches (an address outside its buffer sets a flag
reported as LB_E_BOUNDS and the access is skipped); select it with the
environment variable LBBOIL_LIB. Usage: ``python -m paper_1501_03857_gb300.build``.
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "liblbboil.so")
LIB_CHECKED = os.path.join(OUT_DIR, "liblbboil_checked.so")
SOURCES = ["lb_step3.cu", "lb_aux.cu", "lb_host.cu", "lb_noalloc.cu", "lb_adjoint.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    for c in ("/usr/local/cuda/bin/nvcc",):
        if os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbboil")


def _compile(nvcc, flags, tag, verbose):
    """Start nvcc for every source with `flags`; objects are named by tag."""
    procs = []
    for src in SOURCES:
        obj = os.path.join(OUT_DIR, src.replace(".cu", f"{tag}.o"))
        cmd = [nvcc] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
            print(" ".join(cmd), flush=True)
        procs.append((src, obj, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    return procs


def _link(nvcc, objs, lib):
    tmp = lib + ".tmp"
    r = subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode:
        sys.stdout.write(r.stdout.decode(errors="replace"))
        raise RuntimeError(f"linking {os.path.basename(lib)} failed")
    os.replace(tmp, lib)


def build(verbose: bool = False, extra_flags=None, checked: bool = True) -> str:
    nvcc = nvcc_path()
    os.makedirs(OUT_DIR, exist_ok=True)
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I", os.path.join(ROOT, "include"), "-I", CSRC] + list(extra_flags or [])
    jobs = [("", common, LIB)]
    if checked:
        jobs.append(("_checked", common + ["-DLB_CHECKED"], LIB_CHECKED))
    running = [(tag, lib, _compile(nvcc, flags, tag, verbose)) for tag, flags, lib in jobs]
    failed = []
    for tag, lib, procs in running:
        for src, obj, p in procs:
            out, _ = p.communicate()
            if verbose or p.returncode:
                sys.stdout.write(out.decode(errors="replace"))
            if p.returncode:
                failed.append(src + tag)
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(failed))
    for tag, lib, procs in running:
        objs = [obj for _, obj, _ in procs]
        _link(nvcc, objs, lib)
        for o in objs:
            os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
