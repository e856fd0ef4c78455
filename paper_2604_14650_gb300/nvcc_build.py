"""Builds libplanb.so (and a bounds-checked variant) in-tree with nvcc for sm_103a.

The translation units are compiled in parallel and linked with the static CUDA runtime. Outputs go
to ``paper_2604_14650_gb300/_build/``.
"""
from __future__ import annotations

import os
import platform
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build", platform.machine())
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["builder.cpp", "lookup.cu", "multi_lookup.cu", "learned.cu", "multi.cu", "capi.cu",
           "server.cu", "gpu_builder.cu"]
LIBS = {"libplanb.so": [], "libplanb_checked.so": ["-DPLANB_BOUNDS_CHECK"]}
# the translation units the bounds-checking define changes; the others are compiled once
CHECKED_SOURCES = {"lookup.cu", "multi_lookup.cu"}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(defines):
    return ["-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-O3",
            "-I", INCLUDE, "-I", CSRC, *defines]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> dict:
    """Compiles every library variant; returns {name: path}."""
    os.makedirs(OUT, exist_ok=True)
    cc = nvcc()
    headers = [os.path.join(CSRC, "planb_internal.h"), os.path.join(CSRC, "learned.cuh"),
               os.path.join(CSRC, "primitives.cuh"),
               os.path.join(CSRC, "descent.cuh"), os.path.join(INCLUDE, "planb.h")]
    jobs, links = [], {}
    for lib, defines in LIBS.items():
        objs = []
        for src in SOURCES:
            own = defines if src in CHECKED_SOURCES else []
            tag = "chk" if own else "rel"
            s = os.path.join(CSRC, src)
            o = os.path.join(OUT, f"{os.path.splitext(src)[0]}.{tag}.o")
            objs.append(o)
            if (force or _stale(o, [s, *headers])) and not any(j[-1] == o for j in jobs):
                jobs.append([cc, *_flags(own), "-c", s, "-o", o])
        links[lib] = objs

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)

    with ThreadPoolExecutor(max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        list(ex.map(run, jobs))
    out = {}
    for lib, objs in links.items():
        target = os.path.join(OUT, lib)
        if force or _stale(target, objs):
            tmp = target + f".tmp{os.getpid()}"
            run([cc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"])
            os.replace(tmp, target)
        out[lib] = target
    return out


if __name__ == "__main__":
    for k, v in build(verbose=True).items():
        print(k, v)
