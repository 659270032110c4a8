"""Builds the CUDA library libwc.so in-tree (sm_103a only).

Each translation unit is compiled by nvcc in parallel, then linked into
paper_2206_05269_gb300/_build/libwc.so with the static CUDA runtime.

build(variant="oneslot") builds a test-only copy into _build/oneslot/ with
-DWC_TEST_ONE_SLOT: every hash is a constant, so every key of a table starts
at one home slot (the parity tests' forced-collision build).  Nothing but
those tests loads it.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libwc.so")
SOURCES = ["wc_count.cu", "wc_table.cu", "wc_batch.cu", "wc_api.cu", "wc_batch_api.cu", "wc_noalloc.cu", "wc_ceiling.cu",
           "wc_numeric.cu", "wc_hybrid.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps() -> list[str]:
    hdr = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hdr + [os.path.join(ROOT, "include", "wc.h")]


def _stale(target: str, inputs: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(i) > t for i in inputs)


VARIANTS = {None: [], "oneslot": ["-DWC_TEST_ONE_SLOT"]}


def lib_path(variant: str | None = None) -> str:
    return LIB if variant is None else os.path.join(OUT, variant, "libwc.so")


def build(force: bool = False, verbose: bool = False, variant: str | None = None) -> str:
    if variant not in VARIANTS:
        raise ValueError(f"unknown build variant {variant!r}")
    out = OUT if variant is None else os.path.join(OUT, variant)
    os.makedirs(out, exist_ok=True)
    import fcntl
    with open(os.path.join(out, ".lock"), "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        try:
            return _build(force, verbose, out, VARIANTS[variant], lib_path(variant))
        finally:
            fcntl.flock(lk, fcntl.LOCK_UN)


def _build(force: bool, verbose: bool, out: str, extra: list[str], lib: str) -> str:
    nvcc = _nvcc()
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    deps = _deps()
    objs = []
    jobs = []
    for s in srcs:
        src = os.path.join(CSRC, s)
        obj = os.path.join(out, s.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [src] + deps):
            jobs.append([nvcc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stderr)

    if jobs:
        with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
            list(ex.map(run, jobs))
    if force or _stale(lib, objs):
        tmp = lib + f".{os.getpid()}.tmp"
        run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
