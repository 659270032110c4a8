"""Paper-style parallel CPU word count (a baseline beside the GPU path and
the single-threaded oracle): one hash map per thread over its piece of the
text, merged by hash range, sorted by (count desc, word asc); see
``parallel.cpp``.  Only the benchmark and the tests use it."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libcpu_parallel.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles parallel.cpp with the host C++ compiler (portable flags)."""
    src = os.path.join(_HERE, "parallel.cpp")
    with _lock:
        if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
            return _SO
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-pthread", "-shared", "-fPIC", src, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.cpu_parallel_count.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, u64p, u64p, u64p]
        lib.cpu_parallel_count.restype = ctypes.c_int
        _lib = lib
    return _lib


def count(text: np.ndarray, threads: int | None = None) -> dict:
    """Counts a uint8 text with `threads` threads (default: every core);
    returns distinct words, tokens, the largest count and the seconds taken."""
    t = np.ascontiguousarray(text, dtype=np.uint8)
    threads = threads or os.cpu_count() or 1
    d, n, top = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    lib = _load()
    t0 = time.perf_counter()
    lib.cpu_parallel_count(t.ctypes.data if t.size else None, t.size, threads, ctypes.byref(d), ctypes.byref(n),
                           ctypes.byref(top))
    dt = time.perf_counter() - t0
    return {"distinct": d.value, "tokens": n.value, "top_count": top.value, "seconds": dt, "threads": threads}


def cpu_model() -> str:
    """The host CPU's model name as /proc/cpuinfo gives it (or the machine type)."""
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                k, _, v = ln.partition(":")
                if k.strip() in ("model name", "Model", "Hardware"):
                    return v.strip()
    except OSError:
        pass
    import platform
    return platform.machine()
