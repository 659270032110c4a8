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
    """Compiles parallel.cpp and hybrid.cpp with the host C++ compiler (portable flags)."""
    srcs = [os.path.join(_HERE, f) for f in ("parallel.cpp", "hybrid.cpp")]
    with _lock:
        if not force and os.path.exists(_SO) and all(os.path.getmtime(_SO) >= os.path.getmtime(s) for s in srcs):
            return _SO
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-pthread", "-shared", "-fPIC", *srcs, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.cpu_parallel_count.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, u64p, u64p, u64p]
        lib.cpu_parallel_count.restype = ctypes.c_int
        lib.hybrid_map.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int, u64p, u64p, u64p]
        lib.hybrid_map.restype = ctypes.c_void_p
        lib.hybrid_fill.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        lib.hybrid_fill.restype = ctypes.c_int
        lib.hybrid_free.argtypes = [ctypes.c_void_p]
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


class HybridMap:
    """The paper's CPU map and GPU-reduce preparation (hybrid.cpp): per-document
    dictionaries, grouped into word -> per-document counts, laid out as a
    zero-padded matrix (one row per word).  `seconds` holds the time of each
    host stage."""

    def __init__(self, text: np.ndarray, offsets: np.ndarray, threads: int | None = None):
        self.threads = threads or os.cpu_count() or 1
        t = np.ascontiguousarray(text, dtype=np.uint8)
        o = np.ascontiguousarray(offsets, dtype=np.uint64)
        r, c, wb = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        lib = _load()
        t0 = time.perf_counter()
        self._h = lib.hybrid_map(t.ctypes.data if t.size else None, o.ctypes.data, o.size - 1, self.threads,
                                 ctypes.byref(r), ctypes.byref(c), ctypes.byref(wb))
        self.seconds = {"map_and_group": time.perf_counter() - t0}
        if not self._h:
            raise ValueError("bad hybrid_map arguments")
        self.rows, self.cols, self.word_bytes = r.value, c.value, wb.value

    def fill(self, matrix) -> None:
        """Writes the padded matrix into `matrix` (rows x cols uint32, any
        writable host buffer with a data pointer, e.g. a pinned tensor)."""
        ptr = matrix.data_ptr() if hasattr(matrix, "data_ptr") else matrix.ctypes.data
        t0 = time.perf_counter()
        _load().hybrid_fill(self._h, ptr, self.threads, None, None)
        self.seconds["matrix"] = time.perf_counter() - t0

    def words(self) -> list[bytes]:
        w = np.zeros(max(1, self.word_bytes), dtype=np.uint8)
        o = np.zeros(self.rows + 1, dtype=np.uint64)
        _load().hybrid_fill(self._h, None, 1, w.ctypes.data, o.ctypes.data)
        return [w[o[i]:o[i + 1]].tobytes() for i in range(self.rows)]

    def __del__(self):
        if getattr(self, "_h", None):
            _load().hybrid_free(self._h)
            self._h = None
