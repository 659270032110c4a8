"""Word-frequency oracle (test infrastructure only).

A plain single-threaded CPU implementation of the counting path in
``oracle.cpp``: letters-only tokenisation with ASCII lowercasing, one hash map
per document, per-class and global sums, output sorted by (count desc, word
asc), and the exact class-ratio ranking.  Only the tests, the smoke check and
the benchmark's CPU-baseline arm use it; the CUDA library never does.

Each function cites the passage of the paper it follows (Sec. 2, Sec. 3.1-3.3
and Sec. 4.3 of arXiv 2206.05269); the rule for which bytes are letters is the
fixed letters-only normalisation documented in ``oracle.cpp``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

DOC, CLASS, GLOBAL = 0, 1, 2


def build(force: bool = False) -> str:
    """Compiles oracle.cpp and series.cpp with the host C++ compiler (portable flags)."""
    srcs = [os.path.join(_HERE, f) for f in ("oracle.cpp", "series.cpp")]
    with _lock:
        if not force and os.path.exists(_SO) and all(os.path.getmtime(_SO) >= os.path.getmtime(s) for s in srcs):
            return _SO
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", *srcs, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp = ctypes.c_void_p
        lib.oracle_count.restype = vp
        lib.oracle_count.argtypes = [vp, vp, ctypes.c_uint32, vp, ctypes.c_uint32, ctypes.c_int]
        lib.oracle_merge.restype = vp
        lib.oracle_merge.argtypes = [ctypes.c_uint32, vp, vp, vp, vp]
        lib.oracle_table_size.restype = ctypes.c_int64
        lib.oracle_table_size.argtypes = [vp, ctypes.c_int, ctypes.c_uint32, vp, vp]
        lib.oracle_table_export.restype = ctypes.c_int
        lib.oracle_table_export.argtypes = [vp, ctypes.c_int, ctypes.c_uint32, vp, vp, vp]
        lib.oracle_ratio_topk.restype = ctypes.c_int64
        lib.oracle_ratio_topk.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32, vp, vp, vp]
        lib.oracle_free.argtypes = [vp]
        lib.oracle_series_sum.restype = ctypes.c_double
        lib.oracle_series_sum.argtypes = [ctypes.c_int, ctypes.c_uint64]
        _lib = lib
    return _lib


@dataclasses.dataclass
class Table:
    """A sorted count table: words back to back, offsets [n+1], counts [n]."""
    words: np.ndarray    # uint8
    offs: np.ndarray     # uint64 [n+1]
    counts: np.ndarray   # uint64 [n]

    def __len__(self) -> int:
        return int(self.counts.size)

    def word(self, i: int) -> bytes:
        return self.words[self.offs[i]:self.offs[i + 1]].tobytes()

    def as_list(self) -> list[tuple[bytes, int]]:
        return [(self.word(i), int(self.counts[i])) for i in range(len(self))]

    def as_dict(self) -> dict[bytes, int]:
        return dict(self.as_list())

    @property
    def tokens(self) -> int:
        return int(self.counts.sum())

    @staticmethod
    def from_list(items: list[tuple[bytes, int]]) -> "Table":
        words = b"".join(w for w, _ in items)
        offs = np.zeros(len(items) + 1, dtype=np.uint64)
        offs[1:] = np.cumsum([len(w) for w, _ in items], dtype=np.uint64) if items else []
        return Table(np.frombuffer(words, dtype=np.uint8).copy(), offs,
                     np.array([c for _, c in items], dtype=np.uint64))


def _as_u8(text) -> np.ndarray:
    if isinstance(text, (bytes, bytearray)):
        return np.frombuffer(bytes(text), dtype=np.uint8)
    return np.ascontiguousarray(text, dtype=np.uint8)


class Result:
    def __init__(self, handle, nclasses: int, ndocs: int):
        self._h = handle
        self.nclasses = nclasses
        self.ndocs = ndocs

    def __del__(self):
        if getattr(self, "_h", None):
            _load().oracle_free(self._h)
            self._h = None

    def _table(self, kind: int, idx: int) -> Table:
        lib = _load()
        nb = ctypes.c_uint64()
        n = lib.oracle_table_size(self._h, kind, idx, ctypes.byref(nb), None)
        if n < 0:
            raise IndexError(idx)
        words = np.zeros(max(1, nb.value), dtype=np.uint8)
        offs = np.zeros(n + 1, dtype=np.uint64)
        counts = np.zeros(max(1, n), dtype=np.uint64)
        lib.oracle_table_export(self._h, kind, idx, words.ctypes.data, offs.ctypes.data, counts.ctypes.data)
        return Table(words[:nb.value], offs, counts[:n])

    def doc(self, d: int) -> Table:
        """Per-document table (Sec. 3.1: one dictionary per document)."""
        return self._table(DOC, d)

    def cls(self, c: int) -> Table:
        """Per-class table: the documents of class c summed word by word."""
        return self._table(CLASS, c)

    def glob(self) -> Table:
        """Global table (Sec. 3.2/3.3: all per-document counts summed per key)."""
        return self._table(GLOBAL, 0)

    def ratio_topk(self, c: int, k: int) -> list[tuple[bytes, int, int]]:
        """Top-k words of class c by in-class/out-of-class count ratio (Sec. 4.3
        made exact): (word, cin, cout) in rank order."""
        lib = _load()
        t = self.cls(c)
        idx = np.zeros(max(1, k), dtype=np.uint64)
        cin = np.zeros(max(1, k), dtype=np.uint64)
        cout = np.zeros(max(1, k), dtype=np.uint64)
        n = lib.oracle_ratio_topk(self._h, c, k, idx.ctypes.data, cin.ctypes.data, cout.ctypes.data)
        return [(t.word(int(idx[i])), int(cin[i]), int(cout[i])) for i in range(n)]


def count(text, offsets=None, classes=None, nclasses: int = 0, keep_docs: bool = True) -> Result:
    """Counts words per document, per class and overall.

    text: bytes or uint8 array; offsets: uint64 [ndocs+1] (default: one
    document spanning the whole text); classes: uint32 [ndocs] or None.
    """
    t = _as_u8(text)
    if offsets is None:
        offsets = np.array([0, t.size], dtype=np.uint64)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    ndocs = offsets.size - 1
    cls_ptr = None
    if classes is not None and nclasses > 0:
        classes = np.ascontiguousarray(classes, dtype=np.uint32)
        cls_ptr = classes.ctypes.data
    else:
        nclasses = 0
    buf = t if t.size else np.zeros(1, dtype=np.uint8)
    h = _load().oracle_count(buf.ctypes.data, offsets.ctypes.data, ndocs, cls_ptr, nclasses, int(keep_docs))
    return Result(h, nclasses, ndocs)


def merge(tables: list[Table]) -> Table:
    """Sums tables word by word (Sec. 3.3: "the" counted 10, 4 and 3 times
    in three documents reduces to 17)."""
    lib = _load()
    n = len(tables)
    keep = []
    W = (ctypes.c_void_p * max(1, n))()
    O = (ctypes.c_void_p * max(1, n))()
    C = (ctypes.c_void_p * max(1, n))()
    sizes = np.zeros(max(1, n), dtype=np.uint64)
    for i, t in enumerate(tables):
        w = t.words if t.words.size else np.zeros(1, dtype=np.uint8)
        o = np.ascontiguousarray(t.offs, dtype=np.uint64)
        c = np.ascontiguousarray(t.counts, dtype=np.uint64)
        if c.size == 0:
            c = np.zeros(1, dtype=np.uint64)
        keep += [w, o, c]
        W[i], O[i], C[i] = w.ctypes.data, o.ctypes.data, c.ctypes.data
        sizes[i] = len(t)
    h = lib.oracle_merge(n, ctypes.cast(W, ctypes.c_void_p), ctypes.cast(O, ctypes.c_void_p),
                         ctypes.cast(C, ctypes.c_void_p), sizes.ctypes.data)
    r = Result(h, 0, 0)
    return r.glob()


SERIES_SQRT, SERIES_ALT_HARMONIC = 0, 1


def series_sum(series: int, n: int) -> float:
    """Sec. 4.2's numeric MapReduce: sum_{i=1}^n sqrt(i) (SERIES_SQRT) or
    sum_{i=1}^n (-1)^(i+1)/i (SERIES_ALT_HARMONIC), double-precision terms,
    Neumaier-compensated left-to-right sum (see series.cpp)."""
    if series not in (SERIES_SQRT, SERIES_ALT_HARMONIC) or n < 0:
        raise ValueError("unknown series or negative n")
    return float(_load().oracle_series_sum(series, n))
