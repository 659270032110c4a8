"""Thin Python binding of the C ABI in include/wc.h.

Functions here carry the C names and only marshal arguments: device buffers
are passed as raw pointers (``tensor.data_ptr()``), streams as raw handles
(``torch.cuda.current_stream().cuda_stream``).  Every step of counting runs
in the CUDA library; if the library is missing this module raises instead of
computing anything on the host.

``Table`` and ``Counter`` are small conveniences over the same calls.
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# WC_LIB_PATH selects another build of the same library (the tests' one-slot
# build); there is no host implementation to fall back to either way.
LIB_PATH = os.environ.get("WC_LIB_PATH") or os.path.join(_PKG, "_build", "libwc.so")

WC_OK = 0
WC_ERR_INVALID_ARG = 1
WC_ERR_OOM = 2
WC_ERR_BUDGET = 3
WC_ERR_CAPACITY = 4
WC_ERR_CUDA = 5
WC_ERR_TIMEOUT = 6
WC_ERR_INTERNAL = 7
WC_ERR_UNSUPPORTED = 8

WC_TABLE_DOC, WC_TABLE_CLASS, WC_TABLE_GLOBAL = 0, 1, 2
WC_BATCH_EXACT_BOUNDS = 1

# Every symbol include/wc.h declares (checked by the tests).
EXPORTS = [
    "wc_create", "wc_destroy", "wc_count", "wc_count_ex", "wc_count_host", "wc_count_stream", "wc_count_batched",
    "wc_count_batched_ex", "wc_batch_status",
    "wc_batch_table", "wc_batch_topk", "wc_batch_size", "wc_batch_export",
    "wc_class_ratio_topk", "wc_merge", "wc_topk", "wc_table_status", "wc_table_size",
    "wc_table_export", "wc_table_count_bits", "wc_table_free", "wc_batch_free", "wc_plan_create", "wc_plan_run",
    "wc_plan_free", "wc_count_noalloc", "wc_buffer_alloc", "wc_buffer_free", "wc_mem_usage",
    "wc_series_sum", "wc_batch_vocab", "wc_batch_export_ids", "wc_row_sums", "wc_profile_enable",
    "wc_profile_read", "wc_read_ceiling", "wc_selftest_wait", "wc_status_str", "wc_last_error",
]


class WcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


class WcConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("mem_budget_bytes", ctypes.c_uint64),
                ("count_bits", ctypes.c_int), ("autotune", ctypes.c_int),
                ("tune_cache_path", ctypes.c_char_p)]


class WcCountOpts(ctypes.Structure):
    _fields_ = [("table_slots", ctypes.c_uint64), ("long_slots", ctypes.c_uint64),
                ("arena_bytes", ctypes.c_uint64), ("no_level1", ctypes.c_int)]


_lib = None


def load() -> ctypes.CDLL:
    """Loads libwc.so; raises if it has not been built (no host fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
    lib = ctypes.CDLL(LIB_PATH)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    pvp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "wc_create": (i32, [ctypes.POINTER(WcConfig), pvp]),
        "wc_destroy": (None, [vp]),
        "wc_count": (i32, [vp, vp, u64, vp, pvp]),
        "wc_count_ex": (i32, [vp, vp, u64, ctypes.POINTER(WcCountOpts), vp, pvp]),
        "wc_count_host": (i32, [vp, vp, u64, vp, u64, ctypes.POINTER(WcCountOpts), vp, pvp]),
        "wc_count_stream": (i32, [vp, vp, u64, u64, vp, pvp]),
        "wc_count_batched": (i32, [vp, vp, vp, vp, u32, vp, u32, vp, pvp]),
        "wc_count_batched_ex": (i32, [vp, vp, vp, vp, u32, vp, u32, u32, vp, pvp]),
        "wc_batch_status": (i32, [vp]),
        "wc_batch_table": (i32, [vp, i32, u32, pvp]),
        "wc_batch_topk": (i32, [vp, u32, ctypes.POINTER(u64), ctypes.POINTER(u32), pvp]),
        "wc_batch_size": (i32, [vp, ctypes.POINTER(u64), ctypes.POINTER(u64)]),
        "wc_batch_export": (i32, [vp, vp, vp, vp, vp, vp, vp]),
        "wc_class_ratio_topk": (i32, [vp, vp, u32, u32, vp, vp, vp, vp, ctypes.POINTER(u32)]),
        "wc_merge": (i32, [vp, ctypes.POINTER(ctypes.c_void_p), u32, vp, pvp]),
        "wc_topk": (i32, [vp, vp, u32, vp, pvp]),
        "wc_table_status": (i32, [vp]),
        "wc_table_size": (i32, [vp, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(u64)]),
        "wc_table_export": (i32, [vp, vp, vp, vp, vp]),
        "wc_table_count_bits": (i32, [vp]),
        "wc_table_free": (None, [vp]),
        "wc_batch_free": (None, [vp]),
        "wc_plan_create": (i32, [vp, vp, u32, u32, vp, pvp]),
        "wc_plan_run": (i32, [vp, vp, vp, vp, vp, pvp]),
        "wc_plan_free": (None, [vp]),
        "wc_count_noalloc": (i32, [vp, u64, vp, vp, vp, vp, u64, vp, vp, u64, vp, u64, vp, vp]),
        "wc_series_sum": (i32, [vp, i32, u64, vp, vp]),
        "wc_batch_vocab": (i32, [vp, pvp]),
        "wc_row_sums": (i32, [vp, u64, u64, vp, vp]),
        "wc_batch_export_ids": (i32, [vp, vp, vp, vp, vp, vp]),
        "wc_buffer_alloc": (i32, [vp, u64, vp, pvp]),
        "wc_buffer_free": (i32, [vp, vp, u64, vp]),
        "wc_mem_usage": (i32, [vp, ctypes.POINTER(u64), ctypes.POINTER(u64), i32]),
        "wc_profile_enable": (i32, [vp, i32]),
        "wc_profile_read": (i32, [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(u64), ctypes.POINTER(u64)]),
        "wc_selftest_wait": (i32, [vp, u32, i32, vp]),
        "wc_read_ceiling": (i32, [vp, u64, vp, u32, vp]),
        "wc_status_str": (ctypes.c_char_p, [i32]),
        "wc_last_error": (ctypes.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int, ctx=None, what: str = "") -> None:
    if status != WC_OK:
        lib = load()
        msg = lib.wc_last_error(ctx).decode() if ctx else lib.wc_status_str(status).decode()
        raise WcError(status, f"{what}: {msg}" if what else msg)


# ------------------------------------------------------------------ C names
def wc_create(device: int = 0, mem_budget_bytes: int = 0, count_bits: int = 64, autotune: int = 0,
              tune_cache_path: str | None = None):
    cfg = WcConfig(device, mem_budget_bytes, count_bits, autotune,
                   tune_cache_path.encode() if tune_cache_path else None)
    out = ctypes.c_void_p()
    _check(load().wc_create(ctypes.byref(cfg), ctypes.byref(out)), None, "wc_create")
    return out


def wc_destroy(ctx) -> None:
    load().wc_destroy(ctx)


def wc_count(ctx, d_text: int, nbytes: int, stream: int):
    out = ctypes.c_void_p()
    _check(load().wc_count(ctx, d_text, nbytes, stream, ctypes.byref(out)), ctx, "wc_count")
    return out


def wc_count_ex(ctx, d_text: int, nbytes: int, opts: tuple[int, int, int] | None, stream: int):
    out = ctypes.c_void_p()
    o = WcCountOpts(*(opts or (0, 0, 0)))
    _check(load().wc_count_ex(ctx, d_text, nbytes, ctypes.byref(o), stream, ctypes.byref(out)), ctx,
           "wc_count_ex")
    return out


def wc_count_host(ctx, h_text: int, nbytes: int, d_buf: int | None, piece_bytes: int,
                  opts: tuple[int, int, int] | None, stream: int):
    out = ctypes.c_void_p()
    o = WcCountOpts(*(opts or (0, 0, 0)))
    _check(load().wc_count_host(ctx, h_text, nbytes, d_buf, piece_bytes, ctypes.byref(o), stream, ctypes.byref(out)),
           ctx, "wc_count_host")
    return out


def wc_count_stream(ctx, h_text: int, nbytes: int, chunk_bytes: int, stream: int):
    out = ctypes.c_void_p()
    _check(load().wc_count_stream(ctx, h_text, nbytes, chunk_bytes, stream, ctypes.byref(out)), ctx, "wc_count_stream")
    return out


def wc_count_batched(ctx, d_text: int, d_offsets: int, h_offsets: np.ndarray, ndocs: int, d_class: int | None,
                     nclasses: int, stream: int, flags: int = 0):
    h = np.ascontiguousarray(h_offsets, dtype=np.uint64)
    out = ctypes.c_void_p()
    if flags:
        _check(load().wc_count_batched_ex(ctx, d_text, d_offsets, h.ctypes.data, ndocs, d_class or None, nclasses,
                                          flags, stream, ctypes.byref(out)), ctx, "wc_count_batched_ex")
    else:
        _check(load().wc_count_batched(ctx, d_text, d_offsets, h.ctypes.data, ndocs, d_class or None, nclasses,
                                       stream, ctypes.byref(out)), ctx, "wc_count_batched")
    return out


def wc_batch_status(batch) -> int:
    return load().wc_batch_status(batch)


def wc_batch_size(batch) -> tuple[int, int]:
    n, nb = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().wc_batch_size(batch, ctypes.byref(n), ctypes.byref(nb)), None, "wc_batch_size")
    return n.value, nb.value


def wc_batch_export(batch, ndocs: int, stream: int = 0):
    """Returns (doc_start uint64[ndocs], doc_n uint32[ndocs], words, word offsets, counts uint32)."""
    n, nb = wc_batch_size(batch)
    ds = np.zeros(max(1, ndocs), dtype=np.uint64)
    dn = np.zeros(max(1, ndocs), dtype=np.uint32)
    words = np.zeros(max(1, nb), dtype=np.uint8)
    offs = np.zeros(n + 1, dtype=np.uint64)
    counts = np.zeros(max(1, n), dtype=np.uint32)
    _check(load().wc_batch_export(batch, ds.ctypes.data, dn.ctypes.data, words.ctypes.data, offs.ctypes.data,
                                  counts.ctypes.data, stream), None, "wc_batch_export")
    return ds[:ndocs], dn[:ndocs], words[:nb], offs, counts[:n]


def wc_batch_table(batch, kind: int, idx: int):
    out = ctypes.c_void_p()
    _check(load().wc_batch_table(batch, kind, idx, ctypes.byref(out)), None, "wc_batch_table")
    return out


def wc_batch_topk(batch, ndocs: int, k: int):
    """Per-document top-k rows: (borrowed table handle, first row per document,
    rows per document)."""
    first = np.zeros(max(1, ndocs), dtype=np.uint64)
    n = np.zeros(max(1, ndocs), dtype=np.uint32)
    out = ctypes.c_void_p()
    _check(load().wc_batch_topk(batch, k, first.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                n.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), ctypes.byref(out)),
           None, "wc_batch_topk")
    return out, first[:ndocs], n[:ndocs]


def wc_class_ratio_topk(ctx, batch, cls: int, k: int, stream: int):
    idx = np.zeros(max(1, k), dtype=np.uint64)
    cin = np.zeros(max(1, k), dtype=np.uint64)
    cout = np.zeros(max(1, k), dtype=np.uint64)
    n = ctypes.c_uint32()
    _check(load().wc_class_ratio_topk(ctx, batch, cls, k, stream, idx.ctypes.data, cin.ctypes.data,
                                      cout.ctypes.data, ctypes.byref(n)), ctx, "wc_class_ratio_topk")
    m = n.value
    return idx[:m], cin[:m], cout[:m]


def wc_merge(ctx, tables: list, stream: int):
    arr = (ctypes.c_void_p * max(1, len(tables)))(*[t.value if isinstance(t, ctypes.c_void_p) else t
                                                    for t in tables])
    out = ctypes.c_void_p()
    _check(load().wc_merge(ctx, arr, len(tables), stream, ctypes.byref(out)), ctx, "wc_merge")
    return out


def wc_topk(ctx, table, k: int, stream: int):
    out = ctypes.c_void_p()
    _check(load().wc_topk(ctx, table, k, stream, ctypes.byref(out)), ctx, "wc_topk")
    return out


def wc_table_status(table) -> int:
    return load().wc_table_status(table)


def wc_table_size(table) -> tuple[int, int, int]:
    n, tok, nb = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().wc_table_size(table, ctypes.byref(n), ctypes.byref(tok), ctypes.byref(nb)), None,
           "wc_table_size")
    return n.value, tok.value, nb.value


def wc_table_count_bits(table) -> int:
    return load().wc_table_count_bits(table)


def wc_table_export(table, stream: int = 0):
    """Returns (words uint8, offsets uint64[n+1], counts uint32/uint64[n])."""
    n, _, nb = wc_table_size(table)
    bits = wc_table_count_bits(table)
    words = np.zeros(max(1, nb), dtype=np.uint8)
    offs = np.zeros(n + 1, dtype=np.uint64)
    counts = np.zeros(max(1, n), dtype=np.uint32 if bits == 32 else np.uint64)
    _check(load().wc_table_export(table, words.ctypes.data, offs.ctypes.data, counts.ctypes.data, stream),
           None, "wc_table_export")
    return words[:nb], offs, counts[:n]


def wc_table_free(table) -> None:
    load().wc_table_free(table)


def wc_batch_free(batch) -> None:
    load().wc_batch_free(batch)


def wc_plan_create(ctx, h_offsets: np.ndarray, nclasses: int, stream: int):
    h = np.ascontiguousarray(h_offsets, dtype=np.uint64)
    out = ctypes.c_void_p()
    _check(load().wc_plan_create(ctx, h.ctypes.data, int(h.size - 1), nclasses, stream, ctypes.byref(out)), ctx,
           "wc_plan_create")
    return out


def wc_plan_run(ctx, plan, d_text: int, d_offsets: int, d_class: int | None, stream: int):
    out = ctypes.c_void_p()
    _check(load().wc_plan_run(plan, d_text, d_offsets, d_class or None, stream, ctypes.byref(out)), ctx,
           "wc_plan_run")
    return out


def wc_plan_free(plan) -> None:
    load().wc_plan_free(plan)


NOALLOC_MAX_BYTES = 1 << 20
NOALLOC_ENTRIES = (1 << 17) + (1 << 16) + (1 << 13)
NOALLOC_LONG = 1 << 13


def wc_count_noalloc(d_text: int, nbytes: int, d_khi: int, d_klo: int, d_cnt: int, d_lref: int, out_cap: int,
                     d_loff: int, d_llen: int, long_cap: int, d_arena: int, arena_cap: int, d_meta: int,
                     stream: int) -> None:
    """Single-document count that allocates nothing (caller-owned outputs,
    fixed library scratch); see include/wc.h."""
    _check(load().wc_count_noalloc(d_text, nbytes, d_khi, d_klo, d_cnt, d_lref, out_cap, d_loff, d_llen, long_cap,
                                   d_arena, arena_cap, d_meta, stream), None, "wc_count_noalloc")


WC_SERIES_SQRT, WC_SERIES_ALT_HARMONIC = 0, 1


def wc_series_sum(ctx, series: int, n: int, d_out: int, stream: int) -> None:
    """Sec. 4.2's numeric MapReduce into one device double (asynchronous)."""
    _check(load().wc_series_sum(ctx, series, n, d_out, stream), ctx, "wc_series_sum")


def wc_row_sums(d_matrix: int, rows: int, cols: int, d_sums: int, stream: int) -> None:
    """Row sums of a device uint32 matrix into device uint64 (the hybrid pipeline's reduce)."""
    _check(load().wc_row_sums(d_matrix, rows, cols, d_sums, stream), None, "wc_row_sums")


def wc_buffer_alloc(ctx, nbytes: int, stream: int) -> int:
    """Device buffer from the context's budgeted pool (raises WcError with
    WC_ERR_BUDGET when the budget cannot hold it); returns the pointer."""
    out = ctypes.c_void_p()
    _check(load().wc_buffer_alloc(ctx, nbytes, stream, ctypes.byref(out)), ctx, "wc_buffer_alloc")
    return int(out.value)


def wc_buffer_free(ctx, ptr: int, nbytes: int, stream: int) -> None:
    _check(load().wc_buffer_free(ctx, ptr, nbytes, stream), ctx, "wc_buffer_free")


def wc_mem_usage(ctx, reset: bool = False) -> tuple[int, int]:
    """(bytes the context holds now, peak since creation or the last reset)"""
    u, p = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().wc_mem_usage(ctx, ctypes.byref(u), ctypes.byref(p), int(reset)), ctx, "wc_mem_usage")
    return u.value, p.value


def wc_profile_enable(ctx, enable: bool) -> None:
    _check(load().wc_profile_enable(ctx, int(enable)), ctx, "wc_profile_enable")


def wc_profile_read(ctx) -> tuple[float, float, float, int, int]:
    """(ms in head selection, ms in the main counting kernel, ms in compaction+sort,
    main counting kernels timed, kernels launched)"""
    h, a, b = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    n, k = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().wc_profile_read(ctx, ctypes.byref(h), ctypes.byref(a), ctypes.byref(b), ctypes.byref(n),
                                  ctypes.byref(k)), ctx, "wc_profile_read")
    return h.value, a.value, b.value, n.value, k.value


def wc_read_ceiling(d_text: int, nbytes: int, d_sink: int, sink_words: int, stream: int = 0) -> int:
    """One read-only pass over a device text (the practical HBM limit of any
    single pass); asynchronous, returns the launch status."""
    return load().wc_read_ceiling(d_text, nbytes, d_sink, sink_words, stream)


def wc_selftest_wait(ctx, polls: int, arrive: bool, stream: int = 0) -> int:
    """Runs the bounded device wait on a barrier that is (arrive) or is not
    arrived at; returns the status (WC_OK, or WC_ERR_TIMEOUT)."""
    return load().wc_selftest_wait(ctx, polls, int(arrive), stream)


def wc_status_str(status: int) -> str:
    return load().wc_status_str(status).decode()


def wc_last_error(ctx) -> str:
    return load().wc_last_error(ctx).decode()


# ------------------------------------------------------------------ helpers
def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


class Table:
    """Owns a wc_table handle (or borrows one from a batch, which it keeps
    alive).  An owned table registers with its Counter, which frees it before
    destroying the context: a table must not outlive its context, and Python
    may collect an object (one caught in a reference cycle, say) only after
    its Counter was closed."""

    def __init__(self, handle, owned: bool = True, counter=None, owner=None):
        self.handle = handle
        self.owned = owned
        self._owner = owner  # the batch a borrowed table reads from
        if owned and counter is not None:
            counter._track(self)

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "handle", None) and self.owned:
            wc_table_free(self.handle)
        self.handle = None

    def status(self) -> int:
        return wc_table_status(self.handle)

    def size(self) -> tuple[int, int, int]:
        return wc_table_size(self.handle)

    def export(self, stream=None):
        return wc_table_export(self.handle, _stream_handle(stream))

    def export_into(self, words, offsets, counts, stream=None) -> tuple[int, int]:
        """Exports into caller-owned host tensors (uint8 words, int64 offsets
        of n+1, counts of the table's count width; pinned ones copy fastest),
        each at least the table's size; returns (rows, word bytes)."""
        n, _, nb = self.size()
        if words.numel() < nb or offsets.numel() < n + 1 or counts.numel() < n:
            raise ValueError("export buffers smaller than the table")
        if counts.element_size() * 8 != wc_table_count_bits(self.handle):
            raise ValueError("count buffer width differs from the table's")
        _check(load().wc_table_export(self.handle, words.data_ptr(), offsets.data_ptr(), counts.data_ptr(),
                                      _stream_handle(stream)), None, "wc_table_export")
        return n, nb

    def as_list(self) -> list[tuple[bytes, int]]:
        w, o, c = self.export()
        return [(w[o[i]:o[i + 1]].tobytes(), int(c[i])) for i in range(c.size)]


class Batch:
    """Owns a wc_batch handle (or borrows a plan's, keeping the plan alive);
    an owned batch registers with its Counter like an owned Table."""

    def __init__(self, handle, ndocs: int = 0, owned: bool = True, counter=None, owner=None):
        self.handle = handle
        self.ndocs = ndocs
        self.owned = owned
        self._owner = owner
        if owned and counter is not None:
            counter._track(self)

    def status(self) -> int:
        return wc_batch_status(self.handle)

    def export(self, stream=None):
        return wc_batch_export(self.handle, self.ndocs, _stream_handle(stream))

    def export_into(self, doc_start, doc_n, words, offsets, counts, stream=None) -> tuple[int, int]:
        """Bulk export into caller-owned host tensors (int64 doc_start and
        int32 doc_n of ndocs, uint8 words, int64 offsets of n+1, int32
        counts; pinned ones copy fastest); returns (rows, word bytes)."""
        n, nb = wc_batch_size(self.handle)
        if (doc_start.numel() < self.ndocs or doc_n.numel() < self.ndocs or words.numel() < nb
                or offsets.numel() < n + 1 or counts.numel() < n):
            raise ValueError("export buffers smaller than the batch")
        _check(load().wc_batch_export(self.handle, doc_start.data_ptr(), doc_n.data_ptr(), words.data_ptr(),
                                      offsets.data_ptr(), counts.data_ptr(), _stream_handle(stream)),
               None, "wc_batch_export")
        return n, nb

    def vocab(self) -> Table:
        """The batch's distinct words in word order with global counts
        (borrowed from the batch); a word's id is its row."""
        out = ctypes.c_void_p()
        _check(load().wc_batch_vocab(self.handle, ctypes.byref(out)), None, "wc_batch_vocab")
        return Table(out, owned=False, owner=self)

    def export_ids(self, stream=None):
        """(doc_start uint64[ndocs], doc_n uint32[ndocs], ids uint32[n], counts uint32[n])."""
        n, _ = wc_batch_size(self.handle)
        ds = np.zeros(max(1, self.ndocs), dtype=np.uint64)
        dn = np.zeros(max(1, self.ndocs), dtype=np.uint32)
        ids = np.zeros(max(1, n), dtype=np.uint32)
        counts = np.zeros(max(1, n), dtype=np.uint32)
        _check(load().wc_batch_export_ids(self.handle, ds.ctypes.data, dn.ctypes.data, ids.ctypes.data,
                                          counts.ctypes.data, _stream_handle(stream)), None, "wc_batch_export_ids")
        return ds[:self.ndocs], dn[:self.ndocs], ids[:n], counts[:n]

    def export_ids_into(self, doc_start, doc_n, ids, counts, stream=None) -> int:
        """export_ids into caller-owned host tensors (int64 doc_start, int32
        doc_n, ids and counts; pinned ones copy fastest); returns the rows."""
        n, _ = wc_batch_size(self.handle)
        if doc_start.numel() < self.ndocs or doc_n.numel() < self.ndocs or ids.numel() < n or counts.numel() < n:
            raise ValueError("export buffers smaller than the batch")
        _check(load().wc_batch_export_ids(self.handle, doc_start.data_ptr(), doc_n.data_ptr(), ids.data_ptr(),
                                          counts.data_ptr(), _stream_handle(stream)), None, "wc_batch_export_ids")
        return n

    def doc_lists(self):
        """Per-document [(word, count)] lists from one bulk export."""
        ds, dn, w, o, c = self.export()
        out = []
        for d in range(self.ndocs):
            s0, n = int(ds[d]), int(dn[d])
            out.append([(w[o[i]:o[i + 1]].tobytes(), int(c[i])) for i in range(s0, s0 + n)])
        return out

    def free(self):
        if getattr(self, "handle", None) and self.owned:
            wc_batch_free(self.handle)
        self.handle = None

    def __del__(self):
        self.free()

    def table(self, kind: int, idx: int = 0) -> Table:
        return Table(wc_batch_table(self.handle, kind, idx), owned=False, owner=self)

    def topk(self, k: int):
        """Every document's top-k rows in one table (borrowed from the batch),
        with each document's first row and row count."""
        h, first, n = wc_batch_topk(self.handle, self.ndocs, k)
        return Table(h, owned=False, owner=self), first, n


class DeviceBuffer:
    """A device buffer from a context's budgeted pool (wc_buffer_alloc), seen
    from torch as a uint8 tensor without a copy; free() returns it in stream
    order."""

    def __init__(self, counter, nbytes: int, stream=None):
        import torch
        self.counter = counter
        self.nbytes = max(1, int(nbytes))
        self.ptr = wc_buffer_alloc(counter.ctx, self.nbytes, _stream_handle(stream))
        self.__cuda_array_interface__ = {"shape": (self.nbytes,), "typestr": "|u1", "data": (self.ptr, False),
                                         "version": 3}
        dev = torch.device("cuda", torch.cuda.current_device())
        self.tensor = torch.as_tensor(self, device=dev)

    def free(self, stream=None):
        if getattr(self, "ptr", None) and self.counter.ctx:
            wc_buffer_free(self.counter.ctx, self.ptr, self.nbytes, _stream_handle(stream))
        self.ptr = None
        self.tensor = None


class Counter:
    """A library context plus convenience calls on torch tensors."""

    def __init__(self, device: int = 0, budget: int = 0, count_bits: int = 64, autotune: bool = False,
                 tune_cache_path: str | None = None):
        self._live = weakref.WeakSet()  # owned tables, batches and plans of this context
        self.ctx = wc_create(device, budget, count_bits, int(autotune), tune_cache_path)

    def _track(self, obj) -> None:
        self._live.add(obj)

    def close(self):
        """Frees every table, batch and plan still alive, then the context."""
        for obj in list(getattr(self, "_live", ())):
            obj.free()
        if getattr(self, "ctx", None):
            wc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        self.close()

    def count(self, text, stream=None, opts=None) -> Table:
        """Counts one document held in a uint8 CUDA tensor (asynchronous)."""
        s = _stream_handle(stream)
        return Table(wc_count_ex(self.ctx, text.data_ptr(), text.numel(), opts, s), counter=self)

    def count_host(self, text, stream=None, out=None, piece_bytes: int = 0, opts=None) -> Table:
        """Counts one document held in host memory (a uint8 CPU tensor, pinned
        for the copies to overlap counting): copied to the device piece by
        piece (into `out`, a uint8 CUDA tensor of at least text.numel()
        bytes, or library memory) and each piece counted as it lands."""
        s = _stream_handle(stream)
        n = int(text.numel())
        return Table(wc_count_host(self.ctx, text.data_ptr() if n else None, n,
                                   out.data_ptr() if out is not None else None, piece_bytes, opts, s), counter=self)

    def count_stream(self, text, chunk_bytes: int = 0, stream=None) -> Table:
        """Counts a host text (a uint8 CPU tensor, pinned for overlap) that
        need not fit on the device: chunk by chunk through one device buffer,
        each chunk's table merged into the total (wc_count_stream)."""
        n = int(text.numel())
        return Table(wc_count_stream(self.ctx, text.data_ptr() if n else None, n, chunk_bytes,
                                     _stream_handle(stream)), counter=self)

    def count_host_checked(self, text, stream=None, out=None, piece_bytes: int = 0, retries: int = 4) -> Table:
        """count_host() that waits for the result and counts again with 4x
        capacities on WC_ERR_CAPACITY (as count_checked)."""
        opts = (0, 0, 0)
        for _ in range(retries + 1):
            t = self.count_host(text, stream, out, piece_bytes, opts)
            st = t.status()
            if st != WC_ERR_CAPACITY:
                _check(st, self.ctx, "count_host")
                return t
            n = int(text.numel())
            t.free()
            base = opts if any(opts) else (max(1024, n // 4), max(256, n // 64), max(4096, n // 8))
            opts = tuple(max(1, int(v)) * 4 for v in base)
        raise WcError(WC_ERR_CAPACITY, "capacity retries exhausted")

    def count_checked(self, text, stream=None, opts=None, retries: int = 4) -> Table:
        """count() that waits for the result and recounts with 4x capacities on
        WC_ERR_CAPACITY (the input is still alive, so a recount is exact)."""
        opts = tuple(opts) if opts else (0, 0, 0)
        caps, rest = opts[:3], opts[3:]  # capacity hints; the no_level1 flag is kept as given
        for _ in range(retries + 1):
            t = self.count(text, stream, caps + rest)
            st = t.status()
            if st != WC_ERR_CAPACITY:
                _check(st, self.ctx, "count")
                return t
            n = text.numel()
            t.free()
            base = caps if any(caps) else (max(1024, n // 4), max(256, n // 64), max(4096, n // 8))
            caps = tuple(max(1, int(v)) * 4 for v in base)
        raise WcError(WC_ERR_CAPACITY, "capacity retries exhausted")

    def count_batched(self, text, offsets, h_offsets, classes=None, nclasses: int = 0, stream=None,
                      exact: bool = False) -> Batch:
        s = _stream_handle(stream)
        return Batch(wc_count_batched(self.ctx, text.data_ptr(), offsets.data_ptr(), h_offsets,
                                      int(h_offsets.size - 1), classes.data_ptr() if classes is not None else None,
                                      nclasses, s, WC_BATCH_EXACT_BOUNDS if exact else 0),
                     int(h_offsets.size - 1), counter=self)

    def count_batched_checked(self, text, offsets, h_offsets, classes=None, nclasses: int = 0,
                              stream=None) -> Batch:
        """count_batched() that waits for the result and, on WC_ERR_CAPACITY,
        counts again with capacities at the exact bounds (which cannot
        overflow)."""
        b = self.count_batched(text, offsets, h_offsets, classes, nclasses, stream)
        st = b.status()
        if st == WC_ERR_CAPACITY:
            b.free()
            b = self.count_batched(text, offsets, h_offsets, classes, nclasses, stream, exact=True)
            st = b.status()
        _check(st, self.ctx, "count_batched")
        return b

    def buffer(self, nbytes: int, stream=None) -> DeviceBuffer:
        """Device memory charged against this context's budget."""
        return DeviceBuffer(self, nbytes, stream)

    def mem_usage(self, reset: bool = False) -> tuple[int, int]:
        return wc_mem_usage(self.ctx, reset)

    def plan(self, h_offsets, nclasses: int = 0, stream=None) -> "Plan":
        return Plan(self, h_offsets, nclasses, stream)

    def merge(self, tables: list[Table], stream=None) -> Table:
        return Table(wc_merge(self.ctx, [t.handle for t in tables], _stream_handle(stream)), counter=self)

    def topk(self, table: Table, k: int, stream=None) -> Table:
        return Table(wc_topk(self.ctx, table.handle, k, _stream_handle(stream)), counter=self)


class Plan:
    """Resident batched-count state replayed through a CUDA graph (wc_plan_*)."""

    def __init__(self, counter: Counter, h_offsets, nclasses: int = 0, stream=None):
        self.counter = counter
        self.ndocs = int(np.asarray(h_offsets).size - 1)
        self.handle = wc_plan_create(counter.ctx, h_offsets, nclasses, _stream_handle(stream))
        counter._track(self)

    def run(self, text, offsets, classes=None, stream=None) -> Batch:
        h = wc_plan_run(self.counter.ctx, self.handle, text.data_ptr(), offsets.data_ptr(),
                        classes.data_ptr() if classes is not None else None, _stream_handle(stream))
        return Batch(h, self.ndocs, owned=False, owner=self)

    def free(self):
        if getattr(self, "handle", None):
            wc_plan_free(self.handle)
        self.handle = None

    def __del__(self):
        self.free()
