"""Helpers for the GPU parity tests: device copies and table comparison."""
import numpy as np


def to_dev(data, offset: int = 0):
    """uint8 CUDA tensor holding data; with offset > 0 the tensor starts
    `offset` bytes into a larger allocation (unaligned base pointer)."""
    import torch
    arr = np.frombuffer(data, dtype=np.uint8) if isinstance(data, (bytes, bytearray)) else np.asarray(data, np.uint8)
    buf = torch.empty(arr.size + offset + 16, dtype=torch.uint8, device="cuda:0")
    buf.fill_(ord("x"))  # letters around the slice must not leak into it
    t = buf[offset:offset + arr.size]
    if arr.size:  # from a writable host copy (the bytes object's buffer is read-only)
        t.copy_(torch.from_numpy(np.array(arr, dtype=np.uint8, copy=True)))
    return t


def assert_same(gpu_export, oracle_table, what: str = ""):
    gw, go, gc = gpu_export
    assert gc.size == len(oracle_table), f"{what}: {gc.size} words vs oracle {len(oracle_table)}"
    assert np.array_equal(go.astype(np.uint64), oracle_table.offs), f"{what}: word offsets differ"
    assert np.array_equal(gw, oracle_table.words), f"{what}: word bytes differ"
    assert np.array_equal(gc.astype(np.uint64), oracle_table.counts), f"{what}: counts differ"


def first_diff(gpu_export, oracle_table, limit: int = 5):
    gw, go, gc = gpu_export
    out = []
    for i in range(min(gc.size, len(oracle_table))):
        g = (gw[go[i]:go[i + 1]].tobytes(), int(gc[i]))
        o = (oracle_table.word(i), int(oracle_table.counts[i]))
        if g != o:
            out.append((i, g, o))
            if len(out) >= limit:
                break
    return out
