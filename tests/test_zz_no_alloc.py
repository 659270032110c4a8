"""The allocation-free entry point (wc_count_noalloc) gives the same table as
wc_count and as the oracle.

It exists for callers that may not allocate device memory (another component
owns the device memory, or allocation is forbidden after start-up); its
scratch is a fixed array inside the library.  The test calls it through the C
ABI twice in a row on different documents, because every call reuses the same
array and must clear what the previous call left behind.  A document with
more distinct words than the fixed tables hold must report nonzero status
bits, and the call after it must again be exact.  It runs last so that a
failure here never hides the other tests, and it passes alone as well.
"""
import numpy as np
import pytest

import corpus
import oracle

pytestmark = pytest.mark.gpu


def _words(khi, klo, cnt, lref, loff, llen, arena, n):
    out = []
    for i in range(n):
        r = int(lref[i])
        if r:
            o, ln = int(loff[r - 1]), int(llen[r - 1])
            w = arena[o:o + ln].tobytes()
        else:
            w = (int(khi[i]).to_bytes(8, "big") + int(klo[i]).to_bytes(8, "big")).rstrip(b"\0")
        out.append((w, int(cnt[i])))
    return out


class _Outputs:
    """Caller-owned device buffers for wc_count_noalloc (the caller allocates
    its own inputs and outputs; the library allocates nothing)."""

    def __init__(self, torch, wc, dev):
        self.cap, self.lcap = wc.NOALLOC_ENTRIES, wc.NOALLOC_LONG
        z = lambda n, dt: torch.zeros(n, dtype=dt, device=dev)
        self.khi, self.klo, self.cnt = z(self.cap, torch.int64), z(self.cap, torch.int64), z(self.cap, torch.int64)
        self.lref = z(self.cap, torch.int32)
        self.loff, self.llen = z(self.lcap, torch.int64), z(self.lcap, torch.int64)
        self.arena = z(wc.NOALLOC_MAX_BYTES * 2, torch.uint8)
        self.meta = z(8, torch.int64)

    def count(self, torch, wc, text):
        stream = torch.cuda.current_stream()
        wc.wc_count_noalloc(text.data_ptr(), text.numel(), self.khi.data_ptr(), self.klo.data_ptr(),
                            self.cnt.data_ptr(), self.lref.data_ptr(), self.cap, self.loff.data_ptr(),
                            self.llen.data_ptr(), self.lcap, self.arena.data_ptr(), self.arena.numel(),
                            self.meta.data_ptr(), int(stream.cuda_stream))
        torch.cuda.synchronize()
        m = self.meta.cpu().numpy().view(np.uint64)
        return m, int(m[7]) & 0xFFFFFFFF

    def table(self, m):
        return _words(self.khi.cpu().numpy().view(np.uint64), self.klo.cpu().numpy().view(np.uint64),
                      self.cnt.cpu().numpy().view(np.uint64), self.lref.cpu().numpy(), self.loff.cpu().numpy(),
                      self.llen.cpu().numpy(), self.arena.cpu().numpy(), int(m[0]))


def test_no_alloc_matches_wc_count_and_oracle_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_05269_gb300 import wc
    dev = torch.device("cuda:0")
    ctr = wc.Counter(0)
    out = _Outputs(torch, wc, dev)
    docs = [
        corpus.generate("tiny", ndocs=60, len_max=30, len_tail=0.3, len_tail_mean=8.0).text[:900_000],
        corpus.generate("classes", ndocs=8, seed=77).text[:300_000],
    ]
    for k, data in enumerate(docs):
        text = torch.from_numpy(np.ascontiguousarray(data)).to(dev)
        m, bits = out.count(torch, wc, text)
        assert bits == 0, f"call {k}: status bits {bits}"
        got = out.table(m)
        assert got == ctr.count_checked(text).as_list(), f"call {k}: differs from wc_count"
        want = oracle.count(np.ascontiguousarray(data)).glob().as_list()
        assert got == want, f"call {k}: differs from the oracle"
        assert int(m[3]) == sum(c for _, c in want)
    ctr.close()


def test_no_alloc_overflow_is_reported_and_the_next_call_is_exact():
    """About 1 MiB of distinct four-letter words (some 209,000) overflows the
    fixed 2^17-slot table of words up to 8 letters: the status bits say so.
    The next call clears the shared scratch and is exact again."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_05269_gb300 import wc
    dev = torch.device("cuda:0")
    out = _Outputs(torch, wc, dev)
    rng = np.random.default_rng(9)
    idx = rng.permutation(26 ** 4)[:wc.NOALLOC_MAX_BYTES // 5]
    letters = np.stack([(idx // 26 ** p) % 26 for p in range(4)], axis=1).astype(np.uint8) + ord("a")
    dense = np.concatenate([letters, np.full((idx.size, 1), ord(" "), np.uint8)], axis=1).reshape(-1)
    assert dense.size <= wc.NOALLOC_MAX_BYTES
    _, bits = out.count(torch, wc, torch.from_numpy(dense).to(dev))
    assert bits != 0, "a table overflow must set status bits"
    normal = corpus.generate("tiny", ndocs=20, seed=5).text[:500_000]
    m, bits = out.count(torch, wc, torch.from_numpy(np.ascontiguousarray(normal)).to(dev))
    assert bits == 0, f"status bits {bits} after an overflowing call"
    assert out.table(m) == oracle.count(np.ascontiguousarray(normal)).glob().as_list()


def test_no_alloc_rejects_large_documents():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_05269_gb300 import wc
    lib = wc.load()
    assert lib.wc_count_noalloc(None, wc.NOALLOC_MAX_BYTES + 1, None, None, None, None, 0, None, None, 0, None, 0,
                                None, None) == wc.WC_ERR_UNSUPPORTED
