"""The allocation-free entry point (wc_count_noalloc) gives the same table as
wc_count.

It exists for callers that may not allocate device memory (another component
owns the device memory, or allocation is forbidden after start-up); its
scratch is a fixed array inside the library.  The test calls it through the C
ABI twice in a row on different documents, because every call reuses the same
array and must clear what the previous call left behind.  It runs last so that
a failure here never hides the other tests, and it passes alone as well.
"""
import numpy as np
import pytest

import corpus

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


def test_no_alloc_matches_wc_count_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_05269_gb300 import wc
    dev = torch.device("cuda:0")
    ctr = wc.Counter(0)
    # the caller allocates its own inputs and outputs
    cap, lcap = wc.NOALLOC_ENTRIES, wc.NOALLOC_LONG
    khi = torch.zeros(cap, dtype=torch.int64, device=dev)
    klo = torch.zeros(cap, dtype=torch.int64, device=dev)
    cnt = torch.zeros(cap, dtype=torch.int64, device=dev)
    lref = torch.zeros(cap, dtype=torch.int32, device=dev)
    loff = torch.zeros(lcap, dtype=torch.int64, device=dev)
    llen = torch.zeros(lcap, dtype=torch.int64, device=dev)
    arena = torch.zeros(wc.NOALLOC_MAX_BYTES * 2, dtype=torch.uint8, device=dev)
    meta = torch.zeros(8, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    docs = [
        corpus.generate("tiny", ndocs=60, len_max=30, len_tail=0.3, len_tail_mean=8.0).text[:900_000],
        corpus.generate("classes", ndocs=8, seed=77).text[:300_000],
    ]
    for k, data in enumerate(docs):
        text = torch.from_numpy(np.ascontiguousarray(data)).to(dev)
        wc.wc_count_noalloc(text.data_ptr(), text.numel(), khi.data_ptr(), klo.data_ptr(), cnt.data_ptr(),
                            lref.data_ptr(), cap, loff.data_ptr(), llen.data_ptr(), lcap, arena.data_ptr(),
                            arena.numel(), meta.data_ptr(), int(stream.cuda_stream))
        torch.cuda.synchronize()
        m = meta.cpu().numpy().view(np.uint64)
        assert int(m[7]) & 0xFFFFFFFF == 0, f"call {k}: status bits {int(m[7])}"
        n = int(m[0])
        got = _words(khi.cpu().numpy().view(np.uint64), klo.cpu().numpy().view(np.uint64),
                     cnt.cpu().numpy().view(np.uint64), lref.cpu().numpy(), loff.cpu().numpy(),
                     llen.cpu().numpy(), arena.cpu().numpy(), n)
        want = ctr.count_checked(text).as_list()
        assert got == want, f"call {k}: differs from wc_count"
        assert int(m[3]) == sum(c for _, c in want)
    ctr.close()


def test_no_alloc_rejects_large_documents():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_05269_gb300 import wc
    lib = wc.load()
    assert lib.wc_count_noalloc(None, wc.NOALLOC_MAX_BYTES + 1, None, None, None, None, 0, None, None, 0, None, 0,
                                None, None) == wc.WC_ERR_UNSUPPORTED
