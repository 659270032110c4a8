"""The read-ceiling pass (wc_read_ceiling) reads every byte of the text
exactly once at any alignment: its fold of the bytes equals the same fold
computed on the host."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def host_fold(buf: np.ndarray, base_addr: int) -> int:
    """Bytes before the first 16-byte boundary and after the last whole
    vector added one by one; each whole vector (four little-endian words
    w0..w3) adds (w0 ^ w1) + (w2 ^ w3)."""
    n = buf.size
    head = min((-base_addr) % 16, n)
    nv = (n - head) // 16
    mid = buf[head:head + nv * 16].view(np.uint32).reshape(-1, 4).astype(np.uint64)
    total = int(((mid[:, 0] ^ mid[:, 1]) + (mid[:, 2] ^ mid[:, 3])).sum()) if nv else 0
    total += int(buf[:head].astype(np.uint64).sum()) + int(buf[head + nv * 16:].astype(np.uint64).sum())
    return total % (1 << 64)


@pytest.mark.parametrize("offset", [0, 1, 7, 15])
@pytest.mark.parametrize("size", [0, 1, 15, 16, 17, 4096 + 5, (1 << 22) + 11])
def test_read_ceiling_reads_every_byte_once(offset, size):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_05269_gb300 import wc
    rng = np.random.default_rng(size + offset)
    host = rng.integers(0, 256, size, dtype=np.uint8)
    buf = torch.empty(size + offset + 32, dtype=torch.uint8, device="cuda:0")
    t = buf[offset:offset + size]
    if size:
        t.copy_(torch.from_numpy(host))
    sink = torch.zeros(1024, dtype=torch.int64, device="cuda:0")
    st = wc.wc_read_ceiling(t.data_ptr(), size, sink.data_ptr(), 1024, 0)
    assert st == wc.WC_OK
    torch.cuda.synchronize()
    got = int(sink.cpu().numpy().view(np.uint64).astype(object).sum()) % (1 << 64)
    assert got == host_fold(host, t.data_ptr())
