"""The paper's hybrid pipeline (CPU map, padded count matrix, host -> device
copy, GPU row sums; Sec. 3.3 and Sec. 4.1): the GPU row sums of the matrix
are the oracle's global counts, and wc_row_sums equals the host's row sums on
ragged shapes (columns not a multiple of the unrolled loads, empty rows)."""
import numpy as np
import pytest

import corpus
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def gpu_row_sums(torch, m: np.ndarray) -> np.ndarray:
    from paper_2206_05269_gb300 import wc
    dm = torch.from_numpy(m).to("cuda:0")
    out = torch.full((max(1, m.shape[0]),), -1, dtype=torch.int64, device="cuda:0")
    wc.wc_row_sums(dm.data_ptr(), m.shape[0], m.shape[1], out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return out.cpu().numpy().view(np.uint64)[:m.shape[0]]


@pytest.mark.parametrize("shape", [(1, 1), (7, 33), (100, 127), (3, 1000), (5000, 129), (1, 100_000), (64, 0)])
def test_row_sums_ragged(torch, shape):
    rng = np.random.default_rng(shape[0] * 7 + shape[1])
    m = rng.integers(0, 1 << 32, size=shape, dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(gpu_row_sums(torch, m), m.astype(np.uint64).sum(axis=1))


def test_hybrid_pipeline_equals_oracle(torch):
    from cpu_parallel import HybridMap
    c = corpus.generate("classes", ndocs=200)
    hy = HybridMap(c.text, c.offsets)
    m = torch.empty((hy.rows, hy.cols), dtype=torch.int32).pin_memory()
    hy.fill(m)
    sums = gpu_row_sums(torch, m.numpy().view(np.uint32))
    assert dict(zip(hy.words(), (int(x) for x in sums))) == oracle.count(c.text, c.offsets).glob().as_dict()
