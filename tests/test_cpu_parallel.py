"""The paper-style parallel CPU baseline counts what the oracle counts:
same distinct words, token total and largest count, whatever the thread
count (pieces are cut between words)."""
import numpy as np
import pytest

import corpus
import cpu_parallel
import oracle


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_parallel_baseline_matches_oracle(threads):
    text = corpus.generate("large", size_a=4e6).text
    want = oracle.count(text).glob()
    got = cpu_parallel.count(text, threads)
    assert got["distinct"] == len(want)
    assert got["tokens"] == int(want.counts.sum())
    assert got["top_count"] == int(want.counts[0])


def test_parallel_baseline_edges():
    for s in (b"", b"a", b"abc", b"ab cd", b"x" * 1000, b"Ab-aB ab!"):
        text = np.frombuffer(s, np.uint8)
        want = oracle.count(text).glob()
        got = cpu_parallel.count(text, 5)
        assert got["distinct"] == len(want) and got["tokens"] == int(want.counts.sum())


def test_hybrid_matrix_row_sums_equal_the_oracle():
    """The paper's CPU map + padded matrix: each row's sum (here on the host)
    is the word's total count; the matrix is zero past each count list."""
    import corpus
    import oracle
    from cpu_parallel import HybridMap
    c = corpus.generate("tiny", ndocs=60)
    hy = HybridMap(c.text, c.offsets, threads=4)
    m = np.zeros((hy.rows, hy.cols), dtype=np.uint32)
    hy.fill(m)
    sums = m.astype(np.uint64).sum(axis=1)
    got = dict(zip(hy.words(), (int(x) for x in sums)))
    assert got == oracle.count(c.text, c.offsets).glob().as_dict()
    assert hy.cols == max(int((m[i] > 0).sum()) for i in range(hy.rows))
