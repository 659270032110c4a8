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
