"""Long words (17 letters or more) in single-document counts of 16 MB or
more: the counting kernel queues them and a second kernel inserts them,
first counting each chunk's repeats in a shared table (two queued words are
merged only when hash, length and both 16-letter ends agree, which for words
of at most 32 letters is the whole word).  A queue that fills up (2^21 words
a launch) falls back to inserting in place.  Both paths against the oracle,
with words that share their first or last 16 letters, mixed case, and
lengths on both sides of 32.
"""
import numpy as np
import pytest

import oracle
from gpu_util import assert_same, to_dev

pytestmark = pytest.mark.gpu

LETTERS = np.frombuffer(b"abcdefghijklmnopqrstuvwxyz", np.uint8)


@pytest.fixture(scope="module")
def ctr():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_05269_gb300 import wc
    c = wc.Counter(0)
    yield c
    c.close()


def rand_word(rng, n: int) -> bytes:
    return LETTERS[rng.integers(0, 26, n)].tobytes()


def long_vocab(rng, n: int) -> list[bytes]:
    """n distinct long words: many share a 16-letter head or tail with
    others, lengths 17-24 mostly, some 25-64."""
    heads = [rand_word(rng, 16) for _ in range(40)]
    tails = [rand_word(rng, 16) for _ in range(40)]
    out = set()
    while len(out) < n:
        kind = rng.integers(0, 4)
        mid = rand_word(rng, int(rng.integers(1, 9)) if rng.random() < 0.85 else int(rng.integers(9, 33)))
        if kind == 0:
            w = heads[rng.integers(0, 40)] + mid
        elif kind == 1:
            w = mid + tails[rng.integers(0, 40)]
        elif kind == 2:
            w = heads[rng.integers(0, 40)] + mid + tails[rng.integers(0, 40)]
        else:
            w = rand_word(rng, int(rng.integers(17, 25)))
        out.add(w)
    return sorted(out)


def build_text(rng, vocab: list[bytes], n_long: int, n_short: int, zipf_s: float) -> bytes:
    """n_long long words drawn Zipf(zipf_s) from vocab (a quarter of them
    partly upper-cased), shuffled with n_short short filler words."""
    ranks = np.arange(1, len(vocab) + 1, dtype=np.float64)
    p = ranks ** -zipf_s
    p /= p.sum()
    idx = rng.choice(len(vocab), size=n_long, p=p)
    words = [vocab[i] for i in idx]
    for j in np.nonzero(rng.random(n_long) < 0.25)[0]:  # mixed case: the same word
        a = np.frombuffer(words[j], np.uint8).copy()
        a[rng.random(a.size) < 0.3] -= 32
        words[j] = a.tobytes()
    short = [b"the", b"of", b"and", b"a", b"to", b"in", b"word"]
    words += [short[i] for i in rng.integers(0, len(short), n_short)]
    order = rng.permutation(len(words))
    seps = [b" ", b", ", b"\n", b"-", b"7"]
    sep = rng.integers(0, len(seps), len(words))
    return b"".join(words[j] + seps[int(s)] for j, s in zip(order, sep))


def count_and_check(ctr, data: bytes, what: str):
    t = ctr.count_checked(to_dev(data))
    assert_same(t.export(), oracle.count(data).glob(), what)
    t.free()


def test_deferred_long_words_aggregated(ctr):
    """About 20 MB: dense long words with heavy repeats (each chunk of the
    queue holds the frequent ones many times) among short fillers."""
    rng = np.random.default_rng(5)
    vocab = long_vocab(rng, 3000)
    data = build_text(rng, vocab, n_long=700_000, n_short=600_000, zipf_s=1.1)
    assert len(data) >= 16 << 20
    count_and_check(ctr, data, "deferred long words")


def test_deferred_long_word_queue_overflow(ctr):
    """About 60 MB of long words only: more than the queue holds in one
    launch, so the rest are inserted by the counting kernel itself."""
    rng = np.random.default_rng(6)
    vocab = long_vocab(rng, 2000)
    data = build_text(rng, vocab, n_long=2_300_000, n_short=0, zipf_s=0.9)
    assert len(data) >= 16 << 20
    count_and_check(ctr, data, "deferred long words, queue overflow")
