"""GPU parity of the single-document path (wc_count) against the oracle.

Every case compares the exported table element by element: the same words in
the same order with the same integer counts (bit-exact).
"""
import numpy as np
import pytest

import corpus
import oracle
from gpu_util import assert_same, first_diff, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctr():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_05269_gb300 import wc
    c = wc.Counter(0)
    yield c
    c.close()


def check(ctr, data: bytes, offset: int = 0, opts=None, what: str = ""):
    t = ctr.count_checked(to_dev(data, offset), opts=opts)
    exp = t.export()
    want = oracle.count(data).glob()
    if not (exp[2].size == len(want) and np.array_equal(exp[2].astype(np.uint64), want.counts)
            and np.array_equal(exp[0], want.words)):
        raise AssertionError(f"{what}: first differences {first_diff(exp, want)}")
    assert_same(exp, want, what)
    return exp


EDGE = [
    b"", b" ", b"...", b"a", b"Z", b"1234", b"\xc3\xa9\xc3\xa9", b"abc123def", b"don't",
    b"caf\xc3\xa9 Cafe CAFE", b"@[`{AZaz", b"end word", b"word at start ", b"MiXeD mixed MIXED",
    b"tab\tsep\nnew\rline", b"a b a b a", b"\x00\x00ab\x00", b"\xc1\xda\xe1\xfa",
    bytes(b for i in range(256) for b in (i, 0x20)),
    b"I want to test MapReduce MapReduce is a cool algorithm to test.",
]


@pytest.mark.parametrize("i", range(len(EDGE)))
def test_edge_cases(ctr, i):
    check(ctr, EDGE[i], what=repr(EDGE[i][:40]))


@pytest.mark.parametrize("offset", [0, 1, 3, 7, 8, 15])
def test_unaligned_base(ctr, offset):
    c = corpus.generate("tiny", ndocs=3)
    check(ctr, c.text.tobytes(), offset=offset, what=f"offset {offset}")


def test_words_across_chunk_edges(ctr):
    from paper_2206_05269_gb300.wc import load  # noqa: F401
    rng = np.random.default_rng(11)
    chunk = 16384
    letters = np.frombuffer(b"abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ", np.uint8)
    for trial in range(12):
        n = int(rng.integers(3 * chunk - 40, 3 * chunk + 40))
        # mostly letters with sparse separators: words of every length cross every edge
        text = letters[rng.integers(0, letters.size, n)].copy()
        seps = rng.random(n) < rng.choice([0.02, 0.06, 0.2, 0.5])
        text[seps] = ord(" ")
        # force separators / letters right at the chunk edges
        for e in (chunk, 2 * chunk):
            for d in range(-3, 4):
                if 0 <= e + d < n:
                    text[e + d] = ord(" ") if (trial + d) % 3 == 0 else letters[(trial + d) % 26]
        check(ctr, text.tobytes(), offset=trial % 5, what=f"trial {trial}")


def test_long_words(ctr):
    base = b"abcdefghijklmnop"
    words = [base, base + b"a", base + b"b", base + b"aa", base + b"A", b"x" * 40, b"y" * 17, b"Y" * 17,
             base + b"qrstuvwxyz" * 3]
    rng = np.random.default_rng(5)
    toks = [words[i] for i in rng.integers(0, len(words), 3000)]
    check(ctr, b" ".join(toks), what="long words")
    check(ctr, b"-".join(toks), offset=9, what="long words unaligned")


@pytest.mark.parametrize("n", [100_000, 1 << 20])
def test_single_huge_word(ctr, n):
    data = b"Q" + b"q" * (n - 1)
    check(ctr, data, what=f"{n}-letter word")
    check(ctr, b"ab " + data + b" ab", what=f"{n}-letter word framed")


def test_long_word_recipe(ctr):
    c = corpus.generate("tiny", ndocs=40, len_max=40, len_tail=0.6, len_tail_mean=12.0, glue_prob=0.1,
                        high_prob=0.1, punct_prob=0.3)
    check(ctr, c.text.tobytes(), what="long-word corpus")


@pytest.mark.parametrize("name", ["tiny", "classes"])
def test_workload_as_one_document(ctr, name):
    c = corpus.generate(name)
    exp = check(ctr, c.text.tobytes(), what=name)
    assert int(exp[2].astype(np.uint64).sum()) == c.tokens


def test_large_recipe_64mb(ctr):
    c = corpus.generate("large", size_a=64e6)
    check(ctr, c.text.tobytes(), what="large recipe, 64 MB")


_MID = {}


@pytest.mark.parametrize("no_level1", [0, 1])
@pytest.mark.parametrize("size", [1e6, 4e6, 15e6])
def test_mid_sizes_with_and_without_level1(ctr, size, no_level1):
    """Single documents under 16 MB are counted with the claim-as-you-go
    shared-memory table (no sampling pass); at 1, 4 and 15 MB the table, and
    the all-global path with it switched off, equal the oracle."""
    if size not in _MID:
        c = corpus.generate("large", size_a=size)
        _MID[size] = (c.text.tobytes(), oracle.count(c.text).glob())
    data, want = _MID[size]
    t = ctr.count_checked(to_dev(data), opts=(0, 0, 0, no_level1))
    assert_same(t.export(), want, f"{size / 1e6:.0f} MB, no_level1={no_level1}")


def test_two_contexts_from_two_host_threads():
    """Two contexts, created and used from two host threads at once (kernel
    attributes are set per device under a lock), both count exactly."""
    import threading
    from paper_2206_05269_gb300 import wc
    texts = [corpus.generate("large", size_a=s).text.tobytes() for s in (20e6, 6e6)]
    results, errors = [None, None], []

    def work(i):
        try:
            c = wc.Counter(0)
            for _ in range(3):
                t = c.count_checked(to_dev(texts[i]))
                results[i] = t.export()
                t.free()
            c.close()
        except Exception as e:  # reported below
            errors.append(e)

    th = [threading.Thread(target=work, args=(i,)) for i in range(2)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert not errors, errors
    for i in range(2):
        assert_same(results[i], oracle.count(texts[i]).glob(), f"thread {i}")


def test_large_full_size_against_generator_truth(ctr):
    """The 1e9-byte workload as the benchmark runs it, checked in full against
    the generator's tally (which the oracle is pinned to) and the token count."""
    import torch
    c = corpus.generate("large")
    t = torch.from_numpy(c.text).to("cuda:0")
    table = ctr.count_checked(t)
    w, o, cnt = table.export()
    truth = c.truth()
    items = sorted(truth.items(), key=lambda kv: (-kv[1], kv[0]))
    want = oracle.Table.from_list(items)
    assert_same((w, o, cnt), want, "large full size")
    assert int(cnt.sum()) == c.tokens


def test_capacity_error_then_retry(ctr):
    from paper_2206_05269_gb300 import wc
    c = corpus.generate("tiny", ndocs=20)
    t = to_dev(c.text.tobytes())
    small = ctr.count(t, opts=(64, 64, 64))
    assert small.status() == wc.WC_ERR_CAPACITY
    with pytest.raises(wc.WcError) as e:
        small.size()
    assert e.value.status == wc.WC_ERR_CAPACITY
    small.free()
    check(ctr, c.text.tobytes(), opts=(64, 64, 64), what="after regrow")


def test_small_capacity_heavy_probing(ctr):
    # 4096 slots for ~3k distinct words: long probe chains, exact anyway
    c = corpus.generate("tiny", ndocs=60)
    check(ctr, c.text.tobytes(), opts=(4096, 1024, 1 << 16), what="dense table")


def test_merge_reduce_example(ctr):
    docs = [b" ".join([b"the"] * n) for n in (10, 4, 3)]
    tabs = [ctr.count_checked(to_dev(d)) for d in docs]
    m = ctr.merge(tabs)
    assert m.as_list() == [(b"the", 17)]


def test_merge_equals_concatenation(ctr):
    c = corpus.generate("tiny", ndocs=6, len_max=30, len_tail=0.3, len_tail_mean=8.0)
    docs = [c.text[c.offsets[i]:c.offsets[i + 1]].tobytes() for i in range(c.ndocs)]
    tabs = [ctr.count_checked(to_dev(d)) for d in docs]
    m = ctr.merge(tabs)
    want = oracle.count(b" ".join(docs)).glob()
    assert_same(m.export(), want, "merge")


def test_merge_unsynced_and_chained(ctr):
    """Tables not yet waited for (the merge sizes from their capacities),
    then a chain of merges of merges (sized from the known sizes)."""
    c = corpus.generate("tiny", ndocs=8, len_max=30, len_tail=0.3, len_tail_mean=8.0)
    docs = [c.text[c.offsets[i]:c.offsets[i + 1]].tobytes() for i in range(c.ndocs)]
    devs = [to_dev(d) for d in docs]
    tabs = [ctr.count(t) for t in devs]
    acc = ctr.merge(tabs[:4])
    for t in tabs[4:]:
        acc = ctr.merge([acc, t])
        assert acc.status() == 0
    assert_same(acc.export(), oracle.count(b" ".join(docs)).glob(), "chained merge")


def test_topk(ctr):
    c = corpus.generate("tiny", ndocs=10)
    t = ctr.count_checked(to_dev(c.text.tobytes()))
    want = oracle.count(c.text).glob()
    for k in (1, 7, 100, 10 ** 6):
        top = ctr.topk(t, k)
        assert top.as_list() == want.as_list()[:k]


def test_count_bits_32(ctr):
    from paper_2206_05269_gb300 import wc
    c32 = wc.Counter(0, count_bits=32)
    c = corpus.generate("tiny", ndocs=5)
    t = c32.count_checked(to_dev(c.text.tobytes()))
    w, o, cnt = t.export()
    assert cnt.dtype == np.uint32
    assert_same((w, o, cnt), oracle.count(c.text).glob(), "u32")
    t.free()
    c32.close()


def test_budget_rejects(ctr):
    from paper_2206_05269_gb300 import wc
    small = wc.Counter(0, budget=1 << 20)
    c = corpus.generate("large", size_a=8e6)
    with pytest.raises(wc.WcError) as e:
        small.count(to_dev(c.text.tobytes()))
    assert e.value.status == wc.WC_ERR_BUDGET
    small.close()


@pytest.mark.parametrize("piece", [0, 4096, 65536])
def test_count_from_host_memory_in_pieces(ctr, piece):
    """wc_count_host: the text copied and counted piece by piece equals the
    oracle, with pieces cut mid-text (a 10,000-letter word longer than a
    piece, long words repeated across pieces, words at the nominal cuts)."""
    import torch
    c = corpus.generate("tiny", ndocs=6, len_max=30, len_tail=0.3, len_tail_mean=8.0)
    arr = np.concatenate([c.text, np.frombuffer(b" " + b"Qx" * 5000 + b" tail", dtype=np.uint8), c.text[:70000]])
    host = torch.from_numpy(arr.copy()).pin_memory()
    t = ctr.count_host_checked(host, piece_bytes=piece)
    assert t.as_list() == oracle.count(arr).glob().as_list()


def test_count_from_host_memory_with_head_reuse(ctr):
    """A 64 MB text counted from host memory in 16 MB pieces (the first piece
    picks the shared-memory head, the others reuse it) equals the count of
    the same bytes already on the device."""
    import torch
    c = corpus.generate("large", size_a=64e6)
    host = torch.from_numpy(c.text).pin_memory()
    a = ctr.count_host_checked(host, piece_bytes=16 << 20)
    b = ctr.count_checked(host.to("cuda:0"))
    wa, oa, ca = a.export()
    wb, ob, cb = b.export()
    assert np.array_equal(ca, cb) and np.array_equal(oa, ob) and np.array_equal(wa, wb)


def test_count_from_host_memory_empty(ctr):
    import torch
    t = ctr.count_host_checked(torch.zeros(0, dtype=torch.uint8))
    assert t.size()[0] == 0


@pytest.mark.parametrize("chunk_mb", [1, 3])
def test_count_stream_chunks_equal_one_count(ctr, chunk_mb):
    """A host text counted chunk by chunk through one device buffer and
    merged equals the oracle: chunks cut between words, a word longer than a
    chunk extending its chunk, long words kept by their tables."""
    import torch
    text = corpus.generate("large", size_a=9e6).text
    longword = np.frombuffer(b" " + b"Qz" * (700 << 10) + b" ", np.uint8)  # 1.4 MB word
    full = np.concatenate([text[:4_000_000], longword, text[4_000_000:]])
    host = torch.from_numpy(full).pin_memory()
    t = ctr.count_stream(host, chunk_bytes=chunk_mb << 20)
    assert_same(t.export(), oracle.count(full).glob(), f"stream, {chunk_mb} MB chunks")


def test_count_stream_empty_and_small(ctr):
    import torch
    for data in (b"", b"a", b"The cat; the CAT's hat."):
        arr = np.frombuffer(data, np.uint8) if data else np.zeros(0, np.uint8)
        host = torch.from_numpy(np.array(arr, copy=True))
        t = ctr.count_stream(host)
        assert_same(t.export(), oracle.count(arr).glob(), f"stream {data!r}")


def test_counts_across_digit_boundaries(ctr):
    """Counts just above and below 2^8, 2^16 and 2^24: every count digit the
    token bound leaves in the sort is ordered (count desc, word asc)."""
    parts = [(b"a", (1 << 24) + 1), (b"b", (1 << 24) - 1), (b"c", (1 << 16) + 1), (b"dd", 1 << 16),
             (b"e", (1 << 16) - 1), (b"f", 257), (b"g", 256), (b"h", 255), (b"i", 1)]
    text = b"".join((w + b" ") * n for w, n in parts)
    t = ctr.count_checked(to_dev(text))
    assert t.as_list() == [(w, n) for w, n in parts]


def distinct_words(rng, n: int) -> list[bytes]:
    """n distinct lowercase words of 1-14 letters, in random order."""
    letters = np.frombuffer(b"abcdefghijklmnopqrstuvwxyz", np.uint8)
    seen = set()
    out = []
    while len(out) < n:
        w = letters[rng.integers(0, 26, int(rng.integers(1, 15)))].tobytes()
        if w not in seen:
            seen.add(w)
            out.append(w)
    return out


@pytest.mark.parametrize("ndistinct", [4095, 4096, 4097, 8192, 8193, 12289, 40000, 65537])
def test_distinct_counts_around_sort_tiles(ctr, ndistinct):
    """Tables of exactly 4096 * k - 1 ... 4096 * k + 1 distinct words and
    larger: the sort's runs of 4096 entries and every merge of them.  Most
    counts are 1-3, so runs of equal counts span tiles and are ordered by the
    word; a few words of 17+ letters share their first 16 letters and count."""
    rng = np.random.default_rng(ndistinct)
    words = distinct_words(rng, ndistinct - 6)
    words += [b"sharedprefixabcd" + s for s in (b"zz", b"a", b"mmm", b"b", b"zzz", b"")]
    counts = rng.choice([1, 1, 1, 2, 2, 3, 7, 40], size=len(words))
    counts[-6:] = 2
    tokens = np.repeat(np.arange(len(words)), counts)
    rng.shuffle(tokens)
    data = b" ".join(words[i] for i in tokens)
    exp = check(ctr, data, what=f"{ndistinct} distinct words")
    assert exp[2].size == ndistinct
