"""GPU parity of batched counting (wc_count_batched): per-document, per-class
and global tables and the class-ratio ranking, bit-exact against the oracle."""
import numpy as np
import pytest

import corpus
import oracle
from gpu_util import assert_same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctr():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_05269_gb300 import wc
    c = wc.Counter(0, count_bits=32)
    yield c
    c.close()


def run_batched(ctr, text: np.ndarray, offsets: np.ndarray, classes=None, nclasses=0, checked=False):
    import torch
    dev = torch.device("cuda:0")
    t = torch.from_numpy(np.ascontiguousarray(text, dtype=np.uint8)).to(dev) if text.size else \
        torch.zeros(16, dtype=torch.uint8, device=dev)
    o = torch.from_numpy(np.ascontiguousarray(offsets, dtype=np.uint64).view(np.int64)).to(dev)
    cl = torch.from_numpy(np.ascontiguousarray(classes, dtype=np.uint32).view(np.int32)).to(dev) \
        if classes is not None else None
    h = np.ascontiguousarray(offsets, dtype=np.uint64)
    b = ctr.count_batched_checked(t, o, h, cl, nclasses) if checked else ctr.count_batched(t, o, h, cl, nclasses)
    return b, (t, o, cl)


def test_dense_documents_recount_at_exact_bounds(ctr):
    """Documents denser in distinct words than the capacity estimate (a
    three-byte word per token): the estimated count reports
    WC_ERR_CAPACITY, the count at the exact bounds is exact."""
    from paper_2206_05269_gb300 import wc
    rng = np.random.default_rng(5)
    vocab = [bytes([97 + i % 26, 97 + (i // 26) % 26]) for i in range(676)]
    docs = [b" ".join(vocab[w] for w in rng.permutation(676)[:int(rng.integers(300, 676))]) for _ in range(40)]
    text = np.frombuffer(b"".join(docs), np.uint8)
    offs = np.cumsum([0] + [len(d) for d in docs]).astype(np.uint64)
    r = oracle.count(text, offs)
    b, keep = run_batched(ctr, text, offs)
    assert b.status() == wc.WC_ERR_CAPACITY
    b.free()
    b, keep = run_batched(ctr, text, offs, checked=True)
    check_docs(b, r, len(docs))
    assert_same(b.table(wc.WC_TABLE_GLOBAL).export(), r.glob(), "global")


def check_docs(b, r, ndocs, sample=None):
    from paper_2206_05269_gb300 import wc
    assert b.status() == wc.WC_OK
    ds, dn, w, o, c = b.export()
    docs = range(ndocs) if sample is None else sample
    for d in docs:
        want = r.doc(d)
        s0, n = int(ds[d]), int(dn[d])
        assert n == len(want), f"doc {d}: {n} words vs oracle {len(want)}"
        got_w = w[o[s0]:o[s0 + n]] if n else np.zeros(0, np.uint8)
        assert np.array_equal(got_w, want.words), f"doc {d}: words differ"
        assert np.array_equal((o[s0:s0 + n + 1] - o[s0]).astype(np.uint64), want.offs), f"doc {d}: offsets"
        assert np.array_equal(c[s0:s0 + n].astype(np.uint64), want.counts), f"doc {d}: counts differ"


def test_tiny_workload_docs_and_global(ctr):
    from paper_2206_05269_gb300 import wc
    c = corpus.generate("tiny")
    r = oracle.count(c.text, c.offsets)
    b, keep = run_batched(ctr, c.text, c.offsets)
    check_docs(b, r, c.ndocs)
    g = b.table(wc.WC_TABLE_GLOBAL)
    assert_same(g.export(), r.glob(), "global")
    # a per-document view equals the bulk export
    v = b.table(wc.WC_TABLE_DOC, 7)
    assert v.as_list() == r.doc(7).as_list()


def test_class_workload_tables_and_ratio(ctr):
    from paper_2206_05269_gb300 import wc
    c = corpus.generate("classes")
    r = oracle.count(c.text, c.offsets, c.classes, c.nclasses)
    b, keep = run_batched(ctr, c.text, c.offsets, c.classes, c.nclasses)
    check_docs(b, r, c.ndocs, sample=range(0, c.ndocs, 7))
    assert_same(b.table(wc.WC_TABLE_GLOBAL).export(), r.glob(), "global")
    for k in range(c.nclasses):
        tab = b.table(wc.WC_TABLE_CLASS, k)
        assert_same(tab.export(), r.cls(k), f"class {k}")
        idx, cin, cout = wc.wc_class_ratio_topk(ctr.ctx, b.handle, k, 50, 0)
        want = r.ratio_topk(k, 50)
        ctab = r.cls(k)
        got = [(ctab.word(int(i)), int(a), int(o)) for i, a, o in zip(idx, cin, cout)]
        assert got == want, f"class {k} ratio ranking"


def check_ratio(ctr, b, r, cls, k):
    from paper_2206_05269_gb300 import wc
    idx, cin, cout = wc.wc_class_ratio_topk(ctr.ctx, b.handle, cls, k, 0)
    want = r.ratio_topk(cls, k)
    ctab = r.cls(cls)
    got = [(ctab.word(int(i)), int(a), int(o)) for i, a, o in zip(idx, cin, cout)]
    assert got == want, f"class {cls}, k={k}: ratio ranking"


def test_ratio_topk_every_k(ctr):
    """The ranking for k across the selection's regimes: one sorted slice,
    several rounds of slices, the largest k the rounds take (512), the
    arg-best path above it, and k at and above the class's size."""
    c = corpus.generate("classes", ndocs=120)
    r = oracle.count(c.text, c.offsets, c.classes, c.nclasses)
    b, keep = run_batched(ctr, c.text, c.offsets, c.classes, c.nclasses)
    for cls in range(c.nclasses):
        n = len(r.cls(cls).counts)
        for k in (1, 7, 50, 511, 512, 513, 700, n, n + 5):
            check_ratio(ctr, b, r, cls, k)


def test_ratio_topk_ties(ctr):
    """Many equal ratios (every class draws from one small vocabulary): the
    order falls to cin, then to the word."""
    rng = np.random.default_rng(11)
    vocab = [bytes([97 + i % 26, 97 + (i // 26) % 26]) for i in range(1500)]
    docs, classes = [], []
    for d in range(60):
        words = rng.choice(len(vocab), int(rng.integers(50, 400)))
        docs.append(b" ".join(vocab[w] for w in words))
        classes.append(d % 3)
    text = np.frombuffer(b"\n".join(docs) + b"\n", np.uint8)
    lens = [len(d) + 1 for d in docs]
    offs = np.cumsum([0] + lens).astype(np.uint64)
    cl = np.array(classes, np.uint32)
    r = oracle.count(text, offs, cl, 3)
    b, keep = run_batched(ctr, text, offs, cl, 3, checked=True)
    for cls in range(3):
        for k in (3, 64, 300, 512, 900, 5000):
            check_ratio(ctr, b, r, cls, k)


def test_edges_long_words_spills_and_splits(ctr):
    rng = np.random.default_rng(3)
    docs = [b"", b"   ", b"abc", b"def", b"Abc abc ABC", b"12 34", b"x" * 40 + b" " + b"X" * 40,
            b"-".join([b"abcdefghijklmnopq%c" % (97 + i % 26) + bytes([97 + i // 26]) for i in range(120)]),
            # more distinct words than a small document's shared table holds
            b" ".join(bytes([97 + (i // 676) % 26, 97 + (i // 26) % 26, 97 + i % 26]) for i in range(2000)),
            ]
    # a document above the split threshold (counted in ranges across blocks)
    big = corpus.generate("tiny", ndocs=1, size_a=60000, size_b=60000, len_max=30, len_tail=0.3,
                          len_tail_mean=8.0)
    docs.append(big.text.tobytes())
    # words touching document edges on both sides
    docs += [b"edge", b"word", b"Edge"]
    for _ in range(20):
        n = int(rng.integers(1, 3000))
        arr = rng.choice(np.frombuffer(b"abcXYZ .,\n1\xc3", np.uint8), n)
        docs.append(arr.tobytes())
    text = np.frombuffer(b"".join(docs), np.uint8)
    offs = np.cumsum([0] + [len(d) for d in docs]).astype(np.uint64)
    r = oracle.count(text, offs)
    b, keep = run_batched(ctr, text, offs)
    check_docs(b, r, len(docs))


def test_batched_equals_single_document_counts(ctr):
    c = corpus.generate("batched", ndocs=300)
    b, keep = run_batched(ctr, c.text, c.offsets)
    lists = b.doc_lists()
    from gpu_util import to_dev
    for d in range(0, c.ndocs, 37):
        seg = c.text[c.offsets[d]:c.offsets[d + 1]].tobytes()
        single = ctr.count_checked(to_dev(seg)).as_list()
        assert lists[d] == single, f"doc {d}"


def test_batched_workload_full_size_sampled(ctr):
    """The 100k-document workload as the benchmark runs it: every document's
    table checked for the token invariant, 1,500 sampled documents checked
    word by word against the oracle, the global table against the generator."""
    from paper_2206_05269_gb300 import wc
    c = corpus.generate("batched")
    b, keep = run_batched(ctr, c.text, c.offsets)
    ds, dn, w, o, cnt = b.export()
    rng = np.random.default_rng(1)
    sample = np.sort(rng.choice(c.ndocs, 1500, replace=False))
    sub_docs = [c.text[c.offsets[d]:c.offsets[d + 1]] for d in sample]
    sub_text = np.concatenate(sub_docs)
    sub_offs = np.cumsum([0] + [x.size for x in sub_docs]).astype(np.uint64)
    r = oracle.count(sub_text, sub_offs)
    for j, d in enumerate(sample):
        want = r.doc(j)
        s0, n = int(ds[d]), int(dn[d])
        assert n == len(want)
        assert np.array_equal(cnt[s0:s0 + n].astype(np.uint64), want.counts)
        assert np.array_equal(w[o[s0]:o[s0 + n]], want.words)
    assert int(cnt.astype(np.uint64).sum()) == c.tokens
    g = b.table(wc.WC_TABLE_GLOBAL)
    items = sorted(c.truth().items(), key=lambda kv: (-kv[1], kv[0]))
    assert_same(g.export(), oracle.Table.from_list(items), "global vs generator")


def test_batch_topk_rows_are_each_documents_first_rows(ctr):
    """wc_batch_topk: every document's first min(k, n) rows, gathered into one
    table, equal the oracle's top k of that document (long words included)."""
    c = corpus.generate("tiny", ndocs=40, len_max=30, len_tail=0.3, len_tail_mean=8.0)
    r = oracle.count(c.text, c.offsets)
    b, keep = run_batched(ctr, c.text, c.offsets)
    for k in (1, 7, 100, 100000):
        top, first, n = b.topk(k)
        w, o, cnt = top.export()
        assert cnt.size == int(n.sum())
        for d in range(c.ndocs):
            want = r.doc(d).as_list()[:k]
            s0, m = int(first[d]), int(n[d])
            got = [(w[o[i]:o[i + 1]].tobytes(), int(cnt[i])) for i in range(s0, s0 + m)]
            assert got == want, f"k={k} doc {d}"


def test_class_id_out_of_range_is_an_error(ctr):
    """A class id not below nclasses is rejected when the class tables are
    built (WC_ERR_INVALID_ARG), not read past the class-table array."""
    from paper_2206_05269_gb300 import wc
    c = corpus.generate("tiny", ndocs=12)
    classes = np.zeros(c.ndocs, dtype=np.uint32)
    classes[5] = 3  # nclasses = 2
    b, keep = run_batched(ctr, c.text, c.offsets, classes, 2)
    assert b.status() == wc.WC_OK  # per-document tables do not depend on classes
    with pytest.raises(wc.WcError) as ei:
        b.table(wc.WC_TABLE_CLASS, 0)
    assert ei.value.status == wc.WC_ERR_INVALID_ARG


def test_class_tables_many_distinct_words(ctr):
    """Class and global tables of documents with little vocabulary overlap
    (the first-size estimate is exceeded and the tables are rebuilt at the
    exact bound) still equal the oracle."""
    from paper_2206_05269_gb300 import wc
    c = corpus.generate("classes", ndocs=40, vocab_size=400000, zipf_s=0.6, seed=123)
    r = oracle.count(c.text, c.offsets, c.classes, c.nclasses)
    b, keep = run_batched(ctr, c.text, c.offsets, c.classes, c.nclasses)
    assert_same(b.table(wc.WC_TABLE_GLOBAL).export(), r.glob(), "global")
    for k in range(c.nclasses):
        assert_same(b.table(wc.WC_TABLE_CLASS, k).export(), r.cls(k), f"class {k}")


def test_vocabulary_ids_decode_to_the_oracle():
    """Vocabulary-id export: the vocabulary is the global word set in word
    order with global counts, and every document's (id, count) rows decode to
    the oracle's table of that document, row for row."""
    import torch
    from paper_2206_05269_gb300 import wc
    ctr = wc.Counter(0, count_bits=32)
    c = corpus.generate("batched", ndocs=600)
    docs_extra = [b"", b"x" * 40 + b" Y" * 3, b"-".join([b"abcdefghijklmnopq%c" % (97 + i % 26) for i in range(60)])]
    text = np.concatenate([c.text, np.frombuffer(b"".join(docs_extra), np.uint8)])
    offs = np.concatenate([c.offsets, c.offsets[-1] + np.cumsum([len(d) for d in docs_extra])]).astype(np.uint64)
    b, keep = run_batched(ctr, text, offs, checked=True)
    r = oracle.count(text, offs)
    v = b.vocab()
    vw, vo, vc = v.export()
    vocab = [vw[vo[i]:vo[i + 1]].tobytes() for i in range(vc.size)]
    gd = r.glob().as_dict()
    assert vocab == sorted(gd), "vocabulary: the global words in word order"
    assert [int(x) for x in vc] == [gd[w] for w in vocab], "vocabulary counts"
    ds, dn, ids, counts = b.export_ids()
    ndocs = offs.size - 1
    for d in range(ndocs):
        s0, n = int(ds[d]), int(dn[d])
        got = [(vocab[int(i)], int(k)) for i, k in zip(ids[s0:s0 + n], counts[s0:s0 + n])]
        assert got == r.doc(d).as_list(), f"doc {d}"
    # the same rows as the word export, in the same order
    _, _, w, o, cw = b.export()
    assert np.array_equal(cw, counts)
    assert all(vocab[int(ids[j])] == w[o[j]:o[j + 1]].tobytes() for j in range(0, ids.size, 97))
    b.free()
    ctr.close()
