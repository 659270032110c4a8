"""Pins the oracle to facts that do not come from the oracle itself.

- the worked example of Sec. 2 and the reduce example of Sec. 3.3 (golden
  fixtures with the paper's printed values);
- a library special case: Python's ``re`` + ``bytes.lower`` + ``Counter``;
- brute force over every short string of an alphabet that holds letters, the
  bytes just outside the letter ranges and a high byte whose low 7 bits are a
  letter;
- the generator's own tally of the words it wrote;
- invariants: total count = word starts, class and global sums, document
  permutation, concatenation = merge, the ceil(B/2) bound;
- the class-ratio ranking against exact ``fractions.Fraction`` sorting.
"""
import collections
import fractions
import itertools
import re

import numpy as np
import pytest

import corpus
import oracle
from conftest import read_golden

WORD_RE = re.compile(rb"[A-Za-z]+")


def lib_counts(data: bytes) -> collections.Counter:
    return collections.Counter(w.lower() for w in WORD_RE.findall(data))


def sorted_items(counter) -> list:
    return sorted(counter.items(), key=lambda kv: (-kv[1], kv[0]))


def word_starts(text: np.ndarray) -> int:
    t = np.asarray(text, dtype=np.uint8)
    let = ((t >= 65) & (t <= 90)) | ((t >= 97) & (t <= 122))
    prev = np.concatenate([[False], let[:-1]])
    return int((let & ~prev).sum())


def test_worked_example_sec2():
    rows = read_golden("worked_example_sec2.txt")
    docs = [v.encode() for k, v in rows if k == "doc"]
    parts = [v for k, v in rows if k == "part"]
    printed = []
    for p in parts:
        c = collections.Counter()
        for item in p.split(","):
            w, n = item.split()
            c[w.encode()] += int(n)
        printed.append(c)
    want = printed[0] + printed[1]
    text = b"".join(docs)
    offs = np.cumsum([0] + [len(d) for d in docs]).astype(np.uint64)
    r = oracle.count(text, offs)
    assert r.glob().as_list() == sorted_items(want)
    assert sum(want.values()) == 12 and len(want) == 9
    # per document: the two printed partitions come from splitting the
    # alphabetically sorted 12 words 6/6, which the oracle's tokens reproduce
    toks = sorted(w for d in range(2) for w, c in r.doc(d).as_list() for _ in range(c))
    assert collections.Counter(toks[:6]) == printed[0]
    assert collections.Counter(toks[6:]) == printed[1]
    assert r.doc(0).as_dict() == {b"i": 1, b"want": 1, b"to": 1, b"test": 1, b"mapreduce": 1}
    # the document edge separates "MapReduce" and "MapReduce" even with no byte between
    assert r.glob().as_dict()[b"mapreduce"] == 2


def test_reduce_example_sec3_3():
    rows = dict(read_golden("merge_example_sec3_3.txt"))
    word = rows["word"].encode()
    per_doc = [int(x) for x in rows["per_doc"].split()]
    docs = [b" ".join([word.upper() if i % 2 else word for i in range(n)]) + b"." for n in per_doc]
    text = b"".join(docs)
    offs = np.cumsum([0] + [len(d) for d in docs]).astype(np.uint64)
    r = oracle.count(text, offs)
    assert [r.doc(d).as_dict()[word] for d in range(3)] == per_doc
    assert r.glob().as_dict()[word] == int(rows["total"])
    merged = oracle.merge([r.doc(d) for d in range(3)])
    assert merged.as_list() == [(word, int(rows["total"]))]


@pytest.mark.parametrize("data", [
    b"", b" ", b"...", b"a", b"Z", b"1234", b"\xc3\xa9\xc3\xa9", b"abc123def", b"don't",
    b"caf\xc3\xa9 Cafe CAFE", b"@[`{AZaz", b"x" * 100_000, b"end word", b"word at start ",
    b"MiXeD mixed MIXED", b"tab\tsep\nnew\rline",
])
def test_small_cases_match_library(data):
    r = oracle.count(data)
    assert r.glob().as_list() == sorted_items(lib_counts(data))
    assert r.glob().tokens == word_starts(np.frombuffer(data, dtype=np.uint8)) if data else True


def test_every_byte_classified():
    # exactly the 52 ASCII letters are word bytes; lowercasing maps A-Z to a-z
    data = bytes(b for i in range(256) for b in (i, 0x20))
    got = oracle.count(data).glob().as_dict()
    want = {bytes([c]): 2 for c in range(97, 123)}
    assert got == want


def test_brute_force_short_strings():
    alphabet = [ord("a"), ord("Z"), ord("@"), ord("["), ord("`"), ord("{"), 0xC1, ord(" ")]
    docs = [bytes(s) for n in range(0, 6) for s in itertools.product(alphabet, repeat=n)]
    text = b"".join(docs)
    offs = np.cumsum([0] + [len(d) for d in docs]).astype(np.uint64)
    r = oracle.count(text, offs)
    for d, data in enumerate(docs):
        assert r.doc(d).as_list() == sorted_items(lib_counts(data)), data
    assert r.glob().as_dict() == dict(sum((lib_counts(d) for d in docs), collections.Counter()))


@pytest.mark.parametrize("name", ["tiny", "classes"])
def test_generator_truth_and_invariants(name):
    c = corpus.generate(name)
    r = oracle.count(c.text, c.offsets, c.classes, c.nclasses)
    g = r.glob()
    assert g.as_dict() == c.truth()
    assert g.tokens == c.tokens == word_starts(c.text)
    assert g.tokens <= (c.nbytes + 1) // 2
    # library special case on the whole corpus (document edges are spaces here)
    assert g.as_list() == sorted_items(lib_counts(c.text.tobytes()))
    # class tables are sums of their documents; classes sum to global
    if c.nclasses:
        tot = collections.Counter()
        for k in range(c.nclasses):
            want = collections.Counter()
            for d in np.nonzero(c.classes == k)[0]:
                want.update(r.doc(int(d)).as_dict())
            assert r.cls(k).as_dict() == dict(want) == c.truth(k)
            tot.update(want)
        assert dict(tot) == g.as_dict()
    sample = range(0, c.ndocs, max(1, c.ndocs // 40))
    for d in sample:
        seg = c.text[c.offsets[d]:c.offsets[d + 1]].tobytes()
        assert r.doc(d).as_list() == sorted_items(lib_counts(seg))


def test_permutation_and_concatenation():
    c = corpus.generate("tiny", ndocs=30)
    docs = [c.text[c.offsets[d]:c.offsets[d + 1]].tobytes() for d in range(c.ndocs)]
    rng = np.random.default_rng(7)
    perm = rng.permutation(len(docs))
    text2 = b"".join(docs[i] for i in perm)
    offs2 = np.cumsum([0] + [len(docs[i]) for i in perm]).astype(np.uint64)
    a = oracle.count(c.text, c.offsets).glob()
    b = oracle.count(text2, offs2).glob()
    assert a.as_list() == b.as_list()
    # count(A + sep + B) = merge(count(A), count(B))
    A, B = docs[0], docs[1]
    whole = oracle.count(A + b" " + B).glob()
    merged = oracle.merge([oracle.count(A).glob(), oracle.count(B).glob()])
    assert whole.as_list() == merged.as_list()


def test_document_edge_is_separator():
    text = b"abcdef"
    r = oracle.count(text, np.array([0, 3, 6], dtype=np.uint64))
    assert r.glob().as_dict() == {b"abc": 1, b"def": 1}
    r = oracle.count(text, np.array([0, 6], dtype=np.uint64))
    assert r.glob().as_dict() == {b"abcdef": 1}


def test_tie_order_prefix_first():
    r = oracle.count(b"ab a abc b aa ab a abc b aa")
    assert [w for w, _ in r.glob().as_list()] == [b"a", b"aa", b"ab", b"abc", b"b"]


def _fraction_rank(cls_tab: dict, glob_tab: dict, k: int):
    inf = fractions.Fraction(10 ** 30)

    def key(w):
        cin = cls_tab[w]
        cout = glob_tab[w] - cin
        ratio = inf if cout == 0 else fractions.Fraction(cin, cout)
        return (-ratio, -cin, w)

    return sorted(cls_tab, key=key)[:k]


def test_ratio_ranking_against_fractions():
    c = corpus.generate("classes", ndocs=80, size_a=300, size_b=900, boost_rank_hi=3000)
    r = oracle.count(c.text, c.offsets, c.classes, c.nclasses)
    g = r.glob().as_dict()
    for k in range(c.nclasses):
        got = r.ratio_topk(k, 50)
        want = _fraction_rank(r.cls(k).as_dict(), g, 50)
        assert [w for w, _, _ in got] == want
        for w, cin, cout in got:
            assert cin == r.cls(k).as_dict()[w] and cin + cout == g[w]


# ---------------------------------------------------------------- numeric MapReduce (Sec. 4.2)
def _ulps(a: float, b: float) -> float:
    import math
    return abs(a - b) / math.ulp(max(abs(a), abs(b), 1e-300))


@pytest.mark.parametrize("n", [0, 1, 2, 3, 10, 99, 100, 1000, 4097])
def test_series_alternating_harmonic_exact_rationals(n):
    """A(n) = sum (-1)^(i+1)/i as an exact fraction, rounded once."""
    from fractions import Fraction
    exact = sum((Fraction(1, i) if i % 2 else Fraction(-1, i)) for i in range(1, n + 1))
    got = oracle.series_sum(oracle.SERIES_ALT_HARMONIC, n)
    assert (n == 0 and got == 0.0) or _ulps(got, float(exact)) <= 2.0, (n, got, float(exact))


@pytest.mark.parametrize("n", [0, 1, 2, 10, 1000, 100_000, 1_000_000])
def test_series_sqrt_against_an_exactly_rounded_sum(n):
    """S(n) = sum sqrt(i): math.fsum rounds the exact sum of the double terms once."""
    import math
    want = math.fsum(math.sqrt(i) for i in range(1, n + 1))
    got = oracle.series_sum(oracle.SERIES_SQRT, n)
    assert (n == 0 and got == 0.0) or _ulps(got, want) <= 2.0, (n, got, want)


@pytest.mark.parametrize("n", [10_000, 1_000_000, 10_000_000])
def test_series_sqrt_euler_maclaurin(n):
    """S(n) = 2/3 n^(3/2) + 1/2 n^(1/2) + zeta(-1/2) + n^(-1/2)/24 - n^(-5/2)/1920
    + O(n^(-9/2)), evaluated with 40 significant digits."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    x = mpmath.mpf(n)
    em = (mpmath.mpf(2) / 3 * x ** 1.5 + x ** 0.5 / 2 + mpmath.zeta(-0.5) + x ** -0.5 / 24 - x ** -2.5 / 1920)
    got = oracle.series_sum(oracle.SERIES_SQRT, n)
    assert abs(got - float(em)) <= 1e-14 * float(em), (n, got, float(em))


@pytest.mark.parametrize("n", [1, 2, 1001, 100_000, 10_000_000])
def test_series_alternating_harmonic_closed_form_and_limit(n):
    """A(n) = ln 2 + (-1)^(n+1)/2 * (psi((n+2)/2) - psi((n+1)/2)), and the
    alternating-series bound |A(n) - ln 2| < 1/(n+1) with the sign of the
    first omitted term's opposite."""
    import math
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    sign = 1 if n % 2 else -1
    closed = mpmath.log(2) + sign * (mpmath.digamma(mpmath.mpf(n + 2) / 2) - mpmath.digamma(mpmath.mpf(n + 1) / 2)) / 2
    got = oracle.series_sum(oracle.SERIES_ALT_HARMONIC, n)
    assert abs(got - float(closed)) <= 4e-16 * max(1.0, abs(float(closed))), (n, got, float(closed))
    d = got - math.log(2)
    assert abs(d) < 1.0 / (n + 1) and (d > 0) == (n % 2 == 1)
