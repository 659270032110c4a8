"""Hash collisions never merge two distinct words (GPU against the oracle).

Two kinds of forced collision:
  * long words (33+ letters) that share their first 16 letters, their last
    16 letters and their length but differ in between: the GPU's long-word
    hash covers exactly those parts, so they collide by construction and
    only the byte comparison separates them (single documents and batched
    documents, different and equal counts, mixed case);
  * a test build of the library in which every hash is a constant, so that
    every word of a table starts at one home slot (tests/one_slot_check.py,
    run in its own process against that build).
Every comparison is element by element against the oracle.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import collisions
import oracle
from gpu_util import assert_same, first_diff, to_dev

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def ctr():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_05269_gb300 import wc
    c = wc.Counter(0)
    yield c
    c.close()


def check(ctr, data: bytes, offset: int = 0, what: str = ""):
    exp = ctr.count_checked(to_dev(data, offset)).export()
    want = oracle.count(data).glob()
    if exp[2].size != len(want) or not np.array_equal(exp[0], want.words):
        raise AssertionError(f"{what}: first differences {first_diff(exp, want)}")
    assert_same(exp, want, what)


def test_families_collide_by_construction():
    """The families really share (first 16, last 16, length) and are distinct."""
    for fam in collisions.families():
        assert len(set(fam)) == len(fam)
        assert len({(w[:16], w[-16:], len(w)) for w in fam}) == 1
        assert len(fam[0]) >= 33


@pytest.mark.parametrize("equal", [False, True])
@pytest.mark.parametrize("offset", [0, 3])
def test_long_word_collisions_single_document(ctr, equal, offset):
    data = collisions.collision_text(seed=21 + offset, equal_counts=equal)
    check(ctr, data, offset, f"collisions equal={equal} offset={offset}")


def test_long_word_collisions_many_occurrences(ctr):
    """Thousands of occurrences spread over every block of the counting kernel."""
    data = b"".join(collisions.collision_text(seed=s, filler=4000) for s in range(40))
    check(ctr, data, 0, "collisions, many occurrences")


def test_long_word_collisions_batched(ctr):
    import torch
    from paper_2206_05269_gb300 import wc
    docs = [collisions.collision_text(seed=s, equal_counts=bool(s % 2), filler=50 + 97 * s) for s in range(12)]
    docs.insert(5, b" ".join(collisions.families()[2]))  # one of each 300-letter word, nothing else
    text = np.frombuffer(b"".join(docs), np.uint8)
    offs = np.cumsum([0] + [len(d) for d in docs]).astype(np.uint64)
    dev = torch.device("cuda:0")
    b = ctr.count_batched_checked(torch.from_numpy(text.copy()).to(dev),
                                  torch.from_numpy(offs.view(np.int64).copy()).to(dev), offs)
    r = oracle.count(text, offs)
    lists = b.doc_lists()
    for d in range(len(docs)):
        assert lists[d] == r.doc(d).as_list(), f"doc {d}"
    assert_same(b.table(wc.WC_TABLE_GLOBAL).export(), r.glob(), "global")
    b.free()


def test_one_home_slot_build():
    """The tiny corpus, merges, batches and the long-word families through a
    build whose every hash is a constant (one probe chain per table)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_05269_gb300 import build
    lib = build.build(variant="oneslot")
    env = dict(os.environ, WC_LIB_PATH=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "one_slot_check.py")], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, f"one-slot build differs from the oracle:\n{r.stdout[-3000:]}\n{r.stderr[-3000:]}"
