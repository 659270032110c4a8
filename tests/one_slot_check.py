"""Parity of the one-home-slot test build against the oracle.

Run as a script in its own process with WC_LIB_PATH naming the library built
with -DWC_TEST_ONE_SLOT (tests/test_gpu_collisions.py does this): every hash
of that build is a constant, so every key of a table starts probing at the
same slot, and only the exact comparison of keys and word bytes keeps the
words apart.  Exits 0 after every case matches the oracle bit for bit.
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)


def main() -> int:
    import torch

    import collisions
    import corpus
    import oracle
    from gpu_util import assert_same, to_dev
    from paper_2206_05269_gb300 import wc

    assert os.environ.get("WC_LIB_PATH"), "run with WC_LIB_PATH set to the one-slot build"
    dev = torch.device("cuda:0")
    ctr = wc.Counter(0)

    def single(data: bytes, what: str, offset: int = 0):
        t = ctr.count_checked(to_dev(data, offset))
        assert_same(t.export(), oracle.count(data).glob(), what)
        return t

    # single documents: a slice of the tiny corpus (about 1,900 distinct
    # words in one probe chain), the forced long-word collisions, edge cases
    tiny = corpus.generate("tiny", ndocs=40)
    seg = tiny.text[:int(tiny.offsets[12])].tobytes()
    a = single(seg, "tiny slice, one home slot")
    single(collisions.collision_text(3), "long-word collisions, one home slot", offset=5)
    single(collisions.collision_text(4, equal_counts=True), "equal-count collisions, one home slot")
    for e in (b"", b"a", b"abc123def don't", b"Aa aA AA aa"):
        single(e, repr(e))

    # merge: the reduce of Sec. 3.3 through the same one-slot tables
    seg2 = tiny.text[int(tiny.offsets[12]):int(tiny.offsets[20])].tobytes()
    b = single(seg2, "second slice")
    m = ctr.merge([a, b])
    assert_same(m.export(), oracle.count(seg + b" " + seg2).glob(), "merge, one home slot")

    # batched: per-document shared tables and the spill tables, class and
    # global tables, all keyed through one home slot
    docs = [tiny.text[int(tiny.offsets[d]):int(tiny.offsets[d + 1])].tobytes() for d in range(8)]
    docs += [collisions.collision_text(11), collisions.collision_text(12, equal_counts=True), b"", b"x"]
    text = np.frombuffer(b"".join(docs), np.uint8)
    offs = np.cumsum([0] + [len(d) for d in docs]).astype(np.uint64)
    cls = (np.arange(len(docs)) % 3).astype(np.uint32)
    t = torch.from_numpy(text.copy()).to(dev)
    o = torch.from_numpy(offs.view(np.int64).copy()).to(dev)
    c = torch.from_numpy(cls.view(np.int32).copy()).to(dev)
    bt = ctr.count_batched_checked(t, o, offs, c, 3)
    r = oracle.count(text, offs, cls, 3)
    lists = bt.doc_lists()
    for d in range(len(docs)):
        assert lists[d] == r.doc(d).as_list(), f"batched doc {d}, one home slot"
    for k in range(3):
        assert_same(bt.table(wc.WC_TABLE_CLASS, k).export(), r.cls(k), f"class {k}, one home slot")
    assert_same(bt.table(wc.WC_TABLE_GLOBAL).export(), r.glob(), "global, one home slot")
    bt.free()
    ctr.close()
    print("one-slot build: every case equals the oracle")
    return 0


if __name__ == "__main__":
    sys.exit(main())
