"""Inputs that force hash collisions, for the parity tests.

Long words (17 letters or more) are keyed in the GPU tables by a 64-bit hash
of their first 16 letters, their last 16 letters and their length; equality
is always decided by comparing every byte.  Words of 33 letters or more that
share both 16-letter ends and the length, but differ in between, therefore
get the same hash by construction: only the byte comparison keeps them
apart.  The families below are built that way, in several cases, so that
the comparison (case folded) and the sort's ordering of words that share
their first 16 letters are both exercised.

This module holds no counting arithmetic: it only writes text.
"""
from __future__ import annotations

import numpy as np

HEAD = b"pneumonoultramic"  # 16 letters shared by every family member
TAIL = b"silicovolcanosis"  # 16 letters shared by every family member


def families() -> list[list[bytes]]:
    """Groups of distinct words with equal (first 16, last 16, length)."""
    fam33 = [HEAD + bytes([c]) + TAIL for c in b"abcxyz"]                      # 33 letters
    fam40 = [HEAD + m + TAIL for m in (b"aaaaaaaa", b"aaaaaaab", b"baaaaaaa", b"zzzzzzzz", b"mmmmnnnn")]
    mid = bytearray(b"q" * 268)
    fam300 = []
    for c in b"acegik":  # differ deep inside a 300-letter word
        m = bytearray(mid)
        m[150] = c
        fam300.append(HEAD + bytes(m) + TAIL)
    # the middle of the same length, differing only in its first or last letter
    fam48 = [HEAD + m + TAIL for m in (b"b" + b"o" * 15, b"o" * 15 + b"b", b"o" * 16)]
    return [fam33, fam40, fam300, fam48]


def mixed_case(w: bytes, rng) -> bytes:
    """The same word with some letters upper-cased (it must count as w)."""
    a = np.frombuffer(w, np.uint8).copy()
    up = rng.random(a.size) < 0.3
    a[up] -= 32
    return a.tobytes()


def collision_text(seed: int = 7, equal_counts: bool = False, filler: int = 400) -> bytes:
    """One document: every family member a distinct number of times (or all
    the same number, so the order among them is decided by their bytes
    alone), some occurrences mixed case, shuffled among short filler words,
    with assorted separators."""
    rng = np.random.default_rng(seed)
    toks = []
    for fam in families():
        for i, w in enumerate(fam):
            n = 5 if equal_counts else 2 + 3 * i
            for _ in range(n):
                toks.append(mixed_case(w, rng) if rng.random() < 0.3 else w)
    short = [b"the", b"of", b"and", b"a", b"to", b"pneumonoultramic", b"silicovolcanosis"]
    toks += [short[i] for i in rng.integers(0, len(short), filler)]
    order = rng.permutation(len(toks))
    seps = [b" ", b", ", b"\n", b"-", b"1", b". "]
    out = bytearray()
    for j in order:
        out += toks[j] + seps[int(rng.integers(0, len(seps)))]
    return bytes(out)
