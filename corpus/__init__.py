"""Seeded synthetic corpora for tests and benchmarks.

The generator itself is ``gen.c`` (compiled on first use with the host C
compiler).  It holds none of the counting method: it draws vocabulary ids from
a Zipf law and writes the words, and its tally of drawn ids is an independent
ground truth for the word counts of the text it wrote.

The recipes below give the five workloads the method is measured on (a tiny
per-document corpus, a four-class corpus shaped like the paper's presidential
speech study in Sec. 4.3, a 1e9-byte single-pass corpus, 100k log-normal
documents, and a request pool for serving), plus small variants for tests.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libwcgen.so")
_lock = threading.Lock()
_lib = None


class GenParams(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("vocab_size", ctypes.c_uint32),
        ("len_min", ctypes.c_uint32), ("len_max", ctypes.c_uint32),
        ("len_a", ctypes.c_double), ("len_b", ctypes.c_double), ("len_jitter", ctypes.c_double),
        ("len_tail", ctypes.c_double), ("len_tail_mean", ctypes.c_double),
        ("zipf_s", ctypes.c_double),
        ("cap_prob", ctypes.c_double),
        ("punct_prob", ctypes.c_double),
        ("digit_prob", ctypes.c_double),
        ("glue_prob", ctypes.c_double),
        ("high_prob", ctypes.c_double),
        ("newline_min", ctypes.c_uint32), ("newline_max", ctypes.c_uint32),
        ("nclasses", ctypes.c_uint32),
        ("boost_per_class", ctypes.c_uint32),
        ("boost_rank_lo", ctypes.c_uint32), ("boost_rank_hi", ctypes.c_uint32),
        ("boost_lo", ctypes.c_double), ("boost_hi", ctypes.c_double),
        ("ndocs", ctypes.c_uint32),
        ("size_mode", ctypes.c_uint32),
        ("size_a", ctypes.c_double), ("size_b", ctypes.c_double), ("size_c", ctypes.c_double),
        ("clip_lo", ctypes.c_double), ("clip_hi", ctypes.c_double),
        ("threads", ctypes.c_uint32),
    ]


def build(force: bool = False) -> str:
    """Compiles gen.c into corpus/_build/libwcgen.so (host compiler, portable flags)."""
    src = os.path.join(_HERE, "gen.c")
    with _lock:
        if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
            return _SO
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", src,
                               "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp = ctypes.c_void_p
        lib.gen_create.restype = vp
        lib.gen_create.argtypes = [ctypes.POINTER(GenParams), ctypes.c_char_p, ctypes.c_int]
        lib.gen_bound_bytes.restype = ctypes.c_uint64
        lib.gen_bound_bytes.argtypes = [vp]
        lib.gen_fill.restype = ctypes.c_int64
        lib.gen_fill.argtypes = [vp, vp, ctypes.c_uint64, vp, vp]
        lib.gen_total_tokens.restype = ctypes.c_uint64
        lib.gen_total_tokens.argtypes = [vp]
        lib.gen_ntally.restype = ctypes.c_uint32
        lib.gen_ntally.argtypes = [vp]
        lib.gen_tally.argtypes = [vp, vp]
        lib.gen_vocab_bytes.restype = ctypes.c_uint64
        lib.gen_vocab_bytes.argtypes = [vp]
        lib.gen_vocab.argtypes = [vp, vp, vp]
        lib.gen_expected_len.restype = ctypes.c_double
        lib.gen_expected_len.argtypes = [vp]
        lib.gen_destroy.argtypes = [vp]
        _lib = lib
    return _lib


@dataclasses.dataclass
class Recipe:
    name: str
    seed: int
    vocab_size: int
    len_min: int
    len_max: int
    len_a: float
    len_b: float
    len_jitter: float
    zipf_s: float
    ndocs: int
    size_mode: int            # 0 words U[a,b]; 1 bytes lognormal(median a, sigma c); 2 bytes = a; 3 log-uniform [a,b]
    size_a: float
    size_b: float = 0.0
    size_c: float = 0.0
    len_tail: float = 0.0
    len_tail_mean: float = 0.0
    clip_lo: float = 0.0
    clip_hi: float = 0.0
    cap_prob: float = 0.1
    punct_prob: float = 0.15
    digit_prob: float = 0.0
    glue_prob: float = 0.0
    high_prob: float = 0.0
    newline_min: int = 8
    newline_max: int = 20
    nclasses: int = 1
    boost_per_class: int = 0
    boost_rank_lo: int = 0
    boost_rank_hi: int = 0
    boost_lo: float = 5.0
    boost_hi: float = 20.0

    def params(self, threads: int) -> GenParams:
        p = GenParams()
        for f in dataclasses.fields(self):
            if f.name == "name":
                continue
            setattr(p, f.name, getattr(self, f.name))
        p.threads = threads
        return p

    def scaled(self, **kw) -> "Recipe":
        return dataclasses.replace(self, **kw)


# Workload recipes.  Separators: mostly one space, sometimes 1-2 punctuation
# bytes before it, a newline every 8-20 tokens; the large corpus also carries
# digit runs.  Length parameters are calibrated so that bytes per token match
# each workload's stated size (tiny 2 MB / 0.35M tokens, class 30 MB / 5M,
# large 1e9 B / 170M).
RECIPES = {
    "tiny": Recipe("tiny", 0x5EED0001, 5000, 1, 12, 2.5, 0.55, 1.5, 1.1, 200, 0, 500, 3000),
    "classes": Recipe("classes", 0x5EED0002, 30000, 1, 14, 2.3, 0.55, 1.5, 1.05, 1000, 0, 2000, 8000,
                      nclasses=4, boost_per_class=200, boost_rank_lo=100, boost_rank_hi=30000),
    "large": Recipe("large", 0x5EED0003, 1_000_000, 1, 24, 0.2, 0.6, 2.0, 1.0, 1, 2, 1e9,
                    len_tail=0.15, len_tail_mean=4.0, cap_prob=0.2, punct_prob=0.12, digit_prob=0.03),
    "batched": Recipe("batched", 0x5EED0004, 200_000, 1, 20, 1.5, 0.55, 1.5, 1.1, 100_000, 1, 2048, 0, 1.5,
                      len_tail=0.1, len_tail_mean=3.0, clip_lo=1024, clip_hi=1 << 20),
    "served_pool": Recipe("served_pool", 0x5EED0005, 500_000, 1, 22, 0.3, 0.6, 2.0, 1.0, 1, 2, 2e9,
                          len_tail=0.15, len_tail_mean=4.0, cap_prob=0.15),
}


@dataclasses.dataclass
class Corpus:
    text: np.ndarray          # uint8 [nbytes]
    offsets: np.ndarray       # uint64 [ndocs+1]
    classes: np.ndarray       # uint32 [ndocs]
    nclasses: int
    tokens: int               # generator's own token count
    recipe: Recipe
    _tally: np.ndarray        # uint64 [ntally, vocab]
    _vbytes: np.ndarray
    _voff: np.ndarray

    @property
    def nbytes(self) -> int:
        return int(self.text.size)

    @property
    def ndocs(self) -> int:
        return int(self.classes.size)

    def vocab_word(self, i: int) -> bytes:
        return self._vbytes[self._voff[i]:self._voff[i + 1]].tobytes()

    def truth(self, cls: int | None = None) -> dict[bytes, int]:
        """Ground-truth tally of emitted words: overall, or for one class."""
        if cls is None:
            t = self._tally.sum(axis=0)
        else:
            t = self._tally[cls] if self._tally.shape[0] > 1 else self._tally[0]
        ids = np.nonzero(t)[0]
        return {self.vocab_word(int(i)): int(t[i]) for i in ids}


def generate(recipe: Recipe | str, threads: int | None = None, **overrides) -> Corpus:
    if isinstance(recipe, str):
        recipe = RECIPES[recipe]
    if overrides:
        recipe = recipe.scaled(**overrides)
    lib = _load()
    if threads is None:
        threads = max(1, min(32, os.cpu_count() or 1))
    p = recipe.params(threads)
    err = ctypes.create_string_buffer(200)
    h = lib.gen_create(ctypes.byref(p), err, 200)
    if not h:
        raise RuntimeError(f"corpus generator: {err.value.decode()}")
    try:
        bound = lib.gen_bound_bytes(h)
        buf = np.empty(max(1, bound), dtype=np.uint8)
        offs = np.zeros(recipe.ndocs + 1, dtype=np.uint64)
        cls = np.zeros(max(1, recipe.ndocs), dtype=np.uint32)
        n = lib.gen_fill(h, buf.ctypes.data, buf.size, offs.ctypes.data, cls.ctypes.data)
        if n < 0:
            raise RuntimeError("corpus generator: fill failed")
        text = buf[:n].copy() if n < buf.size // 2 else buf[:n]
        nt = lib.gen_ntally(h)
        tally = np.zeros((nt, recipe.vocab_size), dtype=np.uint64)
        lib.gen_tally(h, tally.ctypes.data)
        vb = np.zeros(lib.gen_vocab_bytes(h), dtype=np.uint8)
        vo = np.zeros(recipe.vocab_size + 1, dtype=np.uint64)
        lib.gen_vocab(h, vb.ctypes.data, vo.ctypes.data)
        return Corpus(text, offs, cls[:recipe.ndocs], recipe.nclasses, int(lib.gen_total_tokens(h)),
                      recipe, tally, vb, vo)
    finally:
        lib.gen_destroy(h)


def expected_word_len(recipe: Recipe | str, **overrides) -> float:
    if isinstance(recipe, str):
        recipe = RECIPES[recipe]
    if overrides:
        recipe = recipe.scaled(**overrides)
    lib = _load()
    p = recipe.params(1)
    p.ndocs = 0
    err = ctypes.create_string_buffer(200)
    h = lib.gen_create(ctypes.byref(p), err, 200)
    if not h:
        raise RuntimeError(err.value.decode())
    try:
        return lib.gen_expected_len(h)
    finally:
        lib.gen_destroy(h)


def poisson_requests(pool: np.ndarray, rate: float, duration: float, lo: int, hi: int, seed: int):
    """Serving request stream: Poisson arrivals at `rate` per second for
    `duration` seconds; sizes log-uniform in [lo, hi] bytes, cut out of the
    pooled corpus at generator-written spaces.  Returns (arrival s, start, end)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        size = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        start = int(rng.integers(0, max(1, pool.size - size)))
        s, e = slice_at_separators(pool, start, size)
        out.append((t, s, e))
    return out


def slice_at_separators(text: np.ndarray, start: int, length: int) -> tuple[int, int]:
    """Widens [start, start+length) to the nearest generator-written space or
    newline on each side, so no word is cut.  Used to cut serving requests out
    of a pooled corpus (the pool recipe never glues words to digits)."""
    n = text.size
    s = max(0, min(start, n))
    e = max(s, min(start + length, n))
    while s > 0 and text[s - 1] not in (0x20, 0x0A):
        s -= 1
    while e < n and text[e - 1] not in (0x20, 0x0A):
        e += 1
    return s, e
