"""Served counting: every request's answer in the continuous-batching mix is
bit-identical to the same request counted alone, and to the oracle."""
import numpy as np
import pytest

import corpus
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctr():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_05269_gb300 import wc
    c = wc.Counter(0, count_bits=32, budget=8 << 30)
    yield c
    c.close()


def make_requests(n_rate=400.0, dur=0.15, lo=1 << 10, hi=1 << 20, pool_bytes=48e6, seed=9):
    import torch
    from paper_2206_05269_gb300.serve import Request
    pool = corpus.generate("served_pool", size_a=pool_bytes).text
    host = torch.from_numpy(pool).pin_memory()
    trip = corpus.poisson_requests(pool, n_rate, dur, lo, hi, seed)
    reqs = [Request(i, a, host[s:e]) for i, (a, s, e) in enumerate(trip)]
    return pool, trip, reqs


def test_mix_equals_alone_and_oracle(ctr):
    from paper_2206_05269_gb300 import serve
    from gpu_util import to_dev
    pool, trip, reqs = make_requests()
    assert len(reqs) >= 20
    answers, stats = serve.serve_batched(ctr, reqs, topk=100, max_inflight=3, big_bytes=512 << 10,
                                         keep_tables=True)
    assert stats["rounds"] >= 2 and stats["large"] >= 1
    alone = []
    for (a, s, e), ans in zip(trip, answers):
        data = pool[s:e].tobytes()
        alone.append(ctr.count_checked(to_dev(data)).as_list())
        assert ans.full and ans.as_list() == alone[-1], f"request {ans.rid} differs alone vs in the mix"
        assert ans.latency >= 0
    for (a, s, e), ans in list(zip(trip, answers))[::5]:
        assert ans.as_list() == oracle.count(pool[s:e]).glob().as_list()
    # the default answer: the top 100 rows gathered on the device
    top, _ = serve.serve_batched(ctr, reqs, topk=100, max_inflight=3, big_bytes=512 << 10)
    for ans, want in zip(top, alone):
        assert not ans.full and ans.as_list() == want[:100], f"request {ans.rid}: top-100 differs"


def test_fifo_path_matches(ctr):
    from paper_2206_05269_gb300 import serve
    pool, trip, reqs = make_requests(n_rate=200.0, dur=0.05, seed=4)
    a1, _ = serve.serve_batched(ctr, reqs, topk=100, keep_tables=True)
    a2, _ = serve.serve_fifo(ctr, reqs, topk=100, keep_tables=True)
    t1, _ = serve.serve_batched(ctr, reqs, topk=100)
    t2, _ = serve.serve_fifo(ctr, reqs, topk=100)
    for x, y, tx, ty in zip(a1, a2, t1, t2):
        assert x.as_list() == y.as_list()
        assert tx.as_list() == ty.as_list() == x.as_list()[:100]


def test_admission_waits_under_a_tight_budget():
    """Request text is charged to the context's budget with the tables: with
    requests of about 250 KB arriving together, each counted as a unit of its
    own on one of six streams, and a budget of two and a half units, units
    wait for admission instead of failing, the context never holds more than
    its budget, and every answer is still the oracle's."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_05269_gb300 import serve, wc
    pool, trip, reqs = make_requests(n_rate=4000.0, dur=0.015, lo=200 << 10, hi=300 << 10, seed=21)
    assert len(reqs) >= 30
    reqs = [serve.Request(r.rid, 0.0, r.data) for r in reqs]  # all waiting at the start
    kw = dict(topk=100, big_bytes=128 << 10, keep_tables=True)
    # one unit's footprint: the largest, counting one unit at a time
    solo = wc.Counter(0, count_bits=32, budget=8 << 30)
    solo.mem_usage(reset=True)
    serve.serve_batched(solo, reqs, max_inflight=1, **kw)
    unit = solo.mem_usage()[1]
    solo.close()
    budget = int(unit * 2.5)
    tight = wc.Counter(0, count_bits=32, budget=budget)
    answers, stats = serve.serve_batched(tight, reqs, max_inflight=6, **kw)
    used, peak = tight.mem_usage()
    tight.close()
    assert stats["large"] == len(reqs)
    assert stats["budget_waits"] > 0, "six streams under a budget of two and a half units must wait"
    assert peak <= budget, f"peak {peak} over the budget {budget}"
    for (a, s, e), ans in zip(trip, answers):
        assert ans.full and ans.as_list() == oracle.count(pool[s:e]).glob().as_list(), f"request {ans.rid}"
