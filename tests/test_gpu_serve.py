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


def test_budget_charges_buffers_until_their_free_has_run():
    """wc_buffer_alloc refuses what the budget cannot hold; a buffer freed in
    stream order stays charged until the stream has passed the free."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_05269_gb300 import wc
    c = wc.Counter(0, count_bits=32, budget=64 << 20)
    s = torch.cuda.Stream()
    a = c.buffer(40 << 20, s)
    with pytest.raises(wc.WcError) as e:
        c.buffer(40 << 20, s)
    assert e.value.status == wc.WC_ERR_BUDGET
    # keep the stream busy (a bounded spin of about 0.2 s), then free in stream order
    with torch.cuda.stream(s):
        torch.cuda._sleep(400_000_000)
    a.free(s)
    assert c.mem_usage()[0] >= 40 << 20, "freed bytes must stay charged until the stream passes the free"
    with pytest.raises(wc.WcError) as e:
        c.buffer(40 << 20, s)
    assert e.value.status == wc.WC_ERR_BUDGET
    s.synchronize()
    assert c.mem_usage()[0] == 0
    b = c.buffer(40 << 20, s)
    assert c.mem_usage()[0] >= 40 << 20
    b.free(s)
    s.synchronize()
    assert c.mem_usage() == (0, c.mem_usage()[1]) and c.mem_usage()[1] <= 64 << 20
    c.close()


def test_admission_waits_under_a_tight_budget():
    """Request text is charged to the context's budget with the tables: with
    requests of about 12 MB arriving together (each a unit of its own, longer
    on the GPU than the loop takes to launch the next), six streams and a
    budget of 1.2 units, units wait for admission instead of failing, the
    context never holds more than its budget, and every answer is still the
    oracle's."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_05269_gb300 import serve, wc
    pool, trip, reqs = make_requests(n_rate=2000.0, dur=0.006, lo=10 << 20, hi=14 << 20, pool_bytes=96e6, seed=21)
    assert len(reqs) >= 6
    reqs = [serve.Request(r.rid, 0.0, r.data) for r in reqs]  # all waiting at the start
    kw = dict(topk=100, big_bytes=4 << 20)
    # one unit's footprint: the largest, counting one unit at a time
    solo = wc.Counter(0, count_bits=32, budget=8 << 30)
    solo.mem_usage(reset=True)
    serve.serve_batched(solo, reqs, max_inflight=1, **kw)
    unit = solo.mem_usage()[1]
    solo.close()
    # 1.2 units: a context's first unit (tables sized from an estimate) and
    # any other never fit together, so the second waits for the first
    budget = int(unit * 1.2)
    tight = wc.Counter(0, count_bits=32, budget=budget)
    answers, stats = serve.serve_batched(tight, reqs, max_inflight=6, **kw)
    used, peak = tight.mem_usage()
    tight.close()
    assert stats["large"] == len(reqs)
    assert stats["budget_waits"] > 0, f"six streams under a budget of 1.2 units must wait: unit {unit}, {stats}"
    assert peak <= budget, f"peak {peak} over the budget {budget}"
    for (a, s, e), ans in zip(trip, answers):
        assert ans.as_list() == oracle.count(pool[s:e]).glob().as_list()[:100], f"request {ans.rid}"
