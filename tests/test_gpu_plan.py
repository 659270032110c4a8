"""GPU parity of plans (wc_plan_create / wc_plan_run): the batched count as
the benchmark times it, captured into a CUDA graph and replayed, under every
per-document kernel shape the autotuner can choose for each size class,
bit-exact against the oracle."""
import json

import numpy as np
import pytest

import corpus
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def docs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    # log-normal sizes with a heavier tail than the batched recipe, so that
    # every size class (up to 8 KB, up to 32 KB, up to 64 KB, split into
    # ranges above) holds documents
    c = corpus.generate("batched", ndocs=1500, size_c=2.0)
    sizes = np.diff(c.offsets.astype(np.int64))
    assert (sizes <= 8 << 10).any() and ((sizes > 8 << 10) & (sizes <= 32 << 10)).any()
    assert ((sizes > 32 << 10) & (sizes <= 64 << 10)).any() and (sizes > 64 << 10).any()
    r = oracle.count(c.text, c.offsets)
    dev = torch.device("cuda:0")
    text = torch.from_numpy(c.text).to(dev)
    offs = torch.from_numpy(c.offsets.view(np.int64)).to(dev)
    return c, r, text, offs


def check(b, c, r):
    from paper_2206_05269_gb300 import wc
    assert b.status() == wc.WC_OK
    ds, dn, w, o, cnt = b.export()
    for d in range(c.ndocs):
        want = r.doc(d)
        s0, n = int(ds[d]), int(dn[d])
        assert n == len(want), f"doc {d}: {n} rows vs {len(want)}"
        assert np.array_equal(cnt[s0:s0 + n].astype(np.uint64), want.counts), f"doc {d}: counts"
        assert np.array_equal(w[o[s0]:o[s0 + n]], want.words), f"doc {d}: words"


@pytest.mark.parametrize("shapes", [(0, 2, 3), (1, 3, 4), (2, 4, 5), (6, 3, 5), (7, 2, 4)])
def test_plan_replay_every_shape(docs, shapes, tmp_path):
    import torch
    from paper_2206_05269_gb300 import wc
    c, r, text, offs = docs
    cache = tmp_path / "tune.json"
    small, medium, large = shapes
    cache.write_text(json.dumps({torch.cuda.get_device_name(0): {"small": small, "medium": medium, "large": large}}))
    ctr = wc.Counter(0, count_bits=32, autotune=True, tune_cache_path=str(cache))
    try:
        plan = ctr.plan(c.offsets, 0)
        check(plan.run(text, offs), c, r)   # captured
        check(plan.run(text, offs), c, r)   # replayed
        plan.free()
    finally:
        ctr.close()


def test_plan_autotune_then_replay(docs, tmp_path):
    """Autotuning times every shape on the plan's own input, keeps the
    fastest per size class (written to the cache) and the replay is exact."""
    import torch
    from paper_2206_05269_gb300 import wc
    c, r, text, offs = docs
    cache = tmp_path / "tune.json"
    ctr = wc.Counter(0, count_bits=32, autotune=True, tune_cache_path=str(cache))
    try:
        plan = ctr.plan(c.offsets, 0)
        check(plan.run(text, offs), c, r)
        check(plan.run(text, offs), c, r)
        plan.free()
    finally:
        ctr.close()
    tuned = json.loads(cache.read_text())[torch.cuda.get_device_name(0)]
    assert tuned["small"] in (0, 1, 2, 6, 7) and tuned["medium"] in (2, 3, 4) and tuned["large"] in (3, 4, 5)
