"""The device-side failure path without a GPU fault: every device wait of
the library is bounded, gives up with a recorded status and leaves the
context usable.  The counting kernel's barrier wait is run on a barrier that
nothing arrives at (and, as a control, on one that is arrived at)."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_same, to_dev

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


def test_wait_arrived_returns_ok(ctr):
    from paper_2206_05269_gb300 import wc
    assert wc.wc_selftest_wait(ctr.ctx, 1000, True) == wc.WC_OK


def test_wait_never_arrived_times_out_and_context_stays_usable(ctr):
    from paper_2206_05269_gb300 import wc
    for polls in (1, 1000, 100000):
        assert wc.wc_selftest_wait(ctr.ctx, polls, False) == wc.WC_ERR_TIMEOUT
        assert "wait" in wc.wc_last_error(ctr.ctx)
    # the context keeps working after the timeouts
    text = np.frombuffer(b"The cat; the CAT's hat. " * 1000, np.uint8)
    t = ctr.count_checked(to_dev(text))
    assert_same(t.export(), oracle.count(text).glob(), "count after timeouts")


def test_wait_poll_limits_are_checked(ctr):
    from paper_2206_05269_gb300 import wc
    assert wc.wc_selftest_wait(ctr.ctx, 0, False) == wc.WC_ERR_INVALID_ARG
    assert wc.wc_selftest_wait(ctr.ctx, (1 << 22) + 1, False) == wc.WC_ERR_INVALID_ARG
