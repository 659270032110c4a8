"""GPU parity of the numeric MapReduce of Sec. 4.2 (wc_series_sum) against
the oracle.

Both sides compute every term as a correctly rounded IEEE double and sum with
Neumaier's compensated additions, whose error is at most about 2u|S| plus
n u^2 sum|x_i| (u = 2^-53); for n <= 1e8 the second part is below 1e-22 of
the sum, so the two results differ by at most about 4u|S| ~ 4.4e-16 |S|.
The tolerance, 1e-14 of the sum (absolute 1e-14 near the alternating sum's
0.69), leaves a factor of twenty over that bound, and is still far below the
error of an uncompensated sum of 1e8 terms.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

NS = [0, 1, 2, 3, 10, 1000, 65536, 123457, 1_000_000, 10_000_000, 100_000_000]


@pytest.fixture(scope="module")
def ctr():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_05269_gb300 import wc
    c = wc.Counter(0)
    yield c
    c.close()


def gpu_sum(ctr, series: int, n: int) -> float:
    import torch
    from paper_2206_05269_gb300 import wc
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda:0")
    wc.wc_series_sum(ctr.ctx, series, n, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return float(out.cpu()[0])


@pytest.mark.parametrize("n", NS)
@pytest.mark.parametrize("series", [0, 1])
def test_series_matches_oracle(ctr, series, n):
    got = gpu_sum(ctr, series, n)
    want = oracle.series_sum(series, n)
    if n == 0:
        assert got == 0.0
        return
    assert abs(got - want) <= 1e-14 * max(1.0, abs(want)), (series, n, got, want)


def test_series_deterministic_and_limits(ctr):
    import math
    a = [gpu_sum(ctr, 1, 12_345_679) for _ in range(3)]
    assert a[0] == a[1] == a[2]
    assert abs(a[0] - math.log(2)) < 1.0 / 12_345_680 and a[0] > math.log(2)  # odd n: above ln 2


def test_series_rejects_bad_arguments(ctr):
    import torch
    from paper_2206_05269_gb300 import wc
    out = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    s = torch.cuda.current_stream().cuda_stream
    lib = wc.load()
    assert lib.wc_series_sum(ctr.ctx, 2, 10, out.data_ptr(), s) == wc.WC_ERR_INVALID_ARG
    assert lib.wc_series_sum(ctr.ctx, 0, 1 << 53, out.data_ptr(), s) == wc.WC_ERR_UNSUPPORTED
    assert lib.wc_series_sum(ctr.ctx, 0, 10, None, s) == wc.WC_ERR_INVALID_ARG
