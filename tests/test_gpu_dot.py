"""FP64 accuracy of the solver's inner products (spx_dot), on data built to cancel.

The conjugate-gradient reductions must stay at FP64 accuracy even inside the
FP32 solve.  spx_dot runs the solver's reduction (per-thread partials, fixed
order grid sum); here its result is compared with math.fsum of the exact
products (a product of two FP32 values is exact in FP64), on vectors whose
terms cancel to about 1e-6 of sum |a_i b_i| over 10^7 terms.  A plain FP32
accumulation would be off by about (terms per thread) 2^-24 sum |a_i b_i|,
far outside the bound asserted here.
"""
import math

import numpy as np
import pytest
import torch

import paper_1906_03489_gb300 as spx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _cancelling(n, dtype, seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1, 1, n) * 10.0 ** rng.integers(-3, 4, n)
    b = rng.uniform(0.5, 1.5, n)
    a, b = a.astype(dtype), b.astype(dtype)
    p = a.astype(np.float64) * b.astype(np.float64)       # exact for FP32 inputs
    # flip the sign of the last term block so the total nearly cancels
    half = n // 2
    a[half:] = -a[:n - half] * (b[:n - half] / b[half:])
    a = a.astype(dtype)
    a[-1] = dtype(0.123)                                   # leave a small remainder
    return a, b


@pytest.mark.parametrize("dtype,bound", [(np.float32, 1e-13), (np.float64, 1e-14)])
@pytest.mark.parametrize("n", [10_000_000, 1_000_003, 17])
def test_dot_matches_exact_sum_on_cancelling_data(dtype, bound, n):
    plan = spx.Plan(3, 1, order=1)
    a, b = _cancelling(n, dtype, 7 + n % 5)
    prods = a.astype(np.float64) * b.astype(np.float64)
    # FP32 products are exact in FP64; FP64 products carry one rounding each,
    # far below the bound (2^-53 |a_i b_i| per term, summed: 1e-16 scale)
    exact = math.fsum(prods)
    scale = math.fsum(np.abs(prods))
    ta = torch.tensor(a, device="cuda")
    tb = torch.tensor(b, device="cuda")
    r1 = spx.dot(plan, ta, tb)
    r2 = spx.dot(plan, ta, tb)
    torch.cuda.synchronize()
    v1, v2 = float(r1), float(r2)
    assert v1 == v2, "the reduction is not reproducible"
    assert abs(v1 - exact) <= bound * scale + 1e-300, (v1, exact, scale)
    if n >= 1_000_000:
        assert abs(exact) < 1e-4 * scale, "the data should cancel"


def test_dot_fp32_beats_plain_fp32_accumulation():
    # the same data summed in FP32 by torch is far less accurate: the test data discriminates
    n = 10_000_000
    plan = spx.Plan(3, 1, order=1)
    a, b = _cancelling(n, np.float32, 3)
    prods = a.astype(np.float64) * b.astype(np.float64)
    exact, scale = math.fsum(prods), math.fsum(np.abs(prods))
    ta, tb = torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda")
    ours = float(spx.dot(plan, ta, tb))
    plain = float(torch.dot(ta, tb))
    assert abs(ours - exact) <= 1e-13 * scale
    assert abs(plain - exact) > 1e3 * abs(ours - exact)


def test_dot_unaligned_views_and_empty():
    plan = spx.Plan(3, 1, order=1)
    a, b = _cancelling(100_001, np.float32, 11)
    ta, tb = torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda")
    prods = a[1:].astype(np.float64) * b[1:].astype(np.float64)
    r = float(spx.dot(plan, ta[1:], tb[1:]))       # 4-byte aligned, not 16: the scalar path
    assert abs(r - math.fsum(prods)) <= 1e-13 * math.fsum(np.abs(prods))
    e = torch.empty(0, device="cuda")
    assert float(spx.dot(plan, e, e)) == 0.0
