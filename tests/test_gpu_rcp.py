"""The FP64 reciprocal that replaces division at every FP64 pivot step
(bt_device_rcp: the hardware seed rcp.approx.ftz.f64 refined by one
third-order Newton step, IEEE division for zero, subnormal, huge and
non-finite x) against IEEE 1/x: within one unit in the last place over the
whole normal range, including both ends of the Newton branch (biased
exponents 1 and 2044) and the first values past them, and exactly IEEE for
the special cases."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _dev_rcp(x, cuda):
    import torch

    import paper_0912_3678_gb300 as bt
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(cuda)
    y = bt.bt_device_rcp(xd)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def _with_exponent(rng, biased, n):
    """n values m * 2^(biased - 1023), m uniform in [1, 2), random sign."""
    m = 1.0 + rng.random(n)
    v = np.ldexp(m, biased - 1023)
    return v * np.where(rng.random(n) < 0.5, -1.0, 1.0)


def test_rcp_within_one_ulp_over_the_normal_range(cuda):
    rng = np.random.default_rng(20091234)
    parts = [_with_exponent(rng, int(e), 64) for e in rng.integers(1, 2047, size=4000)]
    # the ends of the Newton branch and their neighbours
    for e in (1, 2, 3, 2043, 2044, 2045, 2046):
        parts.append(_with_exponent(rng, e, 4096))
    parts.append(np.array([1.0, -1.0, 3.0, 0.1, 2.0 ** 1021, 2.0 ** -1022, np.nextafter(2.0 ** 1022, 0)]))
    x = np.concatenate(parts)
    y = _dev_rcp(x, cuda)
    ref = 1.0 / x
    ulp = np.spacing(np.abs(ref))
    err = np.abs(y - ref) / ulp
    assert np.all(np.isfinite(y))
    assert err.max() <= 1.0, (x[err.argmax()], y[err.argmax()], ref[err.argmax()])


def test_rcp_special_cases_are_ieee(cuda):
    tiny = np.array([5e-324, -5e-324, 2.0 ** -1030, -3.0 * 2.0 ** -1060])   # subnormal
    huge = np.array([2.0 ** 1022, -(2.0 ** 1023), np.finfo(float).max])     # 1/x subnormal or tiny
    x = np.concatenate([np.array([0.0, -0.0, np.inf, -np.inf, np.nan]), tiny, huge])
    y = _dev_rcp(x, cuda)
    with np.errstate(divide="ignore", over="ignore"):
        ref = 1.0 / x
    assert np.isnan(y[4])
    same = ~np.isnan(ref)
    assert np.array_equal(y[same], ref[same])
    assert np.array_equal(np.signbit(y[same]), np.signbit(ref[same]))
