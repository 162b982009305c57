"""The served trace's offered work (host only): a request of the served BVP
stream is N + 1 block rows of order m with nrhs right-hand sides, so it asks
for (N + 1) m nrhs unknowns·RHS.  At 2000 req/s the trace offers about
2.5e10 unknowns·RHS/s (N log-uniform on [1e3, 5e5]: mean 8.0e4; m uniform on
{4, 8, 16}; 1-32 right-hand sides, mean 16.5), ten times what one device
sustains on these kernels; at 200 req/s about 2.3e9."""
import math

import gen


def _offered(duration_s, rate):
    trace = gen.serve_trace(duration_s, rate)
    return len(trace), sum((r.N + 1) * r.m * r.nrhs for r in trace) / duration_s


def test_offered_work_matches_the_trace_recipe():
    # mean of (N + 1) m nrhs from the recipe's distributions (independent draws)
    lo, hi = math.log(1e3), math.log(5e5)
    mean_n = (5e5 - 1e3) / (hi - lo) + 1.0          # log-uniform mean, plus the extra row
    mean_m = (4 + 8 + 16) / 3.0
    mean_r = 16.5
    per_request = mean_n * mean_m * mean_r
    n, w = _offered(10.0, 2000.0)
    assert abs(n / 10.0 - 2000.0) < 3 * math.sqrt(2000.0 * 10.0) / 10.0   # Poisson count
    # the 30 % repeats redraw nothing but nrhs, so the sample mean stays near the recipe's
    assert 0.6 * per_request * 2000.0 < w < 1.6 * per_request * 2000.0
    assert 1.5e10 < w < 4e10


def test_offered_work_at_200_per_second():
    _, w = _offered(10.0, 200.0)
    assert 1.2e9 < w < 4e9
