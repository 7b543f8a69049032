"""Host-side pieces of serving: the request generator and the arrival
process (no GPU)."""
import math

import numpy as np

from paper_2205_07976_gb300 import workloads as W


def test_requests_follow_the_recipe():
    reqs = W.serving_requests(400, seed=1)
    S = np.array([len(r.lambdas) for r in reqs])
    M = np.array([r.umats.shape[0] for r in reqs])
    npix = np.array([r.npix for r in reqs])
    assert S.min() >= 1 and S.max() <= 100 and M.min() >= 1 and M.max() <= 50
    assert 20 < S.mean() < 80 and 10 < M.mean() < 40
    assert npix.min() >= 500 and npix.max() <= 4.2e6
    # log-uniform area: the median is near the geometric mean of the range
    assert 0.4 < np.median(npix) / math.sqrt(1e3 * 4e6) < 2.5
    for r in reqs:
        f0, s0, nf, ns = r.roi
        assert 0 <= f0 and f0 + nf <= 3072 and 0 <= s0 and s0 + ns <= 3072
        assert abs(r.weights.sum() - 1) < 1e-12
        np.testing.assert_allclose(r.axes @ r.axes.T,
                                   np.diag([79.0**2, 79.0**2, 38.0**2]),
                                   atol=1e-9)


def test_poisson_arrivals():
    t = W.poisson_arrivals(20000, rate=50.0, seed=2)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 1 / 50.0) < 0.03 / 50.0
    # exponential gaps: coefficient of variation 1
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.03
