"""Pins of the estimated rejection bound (Section 2.2: a substitute for w_max when no hard
bound on the weights is known) in the oracle.

The estimate is the largest of `sample` log-weights at independent uniformly drawn indices,
so its law is fixed: for distinct values v_(1) < ... < v_(N), P(estimate <= v_(k)) =
(k / N)^sample. With sample = 40 N it equals the true maximum (it misses it with probability
about e^-40), and the rejection resampler with it is partial rejection control with the
exact maximum as the bound, which delivers unit outcome weights."""
import numpy as np
import pytest

import oracle


def test_large_sample_finds_the_maximum_and_pins_the_rejection_outcome():
    rng = np.random.default_rng(3)
    for dtype in (np.float32, np.float64):
        lw = (-rng.exponential(2.0, 50)).astype(dtype)
        est = oracle.estimate_log_wmax(lw, 40 * len(lw), seed=9)
        assert est == float(lw.max())
        st, a, out, e2, viol = oracle.rejection_estimated(lw, 40 * len(lw), seed=9)
        assert st == oracle.OK and e2 == est and viol == 0
        st2, a2, out2 = oracle.partial_rejection_control(lw, float(lw.max()), seed=9)
        assert np.array_equal(a, a2) and np.all(out == 0)


def test_estimate_law_over_seeds():
    """P(estimate <= v_(k)) = (k/N)^s for s = 3, at three k, over 4000 seeds (5 sigma)."""
    rng = np.random.default_rng(5)
    N, s, R = 40, 3, 4000
    lw = np.sort(-rng.exponential(1.0, N))
    ests = np.array([oracle.estimate_log_wmax(lw, s, seed=1000 + r) for r in range(R)])
    assert np.all(np.isin(ests, lw))
    for k in (10, 25, 35):
        p = (k / N) ** s
        got = np.mean(ests <= lw[k - 1])
        assert abs(got - p) <= 5 * np.sqrt(p * (1 - p) / R) + 1e-12, (k, got, p)


def test_single_draw_is_uniform_over_the_particles():
    rng = np.random.default_rng(7)
    N, R = 16, 8000
    lw = -rng.permutation(N).astype(np.float64) - 0.5  # distinct values
    idx = [int(np.nonzero(lw == oracle.estimate_log_wmax(lw, 1, seed=r, step=3))[0][0])
           for r in range(R)]
    counts = np.bincount(idx, minlength=N)
    chi2 = np.sum((counts - R / N) ** 2 / (R / N))
    assert chi2 < 45.0  # chi-square, 15 degrees of freedom: p < 1e-4 beyond 45


def test_special_values_and_violations():
    lw = np.array([-np.inf, np.nan, -3.0, -1.0], np.float64)
    est = oracle.estimate_log_wmax(lw, 200, seed=1)
    assert est == -1.0  # NaN passed over, -inf loses
    assert oracle.estimate_log_wmax(np.full(5, -np.inf), 100, seed=1) == -np.inf
    st, a, out, e, v = oracle.rejection_estimated(np.full(5, -np.inf), 100, seed=1)
    assert st == oracle.ERR_ZERO_WEIGHT and np.array_equal(a, np.arange(5))
    # a small sample misses large weights: every weight above the estimate is a violation,
    # and each delivered particle of such weight carries log(w / v) = lw - estimate
    rng = np.random.default_rng(11)
    lw = (-rng.exponential(1.0, 3000)).astype(np.float32)
    st, a, out, e, v = oracle.rejection_estimated(lw, 4, seed=2)
    assert st == oracle.OK
    assert v == int(np.sum(lw > np.float32(e))) and v > 0
    above = lw[a] > np.float32(e)
    assert np.array_equal(out[above], lw[a][above] - np.float32(e))
    assert np.all(out[~above] == 0)
