"""Pins of the oracle's partial rejection control (Section 2.2, last paragraph): rejection
sampling from v = min(w, v_max) with the bound v_max, and the weighted outcome w/v.

What pins it: with v_max at or above every weight it is the rejection resampler itself
(pinned in test_oracle_laws.py) with unit weights; at small N its per-particle law is the
rejection law of v, checked by chi-square over seeded draws; and the weighted outcome is
unbiased for the target of w, E[sum_i (w/v)^{a_i} 1{a_i = j}] = N w_j / sum(v), checked by
Monte Carlo -- a dropped clamp, an inverted ratio or a weight attached to the wrong particle
fails one of these."""
import numpy as np
import pytest
from scipy import stats

import oracle
import workload


def _lw(w, dtype):
    w = np.asarray(w, dtype=np.float64)
    lw = np.full(len(w), -np.inf, dtype)
    lw[w > 0] = np.log(w[w > 0]).astype(dtype)
    return lw


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_prc_reduces_to_rejection_when_vmax_bounds_all_weights(dtype):
    lw = workload.synthetic_logw(2000, 2.0, seed=4, dtype=dtype)
    for lvmax in (0.0, float(lw.max())):
        st, a, out = oracle.partial_rejection_control(lw, lvmax, seed=9, step=3)
        st_r, a_r = oracle.rejection(lw, lvmax, seed=9, step=3)
        assert st == st_r == oracle.OK
        assert np.array_equal(a, a_r)
        assert np.all(out == 0)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_prc_exact_law_and_unbiased_weighted_outcome(dtype):
    w = np.array([0.2, 0.9, 0.05, 0.0, 0.6])
    lw = _lw(w, dtype)
    wk = np.exp(lw.astype(np.float64))
    N = len(w)
    lvmax = np.log(0.4)
    vmax = np.exp(np.float64(dtype(lvmax)))
    v = np.minimum(wk, vmax)
    piv = v / v.sum()
    law = (1 - v / vmax)[:, None] * piv[None, :] + np.diag(v / vmax)
    R = 30000
    counts = np.zeros((N, N), np.int64)
    wsum = np.zeros(N)
    wsq = np.zeros(N)
    for s in range(R):
        st, a, out = oracle.partial_rejection_control(lw, lvmax, seed=1000 + s)
        assert st == oracle.OK
        counts[np.arange(N), a] += 1
        contrib = np.bincount(a, weights=np.exp(out.astype(np.float64)), minlength=N)
        wsum += contrib
        wsq += contrib**2
    for i in range(N):
        keep = law[i] > 0
        assert counts[i][~keep].sum() == 0
        if keep.sum() == 1:  # w_i >= v_max: particle i always keeps itself
            continue
        p = stats.chisquare(counts[i][keep], law[i][keep] * R).pvalue
        assert p > 1e-5, (i, p)
    mean = wsum / R
    se = np.sqrt(np.maximum(wsq / R - mean**2, 1e-12) / R)
    want = N * wk / v.sum()
    assert np.all(np.abs(mean - want) <= 5 * se + 1e-12), (mean, want)
    # weights above one exactly on the particles whose weight exceeds v_max
    st, a, out = oracle.partial_rejection_control(lw, lvmax, seed=5)
    assert np.array_equal(out > 0, wk[a] > vmax)


def test_prc_fewer_trials_than_rejection_with_a_loose_bound():
    """The point of the heuristic: a v_max near the bulk of the weights raises the acceptance
    probability p = E(v)/v_max (Section 2.2), so the mean trial count falls."""
    lw = workload.synthetic_logw(4096, 3.0, seed=6)
    _, _, t_rej = oracle.rejection(lw, 0.0, seed=2, with_trials=True)
    lvmax = float(np.quantile(lw, 0.9))
    st, _, _, t_prc = oracle.partial_rejection_control(lw, lvmax, seed=2, with_trials=True)
    assert st == oracle.OK
    assert t_prc.mean() < 0.5 * t_rej.mean()
    p = np.minimum(np.exp(lw - lvmax), 1.0).mean()
    w = np.minimum(np.exp(lw - lvmax), 1.0)
    assert abs(t_prc.mean() - np.mean(1 + (1 - w) / p)) < 0.1 * np.mean(1 + (1 - w) / p)


def test_prc_permuted_outcome_carries_the_weights_of_its_ancestors():
    lw = workload.synthetic_logw(5000, 2.5, seed=8)
    lvmax = float(np.quantile(lw, 0.8))
    st, a, out = oracle.partial_rejection_control(lw, lvmax, seed=3)
    st_p, c, out_p = oracle.partial_rejection_control(lw, lvmax, seed=3, permuted=True)
    assert st == st_p == oracle.OK
    assert np.array_equal(np.sort(c), np.sort(a))
    o = np.bincount(a, minlength=len(lw))
    assert np.all(c[o > 0] == np.nonzero(o > 0)[0])
    pairs = sorted(zip(a.tolist(), out.tolist()))
    pairs_p = sorted(zip(c.tolist(), out_p.tolist()))
    assert pairs == pairs_p


def test_prc_statuses():
    lw = np.array([-5.0, -6.0, -7.0])
    st, a, out = oracle.partial_rejection_control(lw, 0.0, seed=1, max_trials=1)
    assert st == oracle.ERR_REJECTION_CAP and a.tolist() == [0, 1, 2]
    st, _, out = oracle.partial_rejection_control(np.array([0.5, -1.0]), 0.0, seed=1)
    assert st == oracle.OK and out.max() == 0.5
    st, _, _ = oracle.partial_rejection_control(np.array([0.0, np.nan]), 0.0, seed=1)
    assert st == oracle.ERR_NONFINITE
