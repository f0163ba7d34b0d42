"""Pins of the oracle's resamplers against the laws and properties the paper and the
mathematics fix: exact transition laws at small N (chi-square over seeded draws), the
unbiasedness condition (Eq. unbiasedness), the TV bound that defines B* (Eq. B), the floor /
ceiling property of systematic offspring, the one-ancestor-per-stratum definition of the
stratified and systematic resamplers (exact rational arithmetic), and numpy library
routines for the primitives."""
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import oracle
import workload
from parity_tools import stratum_u


def _pi(w):
    w = np.asarray(w, dtype=np.float64)
    return w / w.sum()


def _metropolis_kernel(w):
    """Transition matrix of the independent Metropolis kernel of Section 2.1: propose j
    uniformly, accept with probability min(1, w_j/w_k) (always when w_k = 0)."""
    w = np.asarray(w, dtype=np.float64)
    N = len(w)
    P = np.zeros((N, N))
    for k in range(N):
        for j in range(N):
            if j == k:
                continue
            acc = 1.0 if w[k] == 0 else min(1.0, w[j] / w[k])
            P[k, j] = acc / N
        P[k, k] = 1.0 - P[k].sum()
    return P


def _chi2_ok(counts, probs, alpha=1e-5):
    counts = np.asarray(counts, dtype=np.float64)
    probs = np.asarray(probs, dtype=np.float64)
    keep = probs > 0
    assert counts[~keep].sum() == 0, "mass on an outcome of probability zero"
    exp = probs[keep] * counts.sum()
    p = stats.chisquare(counts[keep], exp).pvalue
    return p > alpha, p


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_metropolis_exact_law_small_n(dtype):
    """a^i ~ P^B(i, .) independently, P the kernel above (Section 2.1), at B = 3 where the
    law is still far from pi, including a zero-weight particle."""
    w = np.array([0.1, 0.5, 1.0, 0.0, 0.35])
    lw = np.log(np.where(w > 0, w, 1.0)).astype(dtype)
    lw[w == 0] = -np.inf
    B = 3
    N = len(w)
    # the kernel acts on the weights the oracle actually uses
    wk = np.exp(lw.astype(np.float64))
    PB = np.linalg.matrix_power(_metropolis_kernel(wk), B)
    R = 30000
    counts = np.zeros((N, N), np.int64)
    for s in range(R):
        st, a = oracle.metropolis(lw, B, seed=1000 + s)
        assert st == oracle.OK
        counts[np.arange(N), a] += 1
    for i in range(N):
        ok, p = _chi2_ok(counts[i], PB[i])
        assert ok, (i, p, counts[i], PB[i])


def test_metropolis_bias_shrinks_with_B():
    """Exact offspring bias sum_i |E o_i - N pi_i| of the Metropolis resampler (from P^B)
    decreases as B grows and respects the TV bound (1 - beta)^B per chain (Section 2.1)."""
    lw = workload.synthetic_logw(6, 3.0, seed=5)
    w = np.exp(lw)
    N = len(w)
    pi = _pi(w)
    P = _metropolis_kernel(w)
    beta = np.min(w.mean() / w)
    prev = np.inf
    for B in [1, 2, 4, 8, 16, 32, 64]:
        PB = np.linalg.matrix_power(P, B)
        Eo = PB.sum(axis=0)
        bias = np.abs(Eo - N * pi).sum()
        assert bias <= prev + 1e-15
        prev = bias
        tv = 0.5 * np.abs(PB - pi[None, :]).sum(axis=1).max()
        assert tv <= (1 - beta) ** B + 1e-12


def test_metropolis_B_meets_tv_target():
    """B* of Eq. (B) makes the TV distance of every chain at most eps (Section 2.1)."""
    for y in [0.0, 1.0, 2.0, 3.0]:
        lw = workload.synthetic_logw(6, y, seed=11)
        w = np.exp(lw)
        beta = float(np.min(w.mean() / w))
        for eps in [0.1, 0.01]:
            B = oracle.metropolis_B(eps, beta)
            assert B >= 1
            PB = np.linalg.matrix_power(_metropolis_kernel(w), B)
            tv = 0.5 * np.abs(PB - _pi(w)[None, :]).sum(axis=1).max()
            assert tv <= eps + 1e-12
    # the settings of the experiments (Section 4.1: eps = 1/100, beta = E(w)/w_max)
    Bs = [oracle.metropolis_B(0.01, workload.beta_estimate(y)) for y in np.arange(0, 4.5, 0.5)]
    assert all(b1 <= b2 for b1, b2 in zip(Bs, Bs[1:]))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_rejection_exact_law_and_trials(dtype):
    """P(a^i = j) = [j = i] w_i/w_max + (1 - w_i/w_max) pi_j (Section 2.2, first proposal
    j = i), and E(trials_i) = 1 + (1 - w_i/w_max)/p with p = mean(w)/w_max."""
    w = np.array([0.2, 0.9, 0.05, 0.0, 0.6])
    lw = np.full(len(w), -np.inf, dtype)
    lw[w > 0] = np.log(w[w > 0]).astype(dtype)
    wk = np.exp(lw.astype(np.float64))
    N = len(w)
    pi = _pi(wk)
    law = (1 - wk)[:, None] * pi[None, :] + np.diag(wk)
    R = 30000
    counts = np.zeros((N, N), np.int64)
    tsum = np.zeros(N)
    for s in range(R):
        st, a, t = oracle.rejection(lw, 0.0, seed=77 + s, with_trials=True)
        assert st == oracle.OK
        counts[np.arange(N), a] += 1
        tsum += t
    for i in range(N):
        ok, p = _chi2_ok(counts[i], law[i])
        assert ok, (i, p)
    p = wk.mean()
    et = 1 + (1 - wk) / p
    var = (1 - wk) * (1 + wk) * (1 - p) / p**2 + (1 - wk) / p**2  # generous bound
    assert np.all(np.abs(tsum / R - et) <= 6 * np.sqrt(var / R))


def test_rejection_max_trials_bound():
    """Mean over seeds of the maximum trial count stays below the bound of Section 2.2,
    E(M*_N) < 1 + (1 + log N)/p, plus one for the deterministic first attempt."""
    N = 4096
    lw = workload.synthetic_logw(N, 2.0, seed=3)
    p = np.exp(lw).mean()
    maxes = []
    for s in range(8):
        st, a, t = oracle.rejection(lw, 0.0, seed=s, with_trials=True)
        assert st == oracle.OK
        maxes.append(t.max())
    assert np.mean(maxes) < 2 + (1 + np.log(N)) / p


def test_rejection_status_cap_bound_nonfinite():
    lw = np.array([-5.0, -6.0, -7.0])
    st, a = oracle.rejection(lw, 0.0, seed=1, max_trials=1)
    assert st == oracle.ERR_REJECTION_CAP
    assert a.tolist() == [0, 1, 2]
    st, a = oracle.rejection(np.array([0.5, -1.0]), 0.0, seed=1)
    assert st == oracle.ERR_BOUND_VIOLATED
    st, _ = oracle.rejection(np.array([0.0, np.nan]), 0.0, seed=1)
    assert st == oracle.ERR_NONFINITE
    st, _ = oracle.metropolis(np.array([0.0, np.inf]), 4, seed=1)
    assert st == oracle.ERR_NONFINITE


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_multinomial_exact_law(dtype):
    """a^i ~ pi independently (Appendix B.1), zero weights never selected."""
    w = np.array([0.3, 0.0, 1.0, 0.05, 0.4, 0.25])
    lw = np.full(len(w), -np.inf, dtype)
    lw[w > 0] = np.log(w[w > 0]).astype(dtype)
    pi = _pi(np.exp(lw.astype(np.float64)))
    N = len(w)
    counts = np.zeros((N, N), np.int64)
    for s in range(20000):
        st, a = oracle.multinomial(lw, seed=s)
        assert st == oracle.OK
        counts[np.arange(N), a] += 1
    for i in range(N):
        ok, p = _chi2_ok(counts[i], pi)
        assert ok, (i, p)


def test_multinomial_f32_is_library_composition():
    """Code 5 in binary32 equals the composition of library primitives: numpy's sequential
    cumulative sum and searchsorted(side='right') of u = U * W^N."""
    lw = workload.synthetic_logw(3000, 2.0, seed=8, dtype=np.float32)
    st, w, m = oracle.weights(lw)
    assert st == oracle.OK
    W = np.cumsum(w, dtype=np.float32)
    assert np.array_equal(W, oracle.inclusive_prefix_sum(w))
    seed = 99
    U = np.array([oracle.u01_f32(oracle.draw(seed, i, 0, 0, 0, oracle.MULTINOMIAL))
                  for i in range(len(lw))], np.float32)
    u = U * W[-1]
    want = np.searchsorted(W, u, side="right")
    st, a = oracle.multinomial(lw, seed)
    assert np.array_equal(a, want)


def test_weights_are_max_shifted():
    lw = np.array([-3.0, 2.0, -np.inf, 1.5])
    st, w, m = oracle.weights(lw)
    assert st == oracle.OK and m == 2.0
    assert w[1] == 1.0 and w[2] == 0.0
    np.testing.assert_allclose(w, np.exp(lw - 2.0), rtol=2e-16)
    st, _, _ = oracle.weights(np.array([-np.inf, -np.inf]))
    assert st == oracle.ERR_ZERO_WEIGHT


def _exact_prefix(w):
    acc = Fraction(0)
    out = []
    for v in w:
        acc += Fraction(float(v))
        out.append(acc)
    return out


def _first_reaching(Wf, S, N, t):
    """First j with N W_j / S >= t (exact rationals), i.e. the ancestor of point t."""
    lo, hi = 0, len(Wf)
    while lo < hi:
        mid = (lo + hi) // 2
        if N * Wf[mid] >= t * S:
            hi = mid
        else:
            lo = mid + 1
    return lo


@pytest.mark.parametrize("scheme", ["systematic", "stratified"])
@pytest.mark.parametrize("prec", [0, 1])
def test_one_ancestor_per_stratum_exact(scheme, prec):
    """Output position k takes the particle whose slice of the circle holds the point
    (k + 1 - u_k) W^N / N, one point per stratum (Appendix B.2/B.3, Figure 1): O^i =
    floor(r^i + u) counts exactly the points k + 1 - u <= r^i. Checked against exact rational
    arithmetic; binary64 positions may differ only within 1e-9 of a slice boundary, the
    double-double form nowhere."""
    N = 257
    lw = workload.synthetic_logw(N, 2.0, seed=21)
    lw[5] = -np.inf
    lw[-3:] = -np.inf  # trailing zero weights
    seed = 4242
    if scheme == "systematic":
        st, O, a = oracle.systematic(lw, seed, prec=prec)
        u0 = oracle.u01_f64(oracle.draw(seed, 0, 0, 0, 0, oracle.SYSTEMATIC))
        us = [u0] * N
    else:
        st, O, a = oracle.stratified(lw, seed, prec=prec)
        us = [stratum_u(seed, k, 0, 0, False) for k in range(N)]
    assert st == oracle.OK
    _, w, _ = oracle.weights(lw)
    Wf = _exact_prefix(w)
    S = Wf[-1]
    for k in range(N):
        t = k + 1 - Fraction(us[k])
        want = _first_reaching(Wf, S, N, t)
        if a[k] != want:
            assert prec == 0
            near = min(abs(N * Wf[j] / S - t) for j in range(min(a[k], want), max(a[k], want) + 1))
            assert near < Fraction(1, 10**9), (k, a[k], want)
        assert w[a[k]] > 0


def test_systematic_floor_ceil_and_unbiased_over_u():
    """Systematic offspring satisfy o_i in {floor(N pi_i), ceil(N pi_i)}, and averaging O over
    u on a uniform grid gives N pi_i (Eq. unbiasedness) to the grid's resolution."""
    N = 300
    lw = workload.synthetic_logw(N, 3.0, seed=31)
    _, w, _ = oracle.weights(lw)
    W = oracle.inclusive_prefix_sum(w)
    Npi = N * w / W[-1]
    G = 2048
    osum = np.zeros(N)
    for g in range(G):
        u = (g + 0.5) / G
        O = oracle.systematic_O_given_u(W, u)
        o = oracle.adjacent_difference_i32(O)
        assert o.sum() == N
        assert np.all((o == np.floor(Npi)) | (o == np.ceil(Npi)) | (np.abs(Npi - np.round(Npi)) < 1e-9))
        osum += o
    assert np.max(np.abs(osum / G - Npi)) <= 1.0 / G + 1e-9


def test_stratified_bounds_and_unbiased():
    """Stratified offspring lie in [floor(N pi_i) - 1, ceil(N pi_i) + 1] and are unbiased
    (Monte Carlo over the per-stratum uniforms)."""
    N = 200
    lw = workload.synthetic_logw(N, 2.5, seed=41)
    _, w, _ = oracle.weights(lw)
    W = oracle.inclusive_prefix_sum(w)
    Npi = N * w / W[-1]
    rng = np.random.default_rng(5)
    R = 4000
    osum = np.zeros(N)
    for _ in range(R):
        O = oracle.stratified_O_given_u(W, rng.random(N))
        o = oracle.adjacent_difference_i32(O)
        assert o.sum() == N and o.min() >= 0
        assert np.all(o >= np.floor(Npi) - 1) and np.all(o <= np.ceil(Npi) + 1)
        osum += o
    assert np.max(np.abs(osum / R - Npi)) <= 6 * np.sqrt(0.25 / R) + 1e-9


def test_dd_systematic_matches_exact_rationals():
    """The double-double cumulative offspring equal the exact rational ones."""
    rng = np.random.default_rng(9)
    N = 150
    w = rng.exponential(1.0, N)
    w[[3, 40]] = 0.0
    hi, lo = oracle.dd_prefix(w)
    Wf = _exact_prefix(w)
    for u in [0.0, 0.25, 0.5, float(rng.random())]:
        O = oracle.systematic_O_given_u(hi, u, lo=lo)
        for i in range(N):
            want = min(N, int((N * Wf[i] / Wf[-1] + Fraction(u)) // 1))
            assert O[i] == want


def test_scan_variants_agree_at_small_n():
    """The dtype prefix sum and the double-double prefix sum give the same systematic and
    multinomial output at small N away from boundaries (both are the same method)."""
    lw = workload.synthetic_logw(512, 1.0, seed=2)
    for f in (oracle.systematic, oracle.stratified):
        _, O0, a0 = f(lw, 5, prec=0)
        _, O1, a1 = f(lw, 5, prec=1)
        assert np.sum(O0 != O1) <= 1
    _, m0 = oracle.multinomial(lw, 5, prec=0)
    _, m1 = oracle.multinomial(lw, 5, prec=1)
    assert np.sum(m0 != m1) <= 1


SCHEMES = [oracle.MULTINOMIAL, oracle.STRATIFIED, oracle.SYSTEMATIC, oracle.METROPOLIS,
           oracle.REJECTION]


@pytest.mark.parametrize("scheme", SCHEMES)
def test_unbiasedness_condition(scheme):
    """E(o_i | w) = N w_i / sum w (Eq. unbiasedness) by Monte Carlo; Metropolis run at
    4 B* so that its bias is far below the Monte Carlo error."""
    N = 48
    lw = workload.synthetic_logw(N, 1.5, seed=13)
    w = np.exp(lw)
    Npi = N * w / w.sum()
    B = 4 * oracle.metropolis_B(0.01, float(np.min(w.mean() / w)))
    R = 3000
    osum = np.zeros(N)
    for s in range(R):
        st, a = oracle.resample(scheme, lw, B=B, seed=500 + s, log_wmax=0.0)
        assert st == oracle.OK
        osum += oracle.ancestors_to_offspring(a)
    sd = np.sqrt(Npi * (1 - Npi / N) / R)
    assert np.all(np.abs(osum / R - Npi) <= 5 * sd + 1e-3)


def test_scale_invariance_exact():
    """Adding a constant to every log-weight leaves Metropolis and rejection ancestors
    unchanged when the shifted values are exact (Appendix E: invariance to scaling)."""
    rng = np.random.default_rng(1)
    lw = -np.round(rng.exponential(2.0, 500) * 1024) / 1024
    for c in [16.0, -64.0]:
        _, a0 = oracle.metropolis(lw, 16, seed=3)
        _, a1 = oracle.metropolis(lw + c, 16, seed=3)
        assert np.array_equal(a0, a1)
        _, r0 = oracle.rejection(lw, 0.0, seed=3)
        _, r1 = oracle.rejection(lw + c, c, seed=3)
        assert np.array_equal(r0, r1)


@pytest.mark.parametrize("f32", [True, False])
def test_stratum_uniforms_share_blocks(f32):
    """The oracle's stratum uniforms follow the block mapping (four strata per Philox block at
    24 bits, two at 53), are exact multiples of 2^-24 / 2^-53 in [0, 1), and strata that share
    a block take distinct words of it (so they are independent draws)."""
    seed, step, filt = 987654321, 7, 3
    f = oracle.stratum_u_f32 if f32 else oracle.stratum_u_f64
    per = 4 if f32 else 2
    us = [f(seed, k, step, filt) for k in range(64)]
    for k, u in enumerate(us):
        assert u == stratum_u(seed, k, step, filt, f32)
        assert 0.0 <= u < 1.0
        assert (u * 2.0 ** (24 if f32 else 53)).is_integer()
    # within a block the uniforms are distinct words; blocks do not repeat
    for b in range(0, 64, per):
        assert len(set(us[b:b + per])) == per
    assert len(set(us)) == 64
