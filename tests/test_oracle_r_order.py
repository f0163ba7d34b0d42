"""Pins of the evaluation order of r^i = N W^i / W^N (Codes 7 and 8) in the oracle's
sequential forms: r^i = W^i * c with c = N / W^N rounded once, and r^i = N where W^i = W^N.

The pins use what exact arithmetic fixes: with weights that are exactly 0 or 1 and a power-of-
two ratio N / K (K = number of ones), every prefix sum, c and r^i are exact in binary32 and
binary64, so O^i must equal floor(N W^i / K + u) computed in rational arithmetic; trailing
zero weights must receive no offspring for any N; and O must be non-decreasing."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from parity_tools import stratum_u


def _zero_one_logw(N, K, rng, dtype):
    lw = np.full(N, -np.inf, dtype)
    lw[rng.choice(N, K, replace=False)] = 0.0
    return lw


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_exact_zero_one_weights_match_rationals(dtype):
    rng = np.random.default_rng(17)
    N, K, seed = 1 << 12, 1 << 9, 77
    lw = _zero_one_logw(N, K, rng, dtype)
    W = np.cumsum(lw == 0.0)
    u01 = oracle.u01_f32 if dtype == np.float32 else oracle.u01_f64
    us = Fraction(u01(oracle.draw(seed, 0, 0, 0, 0, oracle.SYSTEMATIC)))
    for prec in (0, 1):
        st, O, _ = oracle.systematic(lw, seed, prec=prec)
        assert st == oracle.OK
        want = [min(N, int((Fraction(N * int(W[i]), K) + us) // 1)) for i in range(N)]
        want[-1] = N
        assert O.tolist() == want
        st, O, _ = oracle.stratified(lw, seed, prec=prec)
        assert st == oracle.OK
        for i in range(N):
            r = Fraction(N * int(W[i]), K)
            k = min(N - 1, int(r // 1))
            uk = Fraction(stratum_u(seed, k, 0, 0, dtype == np.float32))
            o = min(N, k + 1, int((r + uk) // 1))
            assert O[i] == (N if W[i] == K else o), i


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_trailing_zero_weights_receive_no_offspring(dtype):
    """N not a power of two, so c = N / W^N is rounded: the last nonzero particle and every
    zero weight after it still reach O = N."""
    rng = np.random.default_rng(3)
    for N in (1000, 4097, 33333):
        lw = rng.normal(-2.0, 1.5, N).astype(dtype)
        lw[N - 17:] = -np.inf
        for f in (oracle.systematic, oracle.stratified):
            st, O, a = f(lw, 11, prec=0)
            assert st == oracle.OK
            assert np.all(O[N - 18:] == N)
            assert np.all(np.diff(O) >= 0) and O[-1] == N
            assert a.max() < N - 17


def test_cumulative_offspring_non_decreasing_f32_large_n():
    rng = np.random.default_rng(5)
    N = 200_003
    lw = (-(rng.normal(0, 1, N) - 3.0) ** 2 / 2).astype(np.float32)
    for f in (oracle.systematic, oracle.stratified):
        st, O, a = f(lw, 9, prec=0)
        assert st == oracle.OK
        assert np.all(np.diff(O) >= 0) and O[-1] == N
        assert np.all(np.diff(a) >= 0)
