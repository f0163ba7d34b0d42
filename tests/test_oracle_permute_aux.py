"""Pins of the oracle's ancestry permutation (Appendix C, Codes 9 and 10) and auxiliary
conversions (Appendix D, Codes 11 and 12): the postconditions the paper states, the
order-independence of the parallel Permute, and numpy library routines."""
import numpy as np
import pytest

import oracle
import workload


def _adversarial(N, rng):
    yield np.zeros(N, np.int32)                                  # one dominant particle
    yield np.arange(N, dtype=np.int32)                           # identity
    yield np.arange(N - 1, -1, -1, dtype=np.int32)               # reversal
    yield np.concatenate([[0], np.arange(N - 1)]).astype(np.int32)  # one long chain
    yield np.full(N, N - 1, np.int32)
    yield rng.integers(0, N, N).astype(np.int32)
    yield np.sort(rng.integers(0, N, N)).astype(np.int32)
    yield rng.integers(0, max(1, N // 8), N).astype(np.int32)


@pytest.mark.parametrize("N", [1, 2, 3, 17, 256, 1000])
def test_prepermute_is_min_claimant(N):
    """d^j = lowest i with a^i = j, else the sentinel N (Code 10, Prepermute ensures)."""
    rng = np.random.default_rng(N)
    for a in _adversarial(N, rng):
        d = oracle.prepermute(a)
        want = np.full(N, N, np.int32)
        for i in range(N - 1, -1, -1):
            want[a[i]] = i
        assert np.array_equal(d, want)


@pytest.mark.parametrize("N", [1, 2, 3, 17, 256, 1000])
def test_permute_postconditions_and_order_independence(N):
    """c is a permutation of a, o_i > 0 implies c^i = i (Eq. predicate), and the result of
    Code 10 does not depend on the order of its for-each loop. Code 9 also satisfies the
    predicate (with a different arrangement)."""
    rng = np.random.default_rng(100 + N)
    for a in _adversarial(N, rng):
        c = oracle.permute(a)
        assert np.array_equal(np.sort(c), np.sort(a))
        o = np.bincount(a, minlength=N)
        idx = np.nonzero(o > 0)[0]
        assert np.all(c[idx] == idx)
        for _ in range(3):
            order = rng.permutation(N)
            assert np.array_equal(oracle.permute(a, order=order), c)
        s = oracle.permute_serial(a)
        assert np.array_equal(np.sort(s), np.sort(a))
        assert np.all(s[idx] == idx)


def test_permute_on_resampler_outputs():
    lw = workload.synthetic_logw(2048, 3.0, seed=1)
    for scheme in range(5):
        st, a = oracle.resample(scheme, lw, B=60, seed=9, log_wmax=0.0)
        assert st == oracle.OK
        c = oracle.permute(a)
        o = oracle.ancestors_to_offspring(a)
        assert np.array_equal(np.sort(c), np.sort(a))
        assert np.all(c[o > 0] == np.nonzero(o > 0)[0])


@pytest.mark.parametrize("N", [1, 5, 64, 1001])
def test_conversions_against_numpy(N):
    """Code 12 = bincount; inclusive prefix sum = cumsum; adjacent difference = diff;
    Code 11 = repeat; and the round trip a -> o -> O -> a' gives sorted(a)."""
    rng = np.random.default_rng(7 + N)
    for a in _adversarial(N, rng):
        o = oracle.ancestors_to_offspring(a)
        assert np.array_equal(o, np.bincount(a, minlength=N))
        assert o.sum() == N
        O = oracle.inclusive_prefix_sum_i32(o)
        assert np.array_equal(O, np.cumsum(o))
        assert np.array_equal(oracle.adjacent_difference_i32(O), np.diff(O, prepend=0))
        a2 = oracle.cumulative_offspring_to_ancestors(O)
        assert np.array_equal(a2, np.repeat(np.arange(N), o))
        assert np.array_equal(a2, np.sort(a))


def test_conversion_rejects_bad_input():
    with pytest.raises(ValueError):
        oracle.ancestors_to_offspring(np.array([0, 3, 1]))
    with pytest.raises(ValueError):
        oracle.cumulative_offspring_to_ancestors(np.array([1, 1, 2]))
