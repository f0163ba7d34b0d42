"""Full-size parity of the scan-based resamplers (Codes 5, 7, 8 with Code 11) that can fail:
log-weights in {0, -inf}, so every weight is exactly 0 or 1 and every cumulative weight is an
integer below 2^24. All prefix sums are then exact in every accumulation mode, the kernels'
tree sums and tile prefixes give the oracle's sequential sums bit for bit, and with r^i formed
in the same order on both sides (W^i times N / W^N rounded once) the ancestors must be equal:

  * binary32 plain and IEEE binary64: bit-exact against the sequential oracle (prec 0);
  * compensated binary32 and double-float binary64: against the double-double oracle (prec 1),
    bit-exact for compensated binary32 where N / K is a power of two (every product then
    exact) and for its multinomial draws, otherwise equal except where a draw lies within the
    two-float rounding bound of a boundary (counted, at most 64 positions).

Sizes 2^20, 2^22 + 4097 and 2^24 run through the cooperative kernel with several tiles per CTA
and a ragged last tile; the patterns include a power-of-two and an arbitrary count of ones,
long runs of zeros, trailing zeros, all ones and a single one (one run covering every slot). Permute is checked on the same calls."""
import numpy as np
import pytest
import torch

import oracle
from parity_tools import cumulative_mismatches, multinomial_mismatches

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SIZES = [1 << 20, (1 << 22) + 4097, 1 << 24]
MODES = [("f32", np.float32, 0, 0), ("f64n", np.float64, 2, 0),
         ("f32c", np.float32, 1, 1), ("f64", np.float64, 0, 1)]


@pytest.fixture(scope="module")
def h(rs):
    handle = rs.Handle(1 << 24)
    yield handle
    handle.close()


def _pattern(name, N, rng):
    ones = np.zeros(N, bool)
    if name == "quarter":
        ones[rng.choice(N, N // 4, replace=False)] = True
    elif name == "arbitrary":
        ones[rng.choice(N, int(N * 0.3719) + 7, replace=False)] = True
    elif name == "runs":
        pos, on = 0, True
        while pos < N:
            n = int(rng.geometric(1.0 / 300.0))
            ones[pos:pos + n] = on
            pos += n
            on = not on
    elif name == "trailing":
        ones[: N - 10007] = rng.random(N - 10007) < 0.5
    elif name == "all":
        ones[:] = True
    elif name == "one":  # a single particle carries all the weight: one run covers every slot
        ones[int(rng.integers(N))] = True
    return ones


def _lw(ones, dtype):
    lw = np.full(len(ones), -np.inf, dtype)
    lw[ones] = 0.0
    return lw


def _run(rs, h, scheme, lw, prec, permute=False):
    t = torch.from_numpy(lw).to(DEV)
    a = rs.rs_resample(h, scheme, t, seed=31, step=7, prec=prec, permute=permute)
    assert rs.rs_last_error(h) == rs.RS_OK
    return a.cpu().numpy()


def _pow2(x):
    return x > 0 and (x & (x - 1)) == 0


PATTERNS = {1 << 20: ["quarter", "arbitrary", "runs", "trailing", "all", "one"],
            (1 << 22) + 4097: ["arbitrary", "runs", "trailing"],
            1 << 24: ["quarter", "arbitrary", "trailing", "one"]}


@pytest.mark.parametrize("N", SIZES)
@pytest.mark.parametrize("kind,dtype,prec,oprec", MODES)
def test_exact_weights_systematic_stratified(rs, h, N, kind, dtype, prec, oprec):
    rng = np.random.default_rng(N % 1000 + 5)
    for name in PATTERNS[N]:
        ones = _pattern(name, N, rng)
        K = int(ones.sum())
        lw = _lw(ones, dtype)
        # compensated binary32: W, c and u are exact two-floats, so r^i and r^i + u are exact
        # when N / K is a power of two (the double-float mode's 53-bit uniform is a rounded
        # two-float, so it is always compared by the counted rule)
        exact = oprec == 0 or (kind == "f32c" and _pow2(K) and N % K == 0 and _pow2(N // K))
        for sch, f in ((rs.SYSTEMATIC, oracle.systematic), (rs.STRATIFIED, oracle.stratified)):
            a = _run(rs, h, sch, lw, prec)
            st, O_o, a_o = f(lw, 31, step=7, prec=oprec)
            assert st == oracle.OK
            if exact:
                assert np.array_equal(a, a_o), (name, sch, int(np.sum(a != a_o)))
            else:
                O_k = np.cumsum(np.bincount(a, minlength=N))
                n, bad = cumulative_mismatches(kind, sch, lw, O_k, O_o, seed=31, step=7,
                                               oracle_is_sequential=False)
                assert bad == 0, (name, sch, n, bad)
                assert n <= 64, (name, sch, n)
            c = _run(rs, h, sch, lw, prec, permute=True)
            assert np.array_equal(c, oracle.permute(a)), (name, sch)
            assert ones[a].all()


@pytest.mark.parametrize("N", SIZES)
@pytest.mark.parametrize("kind,dtype,prec,oprec", MODES)
def test_exact_weights_multinomial(rs, h, N, kind, dtype, prec, oprec):
    # the oracle's search costs about 1 us per output at 2^24: one pattern there, and the
    # double-double forms up to 2^22 + 4097
    if N == 1 << 24 and oprec == 1:
        pytest.skip("double-double multinomial oracle at 2^24 covered at 2^22 + 4097")
    rng = np.random.default_rng(N % 1000 + 9)
    names = ["arbitrary"] if N == 1 << 24 else PATTERNS[N][:2]
    for name in names:
        ones = _pattern(name, N, rng)
        lw = _lw(ones, dtype)
        a = _run(rs, h, rs.MULTINOMIAL, lw, prec)
        st, a_o = oracle.multinomial(lw, 31, step=7, prec=oprec)
        assert st == oracle.OK
        if kind in ("f32", "f64n", "f32c"):  # u = U * K is exact for f32c (48-bit product)
            assert np.array_equal(a, a_o), (name, int(np.sum(a != a_o)))
        else:
            n, bad = multinomial_mismatches(kind, lw, a, a_o, seed=31, step=7,
                                            oracle_is_sequential=False)
            assert bad == 0 and n <= 64, (name, n, bad)
        c = _run(rs, h, rs.MULTINOMIAL, lw, prec, permute=True)
        assert np.array_equal(c, oracle.permute(a))
        assert ones[a].all()


def test_exact_weights_separate_kernels_agree(rs, h):
    """The separate-kernel form (max, tile sums, prefixes, emission as four launches) gives the
    same bit-exact result as the oracle on exact weights."""
    N = (1 << 22) + 4097
    rng = np.random.default_rng(77)
    ones = _pattern("runs", N, rng)
    lw = _lw(ones, np.float32)
    rs.rs_set_launch_mode(h, rs.LAUNCH_SEPARATE)
    try:
        for sch, f in ((rs.SYSTEMATIC, oracle.systematic), (rs.STRATIFIED, oracle.stratified)):
            a = _run(rs, h, sch, lw, 0)
            assert np.array_equal(a, f(lw, 31, step=7, prec=0)[2])
    finally:
        rs.rs_set_launch_mode(h, rs.LAUNCH_AUTO)
