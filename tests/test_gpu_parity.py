"""GPU parity: the CUDA library (called through the C ABI) against the CPU oracle on the same
seeded inputs. Bit-exact for Metropolis, rejection, Permute and the integer conversions;
the scan-based resamplers may differ only at draws within the rounding bound of a
cumulative-weight boundary (counted, see parity_tools)."""
import numpy as np
import pytest
import torch

import oracle
import workload
from parity_tools import (cumulative_mismatches, multinomial_mismatches, truth_offset,
                          truth_prefix)

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 3, 5, 127, 1000, 4096, 4097, 12289, 65539]
DEV = "cuda:0"


@pytest.fixture(scope="module")
def h(rs):
    handle = rs.Handle(1 << 21)
    yield handle
    handle.close()


def _lw(N, y, dtype, seed=3):
    return workload.synthetic_logw(N, y, seed=seed + N, dtype=dtype)


def _run(rs, h, scheme, lw, **kw):
    t = torch.from_numpy(lw).to(DEV)
    a = rs.rs_resample(h, scheme, t, **kw)
    st = rs.rs_last_error(h)
    return st, a.cpu().numpy()


# ---------------------------------------------------------------------------------------
# Metropolis and rejection: bit-exact
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("N", SIZES)
def test_metropolis_bit_exact(rs, h, dtype, N):
    for y, B in [(0.0, 4), (2.0, 16), (4.0, 64), (2.0, 0), (1.0, 7)]:
        lw = _lw(N, y, dtype)
        st, a = _run(rs, h, rs.METROPOLIS, lw, B=B, seed=11, step=3)
        assert st == rs.RS_OK
        ost, want = oracle.metropolis(lw, B, seed=11, step=3)
        assert np.array_equal(a, want), (y, B, np.sum(a != want))
        st, c = _run(rs, h, rs.METROPOLIS, lw, B=B, seed=11, step=3, permute=True)
        assert st == rs.RS_OK
        assert np.array_equal(c, oracle.permute(want))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("N", SIZES)
def test_rejection_bit_exact(rs, h, dtype, N):
    for y in [0.0, 2.0, 4.0]:
        lw = _lw(N, y, dtype)
        st, a = _run(rs, h, rs.REJECTION, lw, seed=5, step=1, log_wmax=0.0)
        ost, want = oracle.rejection(lw, 0.0, seed=5, step=1)
        assert st == rs.RS_OK and ost == oracle.OK
        assert np.array_equal(a, want), (y, np.sum(a != want))
        st, c = _run(rs, h, rs.REJECTION, lw, seed=5, step=1, log_wmax=0.0, permute=True)
        assert st == rs.RS_OK
        assert np.array_equal(c, oracle.permute(want))


def test_rejection_and_metropolis_statuses(rs, h):
    lw = np.array([-5.0, -6.0, -7.0, -8.0])
    st, a = _run(rs, h, rs.REJECTION, lw, seed=1, max_trials=1)
    ost, want = oracle.rejection(lw, 0.0, seed=1, max_trials=1)
    assert st == rs.RS_ERR_REJECTION_CAP and ost == oracle.ERR_REJECTION_CAP
    assert np.array_equal(a, want)
    lw = np.array([0.5, -1.0, -2.0])
    st, a = _run(rs, h, rs.REJECTION, lw, seed=1)
    ost, want = oracle.rejection(lw, 0.0, seed=1)
    assert st == rs.RS_ERR_BOUND_VIOLATED and ost == oracle.ERR_BOUND_VIOLATED
    assert np.array_equal(a, want)
    for scheme in range(5):
        st, a = _run(rs, h, scheme, np.array([0.0, np.nan, -1.0]), B=4, seed=1)
        assert st == rs.RS_ERR_NONFINITE, scheme
        assert a.min() >= 0 and a.max() < 3
        st, a = _run(rs, h, scheme, np.array([0.0, np.inf, -1.0], np.float32), B=4, seed=1)
        assert st == rs.RS_ERR_NONFINITE, scheme
    for scheme in (rs.MULTINOMIAL, rs.STRATIFIED, rs.SYSTEMATIC):
        st, a = _run(rs, h, scheme, np.full(10, -np.inf), seed=1)
        assert st == rs.RS_ERR_ZERO_WEIGHT
        assert np.array_equal(np.sort(a), np.arange(10))
    assert rs.rs_last_error(h) == rs.RS_OK  # cleared


def test_scale_invariance_bit_exact(rs, h):
    """Adding an exactly representable constant to every log-weight leaves the ancestors of
    the collective-free schemes unchanged (Appendix E)."""
    rng = np.random.default_rng(1)
    lw = -np.round(rng.exponential(2.0, 3000) * 1024) / 1024
    for c in [16.0, -64.0]:
        _, a0 = _run(rs, h, rs.METROPOLIS, lw, B=16, seed=3)
        _, a1 = _run(rs, h, rs.METROPOLIS, lw + c, B=16, seed=3)
        assert np.array_equal(a0, a1)
        _, r0 = _run(rs, h, rs.REJECTION, lw, seed=3, log_wmax=0.0)
        _, r1 = _run(rs, h, rs.REJECTION, lw + c, seed=3, log_wmax=c)
        assert np.array_equal(r0, r1)


# ---------------------------------------------------------------------------------------
# Scan-based resamplers: equal except near boundaries (counted)
# ---------------------------------------------------------------------------------------
KINDS = [("f32", np.float32, 0), ("f32c", np.float32, 1), ("f64", np.float64, 0),
         ("f64n", np.float64, 2)]


def _check_valid_ancestry(a, lw, sorted_expected):
    N = len(lw)
    assert a.min() >= 0 and a.max() < N
    if sorted_expected:
        assert np.all(np.diff(a) >= 0)
    w_zero = lw == -np.inf
    assert not np.any(w_zero[a]), "a zero-weight particle was selected"


@pytest.mark.parametrize("kind,dtype,prec", KINDS)
@pytest.mark.parametrize("scheme", ["systematic", "stratified"])
@pytest.mark.parametrize("N", SIZES)
def test_systematic_stratified_parity(rs, h, kind, dtype, prec, scheme, N):
    sch = rs.SYSTEMATIC if scheme == "systematic" else rs.STRATIFIED
    f = oracle.systematic if scheme == "systematic" else oracle.stratified
    total_mis = 0
    for y in [0.0, 2.0, 4.0]:
        lw = _lw(N, y, dtype)
        if N > 10:
            lw[N // 3] = -np.inf
            lw[-2:] = -np.inf  # trailing zero weights
        st, a = _run(rs, h, sch, lw, seed=21, step=2, prec=prec)
        assert st == rs.RS_OK
        _check_valid_ancestry(a, lw, sorted_expected=True)
        O_k = np.cumsum(np.bincount(a, minlength=N))
        dev, bound = truth_offset(kind, sch, lw, O_k, seed=21, step=2)
        assert dev <= bound, (y, dev, bound)
        for oprec in sorted({0, prec}):
            ost, O_o, _ = f(lw, 21, step=2, prec=oprec)
            assert ost == oracle.OK
            n, bad = cumulative_mismatches(kind, sch, lw, O_k, O_o, seed=21, step=2,
                                           oracle_is_sequential=(oprec == 0))
            assert bad == 0, (y, oprec, n, bad)
            total_mis += n
        # Permute on the kernel's own ancestry is exact
        st, c = _run(rs, h, sch, lw, seed=21, step=2, prec=prec, permute=True)
        assert st == rs.RS_OK
        assert np.array_equal(c, oracle.permute(a))
    if kind in ("f64", "f64n") or N <= 5:
        assert total_mis <= 2


@pytest.mark.parametrize("kind,dtype,prec", KINDS)
@pytest.mark.parametrize("N", SIZES)
def test_multinomial_parity(rs, h, kind, dtype, prec, N):
    total_mis = 0
    for y in [0.0, 2.0, 4.0]:
        lw = _lw(N, y, dtype)
        if N > 10:
            lw[N // 2] = -np.inf
            lw[-1] = -np.inf
        st, a = _run(rs, h, rs.MULTINOMIAL, lw, seed=8, step=4, prec=prec)
        assert st == rs.RS_OK
        _check_valid_ancestry(a, lw, sorted_expected=False)
        for oprec in sorted({0, prec}):
            ost, want = oracle.multinomial(lw, 8, step=4, prec=oprec)
            n, bad = multinomial_mismatches(kind, lw, a, want, seed=8, step=4,
                                            oracle_is_sequential=(oprec == 0))
            assert bad == 0, (y, oprec, n, bad)
            total_mis += n
        st, c = _run(rs, h, rs.MULTINOMIAL, lw, seed=8, step=4, prec=prec, permute=True)
        assert st == rs.RS_OK
        assert np.array_equal(c, oracle.permute(a))
    if kind in ("f64", "f64n"):
        assert total_mis <= 2


@pytest.mark.parametrize("kind,dtype,prec", KINDS)
def test_scan_schemes_deterministic_and_misaligned(rs, h, kind, dtype, prec):
    """Two runs give identical results; a log-weight pointer that is not 16-byte aligned
    (a view starting at element 1) gives the same result as an aligned copy."""
    N = 20001
    lw = _lw(N + 1, 2.0, dtype)
    base = torch.from_numpy(lw).to(DEV)
    view = base[1:]
    aligned = view.clone()
    assert view.data_ptr() % 16 != 0
    for scheme in (rs.MULTINOMIAL, rs.STRATIFIED, rs.SYSTEMATIC):
        a1 = rs.rs_resample(h, scheme, aligned, seed=4, prec=prec).cpu()
        a2 = rs.rs_resample(h, scheme, aligned, seed=4, prec=prec).cpu()
        a3 = rs.rs_resample(h, scheme, view, seed=4, prec=prec).cpu()
        assert rs.rs_last_error(h) == rs.RS_OK
        assert torch.equal(a1, a2) and torch.equal(a1, a3)


def test_degenerate_inputs(rs, h):
    for dtype in (np.float32, np.float64):
        for scheme in range(5):
            # N = 1
            st, a = _run(rs, h, scheme, np.array([-3.0], dtype), B=5, seed=1, log_wmax=0.0)
            assert st == rs.RS_OK and a.tolist() == [0]
            # all equal weights
            lw = np.zeros(777, dtype)
            st, a = _run(rs, h, scheme, lw, B=5, seed=2, log_wmax=0.0)
            assert st == rs.RS_OK
            if scheme in (rs.STRATIFIED, rs.SYSTEMATIC):
                assert np.array_equal(a, np.arange(777))
            # one particle carries all the weight
            lw = np.full(999, -np.inf, dtype)
            lw[123] = -5.0
            st, a = _run(rs, h, scheme, lw, B=5, seed=3, log_wmax=0.0, max_trials=1 << 16)
            if scheme == rs.REJECTION:
                assert st == rs.RS_ERR_REJECTION_CAP or np.all(a == 123)
            elif scheme == rs.METROPOLIS:
                assert st == rs.RS_OK
            else:
                assert st == rs.RS_OK and np.all(a == 123)


# ---------------------------------------------------------------------------------------
# Permute and conversions: bit-exact
# ---------------------------------------------------------------------------------------
def _adversarial(N, rng):
    yield np.zeros(N, np.int32)
    yield np.arange(N, dtype=np.int32)
    yield np.arange(N - 1, -1, -1, dtype=np.int32)
    yield np.concatenate([[0], np.arange(N - 1)]).astype(np.int32)
    yield rng.integers(0, N, N).astype(np.int32)
    yield np.sort(rng.integers(0, N, N)).astype(np.int32)
    yield rng.integers(0, max(1, N // 16), N).astype(np.int32)


@pytest.mark.parametrize("N", [1, 2, 3, 100, 4096, 4097, 70001])
def test_permute_prepermute_exact(rs, h, N):
    rng = np.random.default_rng(N)
    for a in _adversarial(N, rng):
        t = torch.from_numpy(a).to(DEV)
        d = rs.rs_prepermute(h, t).cpu().numpy()
        c = rs.rs_permute(h, t).cpu().numpy()
        assert rs.rs_last_error(h) == rs.RS_OK
        assert np.array_equal(d, oracle.prepermute(a))
        assert np.array_equal(c, oracle.permute(a))


@pytest.mark.parametrize("N", [1, 2, 3, 100, 4096, 4097, 70001])
def test_conversions_exact(rs, h, N):
    rng = np.random.default_rng(7 + N)
    for a in _adversarial(N, rng):
        t = torch.from_numpy(a).to(DEV)
        o = rs.rs_offspring(h, t)
        O = rs.rs_cumulative_offspring(h, o)
        o2 = rs.rs_adjacent_difference(h, O)
        a2 = rs.rs_cumulative_offspring_to_ancestors(h, O)
        assert rs.rs_last_error(h) == rs.RS_OK
        want_o = oracle.ancestors_to_offspring(a)
        assert np.array_equal(o.cpu().numpy(), want_o)
        assert np.array_equal(O.cpu().numpy(), oracle.inclusive_prefix_sum_i32(want_o))
        assert np.array_equal(o2.cpu().numpy(), want_o)
        assert np.array_equal(a2.cpu().numpy(),
                              oracle.cumulative_offspring_to_ancestors(
                                  oracle.inclusive_prefix_sum_i32(want_o)))


def test_conversion_errors_flagged(rs, h):
    t = torch.tensor([0, 5, 1], dtype=torch.int32, device=DEV)
    rs.rs_offspring(h, t)
    assert rs.rs_last_error(h) == rs.RS_ERR_ARG
    O = torch.tensor([1, 1, 2], dtype=torch.int32, device=DEV)  # O[N-1] != N
    rs.rs_cumulative_offspring_to_ancestors(h, O)
    assert rs.rs_last_error(h) == rs.RS_ERR_ARG


# ---------------------------------------------------------------------------------------
# Cumulative weights (float outputs): 1e-12 relative in binary64, 1e-5 in binary32
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("kind,dtype,prec,tol", [("f32", np.float32, 0, 1e-5),
                                                 ("f32c", np.float32, 1, 1e-6),
                                                 ("f64", np.float64, 0, 1e-12),
                                                 ("f64n", np.float64, 2, 1e-12)])
@pytest.mark.parametrize("N", [1, 3, 4096, 4097, 100003])
def test_cumulative_weights(rs, h, kind, dtype, prec, tol, N):
    lw = _lw(N, 3.0, dtype)
    if N > 10:
        lw[5] = -np.inf
    t = torch.from_numpy(lw).to(DEV)
    W, lt = rs.rs_cumulative_weights(h, t, prec=prec)
    assert rs.rs_last_error(h) == rs.RS_OK
    W = W.cpu().numpy().astype(np.float64)
    Wstar, S = truth_prefix(lw)
    nz = Wstar > 0
    rel = np.abs(W[nz] - Wstar[nz]) / Wstar[nz]
    assert rel.max() <= tol, rel.max()
    assert np.all(np.diff(W) >= 0)
    m = float(np.max(lw))
    assert abs(lt.item() - (m + np.log(S))) <= (1e-12 if dtype == np.float64 else 1e-6) * max(1.0, abs(m + np.log(S)))


@pytest.mark.parametrize("N", [1, 4097, 65539])
def test_cumulative_weights_f64_output(rs, h, N):
    """The binary64 output writes every accumulator exactly: equal to the dtype output where
    the accumulator is the dtype (binary32 plain, binary64), rounding to it where it is a
    pair (compensated), and within the two-float accuracy of the double-double truth."""
    for dtype, prec, tol in ((np.float32, rs.PREC_PLAIN, 1e-5), (np.float32, rs.PREC_COMPENSATED,
                              1e-11), (np.float64, rs.PREC_PLAIN, 1e-12),
                             (np.float64, rs.PREC_BINARY64, 1e-12)):
        lw = _lw(N, 3.0, dtype)
        t = torch.from_numpy(lw).to(DEV)
        W, lt = rs.rs_cumulative_weights(h, t, prec=prec)
        W64, lt64 = rs.rs_cumulative_weights_f64(h, t, prec=prec)
        assert rs.rs_last_error(h) == rs.RS_OK
        W, W64 = W.cpu().numpy(), W64.cpu().numpy()
        assert W64.dtype == np.float64 and lt64.item() == lt.item()
        if prec == rs.PREC_COMPENSATED:  # the binary32 output is the pair's high part
            assert np.all(np.abs(W64 - W.astype(np.float64))
                          <= np.spacing(W).astype(np.float64) / 2)
        else:
            assert np.array_equal(W64, W.astype(np.float64))
        Wstar, _ = truth_prefix(lw)
        nz = Wstar > 0
        assert (np.abs(W64[nz] - Wstar[nz]) / Wstar[nz]).max() <= tol
        assert np.all(np.diff(W64) >= 0)


# ---------------------------------------------------------------------------------------
# Full-size workloads (the benchmark's N = 2^20 in both dtypes)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_full_size_collective_free_bit_exact(rs, dtype):
    N = 1 << 20
    with rs.Handle(N) as hh:
        lw = workload.synthetic_logw(N, 2.0, seed=20130116, dtype=dtype)
        st, a = _run(rs, hh, rs.METROPOLIS, lw, B=16, seed=99)
        assert st == rs.RS_OK
        assert np.array_equal(a, oracle.metropolis(lw, 16, seed=99)[1])
        st, a = _run(rs, hh, rs.REJECTION, lw, seed=99, log_wmax=0.0)
        assert st == rs.RS_OK
        assert np.array_equal(a, oracle.rejection(lw, 0.0, seed=99)[1])


@pytest.mark.parametrize("kind,dtype,prec", KINDS)
def test_full_size_scan_schemes(rs, kind, dtype, prec):
    N = 1 << 20
    with rs.Handle(N) as hh:
        lw = workload.synthetic_logw(N, 2.0, seed=20130116, dtype=dtype)
        for sch, f in ((rs.SYSTEMATIC, oracle.systematic), (rs.STRATIFIED, oracle.stratified)):
            st, a = _run(rs, hh, sch, lw, seed=5, prec=prec)
            assert st == rs.RS_OK
            _check_valid_ancestry(a, lw, True)
            O_k = np.cumsum(np.bincount(a, minlength=N))
            _, O_t, _ = f(lw, 5, prec=1)
            n, bad = cumulative_mismatches(kind, sch, lw, O_k, O_t, seed=5,
                                           oracle_is_sequential=False)
            assert bad == 0, (sch, n, bad)
            dev, bound = truth_offset(kind, sch, lw, O_k, seed=5)
            assert dev <= bound, (sch, dev, bound)
            st, c = _run(rs, hh, sch, lw, seed=5, prec=prec, permute=True)
            o = np.bincount(a, minlength=N)
            assert np.all(c[o > 0] == np.nonzero(o > 0)[0])
            assert np.array_equal(np.sort(c), a)
        st, a = _run(rs, hh, rs.MULTINOMIAL, lw, seed=5, prec=prec)
        assert st == rs.RS_OK
        _check_valid_ancestry(a, lw, False)
        _, want = oracle.multinomial(lw, 5, prec=1)
        n, bad = multinomial_mismatches(kind, lw, a, want, seed=5, oracle_is_sequential=False)
        assert bad == 0


def test_f64_decisions_on_binary32_pipes_edge_cases(rs, h):
    """The binary64 Metropolis / rejection kernels decide on the binary32 pipes and fall back
    to exact binary64 evaluation inside the uncertainty band; inputs that force every branch
    (magnitudes where the bound is too loose, values outside the binary32 range, subnormals,
    signed zeros, near-equal log-weights) must still match the oracle bit for bit."""
    rng = np.random.default_rng(12)
    N = 5000
    cases = {
        "huge": -1e5 + rng.normal(0, 3, N),
        "outside_f32": np.where(rng.random(N) < 0.3, -1e39, rng.normal(-3, 1, N)),
        "subnormal": np.where(rng.random(N) < 0.5, 1e-310, -rng.exponential(1.0, N)),
        "signed_zero": np.where(rng.random(N) < 0.5, 0.0, -0.0),
        "near_equal": -2.0 + rng.integers(-3, 4, N) * 2.0 ** -40,
        "tiny_ratio": np.where(rng.random(N) < 0.5, 0.0, -80.0 - rng.random(N) * 20),
        "mixed_inf": np.where(rng.random(N) < 0.2, -np.inf, rng.normal(-1, 2, N)),
    }
    for name, lw in cases.items():
        lw = np.ascontiguousarray(lw, dtype=np.float64)
        st, a = _run(rs, h, rs.METROPOLIS, lw, B=24, seed=77)
        assert st == rs.RS_OK, name
        assert np.array_equal(a, oracle.metropolis(lw, 24, seed=77)[1]), name
        lwr = lw - max(0.0, float(lw.max()))  # keep the rejection bound log w_max = 0 valid
        st, a = _run(rs, h, rs.REJECTION, lwr, seed=78, log_wmax=0.0, max_trials=4096)
        ost, want = oracle.rejection(lwr, 0.0, seed=78, max_trials=4096)
        assert st == (rs.RS_OK if ost == oracle.OK else rs.RS_ERR_REJECTION_CAP), name
        assert np.array_equal(a, want), name


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_log_normaliser_uses_true_maximum(rs, h, dtype):
    """All log-weights negative and far from 0: the maximum used for renormalisation must be
    the true maximum (the first weight of a maximal particle is exactly 1)."""
    lw = np.array([-7.25, -3.5, -9.0, -3.5, -100.0], dtype=dtype)
    t = torch.from_numpy(lw).to(DEV)
    for prec in ([0, 1] if dtype == np.float32 else [0, 2]):
        W, lt = rs.rs_cumulative_weights(h, t, prec=prec)
        assert rs.rs_last_error(h) == rs.RS_OK
        W = W.cpu().numpy().astype(np.float64)
        assert W[1] - W[0] == pytest.approx(1.0, rel=1e-6)
        tol = 1e-12 if dtype == np.float64 else 1e-6
        assert lt.item() == pytest.approx(np.log(np.sum(np.exp(lw.astype(np.float64)))), rel=tol)


def test_argument_checks_on_the_device_path(rs, h):
    """Empty input, capacity, unknown scheme / precision and aliasing are refused on the host
    (RsError), before any kernel runs; the handle stays usable."""
    lw = torch.zeros(8, dtype=torch.float32, device=DEV)
    out = torch.empty(8, dtype=torch.int32, device=DEV)
    with pytest.raises(rs.RsError) as e:
        rs.rs_resample(h, rs.SYSTEMATIC, lw[:0], out=out[:0])
    assert e.value.status == rs.RS_ERR_ARG
    with rs.Handle(4) as small:
        with pytest.raises(rs.RsError) as e:
            rs.rs_resample(small, rs.SYSTEMATIC, lw, out=out)
        assert e.value.status == rs.RS_ERR_CAPACITY
    with pytest.raises(rs.RsError):
        rs.rs_resample(h, 5, lw, out=out)
    with pytest.raises(rs.RsError):
        rs.rs_resample(h, rs.SYSTEMATIC, lw, out=out, prec=rs.PREC_BINARY64)  # binary32 input
    with pytest.raises(rs.RsError):
        rs.rs_resample(h, rs.METROPOLIS, lw, B=-1, out=out)
    with pytest.raises(rs.RsError):
        rs.rs_permute(h, out, out)
    a = rs.rs_resample(h, rs.SYSTEMATIC, lw, out=out)
    assert rs.rs_last_error(h) == rs.RS_OK
    assert a.cpu().tolist() == list(range(8))


def test_binding_refuses_short_output_buffers(rs, h):
    """The binding checks every caller buffer's length against what the kernels write before
    calling the library: a short buffer raises ValueError and nothing is launched."""
    lw = torch.zeros(64, dtype=torch.float32, device=DEV)
    short = torch.empty(63, dtype=torch.int32, device=DEV)
    with pytest.raises(ValueError):
        rs.rs_resample(h, rs.SYSTEMATIC, lw, out=short)
    with pytest.raises(ValueError):
        rs.rs_resample_prc(h, lw, -1.0, out=short)
    with pytest.raises(ValueError):
        rs.rs_offspring(h, torch.zeros(64, dtype=torch.int32, device=DEV), short)
    with pytest.raises(ValueError):
        rs.rs_permute(h, torch.zeros(64, dtype=torch.int32, device=DEV), short)
    with pytest.raises(ValueError):
        rs.rs_cumulative_weights(h, lw, W=torch.empty(63, dtype=torch.float32, device=DEV))
    with pytest.raises(ValueError):
        rs.rs_ess(h, lw, out=torch.empty(0, dtype=torch.float64, device=DEV))
    offs = torch.tensor([0, 32, 64], dtype=torch.int64, device=DEV)
    with pytest.raises(ValueError):
        rs.rs_resample_batched(h, rs.SYSTEMATIC, lw, offs, out=short)
    with pytest.raises(ValueError):
        rs.rs_log_sum_weights_batched(h, lw, offs,
                                      out=torch.empty(1, dtype=torch.float64, device=DEV))
    a = rs.rs_resample(h, rs.SYSTEMATIC, lw)
    assert rs.rs_last_error(h) == rs.RS_OK
    assert a.cpu().tolist() == list(range(64))


def test_convenience_resample_matches_the_handle_call(rs, h):
    lw = torch.from_numpy(workload.synthetic_logw(70001, 2.0, seed=5)).to(DEV)
    for name in ("multinomial", "stratified", "systematic", "metropolis", "rejection"):
        a = rs.resample(lw, name, B=16, seed=3, step=2)
        b = rs.rs_resample(h, rs.SCHEMES[name], lw, B=16, seed=3, step=2, permute=True)
        assert rs.rs_last_error(h) == rs.RS_OK
        assert torch.equal(a, b), name
    bigger = torch.from_numpy(workload.synthetic_logw(3 << 20, 1.0, seed=6)).to(DEV)
    assert rs.resample(bigger, "systematic").numel() == 3 << 20  # the cached handle grows
    bad = torch.tensor([0.0, float("nan")], dtype=torch.float64, device=DEV)
    with pytest.raises(rs.RsError):
        rs.resample(bad, "metropolis", B=4)


def test_philox_throughput_kernel_draws_the_oracle_blocks(rs, h):
    """The measurement kernel behind the Philox roofline runs the resamplers' Philox: the XOR
    of the words of blocks (i, n, 0, 6), i < T, n < J, equals the oracle's."""
    T, J, seed = 1000, 7, 99
    got = rs.rs_philox_throughput(h, T, J, seed=seed).item() & 0xFFFFFFFF
    want = 0
    for i in range(T):
        for n in range(J):
            x = oracle.draw(seed, i, n, 0, 0, 6)
            want ^= int(x[0]) ^ int(x[1]) ^ int(x[2]) ^ int(x[3])
    assert got == want
    with pytest.raises(rs.RsError):
        rs.rs_philox_throughput(h, 0, 1)
    with pytest.raises(rs.RsError):
        rs.rs_philox_throughput(h, 10, 0)


@pytest.mark.parametrize("N", [1, 2, 7, 8, 9, 255, 257, 2**18 - 1, 2**18, 2**18 + 7])
def test_sorted_permute_from_claimed_bits(rs, h, N):
    """The fused stratified/systematic path permutes from one claimed bit per particle and
    follows Code 10's walks from their ends; its output must be Code 10's (oracle.permute of
    the same call's unpermuted ancestors) on degenerate weights too: one particle carrying all
    the weight (first, middle, last), two particles, equal weights, zero weights everywhere
    (every slot then keeps itself), and weights that leave most particles without offspring.
    Sizes on both sides of the four-slots-per-thread threshold and ragged byte tails."""
    rng = np.random.default_rng(1000 + N)
    cases = {"equal": np.zeros(N)}
    for name, k in (("first", 0), ("middle", N // 2), ("last", N - 1)):
        lw = np.full(N, -np.inf)
        lw[k] = -3.0
        cases["one_" + name] = lw
    if N >= 2:
        lw = np.full(N, -np.inf)
        lw[[0, N - 1]] = [-1.0, 0.0]
        cases["two"] = lw
    cases["skewed"] = np.where(rng.random(N) < 0.05, rng.normal(0.0, 1.0, N), -40.0)
    cases["spread"] = rng.normal(0.0, 3.0, N)
    for dtype in (np.float32, np.float64):
        for sch in (rs.SYSTEMATIC, rs.STRATIFIED):
            for name, lw in cases.items():
                x = lw.astype(dtype)
                st0, a = _run(rs, h, sch, x, seed=17, step=N % 5)
                st1, c = _run(rs, h, sch, x, seed=17, step=N % 5, permute=True)
                assert st0 == st1 == rs.RS_OK, (name, st0, st1)
                assert np.all(np.diff(a) >= 0), name
                assert np.array_equal(c, oracle.permute(a)), (name, dtype, sch)
            zero = np.full(N, -np.inf, dtype)
            st, c = _run(rs, h, sch, zero, seed=1, permute=True)
            assert st == rs.RS_ERR_ZERO_WEIGHT
            assert np.array_equal(c, np.arange(N))
    assert rs.rs_last_error(h) == rs.RS_OK
