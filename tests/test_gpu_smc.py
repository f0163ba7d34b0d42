"""GPU tests of the full SMC loop (Code 1) around the resampler: the in-place copy by a permuted
ancestry equals the gather x[c]; the linear-Gaussian propagate-and-weight kernel equals its
formula evaluated on the host from the oracle's Philox words; and the bootstrap filter's log
marginal likelihood agrees with the Kalman filter's closed form (oracle/kalman.py) within
4 seed-to-seed standard deviations, for the systematic, Metropolis and rejection resamplers."""
import math

import numpy as np
import pytest
import torch

import oracle
import workload
from oracle import kalman

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
PHI, SX, SY = workload.LGSSM_PHI, workload.LGSSM_SIGMA_X, workload.LGSSM_SIGMA_Y


@pytest.fixture(scope="module")
def h(rs):
    handle = rs.Handle(1 << 20)
    yield handle
    handle.close()


@pytest.mark.parametrize("scheme", [2, 3, 0])
@pytest.mark.parametrize("D", [1, 3])
def test_copy_in_place_equals_gather(rs, h, scheme, D):
    N = 50003
    lw = torch.from_numpy(workload.synthetic_logw(N, 2.5, seed=4, dtype=np.float32)).to(DEV)
    c = rs.rs_resample(h, scheme, lw, B=32, seed=9, permute=True)
    rng = np.random.default_rng(D)
    x0 = rng.standard_normal((N, D)).astype(np.float32)
    x = torch.from_numpy(x0.copy() if D > 1 else x0[:, 0].copy()).to(DEV)
    rs.rs_copy_ancestors(h, x, c)
    assert rs.rs_last_error(h) == rs.RS_OK
    want = x0[c.cpu().numpy()]
    got = x.cpu().numpy().reshape(N, D)
    assert np.array_equal(got, want)


def test_copy_rejects_an_ancestry_without_the_predicate(rs, h):
    N = 1000
    c = torch.arange(N - 1, -1, -1, dtype=torch.int32, device=DEV)  # c[c_i] != c_i mostly
    x = torch.arange(N, dtype=torch.float32, device=DEV)
    rs.rs_copy_ancestors(h, x, c)
    assert rs.rs_last_error(h) == rs.RS_ERR_ARG


def _normal_host(seed, i, step, filt=0):
    w = oracle.draw(seed, int(i), 0, step, filt, 5)
    u1 = 1.0 - float(int(w[0]) >> 8) * 2.0 ** -24
    u2 = float(int(w[1]) >> 8) * 2.0 ** -24
    return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def test_lgssm_step_matches_host_formula(rs, h):
    N = 4099
    x = torch.empty(N, dtype=torch.float32, device=DEV)
    logw = rs.rs_lgssm_step(h, x, True, PHI, SX, 0.7, SY, seed=3, step=0)
    x0 = x.cpu().numpy().astype(np.float64)
    s0 = SX / math.sqrt(1 - PHI * PHI)
    idx = np.arange(0, N, 37)
    want0 = np.array([s0 * _normal_host(3, i, 0) for i in idx])
    assert np.allclose(x0[idx], want0, rtol=2e-6, atol=2e-6)
    assert np.allclose(logw.cpu().numpy()[idx], -(0.7 - x0[idx]) ** 2 / (2 * SY * SY),
                       rtol=1e-5, atol=1e-6)
    logw = rs.rs_lgssm_step(h, x, False, PHI, SX, -1.3, SY, seed=3, step=5)
    x1 = x.cpu().numpy().astype(np.float64)
    want1 = np.array([PHI * x0[i] + SX * _normal_host(3, i, 5) for i in idx])
    assert np.allclose(x1[idx], want1, rtol=2e-6, atol=4e-6)
    assert rs.rs_last_error(h) == rs.RS_OK


@pytest.mark.parametrize("scheme", [2, 3, 4])
def test_bootstrap_loglik_matches_kalman(rs, h, scheme):
    from paper_1301_4019_gb300 import smc
    T, N = 100, 1 << 16
    _, y = workload.lgssm_simulate(T, PHI, SX, SY, seed=21)
    want = kalman.lgssm_loglik(y, PHI, SX, SY)
    lls = [smc.lgssm_bootstrap(h, y, N, scheme, PHI, SX, SY, seed=s, B=64) for s in range(16)]
    assert rs.rs_last_error(h) == rs.RS_OK
    lls = np.array(lls)
    sd = lls.std(ddof=1)
    assert sd < 0.5
    assert abs(lls.mean() - want) < 4 * sd, (lls.mean(), want, sd)
    # the full-size filter (N = 2^20): its own spread is a quarter of the 2^16 one
    ll = smc.lgssm_bootstrap(h, y, 1 << 20, scheme, PHI, SX, SY, seed=99, B=64)
    assert abs(ll - want) < 4 * sd / 4 + 0.02, (ll, want, sd)


def test_ess_matches_host(rs, h):
    for dtype in (np.float32, np.float64):
        for N, y in ((1, 0.0), (1000, 2.0), (300007, 3.5)):
            lw = workload.synthetic_logw(N, y, seed=N, dtype=dtype)
            if N > 10:
                lw[::7] = -np.inf
            lt = torch.empty(1, dtype=torch.float64, device=DEV)
            e = rs.rs_ess(h, torch.from_numpy(lw).to(DEV), log_total=lt).item()
            assert rs.rs_last_error(h) == rs.RS_OK
            m = float(lw.max())
            w = np.exp(lw.astype(np.float64) - m)
            want = w.sum() ** 2 / (w * w).sum()
            assert abs(e - want) <= 1e-5 * want, (dtype, N, e, want)
            want_lt = m + math.log(math.fsum(w))
            assert abs(lt.item() - want_lt) <= 2e-7 * max(1.0, abs(want_lt)), (lt.item(), want_lt)
    z = torch.full((100,), -np.inf, dtype=torch.float32, device=DEV)
    lt = torch.empty(1, dtype=torch.float64, device=DEV)
    assert rs.rs_ess(h, z, log_total=lt).item() == 0.0
    assert lt.item() == -np.inf
    assert rs.rs_last_error(h) == rs.RS_ERR_ZERO_WEIGHT


@pytest.mark.parametrize("scheme", [2, 4])
def test_adaptive_filter_matches_kalman(rs, h, scheme):
    """Resampling on demand (ESS < N/2): the log-likelihood still agrees with the Kalman
    filter within 4 seed-to-seed standard deviations, with fewer resamplings than steps."""
    from paper_1301_4019_gb300 import smc
    T, N = 100, 1 << 16
    _, y = workload.lgssm_simulate(T, PHI, SX, SY, seed=21)
    want = kalman.lgssm_loglik(y, PHI, SX, SY)
    runs = [smc.lgssm_adaptive(h, y, N, scheme, PHI, SX, SY, 0.5, seed=s) for s in range(16)]
    assert rs.rs_last_error(h) == rs.RS_OK
    lls = np.array([r[0] for r in runs])
    n_res = [r[1] for r in runs]
    assert 0 < min(n_res) and max(n_res) < T - 1
    sd = lls.std(ddof=1)
    assert abs(lls.mean() - want) < 4 * sd, (lls.mean(), want, sd, n_res)


@pytest.mark.parametrize("scheme", [2, 4])
def test_adaptive_graph_equals_host_decisions(rs, h, scheme):
    """The adaptive filter captured as one CUDA graph (conditional nodes decide on the device)
    takes the same resampling decisions as the host-driven loop and computes the same
    particles, weights and log-likelihood, bit for bit, on every replay."""
    from paper_1301_4019_gb300 import smc
    T, N = 60, 1 << 16
    _, y = workload.lgssm_simulate(T, PHI, SX, SY, seed=23)
    ll_host, n_host = smc.lgssm_adaptive(h, y, N, scheme, PHI, SX, SY, 0.5, seed=8)
    assert rs.rs_last_error(h) == rs.RS_OK
    g = smc.AdaptiveGraph(h, y, N, scheme, PHI, SX, SY, 0.5, seed=8)
    for _ in range(3):
        g.replay()
        ll, n = g.result()
        assert rs.rs_last_error(h) == rs.RS_OK
        assert n == n_host and 0 < n < T - 1
        assert ll == ll_host, (ll, ll_host)
    # the graph's particles equal a host-driven run's
    b = smc.LgssmBuffers(N, T)
    ess = torch.empty(1, dtype=torch.float64, device=DEV)
    resample = False
    for t in range(T):
        if resample:
            rs.rs_resample(h, scheme, b.logw, B=64, seed=8, step=t, out=b.c, permute=True,
                           prec=rs.PREC_COMPENSATED, log_wmax=0.0)
            rs.rs_copy_ancestors(h, b.x, b.c)
        rs.rs_lgssm_step(h, b.x, t == 0, PHI, SX, float(y[t]), SY, seed=8, step=t, logw=b.logw,
                         accumulate=(t > 0 and not resample))
        resample = rs.rs_ess(h, b.logw, out=ess).item() < 0.5 * N
    assert torch.equal(g.b.x, b.x) and torch.equal(g.b.logw, b.logw)


def test_capture_if_below_needs_a_capturing_stream(rs, h):
    v = torch.zeros(1, dtype=torch.float64, device=DEV)
    with pytest.raises(rs.RsError):
        rs.rs_capture_if_below(h, v, 1.0)
    with pytest.raises(rs.RsError):
        rs.rs_capture_end_if(h)


# ---------------------------------------------------------------------------------------
# many filters at once (the CSR layout of rs_resample_batched)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("scheme", [2, 3, 4])
def test_batched_filter_equals_single_filters(rs, h, scheme):
    """Every state of filter f of the batched loop (particles, log-weights) equals the
    single-filter loop run on its own with filter = f, bit for bit; the per-filter log-sums
    agree with the single filter's scan-based totals to rounding."""
    from paper_1301_4019_gb300 import smc
    T = 8
    sizes = [1000, 4097, 1, 70001, 12289, 2]
    if scheme == 4:  # a filter of one or two particles can leave rejection with a tiny
        sizes = [1000, 4097, 70001, 12289, 300]  # acceptance probability: its cap is legal
    F = len(sizes)
    Y = np.stack([workload.lgssm_simulate(T, PHI, SX, SY, seed=40 + f)[1] for f in range(F)],
                 axis=1)
    b = smc.BatchedLgssmBuffers(sizes, Y)
    smc.lgssm_batched_launch(h, b, scheme, PHI, SX, SY, seed=6, B=16)
    assert rs.rs_last_error(h) == rs.RS_OK
    x_b, lw_b = b.x.cpu().numpy(), b.logw.cpu().numpy()
    lt_b = b.log_total.cpu().numpy()
    off = np.concatenate([[0], np.cumsum(sizes)])
    for f, N in enumerate(sizes):
        s = smc.lgssm_bootstrap_launch(h, Y[:, f], N, scheme, PHI, SX, SY, seed=6, B=16,
                                       filter=f)
        assert rs.rs_last_error(h) == rs.RS_OK
        assert np.array_equal(s.x.cpu().numpy(), x_b[off[f]:off[f + 1]]), f
        assert np.array_equal(s.logw.cpu().numpy(), lw_b[off[f]:off[f + 1]]), f
        assert np.allclose(s.log_total.cpu().numpy(), lt_b[:, f], rtol=0, atol=2e-5), f


def test_log_sum_batched_matches_host(rs, h):
    rng = np.random.default_rng(3)
    sizes = [5, 0, 1, 1 << 15, 3000, 70001, 4]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    for dtype in (np.float32, np.float64):
        lw = (rng.standard_normal(off[-1]) * 4 - 30).astype(dtype)
        lw[off[2]:off[3]] = -np.inf           # an all-zero filter of one particle
        lw[off[4]:off[4] + 100] = -np.inf     # zero weights inside a filter
        out = rs.rs_log_sum_weights_batched(h, torch.from_numpy(lw).to(DEV),
                                            torch.from_numpy(off).to(DEV)).cpu().numpy()
        assert rs.rs_last_error(h) == rs.RS_OK
        for f in range(len(sizes)):
            seg = lw[off[f]:off[f + 1]].astype(np.float64)
            if seg.size == 0 or np.all(seg == -np.inf):
                assert out[f] == -np.inf, f
                continue
            m = seg.max()
            want = m + math.log(math.fsum(np.exp(seg - m)))
            tol = 4e-7 if dtype == np.float32 else 1e-12
            assert abs(out[f] - want) <= tol * max(1.0, abs(want)), (dtype, f, out[f], want)
    bad = torch.tensor([0.0, float("nan")], dtype=torch.float32, device=DEV)
    rs.rs_log_sum_weights_batched(h, bad, torch.tensor([0, 2], dtype=torch.int64, device=DEV))
    assert rs.rs_last_error(h) == rs.RS_ERR_NONFINITE


def test_ess_batched_matches_host(rs, h):
    """rs_ess_batched: every filter's ESS within 1e-5 of the host's binary64 value, the log
    totals bit-equal to rs_log_sum_weights_batched (same sums), 0 / -inf for empty and
    all-zero filters, 1 for a single particle, and equal to rs_ess on the filter's slice."""
    rng = np.random.default_rng(11)
    sizes = [5, 0, 1, 1 << 15, 3000, 70001, 4, 1]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    offs = torch.from_numpy(off).to(DEV)
    for dtype in (np.float32, np.float64):
        lw = (rng.standard_normal(off[-1]) * 2 - 30).astype(dtype)
        lw[off[2]:off[3]] = -np.inf           # an all-zero filter of one particle
        lw[off[4]:off[4] + 100] = -np.inf     # zero weights inside a filter
        t = torch.from_numpy(lw).to(DEV)
        lt = torch.empty(len(sizes), dtype=torch.float64, device=DEV)
        ess = rs.rs_ess_batched(h, t, offs, log_total=lt).cpu().numpy()
        assert rs.rs_last_error(h) == rs.RS_OK
        ls = rs.rs_log_sum_weights_batched(h, t, offs).cpu().numpy()
        assert np.array_equal(lt.cpu().numpy(), ls)
        only = rs.rs_ess_batched(h, t, offs).cpu().numpy()  # without the log totals
        assert np.array_equal(only, ess)
        for f in range(len(sizes)):
            seg = lw[off[f]:off[f + 1]].astype(np.float64)
            if seg.size == 0 or np.all(seg == -np.inf):
                assert ess[f] == 0.0, f
                continue
            w = np.exp(seg - seg.max())
            want = math.fsum(w) ** 2 / math.fsum(w * w)
            assert abs(ess[f] - want) <= 1e-5 * want, (dtype, f, ess[f], want)
            if seg.size == 1:
                assert ess[f] == 1.0
            if seg.size > 1000:
                one = rs.rs_ess(h, t[off[f]:off[f + 1]]).item()
                assert abs(one - ess[f]) <= 2e-5 * want, (dtype, f, one, ess[f])
    # neither output: refused on the host before any launch
    st = rs.load().rs_ess_batched(h.ptr, rs._dtype_code(t), rs._dev(t, None, "logw"),
                                  rs._dev(offs, torch.int64, "offsets"), len(sizes), None,
                                  None, 0.5, None, None)
    assert st == rs.RS_ERR_ARG
    bad = torch.tensor([0.0, float("nan")], dtype=torch.float32, device=DEV)
    rs.rs_ess_batched(h, bad, torch.tensor([0, 2], dtype=torch.int64, device=DEV))
    assert rs.rs_last_error(h) == rs.RS_ERR_NONFINITE


def test_batched_loglik_matches_kalman(rs, h):
    """32 independent filters of N = 2^14 on the same observations: their log-likelihood
    estimates centre on the Kalman filter's value (4 standard errors of the mean)."""
    from paper_1301_4019_gb300 import smc
    T, F, N = 100, 32, 1 << 14
    _, y = workload.lgssm_simulate(T, PHI, SX, SY, seed=21)
    want = kalman.lgssm_loglik(y, PHI, SX, SY)
    b = smc.BatchedLgssmBuffers([N] * F, np.repeat(y[:, None], F, axis=1))
    smc.lgssm_batched_launch(h, b, 2, PHI, SX, SY, seed=12)
    lls = smc.lgssm_batched_loglik_from(b, SY)
    assert rs.rs_last_error(h) == rs.RS_OK
    sd = lls.std(ddof=1)
    assert sd < 1.0
    assert abs(lls.mean() - want) < 4 * sd / math.sqrt(F), (lls.mean(), want, sd)


@pytest.mark.parametrize("scheme", [0, 2, 3, 4])
@pytest.mark.parametrize("permute", [False, True])
def test_masked_batched_resample(rs, h, scheme, permute):
    """rs_resample_batched_masked: flagged filters get exactly the ancestors of the unmasked
    call, the others the identity; all flags set gives the unmasked call bit for bit."""
    sizes = np.array([1, 300, 4097, 0, 9000, 2, 1024, 70001], np.int64)
    off, lw, _ = workload.ragged_logw(sizes, seed=31, dtype=np.float32)
    t = torch.from_numpy(lw).to(DEV)
    offs = torch.from_numpy(off).to(DEV)
    kw = dict(B=9, seed=5, step=3, permute=permute, log_wmax=0.0)
    full = rs.rs_resample_batched(h, scheme, t, offs, **kw).cpu().numpy()
    flags = np.array([1, 0, 1, 1, 0, 1, 0, 1], np.uint8)
    got = rs.rs_resample_batched(h, scheme, t, offs, resample=torch.from_numpy(flags).to(DEV),
                                 **kw).cpu().numpy()
    ones = rs.rs_resample_batched(h, scheme, t, offs, resample=torch.ones(len(sizes),
                                  dtype=torch.uint8, device=DEV), **kw).cpu().numpy()
    assert rs.rs_last_error(h) == rs.RS_OK
    assert np.array_equal(ones, full)
    for f in range(len(sizes)):
        lo, hi = off[f], off[f + 1]
        want = full[lo:hi] if flags[f] else np.arange(hi - lo, dtype=np.int32)
        assert np.array_equal(got[lo:hi], want), (f, flags[f])


def test_ess_flags_and_weight_reset(rs, h):
    """rs_ess_batched's below flags are ESS_f < threshold * N_f (0 for empty and all-zero
    filters); rs_reset_weights_batched zeroes exactly the flagged filters' log-weights."""
    sizes = np.array([5, 0, 3000, 1, 70001, 300], np.int64)
    off, lw, _ = workload.ragged_logw(sizes, seed=8, dtype=np.float32)
    lw[off[3]:off[4]] = -np.inf
    t = torch.from_numpy(lw).to(DEV)
    offs = torch.from_numpy(off).to(DEV)
    below = torch.empty(len(sizes), dtype=torch.uint8, device=DEV)
    ess = rs.rs_ess_batched(h, t, offs, threshold=0.5, below=below).cpu().numpy()
    assert rs.rs_last_error(h) == rs.RS_OK
    fl = below.cpu().numpy()
    want = (ess < 0.5 * sizes) & (ess > 0)
    assert np.array_equal(fl.astype(bool), want), (fl, ess)
    assert fl.any() and not fl.all()
    rs.rs_reset_weights_batched(h, t, offs, below)
    assert rs.rs_last_error(h) == rs.RS_OK
    after = t.cpu().numpy()
    for f in range(len(sizes)):
        lo, hi = off[f], off[f + 1]
        if fl[f]:
            assert np.all(after[lo:hi] == 0.0)
        else:
            assert np.array_equal(after[lo:hi], lw[lo:hi])
    with pytest.raises(rs.RsError):
        rs.rs_ess_batched(h, t, offs, threshold=1.5, below=below)


@pytest.mark.parametrize("scheme", [2, 4])
def test_batched_adaptive_loglik_matches_kalman(rs, h, scheme):
    """32 adaptive filters of N = 2^14 (each resampling when its own ESS < N/2, decided on the
    device): log-likelihoods centred on Kalman within 4 standard errors, fewer resamplings
    than steps, and with threshold 1 (always below) the filters equal the resample-every-step
    batched loop bit for bit."""
    from paper_1301_4019_gb300 import smc
    T, F, N = 100, 32, 1 << 14
    _, y = workload.lgssm_simulate(T, PHI, SX, SY, seed=21)
    want = kalman.lgssm_loglik(y, PHI, SX, SY)
    Y = np.repeat(y[:, None], F, axis=1)
    b = smc.BatchedLgssmBuffers([N] * F, Y)
    flags = smc.lgssm_batched_adaptive_launch(h, b, scheme, PHI, SX, SY, threshold=0.5,
                                              seed=12)
    lls = smc.lgssm_batched_adaptive_loglik_from(b, flags, SY)
    assert rs.rs_last_error(h) == rs.RS_OK
    n_res = flags[1:].sum(dim=0).cpu().numpy()
    assert np.all(n_res < T - 1) and np.all(n_res > 0)
    sd = lls.std(ddof=1)
    assert sd < 1.0
    assert abs(lls.mean() - want) < 4 * sd / math.sqrt(F), (lls.mean(), want, sd)
    # threshold 1: every filter resamples at every step (ESS < N unless all weights equal)
    a = smc.BatchedLgssmBuffers([N] * 4, Y[:, :4])
    fa = smc.lgssm_batched_adaptive_launch(h, a, scheme, PHI, SX, SY, threshold=1.0, seed=3)
    e = smc.BatchedLgssmBuffers([N] * 4, Y[:, :4])
    smc.lgssm_batched_launch(h, e, scheme, PHI, SX, SY, seed=3)
    assert rs.rs_last_error(h) == rs.RS_OK
    assert bool(fa.all())
    assert torch.equal(a.x, e.x) and torch.equal(a.log_total, e.log_total)
