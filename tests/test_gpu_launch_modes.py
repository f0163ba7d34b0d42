"""GPU tests of the two launch structures of the scan-based resamplers: one cooperative kernel
with grid barriers (LAUNCH_FUSED) and one kernel per pass (LAUNCH_SEPARATE) must give the same
ancestors bit for bit and the same device status, for every accumulation mode, with and
without Permute, at sizes spanning one tile, several tiles with a ragged tail and more tiles
than the fused grid has CTAs. Each mode is also checked
against the oracle in test_gpu_parity.py (the default mode runs the fused kernel there)."""
import numpy as np
import pytest
import torch

import oracle
import workload
from parity_tools import cumulative_mismatches, truth_offset

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
KINDS = [("f32", np.float32, 0), ("f32c", np.float32, 1), ("f64", np.float64, 0),
         ("f64n", np.float64, 2)]


@pytest.fixture(scope="module")
def h(rs):
    handle = rs.Handle((1 << 22) + 4099)
    yield handle
    handle.close()


def _both(rs, h, scheme, t, **kw):
    out = []
    for mode in (rs.LAUNCH_FUSED, rs.LAUNCH_SEPARATE):
        rs.rs_set_launch_mode(h, mode)
        a = rs.rs_resample(h, scheme, t, **kw)
        out.append((rs.rs_last_error(h), a.cpu().numpy()))
    rs.rs_set_launch_mode(h, rs.LAUNCH_AUTO)
    return out


@pytest.mark.parametrize("kind,dtype,prec", KINDS)
@pytest.mark.parametrize("N", [1, 2, 5, 4095, 4097, 70001, 1310723])
def test_fused_equals_separate(rs, h, kind, dtype, prec, N):
    lw = workload.synthetic_logw(N, 3.0, seed=N, dtype=dtype)
    if N > 10:
        lw[N // 5] = -np.inf
        lw[-3:] = -np.inf
    t = torch.from_numpy(lw).to(DEV)
    for scheme in (rs.MULTINOMIAL, rs.STRATIFIED, rs.SYSTEMATIC):
        for permute in (False, True):
            (s1, a1), (s2, a2) = _both(rs, h, scheme, t, seed=17, step=3, prec=prec,
                                       permute=permute)
            assert s1 == s2 == rs.RS_OK
            assert np.array_equal(a1, a2), (scheme, permute)


def test_fused_equals_separate_large_and_misaligned(rs, h):
    """Sizes with more tiles than the fused grid has CTAs, a ragged tail, and a log-weight
    pointer that is not 16-byte aligned; the systematic result of the default mode is also
    checked against the oracle's double-double cumulative offspring."""
    for N in (1 << 22, (1 << 22) + 4097):
        lw = workload.synthetic_logw(N + 1, 1.0, seed=5, dtype=np.float32)
        base = torch.from_numpy(lw).to(DEV)
        view = base[1:]
        assert view.data_ptr() % 16 != 0
        for scheme in (rs.MULTINOMIAL, rs.SYSTEMATIC):
            (s1, a1), (s2, a2) = _both(rs, h, scheme, view, seed=2, permute=True)
            assert s1 == s2 == rs.RS_OK
            assert np.array_equal(a1, a2)
        rs.rs_set_launch_mode(h, rs.LAUNCH_AUTO)
        a = rs.rs_resample(h, rs.SYSTEMATIC, view, seed=2).cpu().numpy()
        assert rs.rs_last_error(h) == rs.RS_OK
        O_k = np.cumsum(np.bincount(a, minlength=N))
        _, O_t, _ = oracle.systematic(lw[1:], 2, prec=1)
        n, bad = cumulative_mismatches("f32", rs.SYSTEMATIC, lw[1:], O_k, O_t, seed=2,
                                       oracle_is_sequential=False)
        assert bad == 0, (N, n, bad)
        dev, bound = truth_offset("f32", rs.SYSTEMATIC, lw[1:], O_k, seed=2)
        assert dev <= bound, (N, dev, bound)


def test_fused_statuses_match_separate(rs, h):
    """NaN / +inf log-weights and all-zero weights are flagged alike by both structures, and
    all-zero weights give the identity ancestry in both."""
    for dtype in (np.float32, np.float64):
        for case in ("nan", "inf", "zero"):
            N = 9000
            lw = workload.synthetic_logw(N, 0.0, seed=1, dtype=dtype)
            if case == "nan":
                lw[4321] = np.nan
            elif case == "inf":
                lw[17] = np.inf
            else:
                lw[:] = -np.inf
            t = torch.from_numpy(lw).to(DEV)
            for scheme in (rs.MULTINOMIAL, rs.STRATIFIED, rs.SYSTEMATIC):
                (s1, a1), (s2, a2) = _both(rs, h, scheme, t, seed=1, permute=True)
                assert s1 == s2 and s1 != rs.RS_OK, (case, scheme)
                assert a1.min() >= 0 and a1.max() < N
                if case == "zero":
                    assert np.array_equal(a1, np.arange(N)) and np.array_equal(a2, a1)


def test_fused_repeated_calls_and_graph_replay(rs, h):
    """The barrier state resets itself: many back-to-back fused calls, and a CUDA graph of
    fused calls replayed several times, all give the first call's result."""
    N = 300007
    lw = torch.from_numpy(workload.synthetic_logw(N, 2.0, seed=9, dtype=np.float32)).to(DEV)
    rs.rs_set_launch_mode(h, rs.LAUNCH_FUSED)
    try:
        want = rs.rs_resample(h, rs.SYSTEMATIC, lw, seed=4, permute=True).clone()
        for _ in range(50):
            a = rs.rs_resample(h, rs.SYSTEMATIC, lw, seed=4, permute=True)
        assert rs.rs_last_error(h) == rs.RS_OK
        assert torch.equal(a, want)
        out = torch.empty(N, dtype=torch.int32, device=DEV)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            rs.rs_resample(h, rs.SYSTEMATIC, lw, seed=4, permute=True, out=out, stream=s)
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=s):
                rs.rs_resample(h, rs.SYSTEMATIC, lw, seed=4, permute=True, out=out, stream=s)
        for _ in range(5):
            out.zero_()
            g.replay()
            torch.cuda.synchronize()
            assert torch.equal(out, want)
        assert rs.rs_last_error(h) == rs.RS_OK
    finally:
        rs.rs_set_launch_mode(h, rs.LAUNCH_AUTO)


def test_launch_mode_argument_checked(rs, h):
    with pytest.raises(rs.RsError):
        rs.rs_set_launch_mode(h, 3)


@pytest.mark.parametrize("N", [1, 1000, 70001, 1310723])
def test_mcmc_and_conversions_equal_across_launch_modes(rs, h, N):
    """Metropolis and rejection (rejection's claim initialisation runs inside one cooperative
    launch by default) and the offspring / integer-scan conversions (the scan is one
    cooperative launch by default) equal their one-kernel-per-step forms bit for bit."""
    for dtype in (np.float32, np.float64):
        t = torch.from_numpy(workload.synthetic_logw(N, 2.5, seed=N + 1, dtype=dtype)).to(DEV)
        for scheme in (rs.METROPOLIS, rs.REJECTION):
            for permute in (False, True):
                (s1, a1), (s2, a2) = _both(rs, h, scheme, t, B=12, seed=5, step=2,
                                           permute=permute, log_wmax=0.0)
                assert s1 == s2 == rs.RS_OK
                assert np.array_equal(a1, a2), (dtype, scheme, permute)
    a = rs.rs_resample(h, rs.MULTINOMIAL, t, seed=3)
    res = []
    for mode in (rs.LAUNCH_FUSED, rs.LAUNCH_SEPARATE):
        rs.rs_set_launch_mode(h, mode)
        o = rs.rs_offspring(h, a)
        O = rs.rs_cumulative_offspring(h, o)
        res.append((rs.rs_last_error(h), o.cpu().numpy(), O.cpu().numpy()))
    rs.rs_set_launch_mode(h, rs.LAUNCH_AUTO)
    assert res[0][0] == res[1][0] == rs.RS_OK
    assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[0][2], res[1][2])
    assert np.array_equal(res[0][1], np.bincount(a.cpu().numpy(), minlength=N))
    assert np.array_equal(res[0][2], np.cumsum(res[0][1]))
