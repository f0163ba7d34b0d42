"""GPU parity of partial rejection control (Section 2.2): the CUDA library (through the C ABI)
against the oracle, bit for bit -- ancestors and outcome log-weights, with and without
Permute, binary32 and binary64, at sizes spanning one warp run, many runs with a ragged tail
and the bench's 2^20 -- plus its relation to the rejection resampler and its statuses."""
import numpy as np
import pytest
import torch

import oracle
import workload

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def h(rs):
    handle = rs.Handle((1 << 20) + 4099)
    yield handle
    handle.close()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("N", [1, 2, 5, 255, 257, 4097, 70001, 1 << 20])
def test_prc_bit_exact(rs, h, dtype, N):
    for y, q in [(2.0, 0.9), (3.0, 0.5), (4.0, 0.99), (1.0, 1.0)]:
        lw = workload.synthetic_logw(N, y, seed=N + 7, dtype=dtype)
        lvmax = float(np.quantile(lw, q)) if N > 1 else float(lw[0]) - 0.5
        t = torch.from_numpy(lw).to(DEV)
        for permute in (False, True):
            a, lo = rs.rs_resample_prc(h, t, lvmax, seed=13, step=2, permute=permute)
            assert rs.rs_last_error(h) == rs.RS_OK
            st, want_a, want_lo = oracle.partial_rejection_control(lw, lvmax, seed=13, step=2,
                                                                   permuted=permute)
            assert st == oracle.OK
            assert np.array_equal(a.cpu().numpy(), want_a), (y, q, permute)
            got = lo.cpu().numpy()
            assert got.dtype == lw.dtype
            assert np.array_equal(got, want_lo), (y, q, permute)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_prc_ancestry_is_rejection_with_the_clamped_bound(rs, h, dtype):
    """Same draws as RS_REJECTION with log_wmax = log v_max: same ancestry, but no bound
    violation is reported, and the outcome weights exceed one exactly where the ancestor's
    weight exceeds v_max."""
    N = 300007
    lw = workload.synthetic_logw(N, 3.0, seed=2, dtype=dtype)
    lvmax = float(np.quantile(lw, 0.7))
    t = torch.from_numpy(lw).to(DEV)
    a, lo = rs.rs_resample_prc(h, t, lvmax, seed=4, step=9)
    assert rs.rs_last_error(h) == rs.RS_OK
    ar = rs.rs_resample(h, rs.REJECTION, t, seed=4, step=9, log_wmax=lvmax)
    assert rs.rs_last_error(h) == rs.RS_ERR_BOUND_VIOLATED
    assert torch.equal(a, ar)
    a_np = a.cpu().numpy()
    bound = lw.dtype.type(lvmax)
    assert np.array_equal(lo.cpu().numpy() > 0, lw[a_np] > bound)


def test_prc_statuses_and_arguments(rs, h):
    lw = np.array([-5.0, -6.0, -7.0], dtype=np.float32)
    t = torch.from_numpy(lw).to(DEV)
    a, lo = rs.rs_resample_prc(h, t, 0.0, seed=1, max_trials=1)
    assert rs.rs_last_error(h) == rs.RS_ERR_REJECTION_CAP
    assert a.cpu().tolist() == [0, 1, 2]
    t = torch.tensor([0.0, float("nan")], dtype=torch.float64, device=DEV)
    rs.rs_resample_prc(h, t, 0.0, seed=1)
    assert rs.rs_last_error(h) == rs.RS_ERR_NONFINITE
    t = torch.zeros(4, dtype=torch.float32, device=DEV)
    with pytest.raises(rs.RsError):
        rs.rs_resample_prc(h, t, float("inf"))
    with pytest.raises(rs.RsError):
        rs.rs_resample_prc(h, t, 0.0, max_trials=0)
    with pytest.raises(rs.RsError):
        rs.rs_resample_prc(h, t, 0.0, logw_out=t)
    assert rs.rs_last_error(h) == rs.RS_OK
