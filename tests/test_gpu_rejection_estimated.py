"""Rejection resampling with an estimated bound (Section 2.2: a substitute for w_max when no
hard bound is known), through the C ABI, against the oracle bit for bit: the estimate (the
largest of `sample` drawn log-weights), the ancestors (partial rejection control with that
bound), the outcome log-weights and the count of log-weights above the estimate."""
import numpy as np
import pytest
import torch

import oracle
import workload

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def h(rs):
    handle = rs.Handle(1 << 20)
    yield handle
    handle.close()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("N", [1, 5, 1000, 4097, 70001, 1 << 20])
def test_estimated_bound_matches_oracle(rs, h, dtype, N):
    for y, sample in [(2.0, 16), (4.0, 1024), (0.0, 1), (3.0, 40 * N)]:
        sample = min(sample, 1 << 22)
        lw = workload.synthetic_logw(N, y, seed=N + 3, dtype=dtype)
        t = torch.from_numpy(lw).to(DEV)
        for permute in (False, True):
            a, out, bound, viol = rs.rs_resample_rejection_estimated(
                h, t, sample, seed=17, step=2, permute=permute)
            st = rs.rs_last_error(h)
            ost, a_o, out_o, est_o, viol_o = oracle.rejection_estimated(
                lw, sample, seed=17, step=2, permuted=permute)
            assert ost == oracle.OK and st == rs.RS_OK
            assert bound.item() == est_o
            assert viol.item() == viol_o
            assert np.array_equal(a.cpu().numpy(), a_o), (y, sample, permute)
            assert np.array_equal(out.cpu().numpy(), out_o), (y, sample, permute)


def test_estimated_bound_special_cases(rs, h):
    # no finite log-weight drawn: the identity, flagged
    t = torch.full((777,), float("-inf"), dtype=torch.float32, device=DEV)
    a, out, bound, viol = rs.rs_resample_rejection_estimated(h, t, 64, seed=1, permute=True)
    assert rs.rs_last_error(h) == rs.RS_ERR_ZERO_WEIGHT
    assert bound.item() == float("-inf") and viol.item() == 0
    assert a.cpu().tolist() == list(range(777)) and torch.all(out == 0)
    # NaN log-weights are passed over by the estimate and flagged by the resampler
    lw = np.array([0.0, np.nan, -1.0, -2.0] * 50, np.float64)
    t = torch.from_numpy(lw).to(DEV)
    a, out, bound, viol = rs.rs_resample_rejection_estimated(h, t, 400, seed=2)
    assert rs.rs_last_error(h) == rs.RS_ERR_NONFINITE
    assert bound.item() == 0.0
    with pytest.raises(rs.RsError):
        rs.rs_resample_rejection_estimated(h, t, 0, seed=2)
