"""GPU parity at the largest size of the measured workloads (N = 2^26 + 1001: past the 2^26 of
the precision study, with a ragged last tile): Metropolis and rejection bit for bit against
the oracle, systematic within the rounding rule of the scan-based schemes, and Permute's
postconditions on every output."""
import numpy as np
import pytest
import torch

import oracle
import workload
from parity_tools import cumulative_mismatches

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
N = (1 << 26) + 1001


@pytest.fixture(scope="module")
def big(rs):
    handle = rs.Handle(N)
    yield handle
    handle.close()


def _permute_ok(a, c):
    """c is a permutation of a (same counts) with o_i > 0 => c_i = i (Code 10)."""
    o = np.bincount(a, minlength=len(a))
    return np.array_equal(np.bincount(c, minlength=len(a)), o) and \
        np.all(c[o > 0] == np.nonzero(o > 0)[0])


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_collective_free_bit_exact_at_max_size(rs, big, dtype):
    """Index arithmetic at the largest size: short chains (B = 2) and mild skew (y = 1) keep
    the oracle's share of the test to seconds."""
    lw = workload.synthetic_logw(N, 1.0, seed=26, dtype=dtype)
    t = torch.from_numpy(lw).to(DEV)
    a = rs.rs_resample(big, rs.METROPOLIS, t, B=2, seed=3, step=1).cpu().numpy()
    assert rs.rs_last_error(big) == rs.RS_OK
    st, want = oracle.metropolis(lw, 2, seed=3, step=1)
    assert st == oracle.OK and np.array_equal(a, want)
    a = rs.rs_resample(big, rs.REJECTION, t, seed=3, step=1, log_wmax=0.0).cpu().numpy()
    assert rs.rs_last_error(big) == rs.RS_OK
    st, want = oracle.rejection(lw, 0.0, seed=3, step=1)
    assert st == oracle.OK and np.array_equal(a, want)
    c = rs.rs_resample(big, rs.REJECTION, t, seed=3, step=1, log_wmax=0.0,
                       permute=True).cpu().numpy()
    assert rs.rs_last_error(big) == rs.RS_OK
    assert _permute_ok(a, c)


@pytest.mark.parametrize("kind,dtype,prec", [("f32c", np.float32, 1), ("f64", np.float64, 0)])
def test_systematic_at_max_size(rs, big, kind, dtype, prec):
    lw = workload.synthetic_logw(N, 2.0, seed=27, dtype=dtype)
    t = torch.from_numpy(lw).to(DEV)
    a = rs.rs_resample(big, rs.SYSTEMATIC, t, seed=9, prec=prec).cpu().numpy()
    assert rs.rs_last_error(big) == rs.RS_OK
    assert np.all(np.diff(a) >= 0) and a[0] >= 0 and a[-1] < N
    O_k = np.cumsum(np.bincount(a, minlength=N))
    assert O_k[-1] == N
    _, O_t, _ = oracle.systematic(lw, 9, prec=1)
    n, bad = cumulative_mismatches(kind, rs.SYSTEMATIC, lw, O_k, O_t, seed=9,
                                   oracle_is_sequential=False)
    assert bad == 0, (n, bad)
    c = rs.rs_resample(big, rs.SYSTEMATIC, t, seed=9, prec=prec, permute=True).cpu().numpy()
    assert rs.rs_last_error(big) == rs.RS_OK
    assert _permute_ok(a, c)
