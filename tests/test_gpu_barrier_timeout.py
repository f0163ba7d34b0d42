"""The bounded grid barrier of the cooperative kernels: a wait that runs out ends the kernel
with RS_ERR_TIMEOUT instead of hanging, rs_last_error reports it and resets the handle's
barrier state, and the next cooperative call is exact again.

The wait is made to run out by a self-check launch whose barrier expects one arrival more
than its CTAs make (a capped device wait that returns; nothing faults or hangs), with the
handle's barrier limit set to 1 ms."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


def _exact_weights(N, seed):
    rng = np.random.default_rng(seed)
    lw = np.full(N, -np.inf, np.float32)
    lw[rng.choice(N, N // 3 + 11, replace=False)] = 0.0
    return lw


def test_barrier_wait_runs_out_and_the_handle_recovers(rs):
    N = (1 << 21) + 4097
    lw = _exact_weights(N, 5)
    t = torch.from_numpy(lw).cuda()
    want = oracle.systematic(lw, 9, step=1, prec=0)[2]
    with rs.Handle(N) as h:
        rs.rs_set_launch_mode(h, rs.LAUNCH_FUSED)
        a = rs.rs_resample(h, rs.SYSTEMATIC, t, seed=9, step=1).cpu().numpy()
        assert rs.rs_last_error(h) == rs.RS_OK
        assert np.array_equal(a, want)
        rs.rs_set_barrier_timeout(h, 1_000_000)  # 1 ms
        for _ in range(2):
            rs.rs_check_barrier_timeout(h)
            assert rs.rs_last_error(h) == rs.RS_ERR_TIMEOUT
            # the barrier state was reset: cooperative calls are exact again (the integer
            # scan of the conversions is cooperative too)
            a = rs.rs_resample(h, rs.SYSTEMATIC, t, seed=9, step=1).cpu().numpy()
            assert rs.rs_last_error(h) == rs.RS_OK
            assert np.array_equal(a, want)
            o = rs.rs_offspring(h, torch.from_numpy(a).cuda())
            O = rs.rs_cumulative_offspring(h, o)
            assert rs.rs_last_error(h) == rs.RS_OK
            assert np.array_equal(O.cpu().numpy(),
                                  np.cumsum(np.bincount(a, minlength=N)).astype(np.int32))
        rs.rs_set_barrier_timeout(h, 10_000_000_000)
        with pytest.raises(rs.RsError):
            rs.rs_set_barrier_timeout(h, 0)
