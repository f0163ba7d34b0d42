"""Host-side bookkeeping of the SMC loops (paper_1301_4019_gb300/smc.py) without a GPU: the
log-likelihood assembled from the per-step log weight totals, for the resample-every-step
batch and for resampling on demand per filter."""
import math
import types

import numpy as np
import torch

from paper_1301_4019_gb300 import smc


def _bufs(lt, sizes):
    return types.SimpleNamespace(log_total=torch.as_tensor(lt, dtype=torch.float64),
                                 sizes=np.asarray(sizes, np.int64))


def test_adaptive_loglik_increments():
    """Increment t = log total_t - log N_f after a resampling (and at t = 0), else minus the
    previous log total (the carried weights); minus T times the Gaussian constant."""
    rng = np.random.default_rng(1)
    T, sizes, sy = 6, [100, 37], 0.5
    lt = rng.normal(size=(T, 2)) + 3.0
    flags = np.array([[1, 1], [0, 1], [1, 0], [0, 0], [1, 1], [0, 1]], np.uint8)
    got = smc.lgssm_batched_adaptive_loglik_from(_bufs(lt, sizes), torch.from_numpy(flags), sy)
    c = 0.5 * math.log(2 * math.pi * sy * sy)
    for f, n in enumerate(sizes):
        want, base = 0.0, math.log(n)
        for t in range(T):
            if t > 0:
                base = math.log(n) if flags[t, f] else lt[t - 1, f]
            want += lt[t, f] - base - c
        assert abs(got[f] - want) < 1e-12, (f, got[f], want)


def test_adaptive_with_every_flag_set_is_the_every_step_likelihood():
    rng = np.random.default_rng(2)
    T, sizes, sy = 9, [64, 4096, 5], 1.3
    lt = rng.normal(size=(T, 3))
    b = _bufs(lt, sizes)
    ones = torch.ones((T, 3), dtype=torch.uint8)
    a = smc.lgssm_batched_adaptive_loglik_from(b, ones, sy)
    e = smc.lgssm_batched_loglik_from(b, sy)
    assert np.allclose(a, e, rtol=0, atol=1e-12)
