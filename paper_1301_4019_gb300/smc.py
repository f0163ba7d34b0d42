"""The bootstrap particle filter (Code 1) on the 1-D linear-Gaussian state-space model, run
through the library's C ABI: for t = 1..T, resample (t > 1, with Permute so that the copy can
run in place, Section 2.3), copy in place, propagate and weight, and accumulate the log of the
mean weight (the filter's estimate of log p(y_t | y_1:t-1), computed with the max-shift of
Appendix E). Every step runs in the library's kernels; this module only sequences the calls.
The adaptive form resamples only when the effective sample size falls below a threshold
(rs_ess) and carries the weights over the other steps.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import (PREC_COMPENSATED, Handle, rs_copy_ancestors, rs_cumulative_weights, rs_ess,
               rs_lgssm_step, rs_resample)


class LgssmBuffers:
    """Device buffers of one filter of N particles over T steps."""

    def __init__(self, N: int, T: int, device=None):
        device = device or torch.device("cuda", torch.cuda.current_device())
        self.x = torch.empty(N, dtype=torch.float32, device=device)
        self.logw = torch.empty(N, dtype=torch.float32, device=device)
        self.c = torch.empty(N, dtype=torch.int32, device=device)
        self.W = torch.empty(N, dtype=torch.float32, device=device)
        self.log_total = torch.empty(T, dtype=torch.float64, device=device)


def lgssm_bootstrap_launch(h: Handle, y, N: int, scheme: int, phi: float, sigma_x: float,
                           sigma_y: float, seed: int = 0, B: int = 64,
                           prec: int = PREC_COMPENSATED, bufs: LgssmBuffers | None = None,
                           stream=None) -> LgssmBuffers:
    """Enqueue the whole filter on the stream (no synchronisation); returns the buffers, whose
    log_total[t] receives log sum_i w_t^i (max-shifted weights, shift added back)."""
    T = len(y)
    b = bufs or LgssmBuffers(N, T)
    for t in range(T):
        if t > 0:
            rs_resample(h, scheme, b.logw, B=B, seed=seed, step=t, out=b.c, permute=True,
                        prec=prec, log_wmax=0.0, stream=stream)
            rs_copy_ancestors(h, b.x, b.c, stream=stream)
        rs_lgssm_step(h, b.x, t == 0, phi, sigma_x, float(y[t]), sigma_y, seed=seed, step=t,
                      logw=b.logw, stream=stream)
        rs_cumulative_weights(h, b.logw, prec=prec, W=b.W, log_total=b.log_total[t:t + 1],
                              stream=stream)
    return b


def lgssm_loglik_from(bufs: LgssmBuffers, N: int, sigma_y: float) -> float:
    """log p-hat(y_1:T) = sum_t [log sum_i w_t^i - log N - log(2 pi sigma_y^2) / 2]."""
    lt = bufs.log_total.cpu().numpy()
    return float(np.sum(lt) - len(lt) * (math.log(N) + 0.5 * math.log(2 * math.pi * sigma_y ** 2)))


def lgssm_bootstrap(h: Handle, y, N: int, scheme: int, phi: float, sigma_x: float,
                    sigma_y: float, seed: int = 0, B: int = 64, prec: int = PREC_COMPENSATED,
                    stream=None) -> float:
    """Run the filter and return its log marginal likelihood estimate."""
    b = lgssm_bootstrap_launch(h, y, N, scheme, phi, sigma_x, sigma_y, seed, B, prec,
                               stream=stream)
    return lgssm_loglik_from(b, N, sigma_y)


def lgssm_adaptive(h: Handle, y, N: int, scheme: int, phi: float, sigma_x: float,
                   sigma_y: float, ess_fraction: float = 0.5, seed: int = 0, B: int = 64,
                   prec: int = PREC_COMPENSATED, stream=None):
    """The bootstrap filter with resampling on demand: after weighting step t, resample at
    step t + 1 only if ESS_t < ess_fraction * N; otherwise the weights carry over and the next
    step adds its log-likelihood to them. Returns (log p-hat(y_1:T), number of resamplings).
    The increment of step t is log sum w_t - log sum w_{t-1} (log N after a resampling). The
    host reads the ESS every step to decide."""
    T = len(y)
    b = LgssmBuffers(N, T)
    ess = torch.empty(1, dtype=torch.float64, device=b.x.device)
    base = math.log(N)
    resample = False
    n_res = 0
    ll = 0.0
    for t in range(T):
        if resample:
            rs_resample(h, scheme, b.logw, B=B, seed=seed, step=t, out=b.c, permute=True,
                        prec=prec, log_wmax=0.0, stream=stream)
            rs_copy_ancestors(h, b.x, b.c, stream=stream)
            base = math.log(N)
            n_res += 1
        rs_lgssm_step(h, b.x, t == 0, phi, sigma_x, float(y[t]), sigma_y, seed=seed, step=t,
                      logw=b.logw, accumulate=(t > 0 and not resample), stream=stream)
        rs_cumulative_weights(h, b.logw, prec=prec, W=b.W, log_total=b.log_total[t:t + 1],
                              stream=stream)
        rs_ess(h, b.logw, out=ess, stream=stream)
        lse = float(b.log_total[t].item())
        ll += lse - base - 0.5 * math.log(2 * math.pi * sigma_y ** 2)
        base = lse
        resample = float(ess.item()) < ess_fraction * N
    return ll, n_res
