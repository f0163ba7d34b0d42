"""The bootstrap particle filter (Code 1) on the 1-D linear-Gaussian state-space model, run
through the library's C ABI: for t = 1..T, resample (t > 1, with Permute so that the copy can
run in place, Section 2.3), copy in place, propagate and weight, and accumulate the log of the
mean weight (the filter's estimate of log p(y_t | y_1:t-1), computed with the max-shift of
Appendix E). Every step runs in the library's kernels; this module only sequences the calls.
The adaptive form resamples only when the effective sample size falls below a threshold
(rs_ess) and carries the weights over the other steps. The batched form runs many independent
filters of different sizes in the CSR layout of rs_resample_batched, one launch per stage.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import (PREC_COMPENSATED, Handle, rs_capture_end_if, rs_capture_if_below,
               rs_copy_ancestors, rs_copy_ancestors_batched, rs_ess,
               rs_lgssm_step, rs_lgssm_step_batched, rs_log_sum_weights_batched, rs_resample,
               rs_resample_batched, rs_smc_loglik_step, rs_smc_mark_resampled, rs_ess_batched,
               rs_reset_weights_batched)


class LgssmBuffers:
    """Device buffers of one filter of N particles over T steps."""

    def __init__(self, N: int, T: int, device=None):
        device = device or torch.device("cuda", torch.cuda.current_device())
        self.x = torch.empty(N, dtype=torch.float32, device=device)
        self.logw = torch.empty(N, dtype=torch.float32, device=device)
        self.c = torch.empty(N, dtype=torch.int32, device=device)
        self.ess = torch.empty(1, dtype=torch.float64, device=device)
        self.log_total = torch.empty(T, dtype=torch.float64, device=device)


def lgssm_bootstrap_launch(h: Handle, y, N: int, scheme: int, phi: float, sigma_x: float,
                           sigma_y: float, seed: int = 0, B: int = 64,
                           prec: int = PREC_COMPENSATED, bufs: LgssmBuffers | None = None,
                           stream=None, filter: int = 0) -> LgssmBuffers:
    """Enqueue the whole filter on the stream (no synchronisation); returns the buffers, whose
    log_total[t] receives log sum_i w_t^i (max-shifted weights, shift added back, from rs_ess).
    ``filter`` is the filter index of every random-number counter."""
    T = len(y)
    b = bufs or LgssmBuffers(N, T)
    for t in range(T):
        if t > 0:
            rs_resample(h, scheme, b.logw, B=B, seed=seed, step=t, out=b.c, permute=True,
                        prec=prec, log_wmax=0.0, filter=filter, stream=stream)
            rs_copy_ancestors(h, b.x, b.c, stream=stream)
        rs_lgssm_step(h, b.x, t == 0, phi, sigma_x, float(y[t]), sigma_y, seed=seed, step=t,
                      filter=filter, logw=b.logw, stream=stream)
        rs_ess(h, b.logw, out=b.ess, log_total=b.log_total[t:t + 1], stream=stream)
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
        rs_ess(h, b.logw, out=ess, log_total=b.log_total[t:t + 1], stream=stream)
        lse = float(b.log_total[t].item())
        ll += lse - base - 0.5 * math.log(2 * math.pi * sigma_y ** 2)
        base = lse
        resample = float(ess.item()) < ess_fraction * N
    return ll, n_res


class AdaptiveGraph:
    """The adaptive filter as one CUDA graph: every resampling decision is a conditional node
    (rs_capture_if_below on the device-side ESS), the likelihood and the resampling count are
    kept on the device (rs_smc_loglik_step, rs_smc_mark_resampled). Same arithmetic and the
    same decisions as lgssm_adaptive, without a host round trip per step; replay() reruns the
    whole filter."""

    def __init__(self, h: Handle, y, N: int, scheme: int, phi: float, sigma_x: float,
                 sigma_y: float, ess_fraction: float = 0.5, seed: int = 0, B: int = 64,
                 prec: int = PREC_COMPENSATED):
        T = len(y)
        self.b = b = LgssmBuffers(N, T)
        dev = b.x.device
        self.ess = torch.empty(1, dtype=torch.float64, device=dev)
        self.base = torch.empty(1, dtype=torch.float64, device=dev)
        self.ll = torch.empty(1, dtype=torch.float64, device=dev)
        self.count = torch.zeros(1, dtype=torch.int32, device=dev)
        log_n = math.log(N)
        c = 0.5 * math.log(2 * math.pi * sigma_y ** 2)

        def enqueue(stream):
            for t in range(T):
                if t > 0:
                    body = rs_capture_if_below(h, self.ess, ess_fraction * N, stream=stream)
                    rs_resample(h, scheme, b.logw, B=B, seed=seed, step=t, out=b.c,
                                permute=True, prec=prec, log_wmax=0.0, stream=body)
                    rs_copy_ancestors(h, b.x, b.c, stream=body)
                    rs_smc_mark_resampled(h, b.logw, self.base, log_n, self.count, stream=body)
                    rs_capture_end_if(h, stream=stream)
                rs_lgssm_step(h, b.x, t == 0, phi, sigma_x, float(y[t]), sigma_y, seed=seed,
                              step=t, logw=b.logw, accumulate=t > 0, stream=stream)
                rs_ess(h, b.logw, out=self.ess, log_total=b.log_total[t:t + 1], stream=stream)
                rs_smc_loglik_step(h, b.log_total[t:t + 1], self.base, self.ll, c, log_n,
                                   t == 0, self.count, stream=stream)

        cs = torch.cuda.Stream()
        cs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cs):
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=cs):
                enqueue(cs)
        torch.cuda.current_stream().wait_stream(cs)

    def replay(self):
        self.graph.replay()

    def result(self):
        """(log p-hat(y_1:T), number of resamplings) of the last replay (synchronises)."""
        return float(self.ll.item()), int(self.count.item())


class BatchedLgssmBuffers:
    """Device buffers of F filters (sizes N_f, CSR offsets) over T steps; Y is T x F."""

    def __init__(self, sizes, Y, device=None):
        device = device or torch.device("cuda", torch.cuda.current_device())
        sizes = np.asarray(sizes, dtype=np.int64)
        total = int(sizes.sum())
        self.sizes = sizes
        self.offsets = torch.from_numpy(np.concatenate([[0], np.cumsum(sizes)])).to(device)
        self.x = torch.empty(total, dtype=torch.float32, device=device)
        self.logw = torch.empty(total, dtype=torch.float32, device=device)
        self.c = torch.empty(total, dtype=torch.int32, device=device)
        self.y = torch.as_tensor(np.asarray(Y, dtype=np.float32), device=device).contiguous()
        self.log_total = torch.empty(self.y.shape, dtype=torch.float64, device=device)


def lgssm_batched_launch(h: Handle, bufs: BatchedLgssmBuffers, scheme: int, phi: float,
                         sigma_x: float, sigma_y: float, seed: int = 0, B: int = 64,
                         prec: int = PREC_COMPENSATED, stream=None) -> BatchedLgssmBuffers:
    """Enqueue F bootstrap filters, filter f observing column f of Y: per step one batched
    resample with Permute, one in-place copy, one propagate-and-weight and one per-filter
    log-sum of the weights (log_total[t, f]). Filter f equals lgssm_bootstrap_launch on its
    own with filter = f in every state it computes (x, weights, ancestors)."""
    b = bufs
    for t in range(b.y.shape[0]):
        if t > 0:
            rs_resample_batched(h, scheme, b.logw, b.offsets, B=B, seed=seed, step=t, out=b.c,
                                permute=True, prec=prec, log_wmax=0.0, stream=stream)
            rs_copy_ancestors_batched(h, b.x, b.c, b.offsets, stream=stream)
        rs_lgssm_step_batched(h, b.x, b.offsets, t == 0, phi, sigma_x, b.y[t], sigma_y,
                              seed=seed, step=t, logw=b.logw, stream=stream)
        rs_log_sum_weights_batched(h, b.logw, b.offsets, out=b.log_total[t], stream=stream)
    return b


def lgssm_batched_adaptive_launch(h: Handle, bufs: BatchedLgssmBuffers, scheme: int,
                                  phi: float, sigma_x: float, sigma_y: float,
                                  threshold: float = 0.5, seed: int = 0, B: int = 64,
                                  prec: int = PREC_COMPENSATED, stream=None) -> torch.Tensor:
    """Enqueue F adaptive bootstrap filters (resampling on demand, Section 4.3), every
    decision taken per filter on the device: before step t >= 1, rs_ess_batched flags the
    filters whose ESS is below threshold * N_f; only those are resampled
    (rs_resample_batched_masked), copied and given equal weights (rs_reset_weights_batched);
    the others carry their weights, to which the step's log-likelihood terms are added. The
    filters that keep their particles skip every pass of the batched resampler.
    Returns the T x F uint8 flags (row 0: the initial draw); log_total[t, f] as in
    lgssm_batched_launch. No host synchronisation."""
    b = bufs
    T, F = b.y.shape[0], b.offsets.numel() - 1
    flags = torch.zeros((T, F), dtype=torch.uint8, device=b.x.device)
    flags[0].fill_(1)
    ess = torch.empty(F, dtype=torch.float64, device=b.x.device)
    for t in range(T):
        if t > 0:
            rs_resample_batched(h, scheme, b.logw, b.offsets, B=B, seed=seed, step=t, out=b.c,
                                permute=True, prec=prec, log_wmax=0.0, resample=flags[t],
                                stream=stream)
            rs_copy_ancestors_batched(h, b.x, b.c, b.offsets, stream=stream)
            rs_reset_weights_batched(h, b.logw, b.offsets, flags[t], stream=stream)
        rs_lgssm_step_batched(h, b.x, b.offsets, t == 0, phi, sigma_x, b.y[t], sigma_y,
                              seed=seed, step=t, logw=b.logw, accumulate=t > 0, stream=stream)
        if t + 1 < T:  # this step's log totals and the next step's decisions, one kernel
            rs_ess_batched(h, b.logw, b.offsets, out=ess, log_total=b.log_total[t],
                           threshold=threshold, below=flags[t + 1], stream=stream)
        else:
            rs_log_sum_weights_batched(h, b.logw, b.offsets, out=b.log_total[t], stream=stream)
    return flags


def lgssm_batched_adaptive_loglik_from(bufs: BatchedLgssmBuffers, flags: torch.Tensor,
                                       sigma_y: float) -> np.ndarray:
    """Per-filter log p-hat(y_1:T) of the adaptive filters: increment t is log sum w_t minus
    log N_f after a resampling (and at t = 0), minus log sum w_{t-1} otherwise (the carried
    weights), less the Gaussian constant."""
    lt = bufs.log_total.cpu().numpy()
    fl = flags.cpu().numpy().astype(bool)
    logn = np.log(bufs.sizes.astype(np.float64))
    base = np.where(fl[1:], logn[None, :], lt[:-1])
    inc = np.concatenate([(lt[0] - logn)[None, :], lt[1:] - base], axis=0)
    return inc.sum(axis=0) - lt.shape[0] * 0.5 * math.log(2 * math.pi * sigma_y ** 2)


def lgssm_batched_loglik_from(bufs: BatchedLgssmBuffers, sigma_y: float) -> np.ndarray:
    """Per-filter log p-hat(y_1:T) from the per-step log weight totals."""
    lt = bufs.log_total.cpu().numpy()
    T = lt.shape[0]
    return (lt.sum(axis=0) - T * (np.log(bufs.sizes.astype(np.float64))
                                  + 0.5 * math.log(2 * math.pi * sigma_y ** 2)))
