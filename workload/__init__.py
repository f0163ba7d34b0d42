"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds none of the resampling arithmetic: it only draws the weight sets of the
paper's experiments (Section 4.1) and the ragged multi-filter layouts, from numpy's PCG64
generator with an explicit seed. The random numbers that the resamplers themselves consume
are not drawn here: each side derives them from (seed, particle, step) with its own
counter-based generator.

Weight sets (Section 4.1): x^i ~ N(0, 1) i.i.d., and the weight of particle i is the
N(y; x^i, 1) likelihood; the log-weight kept here is -(x^i - y)^2 / 2, i.e. the constant
-log(2 pi)/2 is dropped, which every resampler ignores (they are invariant to scaling all
weights by a constant, Appendix E). With this scaling the a-priori bound on the log-weights
is log w_max = 0.
"""
from __future__ import annotations

import math

import numpy as np

DEFAULT_SEED = 20130115


def synthetic_logw(N: int, y: float, seed: int = DEFAULT_SEED, dtype=np.float64) -> np.ndarray:
    """Log-weights -(x - y)^2/2 with x ~ N(0,1), computed in float64 then cast to dtype."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.standard_normal(N)
    lw = -0.5 * (x - float(y)) ** 2
    return lw.astype(dtype)


def expected_weight(y: float) -> float:
    """E(w) for the weight N(y; x, 1) with x ~ N(0,1): the N(y; 0, 2) density (Section 4.1)."""
    return math.exp(-0.25 * y * y) / (2.0 * math.sqrt(math.pi))


def weight_variance(y: float) -> float:
    """V(w) of the same weights (Section 4.1)."""
    return math.exp(-y * y / 3.0) / (math.pi * math.sqrt(12.0)) - expected_weight(y) ** 2


def max_weight() -> float:
    """The a-priori bound w_max = 1/sqrt(2 pi) of the same weights (Section 4.1)."""
    return 1.0 / math.sqrt(2.0 * math.pi)


def beta_estimate(y: float) -> float:
    """beta = E(w)/w_max, the estimate of Eq. (beta2) used to set B (Section 4.1)."""
    return expected_weight(y) / max_weight()


def ragged_sizes(F: int, n_min: int, n_max: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """F filter sizes drawn log-uniformly on [n_min, n_max] (int64)."""
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    u = rng.uniform(math.log(n_min), math.log(n_max), size=F)
    return np.clip(np.floor(np.exp(u)), n_min, n_max).astype(np.int64)


def ragged_logw(sizes: np.ndarray, y_lo: float = 0.0, y_hi: float = 4.0,
                seed: int = DEFAULT_SEED, dtype=np.float32):
    """Concatenated log-weights of F filters in CSR layout: returns (offsets[F+1], logw, y[F]).
    Filter f holds particles offsets[f] .. offsets[f+1]-1 with its own y_f ~ U[y_lo, y_hi]."""
    sizes = np.asarray(sizes, dtype=np.int64)
    rng = np.random.Generator(np.random.PCG64(seed + 2))
    y = rng.uniform(y_lo, y_hi, size=len(sizes))
    offsets = np.zeros(len(sizes) + 1, np.int64)
    np.cumsum(sizes, out=offsets[1:])
    x = rng.standard_normal(int(offsets[-1]))
    yy = np.repeat(y, sizes)
    lw = (-0.5 * (x - yy) ** 2).astype(dtype)
    return offsets, lw, y


# ---------------------------------------------------------------------------------------
# The state-space model of the full SMC loop (Code 1): a 1-D linear-Gaussian model
#   x_1 ~ N(0, sigma_x^2 / (1 - phi^2))  (the stationary law),
#   x_t = phi x_{t-1} + sigma_x eps_t,   y_t = x_t + sigma_y eta_t,   eps, eta ~ N(0, 1).
# ---------------------------------------------------------------------------------------
LGSSM_PHI, LGSSM_SIGMA_X, LGSSM_SIGMA_Y = 0.9, 1.0, 0.5


def lgssm_simulate(T: int, phi: float = LGSSM_PHI, sigma_x: float = LGSSM_SIGMA_X,
                   sigma_y: float = LGSSM_SIGMA_Y, seed: int = DEFAULT_SEED):
    """T steps of the model: (x, y), float64 arrays."""
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    x = np.empty(T)
    x[0] = rng.standard_normal() * sigma_x / math.sqrt(1.0 - phi * phi)
    for t in range(1, T):
        x[t] = phi * x[t - 1] + sigma_x * rng.standard_normal()
    y = x + sigma_y * rng.standard_normal(T)
    return x, y
