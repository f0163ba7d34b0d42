"""Kalman filter for the 1-D linear-Gaussian state-space model of the SMC loop -- TEST
INFRASTRUCTURE (the closed form the bootstrap particle filter's log marginal likelihood is
checked against; only the tests and bench.py's SMC study use it).

Model: x_1 ~ N(0, sigma_x^2 / (1 - phi^2)), x_t = phi x_{t-1} + sigma_x eps_t,
y_t = x_t + sigma_y eta_t. The textbook prediction / update recursion in binary64:
  predict  m_t|t-1 = phi m_t-1,  P_t|t-1 = phi^2 P_t-1 + sigma_x^2   (t > 1)
  evidence log p(y_t | y_1:t-1) = log N(y_t; m_t|t-1, P_t|t-1 + sigma_y^2)
  update   K = P_t|t-1 / (P_t|t-1 + sigma_y^2), m_t = m_t|t-1 + K (y_t - m_t|t-1),
           P_t = (1 - K) P_t|t-1.
Pinned by tests/test_oracle_kalman.py against the joint Gaussian density of y_1:T.
"""
from __future__ import annotations

import math

import numpy as np


def lgssm_loglik(y, phi: float, sigma_x: float, sigma_y: float) -> float:
    """log p(y_1:T) and the per-step increments log p(y_t | y_1:t-1)."""
    return float(np.sum(lgssm_increments(y, phi, sigma_x, sigma_y)))


def lgssm_increments(y, phi: float, sigma_x: float, sigma_y: float) -> np.ndarray:
    y = np.asarray(y, dtype=np.float64)
    out = np.empty(len(y))
    m, P = 0.0, sigma_x * sigma_x / (1.0 - phi * phi)
    r = sigma_y * sigma_y
    for t in range(len(y)):
        if t > 0:
            m, P = phi * m, phi * phi * P + sigma_x * sigma_x
        s = P + r
        e = y[t] - m
        out[t] = -0.5 * (math.log(2.0 * math.pi * s) + e * e / s)
        K = P / s
        m, P = m + K * e, (1.0 - K) * P
    return out
