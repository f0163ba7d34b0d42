"""Pins of the Kalman-filter oracle (oracle/kalman.py): its log marginal likelihood equals the
joint Gaussian density of y_1:T (covariance of the stationary AR(1) process plus observation
noise) computed directly by scipy, and reduces to i.i.d. normals when phi = 0."""
import math

import numpy as np
import pytest

from oracle import kalman
import workload


@pytest.mark.parametrize("T", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("phi,sx,sy", [(0.9, 1.0, 0.5), (0.5, 2.0, 1.5), (-0.7, 0.3, 0.2)])
def test_kalman_equals_joint_gaussian_density(T, phi, sx, sy):
    stats = pytest.importorskip("scipy.stats")
    _, y = workload.lgssm_simulate(T, phi, sx, sy, seed=11 + T)
    s0 = sx * sx / (1.0 - phi * phi)
    idx = np.arange(T)
    cov = s0 * phi ** np.abs(idx[:, None] - idx[None, :]) + sy * sy * np.eye(T)
    want = stats.multivariate_normal(mean=np.zeros(T), cov=cov).logpdf(y)
    assert abs(kalman.lgssm_loglik(y, phi, sx, sy) - want) < 1e-10 * max(1.0, abs(want))


def test_kalman_independent_case():
    y = np.array([0.3, -1.2, 2.5, 0.0])
    s = 1.5 ** 2 + 0.4 ** 2
    want = sum(-0.5 * (math.log(2 * math.pi * s) + v * v / s) for v in y)
    assert abs(kalman.lgssm_loglik(y, 0.0, 1.5, 0.4) - want) < 1e-12
