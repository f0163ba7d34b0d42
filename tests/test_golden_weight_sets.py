"""The seeded input recipe and the choice of B against the constants the paper prints for
its synthetic weight sets (Section 4.1; tests/golden/weight_sets_section4_1.txt): the moments
of the generated weights match the paper's E(w) and V(w), beta is E(w)/w_max, and B from
Eq. (B) with the paper's epsilon meets the total-variation target at every y of the grid."""
import math
import os

import numpy as np
import pytest

import oracle
import workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "weight_sets_section4_1.txt")


def _golden():
    g = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            name, rest = line.split(None, 1)
            g[name] = rest
    return g


def _num(expr: str) -> float:
    """A constant of the fixture, written as in the paper (digits, pi, sqrt, * / ( ) -)."""
    return float(eval(expr, {"__builtins__": {}}, {"pi": math.pi, "sqrt": math.sqrt}))


def _coef(field: str) -> dict:
    out = {}
    for part in field.split()[:2]:
        k, v = part.split("=")
        out[k] = _num(v)
    return out


def test_golden_fixture_is_complete():
    g = _golden()
    for name in ("x_law", "w_max", "E_w", "V_w", "epsilon", "beta", "y_grid", "log2N_grid",
                 "B_fractions_C"):
        assert name in g, name


@pytest.mark.parametrize("y", [0.0, 0.5, 1.0, 2.0, 3.0, 4.0])
def test_generated_weights_have_the_papers_moments(y):
    """Paper weights w = exp(lw) / sqrt(2 pi) from the library's log-weights: sample mean and
    variance within a few standard errors of the printed E(w) and V(w)."""
    g = _golden()
    assert float(y) in [float(v) for v in g["y_grid"].split()[:9]]
    Ew, Vw = _coef(g["E_w"]), _coef(g["V_w"])
    e = Ew["coef"] * math.exp(Ew["exp"] * y * y)
    v = Vw["coef"] * math.exp(Vw["exp"] * y * y) - e * e
    N = 1 << 21
    w = np.exp(workload.synthetic_logw(N, y, seed=11).astype(np.float64)) / math.sqrt(2 * math.pi)
    assert w.max() <= _num(g["w_max"].split()[0])
    se_mean = math.sqrt(v / N)
    assert abs(w.mean() - e) < 6 * se_mean, (y, w.mean(), e)
    m4 = np.mean((w - w.mean()) ** 4)
    se_var = math.sqrt(max(m4 - v * v, 0.0) / N)
    assert abs(w.var() - v) < 6 * se_var + 1e-15, (y, w.var(), v)


def test_beta_and_B_from_the_papers_constants():
    g = _golden()
    eps = float(g["epsilon"].split()[0])
    Ew = _coef(g["E_w"])
    w_max = _num(g["w_max"].split()[0])
    Bs = []
    for y in [float(v) for v in g["y_grid"].split()[:9]]:
        beta = Ew["coef"] * math.exp(Ew["exp"] * y * y) / w_max
        assert workload.beta_estimate(y) == pytest.approx(beta, rel=1e-14)
        B = oracle.metropolis_B(eps, beta)
        assert (1 - beta) ** B <= eps < (1 - beta) ** (B - 1)  # Eq. (B): the smallest such B
        Bs.append(B)
    assert Bs == sorted(Bs)  # heavier skew, more steps
