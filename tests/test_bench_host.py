"""Host logic of bench.py that needs no GPU: the algorithmic amount behind every roofline, the
DRAM-traffic table's source hashing, and the sweep's byte counts."""
import numpy as np
import pytest

import bench

STEP_LABELS = ["fused_multinomial_f32", "fused_stratified_f32", "fused_systematic_f32",
               "fused_multinomial_f64", "fused_stratified_f64", "fused_systematic_f64",
               "search_f32", "search_f64", "metropolis_f32", "metropolis_f64",
               "rejection_f32", "rejection_f64", "permute", "permute_sorted", "fill",
               "offspring", "iscan", "adjacent_difference", "cumoff_to_ancestors"]


def test_every_kernel_of_the_step_has_a_roofline_amount():
    N, B = 1 << 20, 16
    for lab in STEP_LABELS:
        bound, amount, unit = bench.kernel_roofline_units(lab, N, B)
        assert bound in ("hbm", "alu"), lab
        if lab.startswith("rejection_"):
            assert amount is None  # filled in from the expected trial count by run_ours
        else:
            assert amount is not None and amount > 0, lab
    # binary64 inputs move twice the bytes of binary32 ones in the scan kernels
    assert bench.kernel_roofline_units("fused_systematic_f64", N, B)[1] > \
        bench.kernel_roofline_units("fused_systematic_f32", N, B)[1]
    # binary32 chains take two steps from one Philox block, binary64 chains one
    assert bench.kernel_roofline_units("metropolis_f32", N, B) == ("alu", (B + 1) // 2 * N, "Philox")
    assert bench.kernel_roofline_units("metropolis_f64", N, B) == ("alu", B * N, "Philox")


def test_traffic_table_is_keyed_by_the_kernel_sources():
    for lab in STEP_LABELS:
        h = bench.kernel_source_hash(lab)
        assert h is not None and len(h) == 16, lab
        assert h == bench.kernel_source_hash(lab)  # deterministic
    # kernels defined in the same translation unit share a hash
    assert bench.kernel_source_hash("permute") == bench.kernel_source_hash("iscan")
    assert bench.kernel_source_hash("unknown_kernel") is None
    assert bench.ncu_traffic("permute", 1 << 18) is None  # captured at 2^20 only
    for lab, (nbytes, h) in bench.NCU_TRAFFIC.items():
        assert nbytes > 0 and len(h) == 16, lab


def test_sweep_bytes():
    N = 1 << 10
    for scheme in range(5):
        for S in (4, 8):
            assert bench.sweep_hbm_bytes(scheme, S, N) >= (S + 4 + 16) * N
    assert bench.sweep_hbm_bytes(0, 4, N) > bench.sweep_hbm_bytes(2, 4, N)  # stored W


def test_bias_mse_decomposition():
    """||Bias||^2 + tr Var (divisor R) equals the mean squared error over the R vectors."""
    import numpy as np
    rng = np.random.default_rng(4)
    R, N = 7, 5
    o = rng.integers(0, 4, size=(R, N))
    Npi = rng.uniform(0.5, 1.5, size=N)
    b2, mse = bench.bias_mse(o.sum(0) * 1.0, (o * o).sum(0) * 1.0, Npi, R)
    assert mse == pytest.approx(np.mean(((o - Npi) ** 2).sum(1)), rel=1e-12)
    assert b2 == pytest.approx(((o.mean(0) - Npi) ** 2).sum(), rel=1e-12)
    # identical vectors: no variance, the whole error is bias
    same = np.tile(o[:1], (R, 1))
    b2, mse = bench.bias_mse(same.sum(0) * 1.0, (same * same).sum(0) * 1.0, Npi, R)
    assert b2 == pytest.approx(mse, rel=1e-12)


def test_cpu_baseline_on_all_cores_runs_the_oracle():
    import os
    r = bench.cpu_all_cores(1 << 10, 4, 2.0, steps=1)
    assert r["value"] > 0 and r["cores"] == (os.cpu_count() or 1)
    assert "10 independent oracle calls" in r["sample"]


def test_rejection_expected_draws_against_simulation():
    """The expected attempts and binary32 Philox blocks (two attempts per block) of a
    rejection call, against a direct simulation of every particle's attempt count."""
    rng = np.random.default_rng(5)
    N = 2000
    w = np.exp(-0.5 * (rng.standard_normal(N) - 2.0) ** 2)
    attempts, blocks = bench.rejection_expected_draws(w)
    p = w.mean()
    R = 400
    t_sum = 0
    b_sum = 0
    for _ in range(R):
        first = rng.random(N) < w                       # attempt 0 proposes i itself
        more = rng.geometric(p, N)                      # later attempts until one accepts
        T = np.where(first, 1, 1 + more)
        t_sum += T.sum()
        b_sum += ((T + 1) // 2).sum()
    assert abs(t_sum / R - attempts) < 0.01 * attempts
    assert abs(b_sum / R - blocks) < 0.01 * blocks
    assert blocks < attempts
