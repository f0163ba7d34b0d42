"""Exhaustive and dense checks of the shortcuts in the acceptance tests of Codes 2 and 3.

The binary32 test u < exp(delta) first compares u with a band of relative half-width 2^-15
around the hardware ex2 estimate of exp(delta) and evaluates the pinned exp only inside the
band; it decides like the pinned exp exactly when the pinned exp lies inside the band. That
is checked here for every one of the 1,118,633,984 binary32 values delta in [-86.5, 0), on the
device, with the functions the kernels run (rs_check_acceptance mode 0).

The binary64 test is decided on the binary32 pipes with a rigorous error bound and an exact
binary64 fallback; mode 1 compares its decision with the binary64 definition on 2^22 pairs of
log-weights (four magnitudes of lw_k, lw_j - lw_k over [-90, 0)) with uniforms on the 53-bit
grid at, next to and near the boundary exp(lw_j - lw_k)."""
import pytest

pytestmark = pytest.mark.gpu


def test_binary32_band_holds_for_every_delta(rs):
    assert rs.rs_check_acceptance(0) == 0


def test_binary64_decisions_match_the_definition_on_a_dense_grid(rs):
    assert rs.rs_check_acceptance(1, 1 << 22) == 0


def test_check_refuses_bad_arguments(rs):
    with pytest.raises(rs.RsError):
        rs.rs_check_acceptance(2)
    with pytest.raises(rs.RsError):
        rs.rs_check_acceptance(1, 0)
