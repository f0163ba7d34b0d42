"""The exponential of the plain binary32 scans (the weights exp(lw - M) of Codes 5, 7 and 8
summed in plain binary32, formed with the hardware base-2 exponential and the restored error
of its argument) against exp, for every binary32 argument t <= 0, through the C ABI. The
parity tolerance of those sums (parity_tools.KERNEL_C["f32"]) assumes the bound checked here;
every other path uses the pinned exponential, which the oracle shares."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_scan_exp_within_its_bound_for_every_argument(rs):
    bad, max_rel = rs.rs_check_weight_exp()
    assert bad == 0, (bad, max_rel)
    assert 0.0 < max_rel <= rs.SCAN_EXP_REL_ERR, max_rel


def test_scan_exp_check_reports_a_bound_it_does_not_meet(rs):
    _, max_rel = rs.rs_check_weight_exp()
    bad, _ = rs.rs_check_weight_exp(max_rel / 2)
    assert bad > 0


def test_scan_exp_check_refuses_bad_bounds(rs):
    for bound in (0.0, -1.0, float("nan")):
        with pytest.raises(rs.RsError):
            rs.rs_check_weight_exp(bound)


def test_plain_binary32_weights_of_zero_and_minus_inf_are_exact(rs):
    """exp(0) = 1 and exp(-inf) = 0 exactly, so 0/1 weights sum exactly in every mode."""
    lw = np.array([0.0, -np.inf, 0.0, 0.0, -np.inf, 0.0], np.float32)
    with rs.Handle(16) as h:
        W, lt = rs.rs_cumulative_weights(h, torch.from_numpy(lw).to(DEV), prec=0)
        assert rs.rs_last_error(h) == rs.RS_OK
        assert W.cpu().tolist() == [1.0, 1.0, 2.0, 3.0, 3.0, 4.0]
        assert lt.item() == pytest.approx(np.log(4.0), abs=1e-6)
