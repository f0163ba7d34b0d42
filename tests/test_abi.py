"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports every symbol that
the headers under include/ declare, and its host-only calls behave (no GPU needed)."""
import ctypes as C
import math
import os
import re

import pytest

import oracle
import workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    inc = os.path.join(ROOT, "include")
    text = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc))
                   if f.endswith(".h"))
    return sorted(set(re.findall(r"^\s*(?:int|const char\*|void)\s+(rs_\w+)\s*\(", text, re.M)))


def test_library_builds_and_exports_every_declared_symbol():
    import paper_1301_4019_gb300 as rs
    lib = rs.load()
    declared = _declared_symbols()
    assert len(declared) >= 13
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(rs.EXPORTED) == sorted(n for n in declared if n in rs.EXPORTED)
    assert set(rs.EXPORTED) <= set(declared)


def test_metropolis_B_matches_oracle_and_tv_definition():
    import paper_1301_4019_gb300 as rs
    for y in [0, 0.5, 1, 1.5, 2, 2.5, 3, 3.5, 4]:
        beta = workload.beta_estimate(y)
        B = rs.rs_metropolis_B(0.01, beta)
        assert B == oracle.metropolis_B(0.01, beta)
        assert (1 - beta) ** B <= 0.01 < (1 - beta) ** (B - 1)
    with pytest.raises(rs.RsError):
        rs.rs_metropolis_B(0.0, 0.5)
    with pytest.raises(rs.RsError):
        rs.rs_metropolis_B(0.01, 0.0)


def test_host_argument_checks_need_no_gpu():
    import paper_1301_4019_gb300 as rs
    lib = rs.load()
    h = C.c_void_p()
    assert lib.rs_create(C.byref(h), 0, 0) == rs.RS_ERR_ARG
    assert lib.rs_create(None, 10, 0) == rs.RS_ERR_ARG
    assert lib.rs_adjacent_difference(None, None, 10, None, None) == rs.RS_ERR_ARG
    assert lib.rs_resample(None, 0, 0, None, 10, 0, 0, 0, None, 0, None, None) == rs.RS_ERR_ARG
    assert lib.rs_last_error(None, None) == rs.RS_ERR_ARG
    assert lib.rs_destroy(None) == rs.RS_OK
    for code in range(-8, 1):
        assert rs.rs_strerror(code) != "unknown status"
