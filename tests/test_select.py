"""Host tests of the scheme choice from the measured decision matrices (no GPU)."""
import math

import pytest

from paper_1301_4019_gb300 import select


def test_grid_points_return_the_measured_fastest():
    tab = select._table()["us"]
    for dtype, by_y in tab.items():
        for ys, by_n in by_y.items():
            for ns, times in by_n.items():
                N, y = 1 << int(ns), float(ys)
                name, us = select.choose_scheme(N, y=y, dtype=dtype, unbiased=False)
                assert us == pytest.approx(min(times.values()))
                assert times[name] == pytest.approx(us)
                name_u, us_u = select.choose_scheme(N, y=y, dtype=dtype)
                assert name_u != "metropolis"
                assert us_u == pytest.approx(min(v for k, v in times.items()
                                                 if k != "metropolis"))


def test_regimes_of_the_decision_matrix():
    # skewed weights: the scan-based systematic resampler; flat weights at small N: Metropolis
    assert select.choose_scheme(1 << 20, y=4.0)[0] == "systematic"
    assert select.choose_scheme(1 << 12, y=0.0, unbiased=False)[0] == "metropolis"
    # beyond the measured sizes the times scale with N
    t24 = select.estimated_us("systematic", 1 << 24, 2.0)
    assert select.estimated_us("systematic", 1 << 25, 2.0) == pytest.approx(2 * t24)


def test_beta_and_y_agree():
    for y in (0.0, 0.7, 2.0, 3.5):
        assert select.y_of_beta(select.beta_of_y(y)) == pytest.approx(y, abs=1e-12)
        assert select.choose_scheme(1 << 18, y=y) == select.choose_scheme(
            1 << 18, beta=select.beta_of_y(y))
    assert select.y_of_beta(0.9) == 0.0
    with pytest.raises(ValueError):
        select.choose_scheme(100)
    with pytest.raises(ValueError):
        select.choose_scheme(100, y=1.0, dtype="f16")
    assert math.isfinite(select.estimated_us("rejection", 1, 1.3))


def test_table_from_sweep_and_cli(tmp_path):
    """The committed generator of the decision table: rows of a sweep line become
    us[dtype][y][log2 N][scheme]; the CLI writes the same table to the given file."""
    import json
    rows = [{"dtype": dt, "y": y, "log2n": n, "scheme": s, "us": 1.0 + n + k}
            for dt in ("f32", "f64") for y in (0.0, 4.0) for n in (10, 11)
            for k, s in enumerate(select.SCHEME_ORDER)]
    sweep = {"rows": rows, "clocks": {"sm_mhz": 2070.0}}
    t = select.table_from_sweep(sweep)
    assert t["us"]["f64"]["4.0"]["11"]["rejection"] == 16.0
    assert set(t["us"]["f32"]) == {"0.0", "4.0"} and "2070" in t["source"]
    src, out = tmp_path / "sweep.json", tmp_path / "table.json"
    src.write_text("log line\n" + json.dumps(sweep) + "\n")
    select._main(["--from-sweep", str(src), "--out", str(out)])
    assert json.load(open(out)) == json.loads(json.dumps(t))
