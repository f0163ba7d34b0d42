"""Choice of resampler from measured GB300 times: the decision matrices of the paper's
Section 4.4 (Figure 6: the fastest scheme over N and the weight skew y) turned into a lookup.

``decision_gb300.json`` holds the median time per call (with Permute, L2 flushed) of every
scheme over N = 2^10 .. 2^24 and y = 0 .. 4 in binary32 and binary64, as measured by
``bench.py --sweep`` on a GB300 (Metropolis with B from Eq. B, rejection with the a-priori
bound). ``choose_scheme`` interpolates those times to the requested (N, y) and returns the
fastest scheme; with ``unbiased=True`` (the default) the Metropolis resampler, which is biased
for finite B (Section 2.1), is not considered. The skew can be given as y (the workload's
observation, log w = -(y - x)^2 / 2 with x ~ N(0, 1)) or as beta = E(w)/w_max (Eq. beta2),
which for that workload is exp(-y^2/4)/sqrt(2). Host-only, no GPU needed.

The table is regenerated from a sweep's JSON line with
``python -m paper_1301_4019_gb300.select --from-sweep sweep.json`` (``table_from_sweep``).
"""
from __future__ import annotations

import bisect
import json
import math
import os

_TABLE = None
SCHEME_ORDER = ("multinomial", "stratified", "systematic", "metropolis", "rejection")


def _table():
    global _TABLE
    if _TABLE is None:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                               "decision_gb300.json")) as f:
            _TABLE = json.load(f)
    return _TABLE


def beta_of_y(y: float) -> float:
    """beta = E(w)/w_max for log w = -(y - x)^2/2, x ~ N(0, 1), w_max = 1 (Section 4.1)."""
    return math.exp(-y * y / 4.0) / math.sqrt(2.0)


def y_of_beta(beta: float) -> float:
    """Inverse of beta_of_y (0 for beta >= 1/sqrt(2), the flattest weights of the workload)."""
    if not beta > 0.0:
        raise ValueError("beta must be positive")
    r = beta * math.sqrt(2.0)
    return 0.0 if r >= 1.0 else 2.0 * math.sqrt(-math.log(r))


def _interp(xs, ys, x):
    """Piecewise-linear interpolation, clamped at the ends."""
    if x <= xs[0]:
        return ys[0]
    if x >= xs[-1]:
        return ys[-1]
    k = bisect.bisect_right(xs, x) - 1
    t = (x - xs[k]) / (xs[k + 1] - xs[k])
    return ys[k] + t * (ys[k + 1] - ys[k])


def estimated_us(scheme: str, N: int, y: float, dtype: str = "f32") -> float:
    """Time per call interpolated from the measured table: linear in N between measured sizes
    (proportional to N above the largest, flat below the smallest) and linear in y."""
    if N < 1:
        raise ValueError("N must be positive")
    tab = _table()["us"][dtype]
    ygrid = sorted(float(v) for v in tab)
    per_y = []
    for yv in ygrid:
        row = tab[repr(yv) if repr(yv) in tab else str(yv)]
        ns = sorted(int(k) for k in row)
        sizes = [float(1 << n) for n in ns]
        times = [row[str(n)][scheme] for n in ns]
        if N > sizes[-1]:
            per_y.append(times[-1] * N / sizes[-1])
        else:
            per_y.append(_interp(sizes, times, float(N)))
    return _interp(ygrid, per_y, float(y))


def choose_scheme(N: int, y: float | None = None, beta: float | None = None,
                  dtype: str = "f32", unbiased: bool = True):
    """The fastest resampler for N particles and the given skew. Returns (scheme name,
    estimated microseconds per call with Permute)."""
    if (y is None) == (beta is None):
        raise ValueError("give exactly one of y and beta")
    if dtype not in ("f32", "f64"):
        raise ValueError("dtype must be 'f32' or 'f64'")
    if y is None:
        y = y_of_beta(beta)
    if y < 0:
        raise ValueError("y must be non-negative")
    best = None
    for s in SCHEME_ORDER:
        if unbiased and s == "metropolis":
            continue
        t = estimated_us(s, N, y, dtype)
        if best is None or t < best[1]:
            best = (s, t)
    return best


def table_from_sweep(sweep: dict) -> dict:
    """The decision table from the JSON line of ``bench.py --sweep``: the median microseconds
    per call of every (dtype, y, log2 N, scheme) row of the binary32 and binary64 defaults,
    with the sweep's conditions."""
    tab = {}
    for r in sweep["rows"]:
        if r["dtype"] not in ("f32", "f64"):  # (the other accumulation modes: scan schemes only)
            continue
        tab.setdefault(r["dtype"], {}).setdefault(str(float(r["y"])), {}).setdefault(
            str(int(r["log2n"])), {})[r["scheme"]] = r["us"]
    clocks = sweep.get("clocks", {})
    return {"source": "python bench.py --sweep (one GB300, SM %g MHz, with Permute, L2 flushed; "
                      "median microseconds per call)" % clocks.get("sm_mhz", float("nan")),
            "metropolis_B": "Eq. B with eps = 0.01 and beta(y) = exp(-y^2/4)/sqrt(2)",
            "rejection_log_wmax": 0.0, "us": tab}


_ABBREV = {"multinomial": "Mu", "stratified": "St", "systematic": "Sy", "metropolis": "Me",
           "rejection": "Re"}


def sweep_markdown(sweep: dict, ys=(0.0, 2.0, 4.0)) -> str:
    """Markdown tables of a ``bench.py --sweep`` line: microseconds per call and HBM fraction
    per (dtype, scheme) over N at the given y, and the decision matrices (the fastest scheme
    and its time per (y, N), binary32 and binary64)."""
    rows = sweep["rows"]
    sizes = sorted({int(r["log2n"]) for r in rows})
    dtypes = [d for d in ("f32", "f32c", "f64", "f64n") if any(r["dtype"] == d for r in rows)]
    head = "| dtype | scheme | " + " | ".join(f"2^{n}" for n in sizes) + " |"
    rule = "|---|---|" + "---|" * len(sizes)
    by = {(r["dtype"], float(r["y"]), int(r["log2n"]), r["scheme"]): r for r in rows}
    out = []
    for key, title in (("us", "Time per call, microseconds"), ("hbm_frac", "HBM fraction")):
        for y in (ys if key == "us" else (2.0,)):
            out += [f"## {title} at y = {y:g}", "", head, rule]
            for d in dtypes:
                for sch in SCHEME_ORDER:
                    cells = [by.get((d, y, n, sch)) for n in sizes]
                    if all(c is None for c in cells):
                        continue
                    fmt = "{:.1f}" if key == "us" else "{:.3f}"
                    out.append(f"| {d} | {sch} | " + " | ".join(
                        fmt.format(c[key]) if c else "" for c in cells) + " |")
            out.append("")
    small = [n for n in sizes if any("us_graph" in r and int(r["log2n"]) == n for r in rows)]
    if small:
        out += ["## Time per call inside a CUDA graph at y = 2, microseconds", "",
                "| dtype | scheme | " + " | ".join(f"2^{n}" for n in small) + " |",
                "|---|---|" + "---|" * len(small)]
        for d in dtypes:
            for sch in SCHEME_ORDER:
                cells = [by.get((d, 2.0, n, sch)) for n in small]
                if all(c is None or "us_graph" not in c for c in cells):
                    continue
                out.append(f"| {d} | {sch} | " + " | ".join(
                    f"{c['us_graph']:.1f}" if c and "us_graph" in c else "" for c in cells)
                    + " |")
        out.append("")
    ygrid = sorted({float(r["y"]) for r in rows})
    for d in ("f32", "f64"):
        out += [f"## Decision matrix, {d}: fastest scheme and its microseconds", "",
                "| y \\ N | " + " | ".join(f"2^{n}" for n in sizes) + " |",
                "|---|" + "---|" * len(sizes)]
        for y in ygrid:
            cells = []
            for n in sizes:
                best = min(((by[(d, y, n, s)]["us"], s) for s in SCHEME_ORDER
                            if (d, y, n, s) in by), default=None)
                cells.append(f"{_ABBREV[best[1]]} {best[0]:.0f}" if best else "")
            out.append(f"| {y:g} | " + " | ".join(cells) + " |")
        out.append("")
    return "\n".join(out)


def _main(argv=None):
    import argparse
    p = argparse.ArgumentParser(description="Rebuild decision_gb300.json from a sweep.")
    p.add_argument("--from-sweep", required=True, help="file holding bench.py --sweep output")
    p.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                 "decision_gb300.json"))
    p.add_argument("--markdown", action="store_true",
                   help="print the sweep's tables and decision matrices instead")
    a = p.parse_args(argv)
    with open(a.from_sweep) as f:
        sweep = json.loads(f.read().strip().splitlines()[-1])
    if a.markdown:
        print(sweep_markdown(sweep))
        return
    with open(a.out, "w") as f:
        json.dump(table_from_sweep(sweep), f, indent=0, sort_keys=True)


if __name__ == "__main__":
    _main()
