"""Printed values of the paper checked against the oracle's cost model."""
import os

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _rows(name):
    with open(os.path.join(HERE, "golden", name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                yield [c.strip() for c in line.split("|")]


def test_compression_ratios_and_cost_reduction():
    rows = list(_rows("compression_ratios.txt"))
    assert len(rows) == 5
    for cite, n, r, cr, cost in rows:
        n, r, cr, cost = int(n), int(r), float(cr), float(cost)
        assert abs(oracle.cr_als_skew(n, r) - cr) < 0.1, cite
        assert abs(oracle.cost_reduction(n, r) - cost) < 0.1, cite
        assert abs(oracle.cr_als(n, r) - cr / 2) < 0.1, cite


def _half_unit(printed):
    """Half a unit in the last printed place of a figure."""
    return 0.5 * 10.0 ** -(len(printed.split(".")[1]) if "." in printed else 0)


def test_theoretical_and_measured_speedups():
    rows = list(_rows("speedups.txt"))
    assert len(rows) == 3
    for cite, n, r, f, theo, t_g, t_cp, meas in rows:
        red = oracle.cost_reduction(int(n), int(r))
        # Amdahl's law with the oracle's cost reduction brackets the printed
        # theoretical speedup once f and the speedup are taken at their
        # printed precision (97 % means 96.5 % to 97.5 %)
        lo = oracle.amdahl_speedup((float(f) - _half_unit(f)) / 100, red) - _half_unit(theo)
        hi = oracle.amdahl_speedup((float(f) + _half_unit(f)) / 100, red) + _half_unit(theo)
        assert lo <= float(theo) <= hi, (cite, lo, hi)
        # the printed speedup is the ratio of the printed ("about") wall times,
        # each good to half a unit of its last digit
        ratio_lo = (float(t_g) - 0.5) / (float(t_cp) + 0.5)
        ratio_hi = (float(t_g) + 0.5) / (float(t_cp) - 0.5)
        assert ratio_lo - _half_unit(meas) <= float(meas) <= ratio_hi + _half_unit(meas), cite
    # a plausible mistake: the compression ratio 2N^2/(3R) in place of the cost
    # reduction leaves the printed 3D LDC value outside its bracket
    assert oracle.amdahl_speedup(0.975, oracle.cr_als_skew(400, 3200)) - 0.05 > 11.4
    # limits: no contraction share, no gain; an infinite reduction gives 1/(1-f)
    assert oracle.amdahl_speedup(0.0, 50.0) == 1.0
    assert abs(oracle.amdahl_speedup(0.97, 1e300) - 1 / 0.03) < 1e-9
