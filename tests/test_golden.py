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
