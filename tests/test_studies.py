"""Host logic of the temperature scans (no GPU): temperature grids and the
crossing of two curves."""
import math

import pytest

from paper_1202_0635_gb300 import studies, workloads


def test_temperature_grid_spans_the_critical_point():
    t = studies.temperatures(2, workloads.POTTS, 0.9, 1.1, 5)
    tc = 1.0 / math.log(1.0 + math.sqrt(2.0))
    assert t[0] == pytest.approx(0.9 * tc) and t[-1] == pytest.approx(1.1 * tc)
    assert t[2] == pytest.approx(tc)


def test_crossing_of_two_straight_lines():
    # U_small(T) = 1 + T, U_large(T) = 3 T - 1 cross at T = 1.
    temps = [0.8, 0.9, 1.05, 1.2]
    rows = [{"L": 16, "T": T, "U": 1.0 + T} for T in temps] + [{"L": 32, "T": T, "U": 3.0 * T - 1.0} for T in temps]
    assert studies.crossing(rows, "U", 16, 32) == pytest.approx(1.0)


def test_no_crossing_gives_none():
    rows = [{"L": 16, "T": T, "U": 2.0} for T in (1.0, 2.0)] + [{"L": 32, "T": T, "U": 1.0} for T in (1.0, 2.0)]
    assert studies.crossing(rows, "U", 16, 32) is None
