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


def test_m2_of_counts_limits():
    import numpy as np
    L, q = 6, 3
    ordered = np.array([[36, 0, 0]])        # every site in one state: m^2 = 1
    uniform = np.array([[12, 12, 12]])      # equal counts: M^2 = 0
    assert studies.m2_of_counts(ordered, L, q)[0] == pytest.approx(1.0)
    assert studies.m2_of_counts(uniform, L, q)[0] == pytest.approx(0.0)


def test_binder_crossing_and_its_jackknife_error():
    """Synthetic bins whose U(T) are straight lines crossing at T = 1: the
    crossing is found there, and bins that scatter give a positive error."""
    import numpy as np
    temps = [0.8, 0.9, 1.05, 1.2]
    rng = np.random.default_rng(0)
    bins = {}
    for L, slope in ((16, 1.0), (32, 3.0)):
        for T in temps:
            u = 1.0 + slope * (T - 1.0) + 2.0   # both equal 3 at T = 1
            m2 = 0.5 * (1.0 + 1e-3 * rng.standard_normal(20))
            bins[(L, T)] = np.stack([m2, u * m2.mean() ** 2 * np.ones(20)], axis=1)
    t, sig = studies.binder_crossing(bins, 16, 32, temps)
    assert t == pytest.approx(1.0, abs=5e-3)
    assert sig is not None and 0.0 < sig < 0.05
