"""Pins of the integer bond thresholds against closed forms.

Sec. 2 step (ii): p = 1 - exp(-beta J).  At the Potts critical point
beta_c = ln(1 + sqrt q) (Sec. 4) this is p_c = sqrt(q) / (1 + sqrt(q)).
The clock embedding's projections on a mirror axis are sines of multiples
of pi/q, whose exact values are known for q = 4 and q = 6.
"""
import math

import numpy as np
import pytest

from oracle import CLOCK, ISING, POTTS, Oracle, threshold_from_x

TOL = 2.0 ** -32 + 1e-15


def p_of(thr):
    return int(thr) / 2.0 ** 32


@pytest.mark.parametrize("q", [2, 3, 4])
def test_potts_critical_threshold(q):
    Tc = 1.0 / math.log(1.0 + math.sqrt(q))
    thr = Oracle(8, q, POTTS, Tc, 1).thresholds()[0]
    pc = math.sqrt(q) / (1.0 + math.sqrt(q))
    assert 0.0 <= pc - p_of(thr) <= TOL


def test_ising_units_are_potts_units_halved():
    Tc_ising = 2.0 / math.log(1.0 + math.sqrt(2.0))
    thr = Oracle(8, 2, ISING, Tc_ising, 1).thresholds()[0]
    assert 0.0 <= (2.0 - math.sqrt(2.0)) - p_of(thr) <= TOL
    for T in (0.5, 1.0, 2.269185, 3.7):
        a = Oracle(4, 2, ISING, T, 1).thresholds()[0]
        b = Oracle(4, 2, POTTS, T / 2.0, 1).thresholds()[0]
        assert a == b


def test_threshold_edges():
    assert threshold_from_x(0.0) == 0
    assert threshold_from_x(-1.0) == 0
    assert threshold_from_x(1e-12) == 0
    assert threshold_from_x(1e3) == 2 ** 32 - 1
    assert threshold_from_x(math.log(2.0)) in (2 ** 31 - 1, 2 ** 31)


def test_monotone_in_temperature():
    Ts = np.linspace(0.2, 5.0, 60)
    thr = [int(Oracle(4, 3, POTTS, T, 1).thresholds()[0]) for T in Ts]
    assert all(a >= b for a, b in zip(thr, thr[1:]))


def _clock_table(q, T):
    return Oracle(4, q, CLOCK, T, 1).thresholds().reshape(2 * q, 2 * q)


@pytest.mark.parametrize("q", [3, 4, 5, 6, 8])
def test_clock_table_structure(q):
    """Zero on the axis (j = 0, q) and across it (opposite signs); symmetric."""
    t = _clock_table(q, 0.9)
    n = 2 * q
    for a in range(n):
        for b in range(n):
            side_a = 0 if a % q == 0 else (1 if a < q else -1)
            side_b = 0 if b % q == 0 else (1 if b < q else -1)
            if side_a == 0 or side_b == 0 or side_a != side_b:
                assert t[a, b] == 0
            else:
                assert t[a, b] > 0
    assert np.array_equal(t, t.T)


def test_clock_q4_closed_forms():
    """q = 4: |projections| are sin(pi/4) = 1/sqrt 2 and sin(pi/2) = 1."""
    T = 1.3
    K = 1.0 / T
    t = _clock_table(4, T)
    # j = 2: |s| = 1; j = 1, 3: |s| = 1/sqrt(2); 2K s_a s_b
    assert abs(p_of(t[2, 2]) - (1 - math.exp(-2 * K))) <= TOL
    assert abs(p_of(t[1, 1]) - (1 - math.exp(-K))) <= TOL
    assert abs(p_of(t[1, 3]) - (1 - math.exp(-K))) <= TOL
    assert abs(p_of(t[1, 2]) - (1 - math.exp(-math.sqrt(2) * K))) <= TOL
    assert abs(p_of(t[6, 6]) - (1 - math.exp(-2 * K))) <= TOL


def test_clock_q6_closed_forms():
    """q = 6: |projections| are 1/2, sqrt(3)/2 and 1."""
    T = 0.9
    K = 1.0 / T
    t = _clock_table(6, T)
    half, r3 = 0.5, math.sqrt(3) / 2
    cases = {(1, 1): half * half, (1, 3): half, (2, 2): r3 * r3, (3, 3): 1.0,
             (1, 2): half * r3, (2, 4): r3 * r3, (7, 11): half * half, (9, 9): 1.0}
    for (a, b), prod in cases.items():
        assert abs(p_of(t[a, b]) - (1 - math.exp(-2 * K * prod))) <= TOL + 1e-15, (a, b)
