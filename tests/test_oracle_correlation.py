"""Pins of the oracle's correlation counters (clock model, Sec. 4:
G(r,T) = <S_i^x S_{i+r}^x + S_i^y S_{i+r}^y> at r = L/4 and L/2, averaged
over x and y displacements).

  * closed forms: a uniform lattice (G = 1) and a striped lattice
    k = (x + 2 y) mod q, whose pairs at distance r fall in one known class
    per direction;
  * physics: the q = 4 clock model is two decoupled Ising models at
    coupling J/2 (S_i.S_j = (s_i s_j + t_i t_j)/2 after a 45-degree
    rotation), so G_clock4(r, T) equals the Ising correlation at 2T, known
    exactly on the 4 x 4 torus by enumeration.
"""
import math

import numpy as np
import pytest

import exact
from oracle import CLOCK, Oracle, correlations, ncounters

NSIG = 4.5


def corr_blocks(counts, q):
    nclass = q // 2 + 1
    base = q + nclass + 2
    return counts[base:base + nclass], counts[base + nclass:base + 2 * nclass]


def test_counter_row_layout():
    for q in (2, 3, 6, 64):
        nclass = q // 2 + 1
        assert ncounters(q, CLOCK) == q + 3 * nclass + 2


def test_uniform_lattice_is_fully_correlated():
    L, q = 16, 6
    o = Oracle(L, q, CLOCK, 0.9, 1, init="up")
    c = o.counts()
    h4, h2 = corr_blocks(c, q)
    assert h4[0] == 2 * L * L and h4[1:].sum() == 0
    assert h2[0] == 2 * L * L and h2[1:].sum() == 0
    assert np.allclose(correlations(L, q, c), [1.0, 1.0])


def test_striped_lattice_closed_form():
    # k = (x + 2y) mod 8 on L = 24: a pair at distance r differs by r (x) or
    # 2r (y) states.  r = 6: classes 2 and 4 -> G = (cos(pi/2) + cos(pi)) / 2;
    # r = 12: classes 4 and 0 -> G = (cos(pi) + cos(0)) / 2.
    L, q = 24, 8
    y, x = np.mgrid[0:L, 0:L]
    o = Oracle(L, q, CLOCK, 0.9, 1)
    o.spins = (x + 2 * y) % q
    c = o.counts()
    h4, h2 = corr_blocks(c, q)
    N = L * L
    want4 = np.zeros(q // 2 + 1, dtype=np.int64)
    want4[2] += N
    want4[4] += N
    want2 = np.zeros(q // 2 + 1, dtype=np.int64)
    want2[4] += N
    want2[0] += N
    assert np.array_equal(h4, want4) and np.array_equal(h2, want2)
    g4, g2 = correlations(L, q, c)
    assert g4 == pytest.approx(-0.5, abs=1e-12)
    assert g2 == pytest.approx(0.0, abs=1e-12)


@pytest.mark.parametrize("T", [0.8, 1.134593, 2.0])
def test_clock_q4_correlation_equals_ising(T):
    L = 4
    o = Oracle(L, 4, CLOCK, T, 37)
    o.sweep(200)
    rows = o.sweep(100000, record=True)
    g = correlations(L, 4, rows)
    for col, r in ((0, L // 4), (1, L // 2)):
        want = exact.ising_correlation_exact(L, 2.0 * T, r)
        m, e = exact.binned(g[:, col])
        assert abs(m - want) <= NSIG * e + 1e-12, (r, m, e, want)
