"""Statistical pins of the oracle against exact equilibrium results.

A correct Swendsen-Wang chain samples the Boltzmann distribution of
Eq. (1) (Potts) or Eq. (clock); its long-run averages must agree with:
  * brute-force enumeration of small tori (Ising 4x4, Potts q=3 3x3,
    clock q=6 3x3, clock q=4 4x4 through its exact map onto two Ising
    models at coupling J/2);
  * Kaufman's exact finite-torus energy at the Ising critical point
    T_c = 2 / ln(1 + sqrt 2) (Onsager's -sqrt 2 per site as L -> oo);
  * the self-dual point beta_c = ln(1 + sqrt q) of the Potts model
    (Sec. 4), where the FK bond density is 1/2 per bond as L -> oo.
Error bars are binned standard errors; the bound is 4.5 sigma.
"""
import math

import numpy as np
import pytest

import exact
from oracle import CLOCK, ISING, POTTS, Oracle, observables

TC_ISING = 2.0 / math.log(1.0 + math.sqrt(2.0))
NSIG = 4.5


def series(o, n, burn=200):
    o.sweep(burn)
    c = o.sweep(n, record=True)
    return c, observables(o.L, o.q, o.model, c)


def check(x, exact_value, name):
    m, e = exact.binned(x)
    assert abs(m - exact_value) <= NSIG * e + 1e-12, (name, m, e, exact_value)


@pytest.mark.parametrize("T", [TC_ISING, 2.0, 3.0])
def test_ising_4x4_enumeration(T):
    ex = exact.ising_exact(4, T)
    _, obs = series(Oracle(4, 2, ISING, T, 17), 100000)
    for k, key in enumerate(("e", "absm", "m2", "m4")):
        check(obs[:, k], ex[key], key)


@pytest.mark.parametrize("T", [1.0 / math.log(1.0 + math.sqrt(3.0)), 0.6, 1.6])
def test_potts_q3_3x3_enumeration(T):
    ex = exact.potts_exact(3, 3, T)
    _, obs = series(Oracle(3, 3, POTTS, T, 23), 100000)
    check(obs[:, 0], ex["e"], "e")
    check(obs[:, 2], ex["m2"], "m2")


@pytest.mark.parametrize("T", [0.9, 0.5, 1.5])
def test_clock_q6_3x3_enumeration(T):
    ex = exact.clock_exact(3, 6, T)
    _, obs = series(Oracle(3, 6, CLOCK, T, 29), 100000)
    check(obs[:, 0], ex["e"], "e")
    check(obs[:, 2], ex["m2"], "m2")


@pytest.mark.parametrize("T", [0.8, 1.134593, 2.0])
def test_clock_q4_equals_two_ising_models(T):
    """S_i.S_j = (s_i s_j + t_i t_j)/2 for q = 4 after a 45-degree rotation,
    so <E/N>_clock4(T) = <E/N>_Ising(2T) and <m^2>_clock4(T) = <m^2>_Ising(2T)."""
    ex = exact.ising_exact(4, 2.0 * T)
    _, obs = series(Oracle(4, 4, CLOCK, T, 31), 100000)
    check(obs[:, 0], ex["e"], "e")
    check(obs[:, 2], ex["m2"], "m2")


def test_kaufman_matches_enumeration_and_onsager():
    """The Kaufman evaluation used below is itself pinned: brute force on
    3x3 / 4x4 tori, and Onsager's -sqrt 2 with a 1/L approach."""
    for L in (3, 4):
        for T in (1.5, TC_ISING, 3.0):
            assert abs(exact.kaufman_energy(L, T, dps=40) - exact.ising_exact(L, T)["e"]) < 1e-12
    e256 = exact.kaufman_energy(256, TC_ISING, dps=40)
    e512 = exact.kaufman_energy(512, TC_ISING, dps=40)
    assert abs(e512 + math.sqrt(2.0)) < abs(e256 + math.sqrt(2.0)) < 0.004
    assert abs(e512 + math.sqrt(2.0)) < 0.002


@pytest.mark.parametrize("L,n", [(16, 20000), (32, 6000)])
def test_ising_energy_at_tc_matches_kaufman(L, n):
    want = exact.kaufman_energy(L, TC_ISING)
    c, obs = series(Oracle(L, 2, ISING, TC_ISING, 37, init="random"), n)
    check(obs[:, 0], want, "e")
    # FK bond density: <active> = p <equal pairs>, equal pairs = N (2 - e) / 2
    p = 2.0 - math.sqrt(2.0)
    N = L * L
    check(c[:, -2] / (2 * N), p * (2.0 - want) / 4.0, "active")


@pytest.mark.parametrize("q", [3, 4])
def test_potts_self_dual_point(q):
    """At beta_c = ln(1 + sqrt q) the FK bond density tends to 1/2 per bond
    and the equal-neighbour fraction to (1 + q^{-1/2}) / 2.  A 64x64 torus
    carries a finite-size offset of order 1/L (Ising: Kaufman gives
    0.0099 at L=64), so the bound is 2/L."""
    L = 64
    Tc = 1.0 / math.log(1.0 + math.sqrt(q))
    c, _ = series(Oracle(L, q, POTTS, Tc, 41, init="random"), 1500)
    N = L * L
    dens = c[:, -2].mean() / (2 * N)
    eq = c[:, q].mean() / (2 * N)
    assert abs(dens - 0.5) < 2.0 / L
    assert abs(eq - 0.5 * (1 + q ** -0.5)) < 2.0 / L
