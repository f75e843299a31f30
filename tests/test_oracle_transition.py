"""Pins of the oracle's one-sweep transition law.

The exact Swendsen-Wang kernel P(sigma, .) is built by enumerating every
subset of the bonds that can form (Sec. 2 steps (i)-(vii); clock: the
embedded-cluster move of Sec. 4, averaged over the q mirror axes).  The
construction is checked for detailed balance against the Boltzmann
weights of Eq. (1) / Eq. (clock) -- the physics, not the code -- and the
oracle's sampled one-sweep successors are then tested against the exact
rows with a chi-square test.
"""
import math

import numpy as np
import pytest

import exact
from oracle import CLOCK, ISING, POTTS, Oracle


def energy(sigma, L, q, model):
    b = exact.torus_bonds(L)
    s = np.asarray(sigma, dtype=np.int64).reshape(-1)
    a, c = s[b[:, 0]], s[b[:, 1]]
    if model == "clock":
        return -np.cos(2 * np.pi * (a - c) / q).sum()
    return float((a != c).sum())          # Potts Eq. (1), J = 1


def exact_row(L, q, model, sigma, K):
    if model == "clock":
        rows = [exact.sw_transition_row(L, q, "clock", sigma, exact.clock_bond_p(q, K, m), axis=m)
                for m in range(q)]
        codes = np.unique(np.concatenate([r[0] for r in rows]))
        probs = np.zeros(codes.size)
        for c, p in rows:
            probs[np.searchsorted(codes, c)] += p / q
        return codes, probs
    return exact.sw_transition_row(L, q, "potts", sigma, exact.potts_bond_p(K))


def decode(code, N, q):
    out = np.zeros(N, dtype=np.int64)
    for k in range(N - 1, -1, -1):
        out[k] = code % q
        code //= q
    return out


@pytest.mark.parametrize("q,model,T", [(2, "potts", 1.1346), (3, "potts", 0.9), (4, "clock", 0.8),
                                       (6, "clock", 0.9)])
def test_exact_kernel_detailed_balance_2x2(q, model, T):
    """pi(s) P(s, s') = pi(s') P(s', s) with pi ~ exp(-E/T), all pairs of 2x2 states."""
    L, N = 2, 4
    K = 1.0 / T
    states = exact.all_states(N, q).astype(np.int64)
    codes_all = exact.encode(states, q)
    P = np.zeros((codes_all.size, codes_all.size))
    for s, sig in enumerate(states):
        c, p = exact_row(L, q, model, sig, K)
        P[s, c] = p
    assert np.allclose(P.sum(axis=1), 1.0, atol=1e-12)
    E = np.array([energy(s, L, q, model) for s in states])
    pi = np.exp(-K * (E - E.min()))
    pi /= pi.sum()
    flow = pi[:, None] * P
    assert np.allclose(flow, flow.T, atol=1e-13)
    assert np.allclose(pi @ P, pi, atol=1e-13)


def test_exact_kernel_detailed_balance_3x3_pairs():
    """3x3 tori: detailed balance on random pairs reached in one step."""
    rng = np.random.default_rng(5)
    for q, model, T in ((2, "potts", 1.1346), (3, "potts", 0.9), (6, "clock", 0.9)):
        K = 1.0 / T
        for _ in range(3):
            sig = rng.integers(0, q, 9)
            c, p = exact_row(3, q, model, sig, K)
            j = rng.choice(c.size, size=3, replace=False, p=p)
            for jj in j:
                sig2 = decode(int(c[jj]), 9, q)
                c2, p2 = exact_row(3, q, model, sig2, K)
                back = p2[np.searchsorted(c2, exact.encode(sig, q)[0])]
                lhs = math.exp(-K * energy(sig, 3, q, model)) * p[jj]
                rhs = math.exp(-K * energy(sig2, 3, q, model)) * back
                assert abs(lhs - rhs) <= 1e-12 * max(lhs, rhs)


@pytest.mark.parametrize("L,q,model,omodel,T", [
    (2, 2, "potts", POTTS, 1.1346),
    (3, 2, "potts", ISING, 2.269185),
    (3, 3, "potts", POTTS, 0.9950),
    (3, 6, "clock", CLOCK, 0.9),
    (3, 4, "clock", CLOCK, 0.6),
])
def test_oracle_one_step_law(L, q, model, omodel, T):
    N = L * L
    K = 1.0 / T if omodel != ISING else 2.0 / T
    rng = np.random.default_rng(100 + 10 * L + q)
    o = Oracle(L, q, omodel, T, 2024 + q)
    for trial in range(2):
        sig = rng.integers(0, q, N)
        if trial == 0:
            sig[:] = 0 if model != "clock" else 1
        codes, probs = exact_row(L, q, model, sig, K)
        M = 30000
        samples = o.sample_one_step(sig.astype(np.int8), t0=1000 * trial, M=M)
        sc = exact.encode(samples, q)
        pval, bad = exact.chi2_pvalue(sc, codes, probs)
        assert bad == 0
        assert pval > 1e-4, pval
