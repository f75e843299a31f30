"""Pins of the oracle's generator and of its random-number keying.

The expected values come from Triton's own Philox-4x32-10 routine run by
Triton's CPU interpreter (a library routine independent of the oracle),
combined with the keying written in sw_oracle.h.  Connectivity comes from
scipy.sparse.csgraph.
"""
import math
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

from oracle import CLOCK, ISING, POTTS, Oracle, philox4x32_10

pytest.importorskip("triton")

HERE = os.path.dirname(os.path.abspath(__file__))
SEED = 0x9E3779B97F4A7C15
T_NO_BONDS = 1e12          # p = 1 - exp(-1e-12) -> integer threshold 0
TAG_BOND, TAG_STATE, TAG_AXIS, TAG_INIT, TAG_STATE_BIT = 0, 1, 2, 3, 4


def _triton_philox(ctr, seed):
    with tempfile.TemporaryDirectory() as d:
        fin, fout = os.path.join(d, "in.npz"), os.path.join(d, "out.npy")
        np.savez(fin, ctr=np.asarray(ctr, dtype=np.uint32), seed=np.uint64(seed))
        subprocess.run([sys.executable, os.path.join(HERE, "triton_philox.py"), fin, fout], check=True)
        return np.load(fout)


@pytest.fixture(scope="module")
def table():
    """Triton Philox outputs for counters (index, sweep, tag, 0), index < 1024,
    sweep in {0, 3}, every tag, under key SEED."""
    idx = np.arange(1024, dtype=np.uint32)
    rows, keys = [], []
    for t in (0, 3):
        for tag in range(5):
            c = np.zeros((idx.size, 4), dtype=np.uint32)
            c[:, 0] = idx
            c[:, 1] = t
            c[:, 2] = tag
            rows.append(c)
            keys.append((t, tag))
    out = _triton_philox(np.concatenate(rows), SEED).reshape(len(keys), idx.size, 4)
    return {k: out[n] for n, k in enumerate(keys)}


def _mulhi(u, q):
    return ((u.astype(np.uint64) * np.uint64(q)) >> np.uint64(32)).astype(np.int64)


def _bit(lanes, r):
    """One-bit draws of roots r: bit r & 31 of lane (r >> 5) & 3 of the
    STATE_BIT counter r >> 7."""
    r = np.asarray(r, dtype=np.int64)
    return ((lanes[r >> 7, (r >> 5) & 3] >> (r & 31).astype(np.uint32)) & 1).astype(np.int64)


def test_philox_matches_triton_library():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(512, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    for seed in (0, 1, 0xFFFFFFFFFFFFFFFF, SEED):
        want = _triton_philox(ctr, seed)
        key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
        got = np.stack([philox4x32_10(c, key) for c in ctr])
        assert np.array_equal(got, want)


def test_random_start_keying(table):
    for q in (2, 3, 6, 127):
        L = 32
        o = Oracle(L, q, POTTS, 1.0, SEED, init="random")
        want = _mulhi(table[(0, TAG_INIT)][: L * L, 0], q)
        assert np.array_equal(o.spins.reshape(-1), want)


@pytest.mark.parametrize("model,q", [(POTTS, 3), (ISING, 2), (POTTS, 2)])
def test_no_bonds_every_site_draws_its_own_state(table, model, q):
    """With p = 0 every site is a cluster of its own and takes a uniform
    new state -- Sec. 2 steps (v)-(vii): mulhi(u_STATE(site), q) for q > 2,
    the site's STATE_BIT bit for q = 2."""
    L = 32
    o = Oracle(L, q, model, T_NO_BONDS, SEED, init="random")
    assert o.thresholds()[0] == 0
    o.sweep_index = 3
    rec = o.sweep(1, record=True)[0]
    if q == 2:
        want = _bit(table[(3, TAG_STATE_BIT)], np.arange(L * L))
        assert 0.4 < want.mean() < 0.6
    else:
        want = _mulhi(table[(3, TAG_STATE)][: L * L, 0], q)
    assert np.array_equal(o.spins.reshape(-1), want)
    assert np.array_equal(o.labels.reshape(-1), np.arange(L * L))
    nclass = q // 2 + 1 if model == CLOCK else 2
    assert rec[q + nclass] == 0 and rec[q + nclass + 1] == L * L   # active bonds, clusters
    assert o.sweep_index == 4


@pytest.mark.parametrize("L", [32, 31, 5, 2])
def test_bond_lanes_labels_and_root_draws(table, L):
    """All spins equal, p ~ 1/2: the bonds are lanes 2(i&1)+dir of the BOND
    counter (i>>1, sweep); clusters are the connected components; every site
    takes its root's STATE draw."""
    q = 4
    T = 1.0 / math.log(2.0)
    o = Oracle(L, q, POTTS, T, SEED, init="up")
    thr = int(o.thresholds()[0])
    assert abs(thr / 2.0 ** 32 - 0.5) < 1e-9
    o.sweep(1)
    N = L * L
    i = np.arange(N)
    lanes = table[(0, TAG_BOND)][i >> 1]
    right = lanes[i, 2 * (i & 1)] < thr
    down = lanes[i, 2 * (i & 1) + 1] < thr
    bonds = o.bonds.reshape(-1)
    assert np.array_equal(bonds & 1, right.astype(np.uint8))
    assert np.array_equal((bonds >> 1) & 1, down.astype(np.uint8))
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    y, x = i // L, i % L
    a = np.concatenate([i[right], i[down]])
    b = np.concatenate([(y * L + (x + 1) % L)[right], (((y + 1) % L) * L + x)[down]])
    g = coo_matrix((np.ones(a.size), (a, b)), shape=(N, N))
    nc, comp = connected_components(g, directed=False)
    root = np.full(nc, N)
    np.minimum.at(root, comp, i)
    want_labels = root[comp]
    assert np.array_equal(o.labels.reshape(-1), want_labels)
    want_spins = _mulhi(table[(0, TAG_STATE)][want_labels, 0], q)
    assert np.array_equal(o.spins.reshape(-1), want_spins)
    rec = o.counts()
    assert rec[q + 2] == right.sum() + down.sum()   # active bonds (Potts: 2 classes)
    assert rec[q + 3] == nc                          # clusters


def test_clock_axis_and_single_site_reflections(table):
    """Clock, p = 0: the sweep's axis is mulhi(u_AXIS(0, sweep), q); each site
    is reflected k -> (m - k) mod q iff its STATE_BIT bit is set."""
    q, L = 6, 32
    o = Oracle(L, q, CLOCK, T_NO_BONDS, SEED, init="random")
    assert int(o.thresholds().max()) == 0
    before = o.spins.reshape(-1).astype(np.int64)
    o.sweep_index = 3
    o.sweep(1)
    m = int(_mulhi(table[(3, TAG_AXIS)][0:1, 0], q)[0])
    assert o.axis == m
    flip = _bit(table[(3, TAG_STATE_BIT)], np.arange(L * L)).astype(bool)
    want = np.where(flip, (m - before) % q, before)
    assert np.array_equal(o.spins.reshape(-1), want)
    o2 = Oracle(L, q, CLOCK, T_NO_BONDS, SEED, init="random")
    o2.sweep(1)
    assert o2.axis == int(_mulhi(table[(0, TAG_AXIS)][0:1, 0], q)[0])
