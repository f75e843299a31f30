"""Pins of the oracle's cluster search (Sec. 2 step (iv)).

The canonical label of a cluster is its smallest site index (the "proper
label" of the Hoshen-Kopelman passage of Sec. 2).  Checked against
scipy.sparse.csgraph on the bond graphs real sweeps produce, and against
brute force over every bond set of the 2x2 and 3x3 tori.
"""
import math

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

from exact import components_of_subsets, torus_bonds
from oracle import CLOCK, ISING, POTTS, Oracle


def scipy_labels(L, bonds):
    N = L * L
    i = np.arange(N)
    y, x = i // L, i % L
    r = (bonds & 1).astype(bool)
    d = ((bonds >> 1) & 1).astype(bool)
    a = np.concatenate([i[r], i[d]])
    b = np.concatenate([(y * L + (x + 1) % L)[r], (((y + 1) % L) * L + x)[d]])
    g = coo_matrix((np.ones(a.size), (a, b)), shape=(N, N))
    nc, comp = connected_components(g, directed=False)
    root = np.full(nc, N)
    np.minimum.at(root, comp, i)
    return root[comp], nc


@pytest.mark.parametrize("L", [2, 3, 5, 8, 16, 33, 64])
@pytest.mark.parametrize("model,q,T", [(POTTS, 2, 0.6), (POTTS, 2, 1.1346), (POTTS, 3, 2.0),
                                       (ISING, 2, 1.5), (CLOCK, 6, 0.5), (CLOCK, 6, 0.9)])
def test_labels_match_scipy_components(L, model, q, T):
    o = Oracle(L, q, model, T, 1000 + L, init="random")
    for _ in range(4):
        o.sweep(1)
        want, nc = scipy_labels(L, o.bonds.reshape(-1))
        lab = o.labels.reshape(-1)
        assert np.array_equal(lab, want)
        nclass = q // 2 + 1 if model == CLOCK else 2
        assert o.counts()[q + nclass + 1] == nc   # clusters
        assert np.all(lab <= np.arange(L * L))
        assert np.array_equal(lab[lab], lab)


def _all_bond_sets(L):
    N = L * L
    B = 2 * N
    masks = np.arange(1 << B, dtype=np.int64)
    bonds = np.zeros((masks.size, N), dtype=np.uint8)
    for k in range(B):
        site, direction = k // 2, k % 2
        bonds[:, site] |= (((masks >> k) & 1) << direction).astype(np.uint8)
    return masks, bonds


@pytest.mark.parametrize("L", [2, 3])
def test_labels_exhaustive_small_tori(L):
    """Every one of the 2^(2N) bond sets of the 2x2 and 3x3 tori."""
    masks, bonds = _all_bond_sets(L)
    o = Oracle(L, 2, POTTS, 1.0, 1)
    got = o.label_bonds(bonds)
    want = components_of_subsets(L * L, torus_bonds(L), masks)
    assert np.array_equal(got, want)
    # spot-check the brute force itself against scipy
    for s in (0, 1, 7, masks.size // 3, masks.size - 1):
        assert np.array_equal(want[s], scipy_labels(L, bonds[s])[0])
