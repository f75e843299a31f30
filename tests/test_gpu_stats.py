"""Labeling statistics through the C ABI (needs a GB300).

The tile counts are exact functions of one sweep's bonds, so they are
recomputed here from the oracle's bonds of the same sweep: the components
of every 64 x 64 tile's bond graph (scipy), those reaching the tile border
(left and top edges always, right and bottom edges through an active
crossing bond), and the provisional labels of the scan (runs of a 32-column
quadrant row not reached by a down bond from the quadrant row above).  The
global figures depend on thread timing and are checked for consistency.
"""
import math

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

import paper_1202_0635_gb300 as sw
from oracle import POTTS, Oracle

pytestmark = pytest.mark.gpu
TILE, QUAD = 64, 32


def tc(q):
    return 1.0 / math.log(1.0 + math.sqrt(q))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1202_0635_gb300 import build
    build.build()
    sw.lib()


def tile_counts(bonds):
    """(components, open components, provisional labels) summed over tiles."""
    L = bonds.shape[0]
    R, D = (bonds & 1).astype(bool), ((bonds >> 1) & 1).astype(bool)
    comps = opens = labels = 0
    for y0 in range(0, L, TILE):
        for x0 in range(0, L, TILE):
            th, tw = min(TILE, L - y0), min(TILE, L - x0)
            r = R[y0:y0 + th, x0:x0 + tw].copy()
            d = D[y0:y0 + th, x0:x0 + tw].copy()
            cross_r, cross_d = r[:, tw - 1].copy(), d[th - 1, :].copy()
            r[:, tw - 1] = False
            d[th - 1, :] = False
            idx = np.arange(th * tw).reshape(th, tw)
            rows = np.concatenate([idx[:, :-1][r[:, :-1]], idx[:-1, :][d[:-1, :]]])
            cols = np.concatenate([idx[:, 1:][r[:, :-1]], idx[1:, :][d[:-1, :]]])
            g = coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(th * tw, th * tw))
            n, comp = connected_components(g, directed=False)
            comp = comp.reshape(th, tw)
            border = set(comp[0, :]) | set(comp[:, 0]) | set(comp[:, tw - 1][cross_r]) | set(comp[th - 1, :][cross_d])
            comps += n
            opens += len(border)
            for yy in range(th):
                for qx in range(0, tw, QUAD):
                    c1 = min(qx + QUAD, tw)
                    starts = [c for c in range(qx, c1) if c == qx or not r[yy, c - 1]]
                    for i, s in enumerate(starts):
                        e = starts[i + 1] if i + 1 < len(starts) else c1
                        hooked = yy % QUAD != 0 and d[yy - 1, s:e].any()
                        labels += not hooked
    return comps, opens, labels


@pytest.mark.parametrize("L,q,T", [(192, 2, tc(2)), (200, 3, tc(3)), (128, 2, 1e9), (96, 4, 0.3 * tc(4))])
def test_tile_counts_equal_those_of_the_oracle_bonds(L, q, T):
    lat = sw.Lattice(L, q, sw.SW_POTTS, T, 21, init=sw.SW_INIT_RANDOM)
    o = Oracle(L, q, POTTS, T, 21, init="random")
    lat.sweep(5)
    o.sweep(5)
    sw.sw_set_labeling_stats(lat.h, 1)
    lat.sweep(1)
    o.sweep(1)
    assert np.array_equal(lat.spins, o.spins)
    st = sw.sw_get_labeling_stats(lat.h)
    ntiles = ((L + TILE - 1) // TILE) ** 2
    comps, opens, labels = tile_counts(o.bonds)
    assert st["sweeps"] == 1
    assert round(st["components_per_tile"] * ntiles) == comps
    assert round(st["open_per_tile"] * ntiles) == opens
    assert round(st["labels_per_tile"] * ntiles) == labels
    if T > 1e8:   # no bonds: every site is its own component, no union anywhere
        assert comps == L * L and st["unions_per_sweep"] == 0 and st["pairs_per_tile"] == 0
    lat.close()
    o.close()


def test_global_walk_figures_are_consistent():
    lat = sw.Lattice(512, 2, sw.SW_POTTS, tc(2), 3, init=sw.SW_INIT_RANDOM)
    lat.sweep(20)
    sw.sw_set_labeling_stats(lat.h, 1)
    lat.sweep(10)
    st = sw.sw_get_labeling_stats(lat.h)
    assert st["sweeps"] == 10
    assert st["unions_per_sweep"] > 0 and st["walks_per_sweep"] > 0
    assert st["links_per_union"] >= 0 and 0 <= st["retries_per_link"] <= 1
    assert 0 <= st["steps_per_walk"] <= st["max_steps"]
    # Every open component is walked at least once a sweep (its root walk).
    ntiles = (512 // TILE) ** 2
    assert st["walks_per_sweep"] >= st["open_per_tile"] * ntiles - 1e-6
    sw.sw_set_labeling_stats(lat.h, 0)
    with pytest.raises(sw.SwError):
        sw.sw_get_labeling_stats(lat.h)
    lat.close()
