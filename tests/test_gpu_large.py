"""Large lattices (needs a GB300): L = 8192 against the oracle, and the
largest lattice the int32 labels allow (L = 46340, 2.1e9 sites) on sampled
sites and counter invariants.
"""
import math

import numpy as np
import pytest

import paper_1202_0635_gb300 as sw
from oracle import POTTS, Oracle, philox4x32_10

pytestmark = pytest.mark.gpu

TC2 = 1.0 / math.log(1.0 + math.sqrt(2.0))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1202_0635_gb300 import build
    build.build()
    sw.lib()


def test_8192_matches_the_oracle():
    L, q, seed, n = 8192, 2, 5, 3
    g = sw.Lattice(L, q, sw.SW_POTTS, TC2, seed, init=sw.SW_INIT_RANDOM)
    sw.sw_set_record(g.h, 1)
    o = Oracle(L, q, POTTS, TC2, seed, init="random")
    assert np.array_equal(g.spins, o.spins)
    g.sweep(n)
    rec = o.sweep(n, record=True)
    assert np.array_equal(g.spins, o.spins)
    assert np.array_equal(g.take_counts(), rec)
    o.close()
    g.close()


def test_largest_lattice():
    L, q, seed = 46340, 2, 9          # L * L < 2^31: the int32 label limit
    N = L * L
    g = sw.Lattice(L, q, sw.SW_POTTS, TC2, seed, init=sw.SW_INIT_RANDOM)
    s0 = sw.sw_get_spins(g.h, N)
    # Random start on sampled sites: state = mulhi(u_INIT(i).x, q), key = seed.
    rng = np.random.default_rng(3)
    sites = np.concatenate([rng.integers(0, N, 2000), [0, N - 1, N // 2]])
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    want = [(int(philox4x32_10(np.array([i, 0, 3, 0], dtype=np.uint32), key)[0]) * q) >> 32 for i in sites]
    assert np.array_equal(s0[sites], np.array(want, dtype=np.int8))
    sw.sw_set_record(g.h, 1)
    g.sweep(20)
    rows = g.take_counts()
    assert rows.shape == (20, sw.sw_ncounters(q, sw.SW_POTTS))
    for r in rows:
        assert r[0] + r[1] == N                       # state counts
        assert r[2] + r[3] == 2 * N                   # equal + unequal pairs
        assert 0 < r[4] <= 2 * N and 1 <= r[5] <= N   # active bonds, clusters
    # After 20 sweeps at T_c the unequal pairs per site are close to the
    # infinite-lattice value 1 - 1/sqrt(2) (Onsager: <s s'> = 1/sqrt(2)).
    e = rows[-1][3] / N
    assert abs(e - (1.0 - 1.0 / math.sqrt(2.0))) < 0.01
    s1 = sw.sw_get_spins(g.h, N)
    assert s1.min() >= 0 and s1.max() < q
    g.close()
