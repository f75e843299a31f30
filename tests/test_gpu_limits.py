"""Device-side limits through the C ABI (needs a GB300).

* The overflow path of a tile's union-pair list: valid bond patterns almost
  never fill the list (a quadrant row pair yields at most 31 further pairs,
  and only in a pattern no Potts or clock configuration makes likely), so
  the list is shrunk with sw_set_debug_limits and the chain must still
  equal the oracle's, spins, labels and counters after every sweep.
* The bounded device loops: with every data-dependent loop capped at one
  step, a sweep of an ordered lattice cannot finish its walks; the device
  records the error, the host reports SW_ERR_NOT_CONVERGED, it stays sticky
  on that handle, and a fresh handle sweeps bit-exactly again.  No loop can
  run past its cap, so nothing waits on the GPU.
"""
import math

import numpy as np
import pytest

import paper_1202_0635_gb300 as sw
from oracle import CLOCK, POTTS, Oracle

pytestmark = pytest.mark.gpu

MODEL = {POTTS: sw.SW_POTTS, CLOCK: sw.SW_CLOCK}


def tc(q):
    return 1.0 / math.log(1.0 + math.sqrt(q))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1202_0635_gb300 import build
    build.build()
    sw.lib()


def lockstep(lat, o, n):
    sw.sw_set_debug_labels(lat.h, 1)
    sw.sw_set_record(lat.h, 1)
    for k in range(n):
        lat.sweep(1)
        rec = o.sweep(1, record=True)
        assert np.array_equal(lat.spins, o.spins), "spins differ after sweep %d" % (k + 1)
        assert np.array_equal(lat.labels, o.labels), "labels differ after sweep %d" % (k + 1)
        assert np.array_equal(lat.take_counts(), rec), "counters differ after sweep %d" % (k + 1)


@pytest.mark.parametrize("list_cap", [1, 5, 64])
@pytest.mark.parametrize("L,q,model,T", [(128, 3, POTTS, tc(3)), (200, 2, POTTS, tc(2)), (96, 6, CLOCK, 0.9),
                                         (64, 2, POTTS, 0.5 * tc(2))])
def test_union_list_overflow_matches_the_oracle(list_cap, L, q, model, T):
    lat = sw.Lattice(L, q, MODEL[model], T, 31, init=sw.SW_INIT_RANDOM)
    sw.sw_set_debug_limits(lat.h, 0, list_cap)
    o = Oracle(L, q, model, T, 31, init="random")
    lockstep(lat, o, 6)
    lat.close()
    o.close()


def test_union_list_overflow_on_the_union_heavy_colouring():
    """The stripe colouring at T -> 0 (every 32 x 32 quadrant makes 225
    further pairs) with a list of 16 pairs per tile."""
    from test_gpu_parity import stripes32
    L = 128
    spins = np.tile(stripes32(), (L // 32, L // 32))
    lat = sw.Lattice(L, 3, sw.SW_POTTS, 1e-3, 4, init=None)
    lat.spins = spins
    o = Oracle(L, 3, POTTS, 1e-3, 4, init="random")
    o.spins = spins
    sw.sw_set_debug_limits(lat.h, 0, 16)
    lockstep(lat, o, 3)
    lat.close()
    o.close()


def test_loop_cap_reports_not_converged_and_stays_sticky():
    L, T = 512, 0.5 * tc(2)   # ordered: one cluster spans every tile, walks need several steps
    lat = sw.Lattice(L, 2, sw.SW_POTTS, T, 5, init=sw.SW_INIT_RANDOM)
    sw.sw_set_debug_limits(lat.h, 1, 0)
    with pytest.raises(sw.SwError) as err:
        lat.sweep(3)
        sw.sw_synchronize(lat.h)
    assert err.value.code == sw.SW_ERR_NOT_CONVERGED
    for call in (lambda: lat.sweep(1), lat.measure, lambda: sw.sw_synchronize(lat.h)):
        with pytest.raises(sw.SwError) as again:
            call()
        assert again.value.code == sw.SW_ERR_NOT_CONVERGED
    lat.close()
    # The device and a fresh handle are unaffected.
    lat = sw.Lattice(64, 2, sw.SW_POTTS, tc(2), 6, init=sw.SW_INIT_RANDOM)
    o = Oracle(64, 2, POTTS, tc(2), 6, init="random")
    lockstep(lat, o, 4)
    lat.close()
    o.close()


def test_debug_limits_reject_negative_values():
    lat = sw.Lattice(8, 2, sw.SW_POTTS, 1.0, 1)
    with pytest.raises(sw.SwError):
        sw.sw_set_debug_limits(lat.h, -1, 0)
    with pytest.raises(sw.SwError):
        sw.sw_set_debug_limits(lat.h, 0, -3)
    sw.sw_set_debug_limits(lat.h, 0, 0)
    lat.close()
