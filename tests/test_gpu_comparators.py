"""The paper's own GPU labelings (Sec. 3: Hawick et al.'s label equivalence,
Kalentev et al.'s refinement) as comparators (needs a GB300).  They end at
the same canonical labels as the tiled labeling, so the chains must be
identical: spins after every sweep and the labels themselves."""
import math

import numpy as np
import pytest

import paper_1202_0635_gb300 as sw

pytestmark = pytest.mark.gpu

METHODS = [sw.SW_LABEL_HAWICK, sw.SW_LABEL_KALENTEV]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1202_0635_gb300 import build
    build.build()
    sw.lib()


def tc(q):
    return 1.0 / math.log(1.0 + math.sqrt(q))


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("L,q,model,T", [(64, 2, sw.SW_POTTS, tc(2)), (100, 3, sw.SW_POTTS, tc(3)),
                                         (96, 6, sw.SW_CLOCK, 0.9), (36, 2, sw.SW_ISING, 2.269),
                                         (1024, 2, sw.SW_POTTS, tc(2)), (64, 4, sw.SW_POTTS, 0.3)])
def test_comparator_chain_equals_tiled(method, L, q, model, T):
    a = sw.Lattice(L, q, model, T, 77, init=sw.SW_INIT_RANDOM)
    b = sw.Lattice(L, q, model, T, 77, init=sw.SW_INIT_RANDOM)
    sw.sw_set_measure(a.h, 0)
    sw.sw_set_debug_labels(a.h, 1)
    sw.sw_set_measure(b.h, 0)
    sw.sw_set_labeling(b.h, method)
    for k in range(4):
        a.sweep(1)
        b.sweep(1)
        assert np.array_equal(a.spins, b.spins), "spins differ after sweep %d" % (k + 1)
        assert np.array_equal(a.labels, b.labels), "labels differ after sweep %d" % (k + 1)
        assert sw.sw_label_passes(b.h) >= 1
    assert a.sweep_index == b.sweep_index == 4
    a.close()
    b.close()


def test_comparators_are_update_only_and_stay_out_of_batches():
    g = sw.Lattice(32, 2, sw.SW_POTTS, 1.0, 1)
    with pytest.raises(sw.SwError) as e:
        sw.sw_set_labeling(g.h, sw.SW_LABEL_KALENTEV)     # measurement is on
    assert e.value.code == sw.SW_ERR_STATE
    sw.sw_set_measure(g.h, 0)
    sw.sw_set_labeling(g.h, sw.SW_LABEL_KALENTEV)
    with pytest.raises(sw.SwError):
        sw.sw_set_measure(g.h, 1)
    bt = sw.Batch()
    with pytest.raises(sw.SwError):
        sw.sw_batch_attach(bt.b, g.h)
    bt.close()
    g.close()


def test_switching_back_keeps_the_counters_right():
    """Comparator sweeps leave the counter ring as the tiled sweeps do."""
    L, q, T = 128, 3, tc(3)
    a = sw.Lattice(L, q, sw.SW_POTTS, T, 5, init=sw.SW_INIT_RANDOM)
    b = sw.Lattice(L, q, sw.SW_POTTS, T, 5, init=sw.SW_INIT_RANDOM)
    for g in (a, b):
        sw.sw_set_measure(g.h, 0)
    sw.sw_set_labeling(b.h, sw.SW_LABEL_HAWICK)
    a.sweep(5)
    b.sweep(5)
    sw.sw_set_labeling(b.h, sw.SW_LABEL_TILED)
    for g in (a, b):
        sw.sw_set_measure(g.h, 1)
        sw.sw_set_record(g.h, 1)
        g.sweep(3)
    assert np.array_equal(a.take_counts(), b.take_counts())
    assert np.array_equal(a.spins, b.spins)
    a.close()
    b.close()
