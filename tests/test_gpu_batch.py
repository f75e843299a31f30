"""Batched sweeps through the C ABI (needs a GB300): every lattice of a
batch of mixed sizes, models and temperatures follows exactly the chain it
follows alone, and the oracle's."""
import math

import numpy as np
import pytest

import paper_1202_0635_gb300 as sw
from oracle import CLOCK, ISING, POTTS, Oracle

pytestmark = pytest.mark.gpu

MODEL = {POTTS: sw.SW_POTTS, CLOCK: sw.SW_CLOCK, ISING: sw.SW_ISING}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1202_0635_gb300 import build
    build.build()
    sw.lib()


def mixed_replicas(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n):
        kind = rng.integers(0, 3)
        L = int(rng.choice([8, 32, 36, 64, 100, 128, 264]))
        if kind == 0:
            q, model, Tc = 2, POTTS, 1.0 / math.log(1.0 + math.sqrt(2.0))
        elif kind == 1:
            q, model, Tc = 3, POTTS, 1.0 / math.log(1.0 + math.sqrt(3.0))
        else:
            q, model, Tc = 6, CLOCK, 0.9
        out.append((L, q, model, Tc * rng.uniform(0.8, 1.2), 1000 + r))
    return out


@pytest.mark.parametrize("graph", [False, True])
def test_batch_equals_plain_and_oracle(graph):
    reps = mixed_replicas(12, 3)
    b = sw.Batch()
    sw.sw_batch_set_graph(b.b, graph)
    lats = [b.add(L, q, MODEL[m], T, s, init=sw.SW_INIT_RANDOM) for (L, q, m, T, s) in reps]
    for lat in lats:
        sw.sw_set_record(lat.h, 1)
    refs = [Oracle(L, q, m, T, s, init="random") for (L, q, m, T, s) in reps]
    for step in range(6):
        b.sweep(3)
        for (L, q, m, T, s), lat, ref in zip(reps, lats, refs):
            rec = ref.sweep(3, record=True)
            assert np.array_equal(lat.spins, ref.spins), (L, q, m, step)
            assert np.array_equal(lat.take_counts(), rec), (L, q, m, step)
    alone = []
    for (L, q, m, T, s) in reps:
        a = sw.Lattice(L, q, MODEL[m], T, s, init=sw.SW_INIT_RANDOM)
        a.sweep(18)
        alone.append(a.spins.copy())
        a.close()
    for lat, sp in zip(lats, alone):
        assert np.array_equal(lat.spins, sp)
    b.close()


def test_attach_detach_mid_run_keeps_each_chain():
    """Lattices join and leave a running batch (the serving pattern)."""
    Tc = 1.0 / math.log(1.0 + math.sqrt(2.0))
    b = sw.Batch()
    x = b.add(64, 2, sw.SW_POTTS, Tc, 1, init=sw.SW_INIT_RANDOM)
    y = b.add(36, 3, sw.SW_POTTS, 0.9, 2, init=sw.SW_INIT_RANDOM)
    b.sweep(5)
    z = b.add(100, 6, sw.SW_CLOCK, 0.9, 3, init=sw.SW_INIT_RANDOM)
    b.sweep(4)
    b.remove(y)
    b.sweep(3)
    ox = Oracle(64, 2, POTTS, Tc, 1, init="random"); ox.sweep(12)
    oy = Oracle(36, 3, POTTS, 0.9, 2, init="random"); oy.sweep(9)
    oz = Oracle(100, 6, CLOCK, 0.9, 3, init="random"); oz.sweep(7)
    assert np.array_equal(x.spins, ox.spins)
    assert np.array_equal(y.spins, oy.spins)
    assert np.array_equal(z.spins, oz.spins)
    y.sweep(2)   # a detached lattice keeps working alone
    oy.sweep(2)
    assert np.array_equal(y.spins, oy.spins)
    y.close()
    b.close()


def test_graph_rebuilt_when_the_lattice_count_changes():
    """Four 64^2 lattices and one 128^2 lattice have the same tile and merge
    item counts; swapping one set for the other under a captured graph must
    still sweep the new set correctly."""
    Tc = 1.0 / math.log(1.0 + math.sqrt(2.0))
    b = sw.Batch()
    sw.sw_batch_set_graph(b.b, 1)
    small = [b.add(64, 2, sw.SW_POTTS, Tc, 10 + i, init=sw.SW_INIT_RANDOM) for i in range(4)]
    b.sweep(3)
    for lat in small:
        b.remove(lat)
        lat.close()
    big = b.add(128, 2, sw.SW_POTTS, Tc, 20, init=sw.SW_INIT_RANDOM)
    b.sweep(3)
    o = Oracle(128, 2, POTTS, Tc, 20, init="random")
    o.sweep(3)
    assert np.array_equal(big.spins, o.spins)
    o.close()
    b.close()


def test_batch_measure_off_and_labels():
    Tc = 1.0 / math.log(1.0 + math.sqrt(3.0))
    b = sw.Batch()
    sw.sw_batch_set_debug_labels(b.b, 1)
    lats = [b.add(L, 3, sw.SW_POTTS, Tc, 7 + L, init=sw.SW_INIT_RANDOM) for L in (32, 68, 96)]
    refs = [Oracle(L, 3, POTTS, Tc, 7 + L, init="random") for L in (32, 68, 96)]
    b.sweep(2)
    for lat, ref in zip(lats, refs):
        ref.sweep(2)
        assert np.array_equal(lat.labels, ref.labels)
    sw.sw_batch_set_measure(b.b, 0)
    b.sweep(5)
    for lat, ref in zip(lats, refs):
        ref.sweep(5)
        assert np.array_equal(lat.spins, ref.spins)
        assert lat.measure().nmeas == 2
    b.close()


def test_launch_shapes_never_change_results():
    Tc = 1.0 / math.log(1.0 + math.sqrt(2.0))
    ref = None
    for shape in ([8, 16, 16, 16], [1, 1, 1, 1], [4, 32, 8, 4], [6, 3, 64, 2]):
        lat = sw.Lattice(200, 2, sw.SW_POTTS, Tc, 9, init=sw.SW_INIT_RANDOM)
        sw.sw_set_launch_shape(lat.h, shape)
        sw.sw_set_record(lat.h, 1)
        lat.sweep(10)
        got = (lat.spins.copy(), lat.take_counts())
        lat.close()
        if ref is None:
            ref = got
        else:
            assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), shape


def test_autotune_picks_a_cached_shape_and_keeps_the_chain():
    Tc = 1.0 / math.log(1.0 + math.sqrt(3.0))
    lat = sw.Lattice(256, 3, sw.SW_POTTS, Tc, 4, init=sw.SW_INIT_RANDOM)
    shape = sw.sw_autotune(lat.h, 2)
    assert all(1 <= v <= 64 for v in shape)
    t = lat.sweep_index
    # Every candidate ran real sweeps: labeling 3, merge 4, flip 4 (a Potts
    # sweep launches no bond kernel, so its figure is not tuned).
    assert t == 2 * (3 + 4 + 4)
    o = Oracle(256, 3, POTTS, Tc, 4, init="random")
    o.sweep(t)
    assert np.array_equal(lat.spins, o.spins)
    again = sw.Lattice(256, 3, sw.SW_POTTS, Tc, 5, init=sw.SW_INIT_RANDOM)
    assert sw.sw_autotune(again.h, 2) == shape   # cached: no sweeps
    assert again.sweep_index == 0
    lat.close()
    again.close()
    clk = sw.Lattice(128, 6, sw.SW_CLOCK, 0.9, 6, init=sw.SW_INIT_RANDOM)
    sw.sw_autotune(clk.h, 1)
    assert clk.sweep_index == 3 + 4 + 4 + 4   # a clock sweep's bond kernel is tuned as well
    clk.close()
    b = sw.Batch()
    for L in (32, 96, 160):
        b.add(L, 2, sw.SW_POTTS, 1.0 / math.log(1.0 + math.sqrt(2.0)), L, init=sw.SW_INIT_RANDOM)
    bshape = sw.sw_batch_autotune(b.b, 1)
    assert all(1 <= v <= 64 for v in bshape)
    b.close()


def test_sweep_limits_stop_lattices_inside_a_captured_batch():
    """Lattices with sweep limits 5, 9 and none advanced by one graph-launched
    batch equal plain lattices swept 5, 9 and 12 times (spins and counter
    rows); a lattice that joins after 7 sweeps with a limit of 3 does 3.  The
    batch's captured sweep stays valid across the join."""
    specs = [(64, 2, sw.SW_POTTS, 1.0 / math.log(1.0 + math.sqrt(2.0)), 5),
             (100, 3, sw.SW_POTTS, 1.0 / math.log(1.0 + math.sqrt(3.0)), 9),
             (48, 6, sw.SW_CLOCK, 0.9, None)]
    b = sw.Batch()
    sw.sw_batch_set_graph(b.b, 1)
    lats = []
    for i, (L, q, model, T, lim) in enumerate(specs):
        lat = b.add(L, q, model, T, 300 + i, init=sw.SW_INIT_RANDOM)
        if lim is not None:
            sw.sw_set_sweep_limit(lat.h, lim)
        sw.sw_set_record(lat.h, 1)
        lats.append((lat, L, q, model, T, 300 + i, lim if lim is not None else 12))
    b.sweep(7)
    late = b.add(76, 4, sw.SW_POTTS, 1.0 / math.log(3.0), 399, init=sw.SW_INIT_RANDOM)
    sw.sw_set_sweep_limit(late.h, 3)
    sw.sw_set_record(late.h, 1)
    lats.append((late, 76, 4, sw.SW_POTTS, 1.0 / math.log(3.0), 399, 3))
    b.sweep(5)
    for lat, L, q, model, T, seed, want in lats:
        assert lat.sweep_index == want
        ref = sw.Lattice(L, q, model, T, seed, init=sw.SW_INIT_RANDOM)
        sw.sw_set_record(ref.h, 1)
        ref.sweep(want)
        assert np.array_equal(lat.spins, ref.spins)
        assert np.array_equal(lat.take_counts(), ref.take_counts())
        ref.close()
    assert sw.sw_get_sweep_limit(late.h) == 3
    b.close()
