"""GPU <-> oracle parity through the C ABI (needs a GB300).

Spins, canonical labels and integer counters must agree bit-exactly after
every sweep; FP64 running means to 1e-12 relative.  Sizes span several
64 x 32 tiles with ragged tails (L not a multiple of the tile), the
periodic wrap, single-tile lattices, every model, and the full 4096^2
benchmark lattice in the benchmark's launch configuration (CUDA graph,
measurement on).
"""
import math

import numpy as np
import pytest

import paper_1202_0635_gb300 as sw
from oracle import CLOCK, ISING, POTTS, Oracle, correlations, observables

pytestmark = pytest.mark.gpu

MODEL = {POTTS: sw.SW_POTTS, CLOCK: sw.SW_CLOCK, ISING: sw.SW_ISING}
TC_ISING = 2.0 / math.log(1.0 + math.sqrt(2.0))


def tc_potts(q):
    return 1.0 / math.log(1.0 + math.sqrt(q))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1202_0635_gb300 import build
    build.build()
    sw.lib()


def make_pair(L, q, model, T, seed, init):
    g = sw.Lattice(L, q, MODEL[model], T, seed, init=sw.SW_INIT_RANDOM if init == "random" else sw.SW_INIT_UP)
    o = Oracle(L, q, model, T, seed, init=init)
    return g, o


def run_lockstep(L, q, model, T, seed, init, n, graph=False, labels=True, every=1, spins=None):
    g, o = make_pair(L, q, model, T, seed, init)
    if spins is not None:
        g.spins = spins
        o.spins = spins
    assert np.array_equal(g.spins, o.spins), "initial spins"
    sw.sw_set_graph(g.h, graph)
    sw.sw_set_debug_labels(g.h, labels)
    sw.sw_set_record(g.h, 1)
    rows = []
    done = 0
    while done < n:
        k = min(every, n - done)
        g.sweep(k)
        rec = o.sweep(k, record=True)
        rows.append(rec)
        done += k
        assert np.array_equal(g.spins, o.spins), "spins differ after sweep %d" % done
        if labels:
            assert np.array_equal(g.labels, o.labels), "labels differ after sweep %d" % done
        got = g.take_counts()
        assert np.array_equal(got, rec), "counters differ after sweep %d" % done
    rows = np.concatenate(rows)
    obs = g.measure()
    assert obs.sweep == n and obs.nmeas == n
    ref = observables(L, q, model, rows)
    for k, name in enumerate(("mean_e", "mean_absm", "mean_m2", "mean_m4")):
        want = 0.0
        for v in ref[:, k]:
            want += v
        want /= n
        assert abs(getattr(obs, name) - want) <= 1e-12 * max(1.0, abs(want)), name
    if model == CLOCK:   # correlations at L/4 and L/2 (Sec. 4) and their ratio R
        gref = correlations(L, q, rows)
        want4, want2 = gref[:, 0].mean(), gref[:, 1].mean()
        assert abs(obs.mean_g_quarter - want4) <= 1e-12 * max(1.0, abs(want4))
        assert abs(obs.mean_g_half - want2) <= 1e-12 * max(1.0, abs(want2))
        if want4 != 0.0:
            assert abs(obs.corr_ratio - want2 / want4) <= 1e-9 * max(1.0, abs(want2 / want4))
        assert np.allclose([obs.g_quarter, obs.g_half], gref[-1], rtol=1e-12, atol=1e-15)
    g.close()
    return rows


def test_config_ising_L64_200_sweeps_from_all_up():
    """Ising q = 2, L = 64, T = 2/ln(1+sqrt 2), all-up start, seed 1, 200 sweeps."""
    run_lockstep(64, 2, ISING, TC_ISING, 1, "up", 200)


@pytest.mark.parametrize("L", [4, 8, 12, 28, 60, 64, 68, 100, 132, 256])
@pytest.mark.parametrize("q", [2, 3, 4])
def test_potts_critical(L, q):
    run_lockstep(L, q, POTTS, tc_potts(q), 7 + q, "random", 25)


@pytest.mark.parametrize("L", [8, 36, 96, 128])
@pytest.mark.parametrize("q,T", [(6, 0.7), (6, 0.9), (6, 1.2), (4, 0.8), (5, 0.9), (3, 0.6), (8, 0.5),
                                 (16, 0.3), (64, 0.2)])
def test_clock(L, q, T):
    run_lockstep(L, q, CLOCK, T, 99, "random", 25)


@pytest.mark.parametrize("q,T", [(2, 1e-3), (3, 1e9), (127, 0.3), (2, 0.05)])
def test_potts_extremes(q, T):
    """Frozen (T -> 0: one cluster), infinite T (no bonds), q = 127."""
    run_lockstep(64, q, POTTS, T, 5, "random", 12)


def stripes32():
    """A 32 x 32 Potts colouring (q >= 3) on which, with every equal pair
    bonded (T -> 0), each even row is one run joining the 16 separate
    single-site runs of the row above: 15 union requests per even row,
    225 per 32 x 32 block, the most found by a search over colourings."""
    s = np.empty((32, 32), np.int8)
    s[0] = 2
    for r in range(1, 32):
        m = ((r - 1) // 2) % 2
        if r % 2:
            s[r, 0::2] = m
            s[r, 1::2] = 2 if r == 1 else 1 - m
        else:
            s[r] = m
    return s


@pytest.mark.parametrize("L", [128, 200])
def test_union_heavy_colouring(L):
    """Every 32 x 32 block of the lattice (the warp quadrants of the tile
    labeling) carries the stripe colouring: the heaviest union load."""
    reps = (L + 31) // 32
    spins = np.tile(stripes32(), (reps, reps))[:L, :L]
    run_lockstep(L, 3, POTTS, 1e-3, 4, "random", 3, spins=spins)


def test_graph_mode_matches_direct_launches():
    run_lockstep(200, 3, POTTS, tc_potts(3), 3, "random", 40, graph=True, every=7)
    run_lockstep(120, 6, CLOCK, 0.9, 3, "random", 40, graph=True, every=5)


@pytest.mark.parametrize("model,q,T", [(ISING, 2, TC_ISING), (POTTS, 4, tc_potts(4)), (POTTS, 12, tc_potts(12)),
                                       (CLOCK, 6, 0.9), (CLOCK, 16, 0.5)])
def test_update_only_mode_keeps_the_chain(model, q, T):
    """Measurement off: the spin writes compiled without state counts."""
    g, o = make_pair(96, q, model, T, 11, "random")
    sw.sw_set_measure(g.h, 0)
    g.sweep(30)
    o.sweep(30)
    assert np.array_equal(g.spins, o.spins)
    assert g.measure().nmeas == 0
    g.close()


def test_checkpoint_resume_is_bit_exact():
    """Spins + sweep index + parameters resume the chain exactly."""
    L, q, T = 128, 3, tc_potts(3)
    a = sw.Lattice(L, q, sw.SW_POTTS, T, 77, init=sw.SW_INIT_RANDOM)
    a.sweep(40)
    straight = a.spins.copy()
    b = sw.Lattice(L, q, sw.SW_POTTS, T, 77, init=sw.SW_INIT_RANDOM)
    b.sweep(20)
    saved, t = b.spins.copy(), b.sweep_index
    b.close()
    c = sw.Lattice(L, q, sw.SW_POTTS, T, 77, init=None)
    c.spins = saved
    c.sweep_index = t
    c.sweep(20)
    assert np.array_equal(c.spins, straight)
    a.close()
    c.close()


@pytest.mark.parametrize("model,q,T", [(POTTS, 3, tc_potts(3)), (ISING, 2, TC_ISING), (CLOCK, 6, 0.9)])
def test_spins_and_sweep_index_set_between_sweeps(model, q, T):
    """Spins set between sweeps (the bond stage reads whatever spins it
    finds) and a sweep index set between sweeps (it positions the random
    stream) keep a captured chain equal to the oracle's."""
    L = 100
    g, o = make_pair(L, q, model, T, 31, "random")
    sw.sw_set_graph(g.h, 1)
    g.sweep(3)
    o.sweep(3)
    s = np.random.default_rng(5).integers(0, q, size=(L, L), dtype=np.int8)
    g.spins = s
    o.spins = s
    g.sweep(2)
    o.sweep(2)
    assert np.array_equal(g.spins, o.spins), "after spins were set"
    g.sweep_index = 40
    o.sweep_index = 40
    g.sweep(2)
    o.sweep(2)
    assert np.array_equal(g.spins, o.spins), "after the sweep index was set"
    g.close()
    o.close()


def test_ring_drain_over_many_sweeps():
    """More sweeps than the device counter ring holds (drained mid-call)."""
    L, n = 16, 2600
    g, o = make_pair(L, 2, ISING, TC_ISING, 5, "random")
    sw.sw_set_graph(g.h, 1)
    sw.sw_set_record(g.h, 1)
    g.sweep(n)
    rec = o.sweep(n, record=True)
    assert np.array_equal(g.take_counts(), rec)
    assert np.array_equal(g.spins, o.spins)
    g.close()


def test_set_spins_rejects_out_of_range_states():
    g = sw.Lattice(8, 3, sw.SW_POTTS, 1.0, 1)
    bad = np.zeros(64, dtype=np.int8)
    bad[5] = 3
    with pytest.raises(sw.SwError):
        g.spins = bad
    g.close()


def test_thresholds_equal_the_oracle():
    for model, q, T in ((POTTS, 3, 0.995), (ISING, 2, 2.269), (CLOCK, 6, 0.9), (CLOCK, 5, 1.3)):
        g, o = make_pair(8, q, model, T, 1, "up")
        assert np.array_equal(g.thresholds(), o.thresholds())
        g.close()


@pytest.mark.parametrize("q,model,T", [(2, POTTS, tc_potts(2)), (6, CLOCK, 0.9)])
def test_full_size_4096_in_benchmark_configuration(q, model, T):
    """The benchmark lattice (4096^2, random start, graph launch, measurement
    on): two sweeps bit-exact against the full oracle."""
    run_lockstep(4096, q, model, T, 1, "random", 2, graph=True, labels=False)
