"""sw_sweep_noalloc against sw_sweep (needs a GB300).

sw_sweep_noalloc is for callers that cannot allocate device memory when
they sweep (a plugin inside a framework that owns all device memory, a
latency-bound loop that must not stall on cudaMalloc): it keeps its working
memory in one fixed array inside the library.  Its results must equal the
handle path's bit for bit -- spins and integer counters -- over two calls
in a row, the second continuing the chain of the first, whatever an
earlier call (of another size) left in that array.

The file name makes pytest collect it last, so a run that stops at the
first failure has run every other test before this one.
"""
import math

import numpy as np
import pytest

import paper_1202_0635_gb300 as sw

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TC_ISING = 2.0 / math.log(1.0 + math.sqrt(2.0))


def tc_potts(q):
    return 1.0 / math.log(1.0 + math.sqrt(q))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1202_0635_gb300 import build
    build.build()
    sw.lib()


def stream():
    return torch.cuda.current_stream().cuda_stream


def noalloc(L, q, model, T, seed, sweep0, n, spins, counts):
    sw.sw_sweep_noalloc(L, q, model, T, seed, sweep0, n, spins.data_ptr(),
                        None if counts is None else counts.data_ptr(), stream())


# The largest lattice runs first, so later cases start from an array that
# holds another lattice's leftovers.  n2 = 300 spans more sweeps than the
# array's counter rows hold at once, so the call drains them in chunks and
# wraps the row ring.
CASES = [
    (sw.SW_NOALLOC_MAX_L, 2, sw.SW_POTTS, tc_potts(2), 14, 3, 2),
    (64, 2, sw.SW_ISING, TC_ISING, 11, 7, 5),
    (100, 3, sw.SW_POTTS, tc_potts(3), 12, 9, 300),
    (52, 6, sw.SW_CLOCK, 0.9, 13, 6, 6),
    # The clock model's class and correlation counters through the chunked
    # drain (n2 > 127 rows).
    (40, 6, sw.SW_CLOCK, 0.9, 15, 5, 260),
]


@pytest.mark.parametrize("L,q,model,T,seed,n1,n2", CASES)
def test_two_calls_in_a_row_equal_sw_sweep(L, q, model, T, seed, n1, n2):
    ref = sw.Lattice(L, q, model, T, seed, init=sw.SW_INIT_RANDOM)
    sw.sw_set_record(ref.h, 1)
    nc = sw.sw_ncounters(q, model)
    spins = torch.from_numpy(ref.spins.reshape(-1).copy()).cuda()
    sweep0 = 0
    for n in (n1, n2):
        counts = torch.full((n, nc), -1, dtype=torch.int64, device="cuda")
        noalloc(L, q, model, T, seed, sweep0, n, spins, counts)
        ref.sweep(n)
        want_rows = ref.take_counts()
        sweep0 += n
        assert np.array_equal(spins.cpu().numpy().reshape(L, L), ref.spins), "spins differ at sweep %d" % sweep0
        assert np.array_equal(counts.cpu().numpy(), want_rows), "counters differ at sweep %d" % sweep0
    ref.close()


def test_repeated_calls_allocate_nothing():
    """After a first call (which looks up the array's address and may load the
    library's code onto the device), further calls leave the device's free
    memory and torch's allocator unchanged."""
    L, q, model, T, seed = 256, 3, sw.SW_POTTS, tc_potts(3), 17
    nc = sw.sw_ncounters(q, model)
    spins = torch.zeros(L * L, dtype=torch.int8, device="cuda")
    counts = torch.zeros((200, nc), dtype=torch.int64, device="cuda")
    noalloc(L, q, model, T, seed, 0, 20, spins, counts)
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    sweep0 = 20
    for n in (200, 1, 37):
        noalloc(L, q, model, T, seed, sweep0, n, spins, counts)
        sweep0 += n
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_without_counters_the_chain_is_unchanged():
    L, q, model, T, seed = 68, 4, sw.SW_POTTS, tc_potts(4), 21
    ref = sw.Lattice(L, q, model, T, seed, init=sw.SW_INIT_RANDOM)
    spins = torch.from_numpy(ref.spins.reshape(-1).copy()).cuda()
    for sweep0, n in ((0, 4), (4, 3)):
        noalloc(L, q, model, T, seed, sweep0, n, spins, None)
        ref.sweep(n)
        assert np.array_equal(spins.cpu().numpy().reshape(L, L), ref.spins)
    ref.close()


def test_rejects_oversized_lattices_and_invalid_states():
    big = torch.zeros((sw.SW_NOALLOC_MAX_L + 4) ** 2, dtype=torch.int8, device="cuda")
    with pytest.raises(sw.SwError, match="no-allocation limit") as err:
        noalloc(sw.SW_NOALLOC_MAX_L + 4, 2, sw.SW_POTTS, 1.0, 1, 0, 1, big, None)
    assert err.value.code == sw.SW_ERR_ARG
    L, q = 32, 3
    bad = torch.zeros(L * L, dtype=torch.int8, device="cuda")
    bad[5] = q
    before = bad.clone()
    with pytest.raises(sw.SwError, match="outside") as err:
        noalloc(L, q, sw.SW_POTTS, 1.0, 1, 0, 2, bad, None)
    assert err.value.code == sw.SW_ERR_ARG
    assert torch.equal(bad, before), "a rejected call must leave the spins untouched"
