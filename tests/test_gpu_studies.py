"""Physics of the GPU engine beyond the oracle's sizes (needs a GB300): the
moment ratio U of Eq. (U) for L = 64 and 128 crosses at the exact critical
point T_c = 1/ln(1 + sqrt q) of the Potts model (Sec. 4, Fig. 4), within the
crossing's own jackknife error; the labeling statistics against T."""
import pytest

import paper_1202_0635_gb300 as sw
from paper_1202_0635_gb300 import studies, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1202_0635_gb300 import build
    build.build()
    sw.lib()


@pytest.mark.parametrize("q", [2, 3])
def test_binder_crossing_of_64_and_128_is_the_potts_critical_point(q):
    """U(T) of L = 64 and 128 from 20000 sweeps per point: the first crossing
    scanning up in T lies within four jackknife errors (leave one of 20 bins
    out) of the exact T_c, plus 0.1 pct of T_c for the crossing's own
    finite-size shift at these sizes, and the scan pins T_c to half a pct."""
    tc = workloads.critical_temperature(q, workloads.POTTS)
    temps = [tc * (0.97 + 0.0075 * k) for k in range(9)]
    bins = studies.binder_scan(q, [64, 128], temps, sweeps=20000, equil=1000, nbins=20)
    t, sig = studies.binder_crossing(bins, 64, 128, temps)
    assert t is not None and sig is not None
    assert abs(t - tc) <= 4.0 * sig + 1e-3 * tc, (t, sig, tc)
    assert sig < 5e-3 * tc, (t, sig, tc)
    # Ordered side: U of the larger lattice is closer to 1.
    u = {L: bins[(L, temps[0])][:, 1].mean() / bins[(L, temps[0])][:, 0].mean() ** 2 for L in (64, 128)}
    assert u[128] < u[64]


def test_timing_matrix_covers_the_grid():
    """The ns/flip grid: Potts q = 2, 3, 4 at T_c for every size, clock q = 6
    at three temperatures, each update only and with measurement."""
    rows = studies.timing_matrix(sizes=(128, 256), sweeps=4, equil=4)
    assert len(rows) == 3 * 2 + 3
    assert {(r["model"], r["q"]) for r in rows} == {("potts", 2), ("potts", 3), ("potts", 4), ("clock", 6)}
    for r in rows:
        assert r["update_only"] > 0.0 and r["with_measurement"] > 0.0


def test_labeling_statistics_against_temperature():
    """The open components per tile fall below T_c, where one cluster spans
    the lattice, and the tile components grow towards high T."""
    tc = workloads.critical_temperature(2, workloads.POTTS)
    rows = studies.labeling_vs_T(2, sw.SW_POTTS, 256, [0.7 * tc, tc, 1.3 * tc], sweeps=5, equil=20)
    assert [r["sweeps"] for r in rows] == [5, 5, 5]
    comps = [r["components_per_tile"] for r in rows]
    assert comps[0] < comps[1] < comps[2]
    assert rows[0]["open_per_tile"] < rows[2]["open_per_tile"]
