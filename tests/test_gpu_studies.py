"""Physics of the GPU engine beyond the oracle's sizes (needs a GB300): the
moment ratio U of Eq. (U) for L = 32 and 64 crosses at the exact critical
point T_c = 1/ln(1 + sqrt q) of the Potts model (Sec. 4, Fig. 3)."""
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
def test_binder_curves_cross_at_the_potts_critical_point(q):
    temps = studies.temperatures(q, workloads.POTTS, 0.9, 1.1, 9)
    rows = studies.scan(q, sw.SW_POTTS, [32, 64], temps, sweeps=6000, equil=300)
    tc = workloads.critical_temperature(q, workloads.POTTS)
    # Ordered side: U of the larger lattice is closer to 1.
    lo = {r["L"]: r["U"] for r in rows if r["T"] == temps[0]}
    assert lo[64] < lo[32]
    if q == 2:   # the Ising limit U = 3 is approached from below above T_c
        hi = {r["L"]: r["U"] for r in rows if r["T"] == temps[-1]}
        assert hi[64] > hi[32]
    # The first crossing scanning up in T is the critical point.  (For q = 3
    # the disordered limit U = 2 is approached from above, so the curves
    # cross once more further above T_c.)
    t = studies.crossing(rows, "U", 32, 64)
    assert t is not None and abs(t - tc) < 0.03 * tc, (t, tc)


def test_timing_matrix_covers_the_grid():
    """The ns/flip grid: Potts q = 2, 3, 4 at T_c for every size, clock q = 6
    at three temperatures, each update only and with measurement."""
    rows = studies.timing_matrix(sizes=(128, 256), sweeps=4, equil=4)
    assert len(rows) == 3 * 2 + 3
    assert {(r["model"], r["q"]) for r in rows} == {("potts", 2), ("potts", 3), ("potts", 4), ("clock", 6)}
    for r in rows:
        assert r["update_only"] > 0.0 and r["with_measurement"] > 0.0
