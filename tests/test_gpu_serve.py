"""The served path on the GPU: jobs that overlap in one batch give the same
spins and observables as each job run alone (needs a GB300)."""
import numpy as np
import pytest

import paper_1202_0635_gb300 as sw
from paper_1202_0635_gb300 import serve, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1202_0635_gb300 import build
    build.build()
    sw.lib()


class FakeClock:
    def __init__(self, dt=0.002):
        self.t = 0.0
        self.dt = dt

    def __call__(self):
        self.t += self.dt
        return self.t


def test_results_alone_equal_results_in_the_mix():
    jobs = workloads.served_jobs(24, rate=200.0, seed=11, sweep_scale=0.02)
    for j in jobs:
        j["L"] = min(j["L"], 256)
    be = serve.GpuBackend()
    srv = serve.Server(be, budget_bytes=4e9, max_chunk=8)
    srv.run(jobs, clock=FakeClock(), realtime=False)
    be.shutdown()
    assert srv.peak_resident > 1
    for j in jobs:
        mixed = srv.results[j["id"]]
        h = sw.sw_create(j["L"], j["q"], j["model"], j["T"], j["seed"])
        sw.sw_init(h, sw.SW_INIT_RANDOM)
        sw.sw_sweep(h, j["sweeps"])
        o = sw.sw_measure(h)
        spins = sw.sw_get_spins(h, j["L"] * j["L"])
        sw.sw_destroy(h)
        assert mixed["sweeps"] == j["sweeps"] == int(o.sweep)
        assert np.array_equal(mixed["spins"], spins)
        for k in ("mean_e", "mean_absm", "mean_m2", "mean_m4", "binder_u"):
            assert mixed[k] == getattr(o, k), k
