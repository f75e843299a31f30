"""Host logic of the continuous-batching server, on the CPU: the oracle
stands in for the GPU lattices (test infrastructure)."""
import math

import numpy as np
import pytest

from oracle import Oracle, observables
from paper_1202_0635_gb300 import serve, workloads


class OracleBackend:
    def __init__(self):
        self.rows = {}
        self.live = []
        self.opened = []

    def open(self, job):
        o = Oracle(job["L"], job["q"], job["model"], job["T"], job["seed"], init="random")
        self.rows[id(o)] = []
        self.limit = getattr(self, "limit", {})
        self.limit[id(o)] = int(job["sweeps"])   # the device's per-lattice sweep limit
        self.live.append(o)
        self.opened.append(job["id"])
        return o

    def advance(self, k):
        for o in self.live:
            n = min(k, self.limit[id(o)] - o.sweep_index)
            if n > 0:
                self.rows[id(o)].append(o.sweep(n, record=True))

    def result(self, o, L):
        rows = np.concatenate(self.rows[id(o)])
        obs = observables(o.L, o.q, o.model, rows)
        return {"sweeps": o.sweep_index, "nmeas": rows.shape[0], "mean_e": float(obs[:, 0].mean()),
                "mean_m2": float(obs[:, 2].mean()), "spins": o.spins.reshape(-1).copy()}

    def close(self, o):
        self.live.remove(o)
        o.close()


def small_jobs(n, seed=3):
    rng = np.random.default_rng(seed)
    jobs = []
    t = 0.0
    for j in range(n):
        t += float(rng.exponential(0.01))
        q, model = [(2, 0), (3, 0), (6, 1)][rng.integers(0, 3)]
        L = int(rng.choice([8, 12, 16, 24]))
        jobs.append({"id": j, "arrival": t, "q": q, "model": model, "L": L,
                     "T": workloads.critical_temperature(q, model), "sweeps": int(rng.integers(3, 40)), "seed": 50 + j})
    return jobs


class FakeClock:
    def __init__(self, dt=0.004):
        self.t = 0.0
        self.dt = dt

    def __call__(self):
        self.t += self.dt
        return self.t


def test_every_job_runs_exactly_its_sweeps_and_matches_running_alone():
    jobs = small_jobs(14)
    be = OracleBackend()
    srv = serve.Server(be, budget_bytes=1e12, max_chunk=8)
    srv.run(jobs, clock=FakeClock(), realtime=False)
    assert set(srv.results) == {j["id"] for j in jobs}
    assert srv.peak_resident > 1            # jobs really overlapped
    for j in jobs:
        r = srv.results[j["id"]]
        assert r["sweeps"] == j["sweeps"] and r["nmeas"] == j["sweeps"]
        alone = Oracle(j["L"], j["q"], j["model"], j["T"], j["seed"], init="random")
        rows = alone.sweep(j["sweeps"], record=True)
        obs = observables(j["L"], j["q"], j["model"], rows)
        assert np.array_equal(alone.spins.reshape(-1), r["spins"])
        assert r["mean_e"] == pytest.approx(float(obs[:, 0].mean()), rel=1e-12, abs=1e-15)
        assert r["latency"] >= 0


def test_budget_limits_residency_and_admission_is_first_come_first_served():
    jobs = small_jobs(10, seed=8)
    per = max(serve.job_bytes(j["L"], j["q"], j["model"]) for j in jobs)
    be = OracleBackend()
    srv = serve.Server(be, budget_bytes=2 * per, max_chunk=4)
    srv.run(jobs, clock=FakeClock(), realtime=False)
    assert srv.peak_used <= 2 * per
    assert srv.peak_resident < len(jobs)
    assert be.opened == [j["id"] for j in sorted(jobs, key=lambda j: j["arrival"])]
    assert len(srv.results) == len(jobs)


def test_chunk_never_overshoots_a_job():
    be = OracleBackend()
    srv = serve.Server(be, budget_bytes=1e12, max_chunk=16)
    jobs = [{"id": 0, "arrival": 0.0, "q": 2, "model": 0, "L": 8, "T": 1.0, "sweeps": 5, "seed": 1},
            {"id": 1, "arrival": 0.0, "q": 2, "model": 0, "L": 8, "T": 1.0, "sweeps": 37, "seed": 2}]
    srv.run(jobs, clock=FakeClock(), realtime=False)
    assert srv.results[0]["sweeps"] == 5 and srv.results[1]["sweeps"] == 37


def test_oversized_job_is_rejected():
    srv = serve.Server(OracleBackend(), budget_bytes=1000)
    with pytest.raises(ValueError):
        srv.submit({"id": 0, "arrival": 0.0, "q": 2, "model": 0, "L": 64, "T": 1.0, "sweeps": 1, "seed": 0})


def test_workload_recipes_are_seeded_and_shaped():
    a = workloads.served_jobs(50, seed=7)
    b = workloads.served_jobs(50, seed=7)
    assert a == b
    assert all(64 <= j["L"] <= 4096 and j["L"] % 4 == 0 for j in a)
    assert all(100 <= j["sweeps"] <= 2000 for j in a)
    arr = [j["arrival"] for j in a]
    assert arr == sorted(arr)
    reps = workloads.batched_replicas(256, seed=1)
    assert len(reps) == 256 and {r["L"] for r in reps} <= {32, 64, 128, 256, 512, 1024}
    sites = sum(r["L"] ** 2 for r in reps)
    assert 3e7 < sites < 1e8
    assert workloads.critical_temperature(2, 2) == pytest.approx(2.0 / math.log(1.0 + math.sqrt(2.0)))
