"""Continuous-batching server for Swendsen-Wang simulation jobs.

A job asks for `sweeps` Swendsen-Wang sweeps (Komura & Okabe,
arXiv:1202.0635: Potts Sec. 2, clock Sec. 4) of one lattice (q, model, L,
T, seed) from a random start, and gets back its running-mean observables
(energy, magnetisation moments, moment ratio U of Eq. U) and final spins.

Jobs are admitted first-come-first-served while their device memory fits
the HBM budget; admitted lattices stay resident and are advanced together
by one batched launch sequence per sweep (sw_batch).  Every lattice carries
its job's sweep budget on the device (sw_set_sweep_limit), so every engine
step advances all resident jobs by a full chunk of sweeps and a job whose
budget runs out within the chunk simply stops there; a job that arrives
while others run joins the next step and finished jobs leave after it
(continuous batching).  Membership changes rewrite the batch's device
descriptors without recapturing its CUDA graph.  A job's chain depends only
on its own parameters and seed, so its result is the same alone and in any
mix.

    python -m paper_1202_0635_gb300.serve [--jobs 1000] [--rate 200] [--budget-gb 120]
"""
import argparse
import collections
import importlib
import json
import time

import numpy as np

from . import workloads


def job_bytes(L, q, model):
    """Device bytes one resident lattice holds: spins int8 and codes uint16
    per site; per 64 x 64 tile its bond masks (1 KB), open-component entries
    (256 x 8 B), edge bytes, open count and crossing words; the counter ring,
    the clock threshold table and the descriptors.  (Labels are allocated
    only for debug labels, which the server does not use.)"""
    n = L * L
    tiles = ((L + 63) // 64) ** 2
    nclass = q // 2 + 1 if model == 1 else 2
    ring = 1024 * (q + nclass + 2 + (2 * nclass if model == 1 else 0)) * 8
    table = (2 * q) ** 2 * 4 if model == 1 else 0
    return n * (1 + 2) + tiles * (1024 + 256 * 8 + 128 + 4 + 16) + ring + table + 4096


class GpuBackend:
    """Resident lattices in one sw_batch on the current CUDA device."""

    def __init__(self, stream=None, graph=True):
        sw = importlib.import_module(__package__)
        self.sw = sw
        self.b = sw.sw_batch_create(stream)
        sw.sw_batch_set_graph(self.b, graph)

    def open(self, job):
        sw = self.sw
        h = sw.sw_create(job["L"], job["q"], job["model"], job["T"], job["seed"])
        sw.sw_init(h, sw.SW_INIT_RANDOM)
        sw.sw_set_sweep_limit(h, int(job["sweeps"]))
        sw.sw_batch_attach(self.b, h)
        return h

    def advance(self, k):
        self.sw.sw_batch_sweep(self.b, k)

    def result(self, h, L):
        o = self.sw.sw_measure(h)
        return {"sweeps": int(o.sweep), "nmeas": int(o.nmeas), "mean_e": o.mean_e, "mean_absm": o.mean_absm,
                "mean_m2": o.mean_m2, "mean_m4": o.mean_m4, "binder_u": o.binder_u,
                "spins": self.sw.sw_get_spins(h, L * L)}

    def close(self, h):
        self.sw.sw_batch_detach(self.b, h)
        self.sw.sw_destroy(h)

    def shutdown(self):
        if self.b:
            self.sw.sw_batch_destroy(self.b)
            self.b = None


class Server:
    """First-come-first-served admission under an HBM budget, continuous
    batching of every resident job."""

    def __init__(self, backend, budget_bytes=120e9, max_chunk=16):
        self.backend = backend
        self.budget = float(budget_bytes)
        self.max_chunk = int(max_chunk)
        self.pending = collections.deque()
        self.active = {}          # job id -> [job, handle, remaining, bytes]
        self.used = 0.0
        self.results = {}
        self.steps = 0
        self.sweeps_done = 0
        self.peak_resident = 0
        self.peak_used = 0.0

    def submit(self, job):
        need = job_bytes(job["L"], job["q"], job["model"])
        if need > self.budget:
            raise ValueError("job %r needs %.3g bytes, more than the whole budget" % (job["id"], need))
        self.pending.append(job)

    def admit(self, now):
        """Admit arrived jobs in arrival order while the budget holds."""
        admitted = 0
        while self.pending and self.pending[0]["arrival"] <= now:
            job = self.pending[0]
            need = job_bytes(job["L"], job["q"], job["model"])
            if self.used + need > self.budget:
                break
            self.pending.popleft()
            h = self.backend.open(job)
            self.active[job["id"]] = [job, h, int(job["sweeps"]), need]
            self.used += need
            admitted += 1
        self.peak_resident = max(self.peak_resident, len(self.active))
        self.peak_used = max(self.peak_used, self.used)
        return admitted

    def chunk(self):
        """Sweeps for the next engine step: max_chunk, or fewer when every
        resident job needs fewer (jobs stop at their own budget on the
        device)."""
        if not self.active:
            return 0
        return max(1, min(self.max_chunk, max(a[2] for a in self.active.values())))

    def step(self, now_fn):
        """Admit, advance every resident job, retire the finished ones."""
        self.admit(now_fn())
        k = self.chunk()
        if k == 0:
            return 0
        self.backend.advance(k)
        self.steps += 1
        finished = []
        for jid, a in self.active.items():
            done = min(k, a[2])
            self.sweeps_done += done
            a[2] -= done
            if a[2] == 0:
                finished.append(jid)
        for jid in finished:
            job, h, _, need = self.active.pop(jid)
            res = self.backend.result(h, job["L"])
            res["completed"] = now_fn()
            res["latency"] = res["completed"] - job["arrival"]
            self.results[jid] = res
            self.backend.close(h)
            self.used -= need
        return k

    def run(self, jobs, clock=None, realtime=True):
        """Serve every job; arrivals are seconds after the start.  With
        realtime=False the clock jumps to the next arrival when idle."""
        for j in sorted(jobs, key=lambda j: j["arrival"]):
            self.submit(j)
        t0 = time.perf_counter()
        offset = [0.0]

        def now():
            return (time.perf_counter() - t0) + offset[0] if clock is None else clock()

        while self.pending or self.active:
            if not self.active and self.pending and self.pending[0]["arrival"] > now():
                wait = self.pending[0]["arrival"] - now()
                if realtime and clock is None:
                    time.sleep(min(wait, 0.05))
                else:
                    offset[0] += wait
                continue
            self.step(now)
        return time.perf_counter() - t0


def summary(jobs, results, makespan):
    lat = np.array([results[j["id"]]["latency"] for j in jobs])
    flips = float(sum(j["L"] * j["L"] * j["sweeps"] for j in jobs))
    return {"jobs": len(jobs), "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "max_latency_s": float(lat.max()),
            "makespan_s": makespan, "flips": flips, "flips_per_s": flips / makespan}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=1000)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--sweep-scale", type=float, default=1.0)
    ap.add_argument("--max-chunk", type=int, default=16)
    args = ap.parse_args()
    importlib.import_module(__package__).lib()
    jobs = workloads.served_jobs(args.jobs, rate=args.rate, seed=7, sweep_scale=args.sweep_scale)
    backend = GpuBackend()
    srv = Server(backend, budget_bytes=args.budget_gb * 1e9, max_chunk=args.max_chunk)
    makespan = srv.run(jobs)
    backend.shutdown()
    out = summary(jobs, srv.results, makespan)
    out.update({"rate_per_s": args.rate, "budget_gb": args.budget_gb, "sweep_scale": args.sweep_scale,
                "engine_steps": srv.steps, "peak_resident_jobs": srv.peak_resident})
    print(json.dumps(out))


if __name__ == "__main__":
    main()
