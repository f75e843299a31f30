"""Seeded synthetic workloads shaped like the paper's (Komura & Okabe,
arXiv:1202.0635, Sec. 4: lattices up to 4096^2 at or near the critical
temperature).  Only parameters and seeds are generated here; nothing in
this module computes any part of the Swendsen-Wang method.
"""
import math

import numpy as np

POTTS, CLOCK, ISING = 0, 1, 2


def critical_temperature(q, model):
    """Potts: T_c = 1/ln(1 + sqrt q) (J = 1); Ising units: 2/ln(1 + sqrt 2);
    q = 6 clock: 0.9, the upper KT temperature the paper times at."""
    if model == ISING:
        return 2.0 / math.log(1.0 + math.sqrt(2.0))
    if model == CLOCK:
        return 0.9
    return 1.0 / math.log(1.0 + math.sqrt(q))


def batched_replicas(n=256, seed=1):
    """Independent replicas: L uniform in {32, ..., 1024}, model uniform in
    {q=2 Potts, q=3 Potts, q=6 clock}, T = T_c * U(0.8, 1.2), seed 1000 + r."""
    rng = np.random.default_rng(seed)
    sizes = [32, 64, 128, 256, 512, 1024]
    kinds = [(2, POTTS), (3, POTTS), (6, CLOCK)]
    out = []
    for r in range(n):
        L = int(sizes[rng.integers(0, len(sizes))])
        q, model = kinds[rng.integers(0, len(kinds))]
        T = critical_temperature(q, model) * float(rng.uniform(0.8, 1.2))
        out.append({"L": L, "q": q, "model": model, "T": T, "seed": 1000 + r})
    return out


def served_jobs(n=1000, rate=200.0, seed=7, sweep_scale=1.0):
    """Poisson(rate) arrivals of jobs (q in {2, 4 Potts, 6 clock}, L
    log-uniform in [64, 4096] rounded to a multiple of 4, T = T_c * U(0.9,
    1.1), sweeps uniform in {100..2000} (times sweep_scale), seed = job id)."""
    rng = np.random.default_rng(seed)
    kinds = [(2, POTTS), (4, POTTS), (6, CLOCK)]
    t = 0.0
    jobs = []
    for j in range(n):
        t += float(rng.exponential(1.0 / rate))
        q, model = kinds[rng.integers(0, len(kinds))]
        L = int(round(math.exp(rng.uniform(math.log(64), math.log(4096))) / 4.0)) * 4
        L = max(64, min(4096, L))
        T = critical_temperature(q, model) * float(rng.uniform(0.9, 1.1))
        sweeps = max(1, int(round(int(rng.integers(100, 2001)) * sweep_scale)))
        jobs.append({"id": j, "arrival": t, "q": q, "model": model, "L": L, "T": T, "sweeps": sweeps, "seed": j})
    return jobs
