"""Temperature scans on the GPU engine (Komura & Okabe, arXiv:1202.0635,
Sec. 4): the moment ratio U(T) = <M^4>/<M^2>^2 of several sizes (Eq. U; the
crossing of the curves marks the critical point, Fig. 4), with jackknife
errors of U and of the crossing temperature, the time per spin flip against
T with its per-stage split (Figs. 3 and 5), the labeling statistics against
T (the counterpart of the paper's count of labeling passes), the
correlation ratio R(T) = G(L/2)/G(L/4) of the clock model (Fig. 6), and the
time per spin flip over the paper's grid of models and sizes, with and
without the measurement (the two rows of its timing tables).

Every (L, T) point is its own lattice; all of them advance together in one
batch (one launch sequence per sweep), so a scan costs about as much as
its largest lattice.

    python -m paper_1202_0635_gb300.studies --q 2 --L 32 64 128 --sweeps 4000
"""
import argparse
import importlib
import json
import math

import numpy as np

from . import workloads


def _sw():
    return importlib.import_module(__package__)


def temperatures(q, model, lo=0.9, hi=1.1, n=9):
    """n temperatures evenly spaced in [lo, hi] * T_c."""
    tc = workloads.critical_temperature(q, model)
    return [tc * (lo + (hi - lo) * k / (n - 1)) for k in range(n)]


def scan(q, model, sizes, temps, sweeps, equil=200, seed=1):
    """Running means of every (L, T) lattice after `equil` discarded sweeps
    and `sweeps` measured ones: list of dicts (L, T, e, m2, m4, U, clusters,
    and for the clock model G(L/4), G(L/2), R)."""
    sw = _sw()
    b = sw.Batch()
    try:
        points = []
        for i, L in enumerate(sizes):
            for j, T in enumerate(temps):
                lat = b.add(L, q, model, T, seed + 1000 * i + j, init=sw.SW_INIT_RANDOM)
                points.append((L, T, lat))
        sw.sw_batch_set_graph(b.b, 1)
        b.sweep(equil)
        for _, _, lat in points:
            sw.sw_reset_stats(lat.h)
        b.sweep(sweeps)
        out = []
        for L, T, lat in points:
            o = lat.measure()
            row = {"L": L, "T": T, "sweeps": int(o.nmeas), "e": o.mean_e, "m2": o.mean_m2, "m4": o.mean_m4,
                   "U": o.binder_u, "clusters": o.mean_clusters}
            if model == sw.SW_CLOCK:
                row.update({"g_quarter": o.mean_g_quarter, "g_half": o.mean_g_half, "R": o.corr_ratio})
            out.append(row)
        return out
    finally:
        b.close()


def m2_of_counts(counts, L, q):
    """Per-sweep m^2 = M^2 / N^2 of the Potts model from the state counts
    n_k (columns 0 .. q-1 of the counter rows), M^2 = (q sum n_k^2 - N^2) /
    (q - 1) (Sec. 4, Eq. M^2)."""
    n = np.asarray(counts, dtype=np.float64)[:, :q]
    N = float(L) * float(L)
    return (q * (n * n).sum(axis=1) - N * N) / (q - 1) / (N * N)


def binder_scan(q, sizes, temps, sweeps, equil=500, seed=1, nbins=20):
    """Potts moment ratio U = <m^4>/<m^2>^2 (Eq. U; m^4 = (m^2)^2) of every
    (L, T) lattice with the per-sweep values kept: dict (L, T) -> array of
    per-bin means of (m^2, m^4), nbins bins of the measured sweeps."""
    sw = _sw()
    b = sw.Batch()
    try:
        lats = {}
        for i, L in enumerate(sizes):
            for j, T in enumerate(temps):
                lats[(L, T)] = b.add(L, q, sw.SW_POTTS, T, seed + 1000 * i + j, init=sw.SW_INIT_RANDOM)
        sw.sw_batch_set_graph(b.b, 1)
        b.sweep(equil)
        for lat in lats.values():
            lat.measure()
            sw.sw_set_record(lat.h, 1)
        b.sweep(sweeps)
        out = {}
        for (L, T), lat in lats.items():
            m2 = m2_of_counts(lat.take_counts(sweeps + 1), L, q)
            m = len(m2) // nbins * nbins
            out[(L, T)] = np.stack([m2[:m].reshape(nbins, -1).mean(axis=1),
                                    (m2[:m] ** 2).reshape(nbins, -1).mean(axis=1)], axis=1)
        return out
    finally:
        b.close()


def binder_crossing(bins, small, large, temps):
    """Crossing temperature of U(T) of two sizes and its jackknife error
    (leave one bin out of every lattice's series): (T, sigma_T) or (None, None)."""
    def crossing_of(sel):
        rows = []
        for L in (small, large):
            for T in temps:
                b = bins[(L, T)][sel]
                m2, m4 = b[:, 0].mean(), b[:, 1].mean()
                rows.append({"L": L, "T": T, "U": m4 / (m2 * m2)})
        return crossing(rows, "U", small, large)
    nb = next(iter(bins.values())).shape[0]
    full = crossing_of(np.arange(nb))
    if full is None:
        return None, None
    jk = [crossing_of(np.delete(np.arange(nb), k)) for k in range(nb)]
    if any(t is None for t in jk):
        return full, None
    jk = np.array(jk)
    return full, float(math.sqrt((nb - 1) / nb * ((jk - jk.mean()) ** 2).sum()))


def labeling_vs_T(q, model, L, temps, sweeps=50, equil=100, seed=1):
    """Labeling statistics of one lattice at each T (sw_get_labeling_stats):
    tile components, provisional labels and union pairs per tile, unions
    across tile edges, and the walks of the global union-find."""
    sw = _sw()
    out = []
    for T in temps:
        lat = sw.Lattice(L, q, model, T, seed, init=sw.SW_INIT_RANDOM)
        try:
            sw.sw_set_graph(lat.h, 1)
            lat.sweep(equil)
            sw.sw_set_labeling_stats(lat.h, 1)
            lat.sweep(sweeps)
            row = {"T": T}
            row.update(sw.sw_get_labeling_stats(lat.h))
            out.append(row)
        finally:
            lat.close()
    return out


def crossing(rows, key, small, large):
    """Temperature where key(T) of two sizes cross, by linear interpolation
    between the scanned temperatures that bracket the sign change of
    key(large) - key(small); None if the curves do not cross."""
    a = sorted((r["T"], r[key]) for r in rows if r["L"] == small)
    c = sorted((r["T"], r[key]) for r in rows if r["L"] == large)
    diff = [(ta, vc - va) for (ta, va), (tc, vc) in zip(a, c)]
    for (t0, d0), (t1, d1) in zip(diff, diff[1:]):
        if d0 == 0.0:
            return t0
        if d0 * d1 < 0.0:
            return t0 + (t1 - t0) * d0 / (d0 - d1)
    return None


def timing(q, model, L, temps, sweeps=20, equil=50, seed=1):
    """Per-stage device time per spin flip (ns) of one lattice at each T,
    CUDA events around every kernel of direct-launched sweeps."""
    sw = _sw()
    stages = ["bonds", "label", "merge", "flip"]
    out = []
    for T in temps:
        lat = sw.Lattice(L, q, model, T, seed, init=sw.SW_INIT_RANDOM)
        try:
            lat.sweep(equil)
            ms = sw.sw_profile_sweeps(lat.h, sweeps)
        finally:
            lat.close()
        per = {name: ms[k] * 1e6 / (L * L) for k, name in enumerate(stages)}
        out.append({"T": T, "ns_per_flip": sum(per.values()), "stages_ns_per_flip": per})
    return out


def sweep_time(L, q, model, T, measure, sweeps=200, equil=100, seed=1):
    """Device time per spin flip (ns) of graph-launched sweeps of one
    lattice: CUDA events on the lattice's stream around `sweeps` sweeps,
    after `equil` sweeps from a random start."""
    import torch
    sw = _sw()
    s = torch.cuda.Stream()
    lat = sw.Lattice(L, q, model, T, seed, init=sw.SW_INIT_RANDOM, stream=s.cuda_stream)
    try:
        sw.sw_set_measure(lat.h, measure)
        sw.sw_set_graph(lat.h, 1)
        lat.sweep(equil)
        sw.sw_synchronize(lat.h)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        lat.sweep(sweeps)
        e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e6 / sweeps / (L * L)
    finally:
        lat.close()


def timing_matrix(sizes=(1024, 2048, 4096), sweeps=200, equil=100):
    """ns per spin flip, update only and with measurement: Potts q = 2, 3, 4
    at T_c for each size, and the q = 6 clock model at L = max(sizes) and
    T = 0.7, 0.9, 1.2 (below, at and above the upper KT temperature)."""
    sw = _sw()
    rows = []
    for q in (2, 3, 4):
        T = workloads.critical_temperature(q, sw.SW_POTTS)
        for L in sizes:
            rows.append({"model": "potts", "q": q, "L": L, "T": T,
                         "update_only": sweep_time(L, q, sw.SW_POTTS, T, 0, sweeps, equil),
                         "with_measurement": sweep_time(L, q, sw.SW_POTTS, T, 1, sweeps, equil)})
    L = max(sizes)
    for T in (0.7, 0.9, 1.2):
        rows.append({"model": "clock", "q": 6, "L": L, "T": T,
                     "update_only": sweep_time(L, 6, sw.SW_CLOCK, T, 0, sweeps, equil),
                     "with_measurement": sweep_time(L, 6, sw.SW_CLOCK, T, 1, sweeps, equil)})
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--q", type=int, default=2)
    ap.add_argument("--model", choices=["potts", "clock"], default="potts")
    ap.add_argument("--L", type=int, nargs="+", default=[32, 64, 128])
    ap.add_argument("--sweeps", type=int, default=4000)
    ap.add_argument("--equil", type=int, default=500)
    ap.add_argument("--lo", type=float, default=0.9)
    ap.add_argument("--hi", type=float, default=1.1)
    ap.add_argument("--n", type=int, default=9)
    ap.add_argument("--timing-L", type=int, default=1024)
    ap.add_argument("--matrix", action="store_true", help="only the ns/flip grid of models and sizes")
    ap.add_argument("--labeling", action="store_true",
                    help="only the labeling statistics against T at --timing-L (Potts q = 2, 3; clock q = 6)")
    args = ap.parse_args()
    sw = _sw()
    sw.lib()
    if args.matrix:
        print(json.dumps({"ns_per_flip": timing_matrix()}))
        return
    if args.labeling:
        res = {}
        for name, q, model in (("potts_q2", 2, sw.SW_POTTS), ("potts_q3", 3, sw.SW_POTTS), ("clock_q6", 6, sw.SW_CLOCK)):
            res[name] = labeling_vs_T(q, model, args.timing_L, temperatures(q, model, 0.7, 1.3, 7))
        print(json.dumps({"L": args.timing_L, "labeling": res}))
        return
    model = sw.SW_CLOCK if args.model == "clock" else sw.SW_POTTS
    temps = temperatures(args.q, model, args.lo, args.hi, args.n)
    rows = scan(args.q, model, args.L, temps, args.sweeps, args.equil)
    key = "R" if model == sw.SW_CLOCK else "U"
    cross = {"%d-%d" % (a, c): crossing(rows, key, a, c) for a, c in zip(args.L, args.L[1:])}
    print(json.dumps({"q": args.q, "model": args.model, "T_c": workloads.critical_temperature(args.q, model),
                      "points": rows, "crossings_" + key: cross,
                      "timing_L%d" % args.timing_L: timing(args.q, model, args.timing_L, temps)}))


if __name__ == "__main__":
    main()
