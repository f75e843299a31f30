"""ctypes wrapper around the C oracle (test infrastructure only).

Every method is a thin call into sw_oracle.c; the arithmetic lives there.
"""
import ctypes
import os

import numpy as np

from . import build as _build

POTTS, CLOCK, ISING = 0, 1, 2

_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    lib = ctypes.CDLL(path)
    c_u32p = ctypes.POINTER(ctypes.c_uint32)
    c_i64p = ctypes.POINTER(ctypes.c_int64)
    c_i8p = ctypes.POINTER(ctypes.c_int8)
    lib.swo_philox4x32_10.argtypes = [c_u32p, c_u32p, c_u32p]
    lib.swo_threshold_from_x.argtypes = [ctypes.c_double]
    lib.swo_threshold_from_x.restype = ctypes.c_uint32
    lib.swo_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint64]
    lib.swo_create.restype = ctypes.c_void_p
    lib.swo_destroy.argtypes = [ctypes.c_void_p]
    lib.swo_thresholds.argtypes = [ctypes.c_void_p, c_u32p, ctypes.c_int]
    lib.swo_thresholds.restype = ctypes.c_int
    for name in ("swo_init_up", "swo_init_random"):
        getattr(lib, name).argtypes = [ctypes.c_void_p]
    lib.swo_set_spins.argtypes = [ctypes.c_void_p, c_i8p]
    lib.swo_get_spins.argtypes = [ctypes.c_void_p, c_i8p]
    lib.swo_get_labels.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]
    lib.swo_get_bonds.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint8)]
    lib.swo_get_sweep.argtypes = [ctypes.c_void_p]
    lib.swo_get_sweep.restype = ctypes.c_uint64
    lib.swo_set_sweep.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    lib.swo_last_axis.argtypes = [ctypes.c_void_p]
    lib.swo_last_axis.restype = ctypes.c_int
    lib.swo_ncounters.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.swo_ncounters.restype = ctypes.c_int
    lib.swo_sweep.argtypes = [ctypes.c_void_p, ctypes.c_int, c_i64p]
    lib.swo_counts.argtypes = [ctypes.c_void_p, c_i64p]
    lib.swo_correlations.argtypes = [ctypes.c_int, ctypes.c_int, c_i64p, ctypes.POINTER(ctypes.c_double)]
    lib.swo_observables.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, c_i64p,
                                    ctypes.POINTER(ctypes.c_double)]
    lib.swo_sample_one_step.argtypes = [ctypes.c_void_p, c_i8p, ctypes.c_uint64, ctypes.c_int, c_i8p]
    lib.swo_label_bonds.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint8), ctypes.c_int64,
                                    ctypes.POINTER(ctypes.c_int32)]
    _lib = lib
    return lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def philox4x32_10(ctr, key):
    """Philox-4x32-10 of one 4-word counter under a 2-word key."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.swo_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def threshold_from_x(x):
    return int(_load().swo_threshold_from_x(float(x)))


def ncounters(q, model):
    return int(_load().swo_ncounters(int(q), int(model)))


def observables(L, q, model, counts):
    """{E/N, |m|, m^2, m^4} from one counter row (or an array of rows)."""
    lib = _load()
    c = np.ascontiguousarray(counts, dtype=np.int64)
    if c.ndim == 1:
        out = np.zeros(4, dtype=np.float64)
        lib.swo_observables(int(L), int(q), int(model), _ptr(c, ctypes.c_int64), _ptr(out, ctypes.c_double))
        return out
    out = np.zeros((c.shape[0], 4), dtype=np.float64)
    for r in range(c.shape[0]):
        row = np.ascontiguousarray(c[r])
        o = np.zeros(4, dtype=np.float64)
        lib.swo_observables(int(L), int(q), int(model), _ptr(row, ctypes.c_int64), _ptr(o, ctypes.c_double))
        out[r] = o
    return out


def correlations(L, q, counts):
    """Clock model: {G(L/4), G(L/2)} from one counter row (or an array of rows)."""
    lib = _load()
    c = np.ascontiguousarray(counts, dtype=np.int64)
    rows = c[None, :] if c.ndim == 1 else c
    out = np.zeros((rows.shape[0], 2), dtype=np.float64)
    for r in range(rows.shape[0]):
        row = np.ascontiguousarray(rows[r])
        o = np.zeros(2, dtype=np.float64)
        lib.swo_correlations(int(L), int(q), _ptr(row, ctypes.c_int64), _ptr(o, ctypes.c_double))
        out[r] = o
    return out[0] if c.ndim == 1 else out


class Oracle:
    """One periodic L x L lattice advanced by the CPU Swendsen-Wang sweep."""

    def __init__(self, L, q, model, T, seed, init="up"):
        self.lib = _load()
        self.L, self.q, self.model, self.T, self.seed = int(L), int(q), int(model), float(T), int(seed)
        self.N = self.L * self.L
        self.h = self.lib.swo_create(self.L, self.q, self.model, self.T, ctypes.c_uint64(self.seed))
        if not self.h:
            raise ValueError("swo_create rejected L=%d q=%d model=%d T=%r" % (L, q, model, T))
        self.nc = ncounters(q, model)
        if init == "up":
            self.lib.swo_init_up(self.h)
        elif init == "random":
            self.lib.swo_init_random(self.h)
        else:
            raise ValueError(init)

    def close(self):
        if self.h:
            self.lib.swo_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def thresholds(self):
        n = 4 * self.q * self.q if self.model == CLOCK else 1
        out = np.zeros(n, dtype=np.uint32)
        self.lib.swo_thresholds(self.h, _ptr(out, ctypes.c_uint32), n)
        return out

    def sweep(self, n=1, record=False):
        """Run n sweeps; with record=True return the (n, ncounters) int64 rows."""
        if record:
            out = np.zeros((n, self.nc), dtype=np.int64)
            self.lib.swo_sweep(self.h, int(n), _ptr(out, ctypes.c_int64))
            return out
        self.lib.swo_sweep(self.h, int(n), None)
        return None

    def counts(self):
        out = np.zeros(self.nc, dtype=np.int64)
        self.lib.swo_counts(self.h, _ptr(out, ctypes.c_int64))
        return out

    @property
    def spins(self):
        s = np.zeros(self.N, dtype=np.int8)
        self.lib.swo_get_spins(self.h, _ptr(s, ctypes.c_int8))
        return s.reshape(self.L, self.L)

    @spins.setter
    def spins(self, s):
        a = np.ascontiguousarray(np.asarray(s, dtype=np.int8).reshape(-1))
        if a.size != self.N:
            raise ValueError("expected %d spins" % self.N)
        self.lib.swo_set_spins(self.h, _ptr(a, ctypes.c_int8))

    @property
    def labels(self):
        s = np.zeros(self.N, dtype=np.int32)
        self.lib.swo_get_labels(self.h, _ptr(s, ctypes.c_int32))
        return s.reshape(self.L, self.L)

    @property
    def bonds(self):
        s = np.zeros(self.N, dtype=np.uint8)
        self.lib.swo_get_bonds(self.h, _ptr(s, ctypes.c_uint8))
        return s.reshape(self.L, self.L)

    @property
    def sweep_index(self):
        return int(self.lib.swo_get_sweep(self.h))

    @sweep_index.setter
    def sweep_index(self, t):
        self.lib.swo_set_sweep(self.h, ctypes.c_uint64(int(t)))

    @property
    def axis(self):
        return int(self.lib.swo_last_axis(self.h))

    def observables(self, counts=None):
        return observables(self.L, self.q, self.model, self.counts() if counts is None else counts)

    def label_bonds(self, bonds):
        """Canonical labels of given bond sets, shape (nsets, N) uint8 -> (nsets, N) int32."""
        b = np.ascontiguousarray(np.asarray(bonds, dtype=np.uint8).reshape(-1, self.N))
        out = np.zeros(b.shape, dtype=np.int32)
        self.lib.swo_label_bonds(self.h, _ptr(b, ctypes.c_uint8), ctypes.c_int64(b.shape[0]),
                                 _ptr(out, ctypes.c_int32))
        return out

    def sample_one_step(self, sigma, t0, M):
        """M one-sweep successors of sigma, at sweep indices t0 .. t0+M-1."""
        s = np.ascontiguousarray(np.asarray(sigma, dtype=np.int8).reshape(-1))
        out = np.zeros((M, self.N), dtype=np.int8)
        self.lib.swo_sample_one_step(self.h, _ptr(s, ctypes.c_int8), ctypes.c_uint64(int(t0)), int(M),
                                     _ptr(out, ctypes.c_int8))
        return out
