"""GB300 Swendsen-Wang sweep library: thin ctypes binding of include/sw.h.

Every function below has the name of the C entry point it marshals
arguments for; all work happens in libsw_gb300.so (CUDA kernels for
sm_103a).  There is no CPU fallback: importing the binding without the
built library raises.

Komura & Okabe, arXiv:1202.0635: Potts (Sec. 2, Eq. 1) and clock (Sec. 4)
models on periodic L x L lattices, Swendsen-Wang multi-cluster sweeps.
"""
import ctypes
import os

import numpy as np

from .build import LIB as _LIB_PATH

SW_POTTS, SW_CLOCK, SW_ISING = 0, 1, 2
SW_OK, SW_ERR_ARG, SW_ERR_OOM, SW_ERR_CUDA, SW_ERR_NOT_CONVERGED, SW_ERR_STATE = 0, -1, -2, -3, -4, -5
SW_INIT_UP, SW_INIT_RANDOM = 0, 1
SW_LABEL_TILED, SW_LABEL_HAWICK, SW_LABEL_KALENTEV = 0, 1, 2
SW_MAX_Q = 127
SW_MAX_CLOCK_Q = 64
SW_MAX_COUNTERS = SW_MAX_Q + SW_MAX_Q // 2 + 1 + 2
SW_NOALLOC_MAX_L = 1024
SW_NOALLOC_SCRATCH_BYTES = 7 * 1024 * 1024


class SwError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("sw error %d: %s" % (code, msg))
        self.code = code


class sw_obs(ctypes.Structure):
    _fields_ = [
        ("sweep", ctypes.c_uint64),
        ("L", ctypes.c_int32), ("q", ctypes.c_int32), ("model", ctypes.c_int32), ("ncounters", ctypes.c_int32),
        ("counts", ctypes.c_int64 * SW_MAX_COUNTERS),
        ("e", ctypes.c_double), ("absm", ctypes.c_double), ("m2", ctypes.c_double), ("m4", ctypes.c_double),
        ("nmeas", ctypes.c_uint64),
        ("mean_e", ctypes.c_double), ("mean_e2", ctypes.c_double), ("mean_absm", ctypes.c_double),
        ("mean_m2", ctypes.c_double), ("mean_m4", ctypes.c_double),
        ("binder_u", ctypes.c_double),
        ("mean_active", ctypes.c_double), ("mean_clusters", ctypes.c_double),
        ("g_quarter", ctypes.c_double), ("g_half", ctypes.c_double), ("mean_g_quarter", ctypes.c_double),
        ("mean_g_half", ctypes.c_double), ("corr_ratio", ctypes.c_double),
    ]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "counts"}
        d["counts"] = list(self.counts[: self.ncounters])
        return d


_lib = None

# (name, restype, argtypes) of every exported entry point, as declared in include/sw.h.
_H = ctypes.c_void_p
EXPORTS = [
    ("sw_ncounters", ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    ("sw_create", _H, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint64]),
    ("sw_create_ext", _H, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("sw_destroy", ctypes.c_int, [_H]),
    ("sw_last_error", ctypes.c_char_p, []),
    ("sw_init", ctypes.c_int, [_H, ctypes.c_int]),
    ("sw_sweep", ctypes.c_int, [_H, ctypes.c_int]),
    ("sw_measure", ctypes.c_int, [_H, ctypes.POINTER(sw_obs)]),
    ("sw_synchronize", ctypes.c_int, [_H]),
    ("sw_set_measure", ctypes.c_int, [_H, ctypes.c_int]),
    ("sw_set_record", ctypes.c_int, [_H, ctypes.c_int]),
    ("sw_take_counts", ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int64), ctypes.c_int]),
    ("sw_reset_stats", ctypes.c_int, [_H]),
    ("sw_set_debug_labels", ctypes.c_int, [_H, ctypes.c_int]),
    ("sw_get_spins", ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int8), ctypes.c_size_t]),
    ("sw_set_spins", ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int8), ctypes.c_size_t]),
    ("sw_get_labels", ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int32), ctypes.c_size_t]),
    ("sw_device_spins", ctypes.c_void_p, [_H]),
    ("sw_device_labels", ctypes.c_void_p, [_H]),
    ("sw_get_thresholds", ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_uint32), ctypes.c_int]),
    ("sw_get_sweep", ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_uint64)]),
    ("sw_set_sweep", ctypes.c_int, [_H, ctypes.c_uint64]),
    ("sw_set_labeling", ctypes.c_int, [_H, ctypes.c_int]),
    ("sw_label_passes", ctypes.c_int, [_H]),
    ("sw_set_stream", ctypes.c_int, [_H, ctypes.c_void_p]),
    ("sw_set_graph", ctypes.c_int, [_H, ctypes.c_int]),
    ("sw_profile_sweeps", ctypes.c_int, [_H, ctypes.c_int, ctypes.POINTER(ctypes.c_float), ctypes.c_int]),
    ("sw_autotune", ctypes.c_int, [_H, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("sw_set_launch_shape", ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int)]),
    ("sw_set_debug_limits", ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int]),
    ("sw_set_sweep_limit", ctypes.c_int, [_H, ctypes.c_uint64]),
    ("sw_get_sweep_limit", ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_uint64)]),
    ("sw_set_labeling_stats", ctypes.c_int, [_H, ctypes.c_int]),
    ("sw_get_labeling_stats", ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    ("sw_batch_create", ctypes.c_void_p, [ctypes.c_void_p]),
    ("sw_batch_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("sw_batch_attach", ctypes.c_int, [ctypes.c_void_p, _H]),
    ("sw_batch_detach", ctypes.c_int, [ctypes.c_void_p, _H]),
    ("sw_batch_size", ctypes.c_int, [ctypes.c_void_p]),
    ("sw_batch_sweep", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("sw_batch_synchronize", ctypes.c_int, [ctypes.c_void_p]),
    ("sw_batch_set_measure", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("sw_batch_set_graph", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("sw_batch_set_debug_labels", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("sw_batch_profile_sweeps", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                               ctypes.c_int]),
    ("sw_batch_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("sw_batch_set_launch_shape", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    ("sw_sweep_noalloc", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                        ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]),
]


def lib():
    """The loaded CUDA library.  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError("libsw_gb300.so is not built (%s); run __graft_entry__.build()" % _LIB_PATH)
    L = ctypes.CDLL(_LIB_PATH)
    for name, res, args in EXPORTS:
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(rc):
    if rc < 0:
        raise SwError(rc, lib().sw_last_error().decode())
    return rc


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def sw_last_error():
    return lib().sw_last_error().decode()


def sw_ncounters(q, model):
    return lib().sw_ncounters(int(q), int(model))


def sw_create(L, q, model, T, seed):
    h = lib().sw_create(int(L), int(q), int(model), float(T), ctypes.c_uint64(int(seed)))
    if not h:
        raise SwError(SW_ERR_ARG, sw_last_error())
    return h


def sw_create_ext(L, q, model, T, seed, d_spins=None, d_labels=None, stream=None):
    h = lib().sw_create_ext(int(L), int(q), int(model), float(T), ctypes.c_uint64(int(seed)),
                            d_spins, d_labels, stream)
    if not h:
        raise SwError(SW_ERR_ARG, sw_last_error())
    return h


def sw_destroy(h):
    return _check(lib().sw_destroy(h))


def sw_init(h, mode=SW_INIT_UP):
    return _check(lib().sw_init(h, int(mode)))


def sw_sweep(h, n=1):
    return _check(lib().sw_sweep(h, int(n)))


def sw_measure(h):
    o = sw_obs()
    _check(lib().sw_measure(h, ctypes.byref(o)))
    return o


def sw_synchronize(h):
    return _check(lib().sw_synchronize(h))


def sw_set_measure(h, on):
    return _check(lib().sw_set_measure(h, int(bool(on))))


def sw_set_record(h, on):
    return _check(lib().sw_set_record(h, int(bool(on))))


def sw_take_counts(h, max_rows, ncounters):
    out = np.zeros((max_rows, ncounters), dtype=np.int64)
    n = _check(lib().sw_take_counts(h, _p(out, ctypes.c_int64), int(max_rows)))
    return out[:n]


def sw_reset_stats(h):
    return _check(lib().sw_reset_stats(h))


def sw_set_debug_labels(h, on):
    return _check(lib().sw_set_debug_labels(h, int(bool(on))))


def sw_get_spins(h, n):
    out = np.zeros(n, dtype=np.int8)
    _check(lib().sw_get_spins(h, _p(out, ctypes.c_int8), n))
    return out


def sw_set_spins(h, spins):
    a = np.ascontiguousarray(np.asarray(spins, dtype=np.int8).reshape(-1))
    return _check(lib().sw_set_spins(h, _p(a, ctypes.c_int8), a.size))


def sw_get_labels(h, n):
    out = np.zeros(n, dtype=np.int32)
    _check(lib().sw_get_labels(h, _p(out, ctypes.c_int32), n))
    return out


def sw_device_spins(h):
    return lib().sw_device_spins(h)


def sw_device_labels(h):
    return lib().sw_device_labels(h)


def sw_get_thresholds(h, n):
    out = np.zeros(n, dtype=np.uint32)
    m = _check(lib().sw_get_thresholds(h, _p(out, ctypes.c_uint32), int(n)))
    return out[:m]


def sw_get_sweep(h):
    v = ctypes.c_uint64()
    _check(lib().sw_get_sweep(h, ctypes.byref(v)))
    return int(v.value)


def sw_set_sweep(h, t):
    return _check(lib().sw_set_sweep(h, ctypes.c_uint64(int(t))))


def sw_set_stream(h, stream):
    return _check(lib().sw_set_stream(h, stream))


def sw_set_graph(h, on):
    return _check(lib().sw_set_graph(h, int(bool(on))))


def sw_profile_sweeps(h, n):
    """Mean device milliseconds per sweep of each stage over n sweeps."""
    out = np.zeros(8, dtype=np.float32)
    m = _check(lib().sw_profile_sweeps(h, int(n), _p(out, ctypes.c_float), 8))
    return [float(v) for v in out[:m]]


def sw_autotune(h, n=3):
    out = np.zeros(4, dtype=np.int32)
    _check(lib().sw_autotune(h, int(n), _p(out, ctypes.c_int)))
    return [int(v) for v in out]


def sw_set_launch_shape(h, shape):
    a = np.ascontiguousarray(shape, dtype=np.int32)
    return _check(lib().sw_set_launch_shape(h, _p(a, ctypes.c_int)))


def sw_batch_autotune(b, n=3):
    out = np.zeros(4, dtype=np.int32)
    _check(lib().sw_batch_autotune(b, int(n), _p(out, ctypes.c_int)))
    return [int(v) for v in out]


def sw_batch_set_launch_shape(b, shape):
    a = np.ascontiguousarray(shape, dtype=np.int32)
    return _check(lib().sw_batch_set_launch_shape(b, _p(a, ctypes.c_int)))


def sw_batch_create(stream=None):
    b = lib().sw_batch_create(stream)
    if not b:
        raise SwError(SW_ERR_CUDA, sw_last_error())
    return b


def sw_batch_destroy(b):
    return _check(lib().sw_batch_destroy(b))


def sw_batch_attach(b, h):
    return _check(lib().sw_batch_attach(b, h))


def sw_batch_detach(b, h):
    return _check(lib().sw_batch_detach(b, h))


def sw_batch_size(b):
    return _check(lib().sw_batch_size(b))


def sw_batch_sweep(b, n=1):
    return _check(lib().sw_batch_sweep(b, int(n)))


def sw_batch_synchronize(b):
    return _check(lib().sw_batch_synchronize(b))


def sw_batch_set_measure(b, on):
    return _check(lib().sw_batch_set_measure(b, int(bool(on))))


def sw_batch_set_graph(b, on):
    return _check(lib().sw_batch_set_graph(b, int(bool(on))))


def sw_batch_set_debug_labels(b, on):
    return _check(lib().sw_batch_set_debug_labels(b, int(bool(on))))


def sw_batch_profile_sweeps(b, n):
    out = np.zeros(8, dtype=np.float32)
    m = _check(lib().sw_batch_profile_sweeps(b, int(n), _p(out, ctypes.c_float), 8))
    return [float(v) for v in out[:m]]


def sw_set_sweep_limit(h, stop):
    return _check(lib().sw_set_sweep_limit(h, ctypes.c_uint64(int(stop))))


def sw_get_sweep_limit(h):
    out = ctypes.c_uint64(0)
    _check(lib().sw_get_sweep_limit(h, ctypes.byref(out)))
    return int(out.value)


def sw_set_debug_limits(h, loop_cap, list_cap):
    return _check(lib().sw_set_debug_limits(h, int(loop_cap), int(list_cap)))


LABELING_STATS = ("sweeps", "labels_per_tile", "pairs_per_tile", "components_per_tile", "open_per_tile",
                  "unions_per_sweep", "links_per_union", "retries_per_link", "walks_per_sweep", "steps_per_walk",
                  "max_steps")


def sw_set_labeling_stats(h, on):
    return _check(lib().sw_set_labeling_stats(h, int(on)))


def sw_get_labeling_stats(h):
    """The labeling statistics as a dict (names in LABELING_STATS)."""
    out = np.zeros(len(LABELING_STATS), dtype=np.float64)
    m = _check(lib().sw_get_labeling_stats(h, _p(out, ctypes.c_double), len(out)))
    return {k: float(out[i]) for i, k in enumerate(LABELING_STATS[:m])}


def sw_set_labeling(h, method):
    return _check(lib().sw_set_labeling(h, int(method)))


def sw_label_passes(h):
    return _check(lib().sw_label_passes(h))


def sw_sweep_noalloc(L, q, model, T, seed, sweep0, n, d_spins, d_counts=None, stream=None):
    """n sweeps of caller-owned device spins (address d_spins) starting at
    sweep index sweep0, with no device allocation; d_counts (device address
    of n x sw_ncounters int64, or None) receives the per-sweep counters."""
    return _check(lib().sw_sweep_noalloc(int(L), int(q), int(model), float(T), ctypes.c_uint64(int(seed)),
                                         ctypes.c_uint64(int(sweep0)), int(n), d_spins, d_counts, stream))


class Lattice:
    """Owning convenience wrapper over one sw_handle (same calls, fewer arguments)."""

    def __init__(self, L, q, model, T, seed, init=SW_INIT_UP, stream=None, spins=None, labels=None):
        self.L, self.q, self.model, self.T, self.seed = int(L), int(q), int(model), float(T), int(seed)
        self.N = self.L * self.L
        if stream is None and spins is None and labels is None:
            self.h = sw_create(L, q, model, T, seed)
        else:
            self.h = sw_create_ext(L, q, model, T, seed, spins, labels, stream)
        self.nc = sw_ncounters(q, model)
        if init is not None:
            sw_init(self.h, init)

    def close(self):
        if getattr(self, "h", None):
            sw_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n=1):
        return sw_sweep(self.h, n)

    def measure(self):
        return sw_measure(self.h)

    def take_counts(self, max_rows=1 << 20):
        return sw_take_counts(self.h, max_rows, self.nc)

    @property
    def spins(self):
        return sw_get_spins(self.h, self.N).reshape(self.L, self.L)

    @spins.setter
    def spins(self, s):
        sw_set_spins(self.h, s)

    @property
    def labels(self):
        return sw_get_labels(self.h, self.N).reshape(self.L, self.L)

    def thresholds(self):
        n = 4 * self.q * self.q if self.model == SW_CLOCK else 1
        return sw_get_thresholds(self.h, n)

    @property
    def sweep_index(self):
        return sw_get_sweep(self.h)

    @sweep_index.setter
    def sweep_index(self, t):
        sw_set_sweep(self.h, t)


class Batch:
    """Owning convenience wrapper over one sw_batch: lattices added here are
    attached and destroyed with the batch."""

    def __init__(self, stream=None):
        self.b = sw_batch_create(stream)
        self.lattices = []

    def add(self, L, q, model, T, seed, init=SW_INIT_UP):
        lat = Lattice(L, q, model, T, seed, init=init)
        sw_batch_attach(self.b, lat.h)
        self.lattices.append(lat)
        return lat

    def remove(self, lat):
        sw_batch_detach(self.b, lat.h)
        self.lattices.remove(lat)
        return lat

    def sweep(self, n=1):
        return sw_batch_sweep(self.b, n)

    def close(self):
        if getattr(self, "b", None):
            sw_batch_destroy(self.b)
            self.b = None
        for lat in getattr(self, "lattices", []):
            lat.close()
        self.lattices = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
