"""FP64 CPU oracle for PPS silhouette approximation -- test infrastructure.

Only the tests, the smoke check and the CPU-baseline leg of ``bench.py`` use
this package.  The GPU library never imports it; the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, IEEE double, no fused
multiply-add).  This module compiles it with gcc on first use and marshals
numpy arrays through ctypes; it adds no arithmetic of its own.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

METRICS = {"euclidean": 0, "cosine": 1, "manhattan": 2, "canberra": 3}

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_f64p = ctypes.POINTER(ctypes.c_double)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, OpenMP, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.orc_philox4x64_10.argtypes = [_u64p, _u64p, _u64p]
        lib.orc_philox4x64_10.restype = None
        lib.orc_uniform.argtypes = [ctypes.c_uint64] * 4
        lib.orc_uniform.restype = ctypes.c_double
        lib.orc_dist.argtypes = [ctypes.c_int, _f64p, _f64p, ctypes.c_int]
        lib.orc_dist.restype = ctypes.c_double
        lib.orc_pairwise.argtypes = [ctypes.c_int, _f64p, ctypes.c_int64, _f64p, ctypes.c_int64,
                                     ctypes.c_int, _f64p]
        lib.orc_pairwise.restype = None
        lib.orc_cluster_sizes.argtypes = [_i32p, ctypes.c_int64, ctypes.c_int, _i64p]
        lib.orc_cluster_sizes.restype = ctypes.c_int
        lib.orc_exact.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int, _i32p, ctypes.c_int,
                                  ctypes.c_int, _i64p, ctypes.c_int64, _f64p, _f64p, _f64p, _i32p]
        lib.orc_exact.restype = ctypes.c_int
        lib.orc_poisson_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                         ctypes.c_int64, _f64p, _u8p]
        lib.orc_poisson_draw.restype = None
        lib.orc_sample_pps.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int, _i32p, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                       _u8p, _f64p, _f64p, _f64p, _u8p]
        lib.orc_sample_pps.restype = ctypes.c_int
        lib.orc_build_sample.argtypes = [_i32p, ctypes.c_int64, ctypes.c_int, _u8p, _f64p,
                                         _i64p, _i64p, _f64p]
        lib.orc_build_sample.restype = ctypes.c_int64
        lib.orc_estimate.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int, _i32p, ctypes.c_int,
                                     ctypes.c_int, _i64p, _i64p, _f64p, _i64p, ctypes.c_int64,
                                     _f64p, _f64p, _f64p, _f64p, _i32p]
        lib.orc_estimate.restype = ctypes.c_int
        lib.orc_cohsep.argtypes = [_f64p, _i32p, ctypes.c_int64, ctypes.c_int, _f64p, _f64p]
        lib.orc_cohsep.restype = ctypes.c_int
        lib.orc_mean.argtypes = [_f64p, ctypes.c_int64]
        lib.orc_mean.restype = ctypes.c_double
        lib.orc_t_from_eps.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                       ctypes.c_int]
        lib.orc_t_from_eps.restype = ctypes.c_double
        lib.orc_nthreads.argtypes = []
        lib.orc_nthreads.restype = ctypes.c_int
        _lib = lib
        return lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _f64(X):
    return np.ascontiguousarray(X, dtype=np.float64)


def _metric(m):
    return METRICS[m] if isinstance(m, str) else int(m)


def nthreads() -> int:
    return _load().orc_nthreads()


def philox4x64_10(counter, key):
    c = np.ascontiguousarray(counter, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    _load().orc_philox4x64_10(_p(c, _u64p), _p(k, _u64p), _p(out, _u64p))
    return out


def uniform(seed, stream, cid, e) -> float:
    return _load().orc_uniform(seed, stream, cid, e)


def dist(metric, x, y) -> float:
    x = _f64(x); y = _f64(y)
    return _load().orc_dist(_metric(metric), _p(x, _f64p), _p(y, _f64p), x.shape[0])


def pairwise(metric, X, Y):
    X = _f64(X); Y = _f64(Y)
    out = np.empty((X.shape[0], Y.shape[0]), dtype=np.float64)
    _load().orc_pairwise(_metric(metric), _p(X, _f64p), X.shape[0], _p(Y, _f64p), Y.shape[0],
                         X.shape[1], _p(out, _f64p))
    return out


def cluster_sizes(labels, k):
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    sizes = np.zeros(k, dtype=np.int64)
    rc = _load().orc_cluster_sizes(_p(labels, _i32p), labels.shape[0], k, _p(sizes, _i64p))
    if rc != 0:
        raise ValueError("invalid clustering")
    return sizes


def _rows(rows, n):
    if rows is None:
        return None, n
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    return rows, rows.shape[0]


def exact(X, labels, k, metric, rows=None, want_nb=False):
    """Exact s(e), a(e), b(e) (Eq. 1-2) for the listed rows (and the
    neighbouring cluster, the j attaining b, with want_nb)."""
    X = _f64(X)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    n, d = X.shape
    rows, nr = _rows(rows, n)
    s = np.empty(nr); a = np.empty(nr); b = np.empty(nr)
    nb = np.empty(nr, dtype=np.int32) if want_nb else None
    rc = _load().orc_exact(_p(X, _f64p), n, d, _p(labels, _i32p), k, _metric(metric),
                           _p(rows, _i64p), nr, _p(s, _f64p), _p(a, _f64p), _p(b, _f64p),
                           _p(nb, _i32p))
    if rc != 0:
        raise ValueError("invalid arguments")
    return (s, a, b, nb) if want_nb else (s, a, b)


def poisson_draw(seed, stream, cid, prob):
    prob = _f64(prob)
    flag = np.zeros(prob.shape[0], dtype=np.uint8)
    _load().orc_poisson_draw(seed, stream, cid, prob.shape[0], _p(prob, _f64p), _p(flag, _u8p))
    return flag.astype(bool)


def m0_default(k, delta):
    """Expected initial-sample size 2 ln(5k/delta) of Algorithm 1."""
    return 2.0 * np.log(5.0 * k / delta)


class Sample:
    """Phase-1 result: per-element arrays plus the per-cluster sample lists."""

    def __init__(self, in_f0, w0, gamma, p, in_f, offsets, idx, ps):
        self.in_f0, self.w0, self.gamma, self.p, self.in_f = in_f0, w0, gamma, p, in_f
        self.offsets, self.idx, self.ps = offsets, idx, ps

    @property
    def size(self):
        return int(self.offsets[-1])


def sample_pps(X, labels, k, metric, t, m0=None, delta=0.01, seed=0, cid=0, uniform=False):
    """Algorithm 1, Phase 1 (or the uniform variant when uniform=True)."""
    X = _f64(X)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    n, d = X.shape
    if m0 is None or m0 <= 0:
        m0 = m0_default(k, delta)
    in_f0 = np.zeros(n, dtype=np.uint8); in_f = np.zeros(n, dtype=np.uint8)
    w0 = np.zeros(n); gamma = np.zeros(n); p = np.zeros(n)
    lib = _load()
    rc = lib.orc_sample_pps(_p(X, _f64p), n, d, _p(labels, _i32p), k, _metric(metric),
                            float(t), float(m0), seed, cid, 1 if uniform else 0,
                            _p(in_f0, _u8p), _p(w0, _f64p), _p(gamma, _f64p), _p(p, _f64p),
                            _p(in_f, _u8p))
    if rc != 0:
        raise ValueError("invalid arguments")
    offsets = np.zeros(k + 1, dtype=np.int64)
    idx = np.zeros(n, dtype=np.int64)
    ps = np.zeros(n)
    size = lib.orc_build_sample(_p(labels, _i32p), n, k, _p(in_f, _u8p), _p(p, _f64p),
                                _p(offsets, _i64p), _p(idx, _i64p), _p(ps, _f64p))
    return Sample(in_f0.astype(bool), w0, gamma, p, in_f.astype(bool), offsets,
                  idx[:size].copy(), ps[:size].copy())


def build_sample(labels, k, in_f, p):
    """Per-cluster sample lists from per-element flags and probabilities."""
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    in_f = np.ascontiguousarray(in_f, dtype=np.uint8)
    p = _f64(p)
    n = labels.shape[0]
    offsets = np.zeros(k + 1, dtype=np.int64)
    idx = np.zeros(n, dtype=np.int64)
    ps = np.zeros(n)
    size = _load().orc_build_sample(_p(labels, _i32p), n, k, _p(in_f, _u8p), _p(p, _f64p),
                                    _p(offsets, _i64p), _p(idx, _i64p), _p(ps, _f64p))
    return offsets, idx[:size].copy(), ps[:size].copy()


def estimate(X, labels, k, metric, offsets, idx, ps, rows=None, want_w=False, want_nb=False):
    """Algorithm 1, Phase 2: s_hat, a_hat, b_hat (then W_hat if want_w, then the
    neighbouring cluster if want_nb)."""
    X = _f64(X)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    n, d = X.shape
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    ps = _f64(ps)
    rows, nr = _rows(rows, n)
    s = np.empty(nr); a = np.empty(nr); b = np.empty(nr)
    W = np.empty((nr, k)) if want_w else None
    nb = np.empty(nr, dtype=np.int32) if want_nb else None
    rc = _load().orc_estimate(_p(X, _f64p), n, d, _p(labels, _i32p), k, _metric(metric),
                              _p(offsets, _i64p), _p(idx, _i64p), _p(ps, _f64p),
                              _p(rows, _i64p), nr, _p(s, _f64p), _p(a, _f64p), _p(b, _f64p),
                              _p(W, _f64p), _p(nb, _i32p))
    if rc != 0:
        raise ValueError("invalid arguments")
    return (s, a, b) + ((W,) if want_w else ()) + ((nb,) if want_nb else ())


def cohsep(W, labels, k):
    """Cohesion and separation from per-element cluster weights W (n x k)."""
    W = _f64(W)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    coh = np.zeros(1); sep = np.zeros(1)
    rc = _load().orc_cohsep(_p(W, _f64p), _p(labels, _i32p), labels.shape[0], k,
                            _p(coh, _f64p), _p(sep, _f64p))
    if rc != 0:
        raise ValueError("invalid clustering")
    return float(coh[0]), float(sep[0])


def mean(v) -> float:
    v = _f64(v)
    return _load().orc_mean(_p(v, _f64p), v.shape[0])


def t_from_eps(eps, delta, n, k) -> float:
    return _load().orc_t_from_eps(eps, delta, n, k)
