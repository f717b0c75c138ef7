"""Thin Python binding of libsilh (C ABI in include/silh.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Tensors are torch CUDA tensors; the library receives their device
pointers and the current torch stream.  If libsilh.so is missing or fails to
load, every call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsilh.so")

METRICS = {"euclidean": 0, "cosine": 1, "manhattan": 2, "canberra": 3}
DTYPES = {torch.float32: 0, torch.bfloat16: 1}
PRECS = {"fp32": 0, "tf32": 1, "3xtf32": 2, "bf16": 3, "bf16x3": 4}
STATUS = {0: "SILH_OK", -1: "SILH_EINVAL", -2: "SILH_ENOMEM", -3: "SILH_ECUDA",
          -4: "SILH_ECAPACITY", -5: "SILH_ETIMEOUT"}
SILH_ECAPACITY = -4

# exported symbols, as declared in include/silh.h
EXPORTS = ("silh_sample_pps", "silh_estimate", "silh_exact", "silh_global", "silh_t_from_eps",
           "silh_last_error", "silh_version", "silh_kernel_launches", "silh_estimate_noalloc",
           "silh_stream_status", "silh_estimate_batched", "silh_cohsep",
           "silh_estimate_cosine_collapsed", "silh_pipe_rates", "silh_wait_selftest",
           "silh_sample_pps_async", "silh_estimate_async")
SILH_NOALLOC_MAX_COLUMNS = 65536
SILH_NOALLOC_MAX_FLOATS = 2097152


class SilhError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class SilhSample(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("sizes", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
                ("idx", ctypes.c_void_p), ("p", ctypes.c_void_p), ("cap", ctypes.c_int64),
                ("size", ctypes.c_int64)]


class SilhBatchItem(ctypes.Structure):
    _fields_ = [("labels", ctypes.c_void_p), ("sample", ctypes.POINTER(SilhSample)),
                ("s_hat", ctypes.c_void_p)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libsilh.so (raises if it is absent: the product has no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libsilh.so not built at {path}; run paper_2607_01993_b300/build.py")
    lib = ctypes.CDLL(path)
    vp, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    lib.silh_sample_pps.argtypes = [vp, ctypes.c_int, i64, i32, i64, vp, i32, ctypes.c_int, f64,
                                    f64, f64, ctypes.c_uint64, ctypes.c_uint32, i32,
                                    ctypes.POINTER(SilhSample), vp]
    lib.silh_sample_pps.restype = ctypes.c_int
    lib.silh_estimate.argtypes = [vp, ctypes.c_int, i64, i32, i64, vp, i32, ctypes.c_int,
                                  ctypes.c_int, ctypes.POINTER(SilhSample), vp, i64, vp, vp, vp, vp,
                                  vp]
    lib.silh_estimate.restype = ctypes.c_int
    lib.silh_sample_pps_async.argtypes = list(lib.silh_sample_pps.argtypes[:-1]) + [vp, vp, vp]
    lib.silh_sample_pps_async.restype = ctypes.c_int
    lib.silh_estimate_async.argtypes = (list(lib.silh_estimate.argtypes[:10]) + [vp]
                                        + list(lib.silh_estimate.argtypes[10:]))
    lib.silh_estimate_async.restype = ctypes.c_int
    lib.silh_estimate_noalloc.argtypes = list(lib.silh_estimate.argtypes)
    lib.silh_estimate_noalloc.restype = ctypes.c_int
    lib.silh_exact.argtypes = [vp, ctypes.c_int, i64, i32, i64, vp, i32, ctypes.c_int,
                               ctypes.c_int, vp, i64, vp, vp, vp, vp, vp]
    lib.silh_exact.restype = ctypes.c_int
    lib.silh_global.argtypes = [vp, i64, vp, vp]
    lib.silh_global.restype = ctypes.c_int
    lib.silh_t_from_eps.argtypes = [f64, f64, i64, i32]
    lib.silh_t_from_eps.restype = f64
    lib.silh_last_error.argtypes = []
    lib.silh_last_error.restype = ctypes.c_char_p
    lib.silh_version.argtypes = []
    lib.silh_version.restype = ctypes.c_char_p
    lib.silh_estimate_batched.argtypes = [vp, ctypes.c_int, i64, i32, i64, ctypes.c_int,
                                          ctypes.c_int, i32, ctypes.POINTER(SilhBatchItem), i32,
                                          vp]
    lib.silh_estimate_batched.restype = ctypes.c_int
    lib.silh_estimate_cosine_collapsed.argtypes = [vp, ctypes.c_int, i64, i32, i64, vp, i32,
                                                   ctypes.POINTER(SilhSample), vp, i64, vp, vp,
                                                   vp, vp, vp]
    lib.silh_estimate_cosine_collapsed.restype = ctypes.c_int
    lib.silh_pipe_rates.argtypes = [ctypes.POINTER(ctypes.c_double), vp]
    lib.silh_pipe_rates.restype = ctypes.c_int
    lib.silh_cohsep.argtypes = [vp, ctypes.c_int, i64, i32, i64, vp, i32, ctypes.c_int,
                                ctypes.POINTER(SilhSample), vp, vp]
    lib.silh_cohsep.restype = ctypes.c_int
    lib.silh_stream_status.argtypes = [vp]
    lib.silh_stream_status.restype = ctypes.c_int
    lib.silh_wait_selftest.argtypes = [i32, ctypes.c_uint64, vp]
    lib.silh_wait_selftest.restype = ctypes.c_int
    lib.silh_kernel_launches.argtypes = []
    lib.silh_kernel_launches.restype = ctypes.c_uint64
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        raise SilhError(rc, load().silh_last_error().decode())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _data(X):
    if (not X.is_cuda or X.dim() != 2 or (X.stride(1) != 1 and X.shape[1] > 1)
            or X.stride(0) < X.shape[1] or X.dtype not in DTYPES):
        raise ValueError("X must be a 2-D CUDA float32/bfloat16 tensor with unit column stride")
    return DTYPES[X.dtype], X.shape[0], X.shape[1], X.stride(0)


def _labels(labels):
    if not labels.is_cuda or labels.dtype != torch.int32 or not labels.is_contiguous():
        raise ValueError("labels must be a contiguous CUDA int32 tensor")
    return labels


def _rows(rows):
    if rows is None:
        return None, 0
    if not rows.is_cuda or rows.dtype != torch.int64 or not rows.is_contiguous():
        raise ValueError("rows must be a contiguous CUDA int64 tensor")
    return rows, rows.shape[0]


def _out(out, nrows, device):
    """A caller output tensor must hold nrows float32 values on the device."""
    if out is None:
        return torch.empty(nrows, dtype=torch.float32, device=device)
    if (not out.is_cuda or out.dtype != torch.float32 or not out.is_contiguous()
            or out.numel() < nrows):
        raise ValueError(f"out must be a contiguous CUDA float32 tensor of >= {nrows} elements")
    return out


def _empty_rows(rows, nr):
    """An empty row list: nothing to compute (a null pointer would mean all rows)."""
    return rows is not None and nr == 0


@dataclass
class Sample:
    """Sample set of Phase 1: per-cluster lists over device tensors."""
    k: int
    sizes: torch.Tensor      # int64 [k]
    offsets: torch.Tensor    # int64 [k+1]
    idx: torch.Tensor        # int32 [cap]
    p: torch.Tensor          # float64 [cap]
    size: int

    def as_struct(self) -> SilhSample:
        return SilhSample(self.k, self.sizes.data_ptr(), self.offsets.data_ptr(),
                          self.idx.data_ptr(), self.p.data_ptr(), self.idx.shape[0], self.size)

    @staticmethod
    def empty(k: int, cap: int, device) -> "Sample":
        return Sample(k, torch.zeros(k, dtype=torch.int64, device=device),
                      torch.zeros(k + 1, dtype=torch.int64, device=device),
                      torch.zeros(max(cap, 1), dtype=torch.int32, device=device),
                      torch.zeros(max(cap, 1), dtype=torch.float64, device=device), 0)

    @staticmethod
    def from_lists(sizes, offsets, idx, p, device) -> "Sample":
        """A sample built elsewhere (host arrays), e.g. for feeding a fixed sample."""
        idx_t = torch.as_tensor(idx, dtype=torch.int32).to(device)
        return Sample(len(sizes), torch.as_tensor(sizes, dtype=torch.int64).to(device),
                      torch.as_tensor(offsets, dtype=torch.int64).to(device), idx_t,
                      torch.as_tensor(p, dtype=torch.float64).to(device), int(idx_t.shape[0]))


def silh_sample_pps(X, labels, k, metric="euclidean", t=64.0, m0=None, delta=0.01, seed=0,
                    clustering_id=0, uniform=False, cap=None, out=None, stream=None) -> Sample:
    """Algorithm 1, Phase 1 on the GPU (synchronising)."""
    lib = load()
    dt, n, d, ld = _data(X)
    labels = _labels(labels)
    smp = out if out is not None else Sample.empty(k, n if cap is None else cap, X.device)
    st = smp.as_struct()
    rc = lib.silh_sample_pps(_ptr(X), dt, n, d, ld, _ptr(labels), k, METRICS[metric], float(t),
                             -1.0 if m0 is None else float(m0), float(delta), int(seed),
                             int(clustering_id), 1 if uniform else 0, ctypes.byref(st),
                             _stream(stream))
    if rc == SILH_ECAPACITY and out is None:
        return silh_sample_pps(X, labels, k, metric, t, m0, delta, seed, clustering_id, uniform,
                               cap=int(st.size), stream=stream)
    _check(rc)
    smp.size = int(st.size)
    return smp


def silh_sample_pps_async(X, labels, k, metric="euclidean", t=64.0, m0=None, delta=0.01, seed=0,
                          clustering_id=0, uniform=False, cap=None, out=None, d_size=None,
                          d_status=None, stream=None):
    """Algorithm 1, Phase 1, enqueued without host synchronisation.

    Returns (sample, d_size, d_status): |S| and the status stay on the device
    (int64 / int32 CUDA tensors) until the caller reads them; sample.size is
    left at -1.  cap defaults to n (always enough)."""
    lib = load()
    dt, n, d, ld = _data(X)
    labels = _labels(labels)
    smp = out if out is not None else Sample.empty(k, n if cap is None else cap, X.device)
    if d_size is None:
        d_size = torch.empty(1, dtype=torch.int64, device=X.device)
    if d_status is None:
        d_status = torch.empty(1, dtype=torch.int32, device=X.device)
    st = smp.as_struct()
    _check(lib.silh_sample_pps_async(_ptr(X), dt, n, d, ld, _ptr(labels), k, METRICS[metric],
                                     float(t), -1.0 if m0 is None else float(m0), float(delta),
                                     int(seed), int(clustering_id), 1 if uniform else 0,
                                     ctypes.byref(st), _ptr(d_size), _ptr(d_status),
                                     _stream(stream)))
    smp.size = -1
    return smp, d_size, d_status


def _outputs(nrows, device, want_ab, want_nb):
    a = torch.empty(nrows, dtype=torch.float32, device=device) if want_ab else None
    b = torch.empty(nrows, dtype=torch.float32, device=device) if want_ab else None
    nb = torch.empty(nrows, dtype=torch.int32, device=device) if want_nb else None
    return a, b, nb


def _ret(s, a, b, nb, want_ab, want_nb):
    """s; (s, a, b) with want_ab; (s, nb) with want_nb; (s, a, b, nb) with both."""
    out = (s,) + ((a, b) if want_ab else ()) + ((nb,) if want_nb else ())
    return out if len(out) > 1 else s


def silh_estimate_async(X, labels, k, sample: Sample, d_size, metric="euclidean", prec="fp32",
                        rows=None, want_ab=False, out=None, stream=None, want_nb=False):
    """Phase 2 for a sample whose size is on the device (d_size, int64 CUDA)."""
    lib = load()
    dt, n, d, ld = _data(X)
    labels = _labels(labels)
    rows, nr = _rows(rows)
    nrows = n if rows is None else nr
    s = _out(out, nrows, X.device)
    a, b, nb = _outputs(nrows, X.device, want_ab, want_nb)
    if _empty_rows(rows, nr):
        return _ret(s, a, b, nb, want_ab, want_nb)
    st = sample.as_struct()
    _check(lib.silh_estimate_async(_ptr(X), dt, n, d, ld, _ptr(labels), k, METRICS[metric],
                                   PRECS[prec], ctypes.byref(st), _ptr(d_size), _ptr(rows), nr,
                                   _ptr(s), _ptr(a), _ptr(b), _ptr(nb), _stream(stream)))
    return _ret(s, a, b, nb, want_ab, want_nb)


def silh_estimate(X, labels, k, sample: Sample, metric="euclidean", prec="fp32", rows=None,
                  want_ab=False, out=None, stream=None, want_nb=False):
    """Algorithm 1, Phase 2: s_hat (and a_hat, b_hat; the neighbouring cluster
    with want_nb) for all rows or a row list."""
    lib = load()
    dt, n, d, ld = _data(X)
    labels = _labels(labels)
    rows, nr = _rows(rows)
    nrows = n if rows is None else nr
    s = _out(out, nrows, X.device)
    a, b, nb = _outputs(nrows, X.device, want_ab, want_nb)
    if _empty_rows(rows, nr):
        return _ret(s, a, b, nb, want_ab, want_nb)
    st = sample.as_struct()
    _check(lib.silh_estimate(_ptr(X), dt, n, d, ld, _ptr(labels), k, METRICS[metric],
                             PRECS[prec], ctypes.byref(st), _ptr(rows), nr, _ptr(s), _ptr(a),
                             _ptr(b), _ptr(nb), _stream(stream)))
    return _ret(s, a, b, nb, want_ab, want_nb)


def silh_estimate_noalloc(X, labels, k, sample: Sample, metric="euclidean", prec="fp32",
                          rows=None, want_ab=False, out=None, stream=None, want_nb=False):
    """silh_estimate through the no-allocation entry point (fixed device scratch).

    For callers that cannot allocate device memory during the call; the output
    tensors are allocated here only when the caller does not pass them.
    """
    lib = load()
    dt, n, d, ld = _data(X)
    labels = _labels(labels)
    rows, nr = _rows(rows)
    nrows = n if rows is None else nr
    s = _out(out, nrows, X.device)
    a, b, nb = _outputs(nrows, X.device, want_ab, want_nb)
    if _empty_rows(rows, nr):
        return _ret(s, a, b, nb, want_ab, want_nb)
    st = sample.as_struct()
    _check(lib.silh_estimate_noalloc(_ptr(X), dt, n, d, ld, _ptr(labels), k, METRICS[metric],
                                     PRECS[prec], ctypes.byref(st), _ptr(rows), nr, _ptr(s),
                                     _ptr(a), _ptr(b), _ptr(nb), _stream(stream)))
    return _ret(s, a, b, nb, want_ab, want_nb)


def silh_estimate_cosine_collapsed(X, labels, k, sample: Sample, rows=None, want_ab=False,
                                   out=None, stream=None, want_nb=False):
    """Cosine Phase 2 in O(n k d) (parallel-axis collapse of the weighted sums)."""
    lib = load()
    dt, n, d, ld = _data(X)
    labels = _labels(labels)
    rows, nr = _rows(rows)
    nrows = n if rows is None else nr
    s = _out(out, nrows, X.device)
    a, b, nb = _outputs(nrows, X.device, want_ab, want_nb)
    if _empty_rows(rows, nr):
        return _ret(s, a, b, nb, want_ab, want_nb)
    st = sample.as_struct()
    _check(lib.silh_estimate_cosine_collapsed(_ptr(X), dt, n, d, ld, _ptr(labels), k,
                                              ctypes.byref(st), _ptr(rows), nr, _ptr(s), _ptr(a),
                                              _ptr(b), _ptr(nb), _stream(stream)))
    return _ret(s, a, b, nb, want_ab, want_nb)


def pipe_rates(stream=None):
    """Measured lane-operations per second per SM of the arithmetic pipes."""
    lib = load()
    out = (ctypes.c_double * 6)()
    _check(lib.silh_pipe_rates(out, _stream(stream)))
    return dict(zip(("ffma", "ffma2_lanes", "mufu_rcp", "mufu_sqrt", "fmnmx", "dfma"), list(out)))


BATCH_VARIANTS = 4   # tile shapes of the batched sweep (see include/silh.h)


def silh_estimate_batched(X, items, metric="euclidean", variant=-1, outs=None, stream=None,
                          prec="fp32"):
    """Phase 2 for many clusterings of X in one persistent launch.

    items: list of (labels, sample) pairs (int32 CUDA labels, Sample from
    silh_sample_pps on those labels).  Returns one FP32 s_hat tensor per item.
    prec "fp32" runs the CUDA-core sweep (variant picks its tile shape);
    "tf32" / "3xtf32" / "bf16" / "bf16x3" with the Euclidean or cosine
    distance and d <= 64 run the tensor-core sweep, each item equal to
    silh_estimate with that prec.  Asynchronous and graph-capturable when outs
    are preallocated.
    """
    lib = load()
    dt, n, d, ld = _data(X)
    if outs is None:
        outs = [torch.empty(n, dtype=torch.float32, device=X.device) for _ in items]
    if len(outs) != len(items):
        raise ValueError("one output tensor per item")
    outs = [_out(o, n, X.device) for o in outs]
    structs = [smp.as_struct() for _, smp in items]
    arr = (SilhBatchItem * len(items))()
    for i, ((labels, _), st, out) in enumerate(zip(items, structs, outs)):
        arr[i].labels = _labels(labels).data_ptr()
        arr[i].sample = ctypes.pointer(st)
        arr[i].s_hat = out.data_ptr()
    _check(lib.silh_estimate_batched(_ptr(X), dt, n, d, ld, METRICS[metric], PRECS[prec],
                                     len(items), arr, int(variant), _stream(stream)))
    return outs


def silh_exact(X, labels, k, metric="euclidean", prec="fp32", rows=None, want_ab=False,
               stream=None, want_nb=False):
    """Exact silhouette (Eq. 1-2) of all rows or a row list."""
    lib = load()
    dt, n, d, ld = _data(X)
    labels = _labels(labels)
    rows, nr = _rows(rows)
    nrows = n if rows is None else nr
    s = torch.empty(nrows, dtype=torch.float32, device=X.device)
    a, b, nb = _outputs(nrows, X.device, want_ab, want_nb)
    if _empty_rows(rows, nr):
        return _ret(s, a, b, nb, want_ab, want_nb)
    _check(lib.silh_exact(_ptr(X), dt, n, d, ld, _ptr(labels), k, METRICS[metric], PRECS[prec],
                          _ptr(rows), nr, _ptr(s), _ptr(a), _ptr(b), _ptr(nb), _stream(stream)))
    return _ret(s, a, b, nb, want_ab, want_nb)


def silh_cohsep(X, labels, k, sample: Sample, metric="euclidean", stream=None):
    """Estimated cohesion and separation; returns a 2-element float64 CUDA tensor."""
    lib = load()
    dt, n, d, ld = _data(X)
    labels = _labels(labels)
    out = torch.empty(2, dtype=torch.float64, device=X.device)
    st = sample.as_struct()
    _check(lib.silh_cohsep(_ptr(X), dt, n, d, ld, _ptr(labels), k, METRICS[metric],
                           ctypes.byref(st), _ptr(out), _stream(stream)))
    return out


def silh_global(s, out=None, stream=None):
    """FP64 mean of s (Eq. 3 / 6 / 7); returns a 1-element float64 CUDA tensor."""
    lib = load()
    if not s.is_cuda or s.dtype != torch.float32 or not s.is_contiguous():
        raise ValueError("s must be a contiguous CUDA float32 tensor")
    o = out if out is not None else torch.empty(1, dtype=torch.float64, device=s.device)
    _check(lib.silh_global(_ptr(s), s.numel(), _ptr(o), _stream(stream)))
    return o


def silh_t_from_eps(eps, delta, n, k) -> float:
    return load().silh_t_from_eps(eps, delta, n, k)


def silh_stream_status(stream=None):
    """Synchronise the stream; raise SilhError(SILH_ETIMEOUT) if a bounded device
    wait gave up since the previous check."""
    _check(load().silh_stream_status(_stream(stream)))


def wait_selftest(arrive: bool, timeout_ns: int = 1_000_000, stream=None):
    """Launch the bounded-wait self-test kernel (asynchronous); read the outcome
    with silh_stream_status."""
    _check(load().silh_wait_selftest(1 if arrive else 0, int(timeout_ns), _stream(stream)))


def kernel_launches() -> int:
    """Kernels launched by libsilh so far in this process."""
    return int(load().silh_kernel_launches())


def version() -> str:
    return load().silh_version().decode()
