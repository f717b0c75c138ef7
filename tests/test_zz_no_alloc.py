"""silh_estimate_noalloc, the entry point for callers that cannot allocate.

Some callers of this library cannot allocate device memory during a call: a host
framework that has already reserved the whole device for its own allocator, a
latency-bound serving loop that cannot take an allocation (or its failure) in
the middle of a stream, code running inside an allocator callback.  For them
silh_estimate_noalloc runs Phase 2 with its scratch in a fixed device array of
the library.  These tests call it through the C ABI and compare it with the
allocating silh_estimate, on two calls in a row, within the tolerance the other
parity tests use, check that a call takes no memory from the device's
stream-ordered pool and leaves free device memory unchanged, and check the
documented precision rule (FP32 on CUDA cores whatever mode is asked for).
The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2607_01993_b300 import silh, synth

pytestmark = pytest.mark.gpu
S_TOL = 1e-5     # the GPU parity tolerance on s_hat


def _data(n, d, k, seed):
    X, lab, _ = synth.gaussian_mixture(n, d, k, seed=seed, sizes=synth.zipf_sizes(n, k),
                                       sigma_range=(0.5, 3.0))
    return torch.from_numpy(X).cuda(), torch.from_numpy(lab).cuda()


def _close(a, b):
    assert torch.isfinite(a).all()
    assert (a - b).abs().max().item() <= S_TOL


def test_noalloc_matches_estimate_on_two_calls_in_a_row():
    X1, l1 = _data(40000, 32, 16, seed=31)
    X2, l2 = _data(9000, 13, 5, seed=32)
    s1 = silh.silh_sample_pps(X1, l1, 16, "euclidean", t=128.0, seed=1)
    s2 = silh.silh_sample_pps(X2, l2, 5, "canberra", t=64.0, m0=10.0, seed=2)
    assert s1.size * 32 <= silh.SILH_NOALLOC_MAX_FLOATS
    # first call, then a second one with a different shape and metric
    n1 = silh.silh_estimate_noalloc(X1, l1, 16, s1, "euclidean", want_ab=True)
    n2 = silh.silh_estimate_noalloc(X2, l2, 5, s2, "canberra", want_ab=True)
    r1 = silh.silh_estimate(X1, l1, 16, s1, "euclidean", want_ab=True)
    r2 = silh.silh_estimate(X2, l2, 5, s2, "canberra", want_ab=True)
    for got, want in zip(n1 + n2, r1 + r2):
        _close(got, want)
    # and once more on the first problem after the second overwrote the scratch
    n1b = silh.silh_estimate_noalloc(X1, l1, 16, s1, "euclidean")
    _close(n1b, r1[0])


def test_noalloc_row_subset_and_oracle():
    X, l = _data(5000, 8, 4, seed=33)
    smp = silh.silh_sample_pps(X, l, 4, "manhattan", t=64.0, m0=16.0, seed=3)
    rows = torch.arange(0, 5000, 7, dtype=torch.int64, device="cuda")
    got = silh.silh_estimate_noalloc(X, l, 4, smp, "manhattan", rows=rows)
    want = silh.silh_estimate(X, l, 4, smp, "manhattan", rows=rows)
    _close(got, want)
    Xh = X.cpu().numpy().astype(np.float64)
    lab = l.cpu().numpy()
    os_ = oracle.sample_pps(Xh, lab, 4, "manhattan", t=64.0, m0=16.0, seed=3)
    s_o, _, _ = oracle.estimate(Xh, lab, 4, "manhattan", os_.offsets, os_.idx, os_.ps,
                                rows=rows.cpu().numpy())
    assert np.abs(got.cpu().numpy() - s_o).max() <= S_TOL


def test_noalloc_runs_fp32_whatever_the_precision():
    # A tensor-core precision is accepted but the distances stay FP32 on the CUDA
    # cores: equal to silh_estimate(prec="fp32") bit for bit, and within the FP32
    # tolerance of the oracle, while silh_estimate(prec="bf16") itself is not.
    X, l = _data(20000, 24, 8, seed=35)
    smp = silh.silh_sample_pps(X, l, 8, "euclidean", t=96.0, seed=5)
    ref = silh.silh_estimate(X, l, 8, smp, "euclidean", prec="fp32")
    for prec in ("3xtf32", "bf16", "bf16x3", "tf32"):
        got = silh.silh_estimate_noalloc(X, l, 8, smp, "euclidean", prec=prec)
        assert torch.equal(got, ref), prec
    rows = torch.arange(0, 20000, 13, dtype=torch.int64, device="cuda")
    Xh = X.cpu().numpy().astype(np.float64)
    lab = l.cpu().numpy()
    off = smp.offsets.cpu().numpy()
    idx = smp.idx[: smp.size].cpu().numpy().astype(np.int64)
    ps = smp.p[: smp.size].cpu().numpy()
    s_o, _, _ = oracle.estimate(Xh, lab, 8, "euclidean", off, idx, ps, rows=rows.cpu().numpy())
    got = silh.silh_estimate_noalloc(X, l, 8, smp, "euclidean", prec="3xtf32", rows=rows)
    assert np.abs(got.cpu().numpy() - s_o).max() <= S_TOL


def _cudart():
    for name in ("libcudart.so.13", "libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("libcudart not found by the dynamic loader")


def test_noalloc_takes_no_device_memory_during_a_call():
    # The property the entry point exists for: with its outputs in place, a call
    # neither draws on the device's stream-ordered pool (whose high-water mark is
    # reset just before) nor changes the free device memory.
    rt = _cudart()
    X, l = _data(30000, 16, 12, seed=36)
    smp = silh.silh_sample_pps(X, l, 12, "canberra", t=64.0, seed=6)
    out = torch.empty(30000, dtype=torch.float32, device="cuda")
    silh.silh_estimate_noalloc(X, l, 12, smp, "canberra", out=out)      # loads, maps
    torch.cuda.synchronize()
    dev = torch.cuda.current_device()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    USED_CURRENT, USED_HIGH = 7, 8          # cudaMemPoolAttr values
    used0, high, zero = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64(0)
    assert rt.cudaMemPoolGetAttribute(pool, USED_CURRENT, ctypes.byref(used0)) == 0
    assert rt.cudaMemPoolSetAttribute(pool, USED_HIGH, ctypes.byref(zero)) == 0
    free0, total = ctypes.c_size_t(), ctypes.c_size_t()
    assert rt.cudaMemGetInfo(ctypes.byref(free0), ctypes.byref(total)) == 0
    silh.silh_estimate_noalloc(X, l, 12, smp, "canberra", out=out)
    torch.cuda.synchronize()
    free1 = ctypes.c_size_t()
    assert rt.cudaMemGetInfo(ctypes.byref(free1), ctypes.byref(total)) == 0
    assert rt.cudaMemPoolGetAttribute(pool, USED_HIGH, ctypes.byref(high)) == 0
    assert high.value <= used0.value, (high.value, used0.value)
    assert free1.value == free0.value
    # the allocating entry point, by contrast, does draw on the pool
    assert rt.cudaMemPoolSetAttribute(pool, USED_HIGH, ctypes.byref(zero)) == 0
    silh.silh_estimate(X, l, 12, smp, "canberra", out=out)
    torch.cuda.synchronize()
    assert rt.cudaMemPoolGetAttribute(pool, USED_HIGH, ctypes.byref(high)) == 0
    assert high.value > used0.value


def test_noalloc_rejects_samples_beyond_its_scratch():
    n = silh.SILH_NOALLOC_MAX_COLUMNS + 100
    X, l = _data(n, 4, 2, seed=34)
    # every element sampled with p = 1: |S| = n > the no-alloc maximum
    lab = l.cpu().numpy()
    offsets = np.concatenate([[0], np.cumsum(np.bincount(lab, minlength=2))])
    idx = np.concatenate([np.flatnonzero(lab == 0), np.flatnonzero(lab == 1)])
    smp = silh.Sample.from_lists(np.bincount(lab, minlength=2), offsets, idx, np.ones(n),
                                 X.device)
    with pytest.raises(silh.SilhError) as ei:
        silh.silh_estimate_noalloc(X, l, 2, smp, "euclidean")
    assert ei.value.status == silh.SILH_ECAPACITY
    assert "no-alloc" in str(ei.value)
