"""silh_estimate_noalloc, the entry point for callers that cannot allocate.

Some callers of this library cannot allocate device memory during a call: a host
framework that has already reserved the whole device for its own allocator, a
latency-bound serving loop that cannot take an allocation (or its failure) in
the middle of a stream, code running inside an allocator callback.  For them
silh_estimate_noalloc runs Phase 2 with its scratch in a fixed device array of
the library.  These tests call it through the C ABI and compare it with the
allocating silh_estimate, on two calls in a row, within the tolerance the other
parity tests use.  The file is named to be collected last.
"""
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
