"""Edge cases at the limits of the boundary, each against the oracle.

d = 128 (largest), d = 1 (smallest), k = 8192 (largest: clusters of two or
three points), one cluster holding all but a few singletons, empty row lists,
and caller output tensors that are too small (refused in the binding).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_01993_b300 import silh, synth
from test_gpu_parity import _assert_close, _host_values, _to_dev, assert_same_sample

pytestmark = pytest.mark.gpu

METRICS = ["euclidean", "cosine", "manhattan", "canberra"]


def _oracle_lists(os_, lab, k):
    """The oracle's sample lists on the device (Phase 2 compared on one sample)."""
    return silh.Sample.from_lists(np.bincount(lab, minlength=k), os_.offsets, os_.idx, os_.ps,
                                  "cuda")


@pytest.mark.parametrize("metric", METRICS)
def test_widest_rows_d128(metric):
    X, lab, _ = synth.gaussian_mixture(3000, 128, 5, seed=31, sizes=[1500, 700, 500, 250, 50])
    if metric == "canberra":
        X = synth.abs_shift(X)
    Xt, lt = _to_dev(X, lab)
    Xh = _host_values(Xt)
    gs = silh.silh_sample_pps(Xt, lt, 5, metric, t=48.0, m0=8.0, seed=5)
    os_ = oracle.sample_pps(Xh, lab, 5, metric, t=48.0, m0=8.0, seed=5)
    assert_same_sample(gs, os_, 5, 5, 0, metric, lab)
    s = silh.silh_estimate(Xt, lt, 5, _oracle_lists(os_, lab, 5), metric)
    s_o, _, _ = oracle.estimate(Xh, lab, 5, metric, os_.offsets, os_.idx, os_.ps)
    _assert_close(s, s_o)
    rows = torch.arange(0, 3000, 7, dtype=torch.int64, device="cuda")
    se = silh.silh_exact(Xt, lt, 5, metric, rows=rows)
    se_o, _, _ = oracle.exact(Xh, lab, 5, metric, rows=rows.cpu().numpy())
    _assert_close(se, se_o)


@pytest.mark.parametrize("metric", ["euclidean", "manhattan"])
def test_single_coordinate_d1(metric):
    rng = np.random.default_rng(32)
    X = np.concatenate([rng.normal(0, 1, 400), rng.normal(6, 1, 300),
                        rng.normal(-5, 2, 300)]).astype(np.float32).reshape(-1, 1)
    lab = np.repeat(np.arange(3, dtype=np.int32), [400, 300, 300])
    Xt, lt = _to_dev(X, lab)
    Xh = _host_values(Xt)
    gs = silh.silh_sample_pps(Xt, lt, 3, metric, t=40.0, m0=8.0, seed=6)
    os_ = oracle.sample_pps(Xh, lab, 3, metric, t=40.0, m0=8.0, seed=6)
    assert_same_sample(gs, os_, 3, 6, 0, metric, lab)
    s = silh.silh_estimate(Xt, lt, 3, _oracle_lists(os_, lab, 3), metric)
    s_o, _, _ = oracle.estimate(Xh, lab, 3, metric, os_.offsets, os_.idx, os_.ps)
    _assert_close(s, s_o)
    se = silh.silh_exact(Xt, lt, 3, metric)
    se_o, _, _ = oracle.exact(Xh, lab, 3, metric)
    _assert_close(se, se_o)


def test_largest_k():
    """k = SILH_MAX_K = 8192 clusters of two or three points each."""
    k = 8192
    rng = np.random.default_rng(33)
    n = 20000
    lab = (np.arange(n) % k).astype(np.int32)
    X = (rng.normal(0, 1, (n, 4)) + 3.0 * rng.normal(0, 1, (k, 4))[lab]).astype(np.float32)
    Xt, lt = _to_dev(X, lab)
    Xh = _host_values(Xt)
    gs = silh.silh_sample_pps(Xt, lt, k, "euclidean", t=8.0, seed=7)
    assert gs.size == n                      # every cluster is below t: F_j = C_j, p = 1
    os_ = oracle.sample_pps(Xh, lab, k, "euclidean", t=8.0, seed=7)
    rows = np.arange(0, n, 53, dtype=np.int64)
    s = silh.silh_estimate(Xt, lt, k, gs, "euclidean", rows=torch.from_numpy(rows).cuda())
    s_o, _, _ = oracle.estimate(Xh, lab, k, "euclidean", os_.offsets, os_.idx, os_.ps, rows=rows)
    _assert_close(s, s_o)
    se = silh.silh_exact(Xt, lt, k, "euclidean", rows=torch.from_numpy(rows).cuda())
    se_o, _, _ = oracle.exact(Xh, lab, k, "euclidean", rows=rows)
    _assert_close(se, se_o)
    np.testing.assert_allclose(s_o, se_o, atol=1e-12)   # p = 1 everywhere: estimate = exact
    with pytest.raises(RuntimeError):
        silh.silh_sample_pps(Xt, lt, k + 1, "euclidean", t=8.0)


def test_one_big_cluster_and_singletons():
    X, _, _ = synth.gaussian_mixture(2000, 6, 1, seed=34)
    lab = np.zeros(2000, dtype=np.int32)
    lab[[3, 500, 1999]] = [1, 2, 3]
    Xt, lt = _to_dev(X, lab)
    Xh = _host_values(Xt)
    for metric in METRICS[:2]:
        gs = silh.silh_sample_pps(Xt, lt, 4, metric, t=64.0, seed=8)
        os_ = oracle.sample_pps(Xh, lab, 4, metric, t=64.0, seed=8)
        assert_same_sample(gs, os_, 4, 8, 0, metric, lab)
        for prec in ("fp32", "3xtf32"):
            s = silh.silh_estimate(Xt, lt, 4, _oracle_lists(os_, lab, 4), metric, prec=prec)
            s_o, _, _ = oracle.estimate(Xh, lab, 4, metric, os_.offsets, os_.idx, os_.ps)
            _assert_close(s, s_o)
            assert s[3].item() == 0.0 and s[500].item() == 0.0 and s[1999].item() == 0.0


def test_empty_row_list_and_short_outputs():
    X, lab, _ = synth.tiny(seed=0)
    Xt, lt = _to_dev(X, lab)
    gs = silh.silh_sample_pps(Xt, lt, 4, "euclidean", t=64.0, m0=16.0, seed=0)
    empty = torch.empty(0, dtype=torch.int64, device="cuda")
    launches = silh.kernel_launches()
    assert silh.silh_estimate(Xt, lt, 4, gs, "euclidean", rows=empty).numel() == 0
    assert silh.silh_exact(Xt, lt, 4, "euclidean", rows=empty).numel() == 0
    assert silh.silh_estimate_cosine_collapsed(Xt, lt, 4, gs, rows=empty).numel() == 0
    assert silh.kernel_launches() == launches
    short = torch.empty(10, dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        silh.silh_estimate(Xt, lt, 4, gs, "euclidean", out=short)
    with pytest.raises(ValueError):
        silh.silh_estimate_batched(Xt, [(lt, gs)], "euclidean", outs=[short])


def test_scratch_exhaustion_is_enomem_and_the_context_survives():
    """A sample whose column operand cannot fit in device memory (its stated
    size, 2^40 columns, is checked before anything is launched) returns
    SILH_ENOMEM; the next call on the same context works."""
    import ctypes
    lib = silh.load()
    X, lab, _ = synth.tiny(seed=0)
    Xt, lt = _to_dev(X, lab)
    n, d = X.shape
    gs = silh.silh_sample_pps(Xt, lt, 4, "manhattan", t=64.0, m0=16.0, seed=0)
    torch.cuda.synchronize()
    huge = silh.SilhSample(4, gs.sizes.data_ptr(), gs.offsets.data_ptr(), gs.idx.data_ptr(),
                           gs.p.data_ptr(), 1 << 40, 1 << 40)
    s = torch.empty(n, dtype=torch.float32, device="cuda")
    launches = silh.kernel_launches()
    rc = lib.silh_estimate(Xt.data_ptr(), 0, n, d, d, lt.data_ptr(), 4, 2, 0, ctypes.byref(huge),
                           None, 0, s.data_ptr(), None, None, None, None)
    assert rc == -2, (rc, lib.silh_last_error())
    assert silh.kernel_launches() == launches
    s2 = silh.silh_estimate(Xt, lt, 4, gs, "manhattan")
    torch.cuda.synchronize()
    assert torch.isfinite(s2).all()
