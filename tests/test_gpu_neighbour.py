"""The neighbouring cluster (the j != C attaining b_hat, Eq. 8 / Eq. 2) through
every entry point that returns it, against the FP64 oracle.

Where the GPU and the oracle name different clusters, the two clusters'
ratios W_j / |Cj| must agree within the arithmetic's tolerance (the GPU's
choice, evaluated by the oracle, is within that relative tolerance of the
oracle's b), i.e. the GPU's cluster also attains b within that tolerance.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_01993_b300 import silh, synth
from test_gpu_parity import _host_values, _to_dev

pytestmark = pytest.mark.gpu
METRICS = ["euclidean", "cosine", "manhattan", "canberra"]


def _data(metric, seed=21):
    X, lab, _ = synth.gaussian_mixture(3001, 13, 6, seed=seed, sigma=2.5,
                                       sizes=[1200, 700, 500, 400, 180, 21])
    if metric == "canberra":
        X = synth.abs_shift(X)
    return X, lab, 6


def _check(nb_g, lab_rows, b_o, nb_o, W_o, sizes, tol):
    nb_g = nb_g.cpu().numpy().astype(np.int64)
    assert (nb_g >= 0).all() and (nb_g < len(sizes)).all()
    assert (nb_g != lab_rows).all()
    diff = np.nonzero(nb_g != nb_o)[0]
    ratio = W_o[diff, nb_g[diff]] / sizes[nb_g[diff]]
    assert (ratio <= b_o[diff] * (1.0 + tol)).all(), "neighbour differs beyond a near-tie"
    return len(diff)


def _full_sample(lab, k):
    """F_j = C_j with p = 1: the oracle's estimate is then the exact W."""
    idx = np.argsort(lab, kind="stable").astype(np.int64)
    offsets = np.concatenate([[0], np.cumsum(np.bincount(lab, minlength=k))]).astype(np.int64)
    return offsets, idx, np.ones(len(idx))


@pytest.mark.parametrize("metric", METRICS)
def test_estimate_neighbour_cuda_cores(metric):
    X, lab, k = _data(metric)
    Xt, lt = _to_dev(X, lab)
    Xh = _host_values(Xt)
    os_ = oracle.sample_pps(Xh, lab, k, metric, t=64.0, seed=2, cid=1)
    smp = silh.Sample.from_lists(np.bincount(lab, minlength=k), os_.offsets, os_.idx, os_.ps,
                                 Xt.device)
    sizes = np.bincount(lab, minlength=k).astype(np.float64)
    _, _, b_o, W_o, nb_o = oracle.estimate(Xh, lab, k, metric, os_.offsets, os_.idx, os_.ps,
                                           want_w=True, want_nb=True)
    s, nb = silh.silh_estimate(Xt, lt, k, smp, metric, want_nb=True)
    _check(nb, lab, b_o, nb_o, W_o, sizes, 1e-5)
    # row list (reversed, every third row), the no-alloc and asynchronous entry points
    rows = np.arange(len(lab))[::-3].copy()
    rt = torch.from_numpy(rows).cuda()
    _, nb_r = silh.silh_estimate(Xt, lt, k, smp, metric, rows=rt, want_nb=True)
    assert torch.equal(nb_r, nb[rt])
    _, _, _, nb_n = silh.silh_estimate_noalloc(Xt, lt, k, smp, metric, want_ab=True,
                                               want_nb=True)
    assert torch.equal(nb_n, nb)
    d_size = torch.tensor([smp.size], dtype=torch.int64, device="cuda")
    _, nb_a = silh.silh_estimate_async(Xt, lt, k, smp, d_size, metric, want_nb=True)
    assert torch.equal(nb_a, nb)


@pytest.mark.parametrize("metric", ["euclidean", "cosine"])
@pytest.mark.parametrize("prec", ["3xtf32", "tf32"])
def test_estimate_neighbour_tensor_cores(metric, prec):
    X, lab, k = _data(metric, seed=22)
    Xt, lt = _to_dev(X, lab)
    Xh = _host_values(Xt)
    os_ = oracle.sample_pps(Xh, lab, k, metric, t=64.0, seed=3, cid=0)
    smp = silh.Sample.from_lists(np.bincount(lab, minlength=k), os_.offsets, os_.idx, os_.ps,
                                 Xt.device)
    sizes = np.bincount(lab, minlength=k).astype(np.float64)
    _, _, b_o, W_o, nb_o = oracle.estimate(Xh, lab, k, metric, os_.offsets, os_.idx, os_.ps,
                                           want_w=True, want_nb=True)
    tol = 1e-5 if prec == "3xtf32" else 2e-3
    s, a, b, nb = silh.silh_estimate(Xt, lt, k, smp, metric, prec=prec, want_ab=True,
                                     want_nb=True)
    _check(nb, lab, b_o, nb_o, W_o, sizes, tol)
    rows = np.array([0, 17, 3000, 2999, 1500, 1201])
    rt = torch.from_numpy(rows).cuda()
    _, nb_r = silh.silh_estimate(Xt, lt, k, smp, metric, prec=prec, rows=rt, want_nb=True)
    assert torch.equal(nb_r, nb[rt])
    if metric == "cosine" and prec == "3xtf32":
        _, nb_c = silh.silh_estimate_cosine_collapsed(Xt, lt, k, smp, want_nb=True)
        _check(nb_c, lab, b_o, nb_o, W_o, sizes, 1e-5)


@pytest.mark.parametrize("metric,prec", [(m, "fp32") for m in METRICS]
                         + [("euclidean", "3xtf32"), ("cosine", "3xtf32")])
def test_exact_neighbour(metric, prec):
    X, lab, _ = synth.gaussian_mixture(1500, 13, 5, seed=23, sigma=2.5,
                                       sizes=[600, 400, 300, 190, 10])
    if metric == "canberra":
        X = synth.abs_shift(X)
    k = 5
    Xt, lt = _to_dev(X, lab)
    Xh = _host_values(Xt)
    sizes = np.bincount(lab, minlength=k).astype(np.float64)
    off, idx, ps = _full_sample(lab, k)
    _, _, b_o, W_o, nb_o = oracle.estimate(Xh, lab, k, metric, off, idx, ps, want_w=True,
                                           want_nb=True)
    _, nb_x = oracle.exact(Xh, lab, k, metric, want_nb=True)[2:]
    assert np.array_equal(nb_o, nb_x)
    s, nb = silh.silh_exact(Xt, lt, k, metric, prec=prec, want_nb=True)
    _check(nb, lab, b_o, nb_o, W_o, sizes, 1e-5)
    rows = np.array([5, 0, 1499, 700])
    _, nb_r = silh.silh_exact(Xt, lt, k, metric, prec=prec,
                              rows=torch.from_numpy(rows).cuda(), want_nb=True)
    _check(nb_r, lab[rows], b_o[rows], nb_o[rows], W_o[rows], sizes, 1e-5)
