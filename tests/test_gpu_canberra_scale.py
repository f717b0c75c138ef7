"""Canberra at any scale (Sec. 5.1.1): every term |x_c - y_c| / (|x_c| + |y_c|)
is unchanged when both points are multiplied by the same factor, and the FP64
oracle evaluates it at any magnitude.  The GPU must agree with the oracle on
the same data scaled by 1e-20 ... 1e18 (Phase 1 sample, Phase 2 estimate,
exact silhouette, batched and no-alloc calls, cohesion/separation), and on
data whose coordinates span more than FP32's pairwise range (tiny nonzero
coordinates, denormals, zeros beside magnitudes near 1e25), and on data of
either sign, all negative, with exact zeros, with magnitudes 2^35 apart, and at
row lengths with and without padding.  Tolerances are those of the other
parity tests (1e-5 on s, 1e-5 relative on a, b).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_01993_b300 import silh, synth
from test_gpu_parity import S_TOL, _assert_close, _host_values, _to_dev, assert_same_sample

pytestmark = pytest.mark.gpu
SCALES = [1e-20, 1e-12, 1e12, 1e18]


def _ragged(seed=3):
    X, lab, _ = synth.gaussian_mixture(5003, 13, 6, seed=seed,
                                       sizes=[2500, 1200, 700, 550, 30, 23])
    lab = lab.copy()
    lab[17] = 6                                   # singleton cluster
    return synth.abs_shift(X), lab, 7


def _scaled(scale):
    X, lab, k = _ragged()
    Xs = (X.astype(np.float64) * scale).astype(np.float32)
    assert np.isfinite(Xs).all() and (Xs != 0).all()
    return Xs, lab, k


def _wide_range():
    """Coordinates far apart in magnitude: tiny nonzero values (1e-30, FP32
    denormals near 1e-40), exact zeros, and a few rows near 1e25."""
    X, lab, k = _ragged(seed=13)
    X = X.copy()
    rng = np.random.default_rng(5)
    n = X.shape[0]
    X[rng.choice(n, 200, replace=False), 0] = 1e-30
    X[rng.choice(n, 150, replace=False), 3] = 1e-40
    X[rng.choice(n, 300, replace=False), 5] = 0.0
    X[rng.choice(n, 20, replace=False), 7] *= 1e25
    return X.astype(np.float32), lab, k


def _mixed_sign():
    """Coordinates of both signs (no |x| + 1 shift)."""
    X, lab, _ = synth.gaussian_mixture(5003, 13, 6, seed=3,
                                       sizes=[2500, 1200, 700, 550, 30, 23])
    return X.astype(np.float32), lab, 6


def _negative():
    """Every coordinate negative."""
    X, lab, k = _ragged(seed=21)
    return (-X).astype(np.float32), lab, k


def _with_zeros():
    """Positive data with exact zeros in one coordinate (0/0 terms are 0)."""
    X, lab, k = _ragged(seed=22)
    X = X.copy()
    X[np.random.default_rng(6).choice(X.shape[0], 400, replace=False), 2] = 0.0
    return X, lab, k


def _spread():
    """Positive data with a few coordinates ~1e-9 against a largest ~20
    (2^-35 of the scale: not tiny, far below the bulk)."""
    X, lab, k = _ragged(seed=23)
    X = X.copy()
    X[np.random.default_rng(7).choice(X.shape[0], 100, replace=False), 4] = 1e-9
    return X, lab, k


def _positive(d):
    """Positive data at d = 32 (no padding) and d = 5 (three padding slots of
    eight)."""
    def make():
        X, lab, _ = synth.gaussian_mixture(5003, d, 5, seed=d, sizes=[2000, 1500, 800, 680, 23],
                                           sigma=2.0)
        return synth.abs_shift(X), lab, 5
    return make


def _cases():
    return ([("scale%g" % s, lambda s=s: _scaled(s)) for s in SCALES] + [("wide", _wide_range)]
            + [("mixed_sign", _mixed_sign), ("negative", _negative), ("zeros", _with_zeros),
               ("spread", _spread), ("positive_d32", _positive(32)), ("positive_d5", _positive(5))])


@pytest.mark.parametrize("name,make", _cases(), ids=[c[0] for c in _cases()])
def test_canberra_sample_and_estimate_match_oracle(name, make):
    X, lab, k = make()
    Xt, lt = _to_dev(X, lab)
    Xh = _host_values(Xt)
    gs = silh.silh_sample_pps(Xt, lt, k, "canberra", t=40.0, m0=8.0, seed=3, clustering_id=2)
    os_ = oracle.sample_pps(Xh, lab, k, "canberra", t=40.0, m0=8.0, seed=3, cid=2)
    assert assert_same_sample(gs, os_, k, 3, 2, "canberra", lab) <= 1
    smp = silh.Sample.from_lists(np.bincount(lab, minlength=k), os_.offsets, os_.idx, os_.ps,
                                 Xt.device)
    s, a, b = silh.silh_estimate(Xt, lt, k, smp, "canberra", want_ab=True)
    s_o, a_o, b_o = oracle.estimate(Xh, lab, k, "canberra", os_.offsets, os_.idx, os_.ps)
    _assert_close(s, s_o, a, a_o, b, b_o)
    # rows listed out of order, and the no-alloc entry point on the same sample
    rows = torch.arange(n := X.shape[0], dtype=torch.int64, device="cuda").flip(0)[::3].contiguous()
    s_r = silh.silh_estimate(Xt, lt, k, smp, "canberra", rows=rows)
    _assert_close(s_r, s_o[rows.cpu().numpy()])
    s_n = silh.silh_estimate_noalloc(Xt, lt, k, smp, "canberra")
    assert torch.equal(s_n, s)
    assert n == len(lab)


@pytest.mark.parametrize("name,make", _cases(), ids=[c[0] for c in _cases()])
def test_canberra_exact_matches_oracle(name, make):
    X, lab, k = make()
    Xt, lt = _to_dev(X, lab)
    Xh = _host_values(Xt)
    s, a, b = silh.silh_exact(Xt, lt, k, "canberra", want_ab=True)
    s_o, a_o, b_o = oracle.exact(Xh, lab, k, "canberra")
    _assert_close(s, s_o, a, a_o, b, b_o)
    rows = torch.tensor([17, 0, 4000, 5002, 123], dtype=torch.int64, device="cuda")
    s_r = silh.silh_exact(Xt, lt, k, "canberra", rows=rows)
    _assert_close(s_r, s_o[rows.cpu().numpy()])


@pytest.mark.parametrize("name,make", _cases(), ids=[c[0] for c in _cases()])
def test_canberra_batched_and_cohsep_match_single_calls(name, make):
    X, lab, k = make()
    Xt, lt = _to_dev(X, lab)
    Xh = _host_values(Xt)
    lab2 = synth.nearest_centre_labels(X.astype(np.float64), 5, seed=8)
    l2 = torch.from_numpy(lab2.astype(np.int32)).cuda()
    k2 = int(lab2.max()) + 1
    s1 = silh.silh_sample_pps(Xt, lt, k, "canberra", t=40.0, m0=8.0, seed=4)
    s2 = silh.silh_sample_pps(Xt, l2, k2, "canberra", t=40.0, m0=8.0, seed=5)
    outs = silh.silh_estimate_batched(Xt, [(lt, s1), (l2, s2)], "canberra")
    torch.cuda.synchronize()
    assert torch.equal(outs[0], silh.silh_estimate(Xt, lt, k, s1, "canberra"))
    assert torch.equal(outs[1], silh.silh_estimate(Xt, l2, k2, s2, "canberra"))
    cs = silh.silh_cohsep(Xt, lt, k, s1, "canberra").cpu().numpy()
    off = s1.offsets.cpu().numpy()
    idx = s1.idx[: s1.size].cpu().numpy().astype(np.int64)
    ps = s1.p[: s1.size].cpu().numpy()
    _, _, _, Wh = oracle.estimate(Xh, lab, k, "canberra", off, idx, ps, want_w=True)
    coh, sep = oracle.cohsep(Wh, lab, k)
    np.testing.assert_allclose(cs, [coh, sep], rtol=1e-5)
    assert S_TOL == 1e-5
