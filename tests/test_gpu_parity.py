"""GPU path (through the C ABI) against the FP64 oracle, element by element.

Sample sets must be identical: both sides take the inclusion decision
u < p_e with FP64-class p_e.  The oracle evaluates every distance in FP64 and
sums W sequentially; the GPU evaluates Euclidean, Manhattan and Canberra
distances in double-float arithmetic (relative error below 2^-42 for d <= 128),
cosine in FP64, sums W in a fixed tree and multiplies by 1/W.  A sequential or
tree sum of N positive terms is within (N - 1) u of the exact sum
(u = 2^-53); the per-distance errors (<= (d + 2) u in the oracle, < 2^-42 on the
GPU) and the 1/W rounding add at most (2d + 8) u + 2^-41, so p_e agrees within
tie(j) = (2 |Cj| + 2 * 128 + 64) u + 2^-40 relative.  Cosine evaluates
1 - <x,y>/(|x||y|), whose absolute error (below 40 u on either side) is not
relative to the distance; relative to W and to a maximising ratio d/W >= 1/|Cj|
it adds 80 u |Cj| / min W(e0) over the cluster's initial sample.  An element
may be in one sample and not the other only if |u - p_e| <= tie(j) p_e, and
such elements are counted.  Silhouette values must agree within 1e-5 absolute (FP32
arithmetic on the GPU), a_hat/b_hat within 1e-5 relative.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_01993_b300 import silh, synth

pytestmark = pytest.mark.gpu
METRICS = ["euclidean", "cosine", "manhattan", "canberra"]
S_TOL = 1e-5
AB_RTOL = 1e-5
U64 = 2.0 ** -53


def tie_band(cluster_size):
    return (2.0 * cluster_size + 2 * 128 + 64.0) * U64 + 2.0 ** -40


def _to_dev(X, lab, dtype=torch.float32):
    Xt = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda().to(dtype)
    return Xt, torch.from_numpy(lab.astype(np.int32)).cuda()


def _host_values(Xt):
    return Xt.float().cpu().numpy().astype(np.float64)


def assert_same_sample(gs: silh.Sample, os_: oracle.Sample, k, seed, cid, metric=None, labels=None):
    g_off = gs.offsets.cpu().numpy()
    g_idx = gs.idx[: gs.size].cpu().numpy().astype(np.int64)
    g_p = gs.p[: gs.size].cpu().numpy()
    sizes = gs.sizes.cpu().numpy()
    ties = 0
    gp = dict(zip(g_idx.tolist(), g_p.tolist()))
    for j in range(k):
        tie = tie_band(sizes[j])
        if metric == "cosine" and labels is not None:
            f0 = os_.in_f0 & (labels == j)
            if f0.any():
                tie += 80.0 * U64 * sizes[j] / os_.w0[f0].min()
        a = g_idx[g_off[j]:g_off[j + 1]]
        b = os_.idx[os_.offsets[j]:os_.offsets[j + 1]]
        assert (np.diff(a) > 0).all(), "GPU list not ascending"
        diff = np.setxor1d(a, b)
        for e in diff:
            u = oracle.uniform(seed, 1, cid, int(e))
            assert abs(u - os_.p[e]) <= tie * os_.p[e], f"element {e} differs outside tie band"
            ties += 1
        both = np.intersect1d(a, b)
        got = np.array([gp[e] for e in both])
        np.testing.assert_allclose(got, os_.p[both], rtol=tie, atol=0)
    return ties


def _assert_close(s_g, s_o, a_g=None, a_o=None, b_g=None, b_o=None):
    s_g = s_g.cpu().numpy().astype(np.float64)
    assert np.isfinite(s_g).all()
    err = np.abs(s_g - s_o).max()
    assert err <= S_TOL, f"max |s diff| = {err}"
    if a_g is not None:
        np.testing.assert_allclose(a_g.cpu().numpy(), a_o, rtol=AB_RTOL, atol=1e-30)
        np.testing.assert_allclose(b_g.cpu().numpy(), b_o, rtol=AB_RTOL, atol=1e-30)


def _case(name):
    if name == "tiny":
        X, lab, _ = synth.tiny(seed=0)
        return X, lab, 4, dict(t=64.0, m0=16.0, seed=0)
    if name == "ragged":
        X, lab, _ = synth.gaussian_mixture(5003, 13, 6, seed=3, sizes=[2500, 1200, 700, 550, 30, 23])
        lab = lab.copy()
        lab[17] = 6                                   # singleton cluster
        return X, lab, 7, dict(t=40.0, m0=8.0, seed=3)
    if name == "multitile":
        X, lab, _ = synth.gaussian_mixture(40000, 32, 16, seed=4,
                                           sizes=synth.zipf_sizes(40000, 16), sigma_range=(0.5, 3))
        return X, lab, 16, dict(t=128.0, m0=None, seed=4)
    raise KeyError(name)


@pytest.mark.parametrize("case", ["tiny", "ragged", "multitile"])
@pytest.mark.parametrize("metric", METRICS)
def test_sample_pps_matches_oracle(case, metric):
    X, lab, k, kw = _case(case)
    if metric == "canberra":
        X = synth.abs_shift(X)
    Xt, lt = _to_dev(X, lab)
    gs = silh.silh_sample_pps(Xt, lt, k, metric, t=kw["t"], m0=kw["m0"], seed=kw["seed"],
                              clustering_id=5)
    os_ = oracle.sample_pps(_host_values(Xt), lab, k, metric, t=kw["t"], m0=kw["m0"],
                            seed=kw["seed"], cid=5)
    np.testing.assert_array_equal(gs.sizes.cpu().numpy(), np.bincount(lab, minlength=k))
    ties = assert_same_sample(gs, os_, k, kw["seed"], 5, metric, lab)
    assert ties <= 1


@pytest.mark.parametrize("case", ["tiny", "ragged", "multitile"])
@pytest.mark.parametrize("metric", METRICS)
def test_estimate_matches_oracle_on_oracle_sample(case, metric):
    X, lab, k, kw = _case(case)
    if metric == "canberra":
        X = synth.abs_shift(X)
    Xt, lt = _to_dev(X, lab)
    Xh = _host_values(Xt)
    os_ = oracle.sample_pps(Xh, lab, k, metric, t=kw["t"], m0=kw["m0"], seed=kw["seed"])
    smp = silh.Sample.from_lists(np.bincount(lab, minlength=k), os_.offsets, os_.idx, os_.ps,
                                 Xt.device)
    s, a, b = silh.silh_estimate(Xt, lt, k, smp, metric, want_ab=True)
    s_o, a_o, b_o = oracle.estimate(Xh, lab, k, metric, os_.offsets, os_.idx, os_.ps)
    _assert_close(s, s_o, a, a_o, b, b_o)


@pytest.mark.parametrize("metric", METRICS)
def test_end_to_end_tiny(metric):
    """Phase 1 + Phase 2 + global on the GPU vs the oracle, tiny workload."""
    X, lab, k, kw = _case("tiny")
    if metric == "canberra":
        X = synth.abs_shift(X)
    Xt, lt = _to_dev(X, lab)
    Xh = _host_values(Xt)
    gs = silh.silh_sample_pps(Xt, lt, k, metric, t=64.0, m0=16.0, seed=0)
    s = silh.silh_estimate(Xt, lt, k, gs, metric)
    g = silh.silh_global(s).item()
    os_ = oracle.sample_pps(Xh, lab, k, metric, t=64.0, m0=16.0, seed=0)
    assert_same_sample(gs, os_, k, 0, 0, metric, lab)
    s_o, _, _ = oracle.estimate(Xh, lab, k, metric, os_.offsets, os_.idx, os_.ps)
    _assert_close(s, s_o)
    assert abs(g - oracle.mean(s_o)) <= S_TOL / 10


@pytest.mark.parametrize("case", ["tiny", "ragged"])
@pytest.mark.parametrize("metric", METRICS)
def test_exact_matches_oracle(case, metric):
    X, lab, k, _ = _case(case)
    if metric == "canberra":
        X = synth.abs_shift(X)
    Xt, lt = _to_dev(X, lab)
    Xh = _host_values(Xt)
    s, a, b = silh.silh_exact(Xt, lt, k, metric, want_ab=True)
    s_o, a_o, b_o = oracle.exact(Xh, lab, k, metric)
    _assert_close(s, s_o, a, a_o, b, b_o)
    g = silh.silh_global(s).item()
    assert abs(g - oracle.mean(s_o)) <= S_TOL / 10


@pytest.mark.parametrize("d", [27, 32])
@pytest.mark.parametrize("metric", ["manhattan", "canberra"])
def test_exact_32_element_rows_match_oracle(metric, d):
    """Exact silhouette (Eq. 1-2) of 32-element rows on CUDA cores, whose
    symmetric kernel takes blocks of columns inside one cluster without
    per-column checks: cluster ends inside column blocks, row tiles that span
    clusters, a 4-point cluster, a ragged last tile, several column tiles per
    block; all rows element by element, and a row list."""
    sizes = [1201, 777, 513, 389, 250, 203, 4]
    X, lab, _ = synth.gaussian_mixture(sum(sizes), d, len(sizes), seed=31, sizes=sizes,
                                       sigma_range=(0.5, 3.0))
    if metric == "canberra":
        X = synth.abs_shift(X)
    k = len(sizes)
    Xt, lt = _to_dev(X, lab)
    Xh = _host_values(Xt)
    s, a, b = silh.silh_exact(Xt, lt, k, metric, want_ab=True)
    s_o, a_o, b_o = oracle.exact(Xh, lab, k, metric)
    _assert_close(s, s_o, a, a_o, b, b_o)
    rows = np.array([3336, 0, 1700, 2999, 5, 1201])
    sr = silh.silh_exact(Xt, lt, k, metric, rows=torch.from_numpy(rows).cuda())
    _assert_close(sr, s_o[rows])


def test_bf16_storage_matches_oracle_on_rounded_values():
    X, lab, k, kw = _case("multitile")
    Xt, lt = _to_dev(X, lab, torch.bfloat16)
    Xh = _host_values(Xt)           # the BF16-rounded values, exactly
    gs = silh.silh_sample_pps(Xt, lt, k, "euclidean", t=128.0, seed=4)
    os_ = oracle.sample_pps(Xh, lab, k, "euclidean", t=128.0, seed=4)
    assert_same_sample(gs, os_, k, 4, 0)
    rows = torch.arange(0, 40000, 97, dtype=torch.int64, device="cuda")
    s = silh.silh_estimate(Xt, lt, k, gs, "euclidean", rows=rows)
    s_o, _, _ = oracle.estimate(Xh, lab, k, "euclidean", os_.offsets, os_.idx, os_.ps,
                                rows=rows.cpu().numpy())
    _assert_close(s, s_o)


def test_row_subset_equals_full_rows():
    X, lab, k, kw = _case("ragged")
    Xt, lt = _to_dev(X, lab)
    gs = silh.silh_sample_pps(Xt, lt, k, "manhattan", t=40.0, m0=8.0, seed=1)
    s_all = silh.silh_estimate(Xt, lt, k, gs, "manhattan")
    rows = torch.tensor([17, 0, 5002, 1234, 17], dtype=torch.int64, device="cuda")
    s_sub = silh.silh_estimate(Xt, lt, k, gs, "manhattan", rows=rows)
    assert torch.equal(s_sub, s_all[rows])
    assert s_all[17].item() == 0.0                   # singleton


def test_uniform_variant_matches_oracle():
    X, lab, k, kw = _case("multitile")
    Xt, lt = _to_dev(X, lab)
    gs = silh.silh_sample_pps(Xt, lt, k, "euclidean", t=128.0, seed=9, uniform=True)
    os_ = oracle.sample_pps(_host_values(Xt), lab, k, "euclidean", t=128.0, seed=9, uniform=True)
    assert_same_sample(gs, os_, k, 9, 0)


@pytest.mark.parametrize("metric", METRICS)
def test_empty_initial_sample_matches_oracle(metric):
    """Clusters larger than t with an empty initial sample (m0 = 1e-3): the
    device must take the gamma = 1/|Cj| branch of the oracle, giving the same
    sample (probabilities min(1, t/|Cj|)) and the same estimate."""
    X, lab, k, _ = _case("ragged")
    if metric == "canberra":
        X = synth.abs_shift(X)
    Xt, lt = _to_dev(X, lab)
    Xh = _host_values(Xt)
    gs = silh.silh_sample_pps(Xt, lt, k, metric, t=40.0, m0=1e-3, seed=11, clustering_id=3)
    os_ = oracle.sample_pps(Xh, lab, k, metric, t=40.0, m0=1e-3, seed=11, cid=3)
    assert not os_.in_f0.any()
    sizes = np.bincount(lab, minlength=k)
    big = sizes[lab] > 40.0
    assert big.sum() > 4000
    np.testing.assert_allclose(os_.p[big], 40.0 / sizes[lab][big], rtol=2.0 ** -52, atol=0)
    assert assert_same_sample(gs, os_, k, 11, 3, metric, lab) == 0
    s, a, b = silh.silh_estimate(Xt, lt, k, gs, metric, want_ab=True)
    s_o, a_o, b_o = oracle.estimate(Xh, lab, k, metric, os_.offsets, os_.idx, os_.ps)
    _assert_close(s, s_o, a, a_o, b, b_o)


def test_invalid_clusterings_raise():
    X, lab, k, _ = _case("tiny")
    Xt, lt = _to_dev(X, lab)
    with pytest.raises(silh.SilhError) as ei:
        silh.silh_exact(Xt, lt, 5, "euclidean")                  # cluster 4 empty
    assert ei.value.status == -1
    bad = lt.clone(); bad[3] = 9
    with pytest.raises(silh.SilhError):
        silh.silh_sample_pps(Xt, bad, 4, "euclidean", t=64.0)    # label out of range
    with pytest.raises(silh.SilhError):
        silh.silh_sample_pps(Xt, lt, 1, "euclidean", t=64.0)     # k = 1
    with pytest.raises(silh.SilhError):
        silh.silh_sample_pps(Xt, lt, 4, "euclidean", t=0.0)      # t <= 0
    # the context is still usable afterwards
    s = silh.silh_exact(Xt, lt, 4, "euclidean")
    assert torch.isfinite(s).all()


def test_capacity_error_reports_needed_size():
    X, lab, k, _ = _case("tiny")
    Xt, lt = _to_dev(X, lab)
    out = silh.Sample.empty(4, 10, Xt.device)
    with pytest.raises(silh.SilhError) as ei:
        silh.silh_sample_pps(Xt, lt, 4, "euclidean", t=64.0, m0=16.0, out=out)
    assert ei.value.status == silh.SILH_ECAPACITY
    full = silh.silh_sample_pps(Xt, lt, 4, "euclidean", t=64.0, m0=16.0)
    assert full.size > 10


def _degenerate():
    """Zero rows, exact-zero coordinates, a cluster of identical points (its
    W(e0) = 0, so gamma falls back to 1/|Cj|) and a singleton."""
    X, lab, _ = synth.gaussian_mixture(600, 5, 3, seed=21, sizes=[300, 200, 100])
    X = X.copy()
    lab = np.concatenate([lab, np.full(50, 3, np.int32), [4]]).astype(np.int32)
    X = np.concatenate([X, np.tile(np.array([[1.5, -2.0, 0.0, 3.0, 0.25]], np.float32), (50, 1)),
                        np.array([[0.5, 0.5, 0.5, 0.5, 0.5]], np.float32)])
    X[10] = 0.0                     # zero vector (cosine distance 1 to everything)
    X[20, 1] = 0.0
    X[21, :2] = 0.0                 # Canberra 0/0 terms where paired with zeros
    X[300:310, 2] = 0.0
    return np.ascontiguousarray(X), lab, 5


@pytest.mark.parametrize("metric", METRICS)
def test_degenerate_inputs_match_oracle(metric):
    X, lab, k = _degenerate()
    Xt, lt = _to_dev(X, lab)
    Xh = _host_values(Xt)
    gs = silh.silh_sample_pps(Xt, lt, k, metric, t=20.0, m0=6.0, seed=2)
    os_ = oracle.sample_pps(Xh, lab, k, metric, t=20.0, m0=6.0, seed=2)
    assert_same_sample(gs, os_, k, 2, 0, metric, lab)
    s, a, b = silh.silh_estimate(Xt, lt, k, gs, metric, want_ab=True)
    s_o, a_o, b_o = oracle.estimate(Xh, lab, k, metric, os_.offsets, os_.idx, os_.ps)
    _assert_close(s, s_o)
    np.testing.assert_allclose(a.cpu().numpy(), a_o, rtol=AB_RTOL, atol=1e-6)
    se = silh.silh_exact(Xt, lt, k, metric)
    se_o, _, _ = oracle.exact(Xh, lab, k, metric)
    _assert_close(se, se_o)
    assert s[-1].item() == 0.0 and se[-1].item() == 0.0     # singleton


# ------------------------------------------------ tensor-core (tcgen05) sweep

# Plain TF32 keeps 11 significant bits of each coordinate, so inner products
# carry ~2^-11 relative error; its stated bound on s_hat is 2e-3.  Split TF32
# (3 MMAs) plus the FP32 recompute of close pairs is held to the FP32 bound.
# Split BF16 keeps ~17 significant bits of each coordinate (inner products to
# ~2^-17 |x||y|): 2e-5.  Plain BF16 rounds each coordinate to 8 bits: 5e-3.
TC_TOL = {"3xtf32": S_TOL, "tf32": 2e-3, "bf16x3": 2e-5, "bf16": 5e-3}
TC_PRECS = ["3xtf32", "tf32", "bf16x3", "bf16"]


def _tc_case(name):
    if name == "wide":     # d = 50: two 128-byte TF32 K blocks, one BF16 block of 4 K steps
        X, lab, _ = synth.gaussian_mixture(12000, 50, 8, seed=9, sizes=synth.zipf_sizes(12000, 8),
                                           sigma_range=(0.5, 3))
        return X, lab, 8, dict(t=96.0, m0=None, seed=9)
    if name in ("voronoi", "voronoi_wide"):
        # Nearest-centre labels cut each mixture component into several clusters,
        # so many pairs across clusters are close against |x|^2 + |y|^2: most
        # column chunks take the direct FP32 recompute (d = 16: one column per
        # lane over 4 of 8 coordinate groups; d = 50: the two-slot TF32 form and,
        # for BF16 operands, each lane its own row).  Two zero rows meet it too.
        d, n, comps, k, seed = (16, 9000, 6, 40, 11) if name == "voronoi" else (50, 6000, 4, 24, 13)
        X, _, _ = synth.gaussian_mixture(n, d, comps, seed=seed, sigma=1.5)
        X = X.copy()
        X[[5, 777]] = 0.0
        lab = synth.nearest_centre_labels(X, k, seed=seed + 1)
        return X, lab, k, dict(t=48.0, m0=None, seed=seed)
    return _case(name)


@pytest.mark.parametrize("prec", TC_PRECS)
@pytest.mark.parametrize("case", ["tiny", "ragged", "multitile", "wide", "voronoi", "voronoi_wide"])
@pytest.mark.parametrize("metric", ["euclidean", "cosine"])
def test_tensor_core_estimate_matches_oracle(case, metric, prec):
    X, lab, k, kw = _tc_case(case)
    Xt, lt = _to_dev(X, lab)
    Xh = _host_values(Xt)
    os_ = oracle.sample_pps(Xh, lab, k, metric, t=kw["t"], m0=kw["m0"], seed=kw["seed"])
    smp = silh.Sample.from_lists(np.bincount(lab, minlength=k), os_.offsets, os_.idx, os_.ps,
                                 Xt.device)
    launches = silh.kernel_launches()
    s, a, b = silh.silh_estimate(Xt, lt, k, smp, metric, prec=prec, want_ab=True)
    silh.silh_stream_status()
    assert silh.kernel_launches() > launches
    s_o, a_o, b_o = oracle.estimate(Xh, lab, k, metric, os_.offsets, os_.idx, os_.ps)
    s_g = s.cpu().numpy().astype(np.float64)
    assert np.isfinite(s_g).all()
    assert np.abs(s_g - s_o).max() <= TC_TOL[prec]
    if prec == "3xtf32":
        np.testing.assert_allclose(a.cpu().numpy(), a_o, rtol=AB_RTOL, atol=1e-7)
        np.testing.assert_allclose(b.cpu().numpy(), b_o, rtol=AB_RTOL, atol=1e-7)
    if prec == "bf16x3":
        np.testing.assert_allclose(a.cpu().numpy(), a_o, rtol=2 * AB_RTOL, atol=1e-7)
        np.testing.assert_allclose(b.cpu().numpy(), b_o, rtol=2 * AB_RTOL, atol=1e-7)


@pytest.mark.parametrize("prec", ["3xtf32", "bf16x3"])
@pytest.mark.parametrize("case", ["tiny", "ragged", "wide", "voronoi", "voronoi_wide"])
@pytest.mark.parametrize("metric", ["euclidean", "cosine"])
def test_tensor_core_exact_matches_oracle(case, metric, prec):
    X, lab, k, _ = _tc_case(case)
    if case == "wide":
        X, lab = X[:3000], lab[:3000]
        k = int(lab.max()) + 1
        assert (np.bincount(lab, minlength=k) > 0).all()
    Xt, lt = _to_dev(X, lab)
    Xh = _host_values(Xt)
    s, a, b = silh.silh_exact(Xt, lt, k, metric, prec=prec, want_ab=True)   # each pair once
    silh.silh_stream_status()
    s_o, a_o, b_o = oracle.exact(Xh, lab, k, metric)
    s_g = s.cpu().numpy().astype(np.float64)
    assert np.isfinite(s_g).all()
    assert np.abs(s_g - s_o).max() <= TC_TOL[prec]
    np.testing.assert_allclose(a.cpu().numpy(), a_o, rtol=2 * AB_RTOL, atol=1e-7)
    np.testing.assert_allclose(b.cpu().numpy(), b_o, rtol=2 * AB_RTOL, atol=1e-7)
    # a row list takes the row-streaming tensor-core sweep instead
    rows = np.arange(0, X.shape[0], 5, dtype=np.int64)
    sr = silh.silh_exact(Xt, lt, k, metric, prec=prec, rows=torch.from_numpy(rows).cuda())
    assert np.abs(sr.cpu().numpy().astype(np.float64) - s_o[rows]).max() <= TC_TOL[prec]


@pytest.mark.parametrize("prec", ["3xtf32", "bf16x3"])
@pytest.mark.parametrize("metric", ["euclidean", "cosine"])
def test_tensor_core_rows_degenerate_and_bf16(metric, prec):
    X, lab, k = _degenerate()
    Xt, lt = _to_dev(X, lab)
    Xh = _host_values(Xt)
    gs = silh.silh_sample_pps(Xt, lt, k, metric, t=20.0, m0=6.0, seed=2)
    os_ = oracle.sample_pps(Xh, lab, k, metric, t=20.0, m0=6.0, seed=2)
    assert_same_sample(gs, os_, k, 2, 0, metric, lab)
    rows = torch.tensor([650, 3, 10, 21, 600, 0, 640], dtype=torch.int64, device="cuda")
    s = silh.silh_estimate(Xt, lt, k, gs, metric, prec=prec, rows=rows)
    s_o, _, _ = oracle.estimate(Xh, lab, k, metric, os_.offsets, os_.idx, os_.ps,
                                rows=rows.cpu().numpy())
    assert np.abs(s.cpu().numpy().astype(np.float64) - s_o).max() <= TC_TOL[prec]
    # BF16 storage through the tensor-core path
    X2, lab2, k2, kw2 = _case("multitile")
    Xb, lb = _to_dev(X2, lab2, torch.bfloat16)
    Xbh = _host_values(Xb)
    os2 = oracle.sample_pps(Xbh, lab2, k2, metric, t=128.0, seed=4)
    smp2 = silh.Sample.from_lists(np.bincount(lab2, minlength=k2), os2.offsets, os2.idx, os2.ps,
                                  Xb.device)
    r2 = torch.arange(0, 40000, 131, dtype=torch.int64, device="cuda")
    s2 = silh.silh_estimate(Xb, lb, k2, smp2, metric, prec=prec, rows=r2)
    s2_o, _, _ = oracle.estimate(Xbh, lab2, k2, metric, os2.offsets, os2.idx, os2.ps,
                                 rows=r2.cpu().numpy())
    assert np.abs(s2.cpu().numpy().astype(np.float64) - s2_o).max() <= TC_TOL[prec]
    silh.silh_stream_status()


# ------------------------------------------------- cohesion and separation

COHSEP_TOL = 1e-5     # relative: FP32 distances (<= a few ulp each), FP64 sums


@pytest.mark.parametrize("case", ["tiny", "ragged", "multitile"])
@pytest.mark.parametrize("metric", METRICS)
def test_cohsep_matches_oracle_on_oracle_sample(case, metric):
    X, lab, k, kw = _case(case)
    if metric == "canberra":
        X = synth.abs_shift(X)
    Xt, lt = _to_dev(X, lab)
    Xh = _host_values(Xt)
    os_ = oracle.sample_pps(Xh, lab, k, metric, t=kw["t"], m0=kw["m0"], seed=kw["seed"])
    smp = silh.Sample.from_lists(np.bincount(lab, minlength=k), os_.offsets, os_.idx, os_.ps,
                                 Xt.device)
    out = silh.silh_cohsep(Xt, lt, k, smp, metric).cpu().numpy()
    _, _, _, Wh = oracle.estimate(Xh, lab, k, metric, os_.offsets, os_.idx, os_.ps, want_w=True)
    coh, sep = oracle.cohsep(Wh, lab, k)
    assert out[0] == pytest.approx(coh, rel=COHSEP_TOL)
    assert out[1] == pytest.approx(sep, rel=COHSEP_TOL)


def test_cohsep_all_sampled_is_exact_and_bf16():
    """t above every cluster size: the estimate is the exact Coh/Sep; BF16 storage."""
    X, lab, k, _ = _case("ragged")
    for dtype in (torch.float32, torch.bfloat16):
        Xt, lt = _to_dev(X, lab, dtype)
        Xh = _host_values(Xt)
        gs = silh.silh_sample_pps(Xt, lt, k, "manhattan", t=1e9, seed=1)
        assert gs.size == X.shape[0]
        out = silh.silh_cohsep(Xt, lt, k, gs, "manhattan").cpu().numpy()
        os_ = oracle.sample_pps(Xh, lab, k, "manhattan", t=1e9, seed=1)
        _, _, _, W = oracle.estimate(Xh, lab, k, "manhattan", os_.offsets, os_.idx, os_.ps,
                                     want_w=True)
        coh, sep = oracle.cohsep(W, lab, k)
        assert out[0] == pytest.approx(coh, rel=COHSEP_TOL)
        assert out[1] == pytest.approx(sep, rel=COHSEP_TOL)


# ---------------------------------------- cosine: parallel-axis collapse

@pytest.mark.parametrize("case", ["tiny", "ragged", "multitile"])
def test_cosine_collapsed_matches_oracle(case):
    """The O(n k d) cosine path against the oracle's per-pair Eq. 8 estimate."""
    X, lab, k, kw = _case(case)
    Xt, lt = _to_dev(X, lab)
    Xh = _host_values(Xt)
    os_ = oracle.sample_pps(Xh, lab, k, "cosine", t=kw["t"], m0=kw["m0"], seed=kw["seed"])
    smp = silh.Sample.from_lists(np.bincount(lab, minlength=k), os_.offsets, os_.idx, os_.ps,
                                 Xt.device)
    s, a, b = silh.silh_estimate_cosine_collapsed(Xt, lt, k, smp, want_ab=True)
    s_o, a_o, b_o = oracle.estimate(Xh, lab, k, "cosine", os_.offsets, os_.idx, os_.ps)
    _assert_close(s, s_o, a, a_o, b, b_o)


def test_cosine_collapsed_degenerate_bf16_and_rows():
    """Zero vectors (distance 1 to everything), identical points, a singleton;
    BF16 storage; a row subset equals the same rows of the full output."""
    X, lab, k = _degenerate()
    for dtype in (torch.float32, torch.bfloat16):
        Xt, lt = _to_dev(X, lab, dtype)
        Xh = _host_values(Xt)
        gs = silh.silh_sample_pps(Xt, lt, k, "cosine", t=20.0, m0=6.0, seed=2)
        os_ = oracle.sample_pps(Xh, lab, k, "cosine", t=20.0, m0=6.0, seed=2)
        assert_same_sample(gs, os_, k, 2, 0, "cosine", lab)
        s = silh.silh_estimate_cosine_collapsed(Xt, lt, k, gs)
        s_o, _, _ = oracle.estimate(Xh, lab, k, "cosine", os_.offsets, os_.idx, os_.ps)
        _assert_close(s, s_o)
        assert s[-1].item() == 0.0
        rows = torch.tensor([10, 0, 650, 599, 10], dtype=torch.int64, device=Xt.device)
        sr = silh.silh_estimate_cosine_collapsed(Xt, lt, k, gs, rows=rows)
        assert torch.equal(sr, s[rows])


# ------------------------------------------------------ boundary checks

def test_pageable_host_buffers_are_rejected_before_any_launch():
    """A pageable host pointer in place of device memory is SILH_EINVAL, with
    nothing launched (the check is on the host, before the first kernel)."""
    import ctypes
    lib = silh.load()
    X, lab, k, _ = _case("tiny")
    Xt, lt = _to_dev(X, lab)
    n, d = X.shape
    gs = silh.silh_sample_pps(Xt, lt, k, "euclidean", t=64.0, m0=16.0, seed=0)
    torch.cuda.synchronize()
    Xh = np.ascontiguousarray(X, dtype=np.float32)
    lh = np.ascontiguousarray(lab, dtype=np.int32)
    sh = np.zeros(n, dtype=np.float32)
    s = torch.empty(n, dtype=torch.float32, device="cuda")
    g = torch.empty(1, dtype=torch.float64, device="cuda")
    st = gs.as_struct()
    launches = silh.kernel_launches()
    cases = [
        lib.silh_estimate(Xh.ctypes.data, 0, n, d, d, lt.data_ptr(), k, 0, 0, ctypes.byref(st),
                          None, 0, s.data_ptr(), None, None, None, None),
        lib.silh_estimate(Xt.data_ptr(), 0, n, d, d, lh.ctypes.data, k, 0, 0, ctypes.byref(st),
                          None, 0, s.data_ptr(), None, None, None, None),
        lib.silh_estimate(Xt.data_ptr(), 0, n, d, d, lt.data_ptr(), k, 0, 0, ctypes.byref(st),
                          None, 0, sh.ctypes.data, None, None, None, None),
        lib.silh_exact(Xh.ctypes.data, 0, n, d, d, lt.data_ptr(), k, 0, 0, None, 0,
                       s.data_ptr(), None, None, None, None),
        lib.silh_global(sh.ctypes.data, n, g.data_ptr(), None),
        lib.silh_global(s.data_ptr(), n, sh.ctypes.data, None),
    ]
    assert all(rc == -1 for rc in cases), cases
    assert b"device-accessible" in lib.silh_last_error()
    smp = silh.Sample.empty(k, n, "cuda")
    st2 = smp.as_struct()
    rc = lib.silh_sample_pps(Xh.ctypes.data, 0, n, d, d, lt.data_ptr(), k, 0, 64.0, 16.0, 0.01,
                             0, 0, 0, ctypes.byref(st2), None)
    assert rc == -1
    assert silh.kernel_launches() == launches
