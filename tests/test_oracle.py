"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: numpy's
Philox known answers, scipy/sklearn on tiny inputs, the printed worked example,
identities and bounds proved in the paper, and statistical properties of the
estimator.  None of these tests touches the GPU library.
"""
import math
import os

import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle
from paper_2607_01993_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SCIPY = {"euclidean": "euclidean", "cosine": "cosine", "manhattan": "cityblock",
         "canberra": "canberra"}


def _blobs(n, d, k, seed, sigma=1.0, shift=False):
    X, lab, _ = synth.gaussian_mixture(n, d, k, seed=seed, sigma=sigma)
    if shift:
        X = synth.abs_shift(X)
    return X.astype(np.float64), lab


# ------------------------------------------------------------------ RNG

@pytest.mark.parametrize("key", [0, 5, 0xDEADBEEFCAFEF00D])
@pytest.mark.parametrize("ctr", [(1, 0, 0, 0), (7, 1, 3, 0), (123456789, 2, 99, 5)])
def test_philox_matches_numpy_known_answers(key, ctr):
    # numpy's Philox (4x64, 10 rounds) advances its counter by one before
    # producing each block, so the block at counter c is numpy's first block
    # when numpy starts at c - 1.
    c = list(ctr)
    start = [c[0] - 1] + c[1:]
    g = np.random.Philox(key=np.array([key, 0], dtype=np.uint64),
                         counter=np.array(start, dtype=np.uint64))
    want = g.random_raw(4)
    got = oracle.philox4x64_10(c, [key, 0])
    assert list(got) == list(want)


@pytest.mark.parametrize("seed,stream,cid,e", [(0, 0, 0, 1), (0, 1, 0, 17), (42, 1, 7, 999)])
def test_uniform_matches_numpy_double_conversion(seed, stream, cid, e):
    # numpy's Generator.random() maps a 64-bit word to [0,1) as (w >> 11) * 2^-53,
    # the same conversion the oracle documents.
    g = np.random.Generator(np.random.Philox(
        key=np.array([seed, 0], dtype=np.uint64),
        counter=np.array([e - 1, stream, cid, 0], dtype=np.uint64)))
    assert oracle.uniform(seed, stream, cid, e) == g.random()


def test_uniform_is_uniform():
    u = np.array([oracle.uniform(3, 0, 0, e) for e in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    hist, _ = np.histogram(u, bins=20, range=(0, 1))
    chi2 = ((hist - 1000.0) ** 2 / 1000.0).sum()
    assert chi2 < 50.0  # 19 dof; p ~ 1e-4


# ------------------------------------------------------------ distances

@pytest.mark.parametrize("metric", ["euclidean", "cosine", "manhattan", "canberra"])
def test_distances_match_scipy(metric):
    rng = np.random.default_rng(1)
    X = rng.standard_normal((40, 7))
    Y = rng.standard_normal((30, 7))
    if metric == "canberra":
        X[3, 2] = 0.0
        Y[5, 2] = 0.0   # 0/0 term -> 0 (scipy convention)
    got = oracle.pairwise(metric, X, Y)
    want = cdist(X, Y, SCIPY[metric])
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_cosine_zero_vector_is_one():
    assert oracle.dist("cosine", [0.0, 0.0], [1.0, 2.0]) == 1.0


# ------------------------------------------------------ exact silhouette

def _figure1():
    rows, sc = [], None
    with open(os.path.join(GOLDEN, "figure1.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] == "s_C":
                sc = float(parts[1])
            else:
                rows.append(parts)
    X = np.array([[float(r[1]), float(r[2])] for r in rows])
    lab = np.array([int(r[3]) for r in rows], dtype=np.int32)
    printed = np.array([float(r[4]) for r in rows])
    return X, lab, printed, sc


def test_figure1_worked_example():
    X, lab, printed, sc = _figure1()
    s, a, b = oracle.exact(X, lab, 4, "euclidean")
    # panel (b) prints two decimals
    assert np.abs(s - printed).max() <= 0.005 + 1e-12
    assert s[14] == 0.0                       # singleton e15 (Sec. 2)
    assert s[13] < 0                           # e14 is closer to another cluster
    assert abs(oracle.mean(s) - sc) <= 0.5e-5  # s(C) printed to 5 decimals


@pytest.mark.parametrize("metric", ["euclidean", "cosine", "manhattan", "canberra"])
def test_exact_matches_sklearn(metric):
    silhouette_samples = pytest.importorskip("sklearn.metrics").silhouette_samples
    X, lab = _blobs(120, 5, 4, seed=3, sigma=3.0, shift=(metric == "canberra"))
    # add a singleton cluster
    lab = lab.copy()
    lab[7] = 4
    s, a, b = oracle.exact(X, lab, 5, metric)
    want = silhouette_samples(X, lab, metric=SCIPY[metric])
    np.testing.assert_allclose(s, want, rtol=1e-10, atol=1e-12)
    assert s[7] == 0.0
    assert (s >= -1).all() and (s <= 1).all()


def test_exact_row_subset_equals_full_rows():
    X, lab = _blobs(90, 4, 3, seed=4)
    rows = np.array([5, 0, 88, 41])
    s_all, _, _ = oracle.exact(X, lab, 3, "manhattan")
    s_sub, _, _ = oracle.exact(X, lab, 3, "manhattan", rows=rows)
    np.testing.assert_array_equal(s_sub, s_all[rows])


def test_invalid_clusterings_rejected():
    X, lab = _blobs(20, 3, 2, seed=0)
    with pytest.raises(ValueError):
        oracle.exact(X, lab, 3, "euclidean")        # cluster 2 empty
    bad = lab.copy(); bad[0] = 2
    with pytest.raises(ValueError):
        oracle.exact(X, bad, 2, "euclidean")        # label out of range
    with pytest.raises(ValueError):
        oracle.exact(X, np.zeros(20, np.int32), 1, "euclidean")  # k = 1


# --------------------------------------------------------------- Phase 1

def _cluster_weights(X, lab, k, metric):
    """W_j(e) for every e and j by brute force with scipy (Eq. 4)."""
    D = cdist(X, X, SCIPY[metric])
    return np.stack([D[:, lab == j].sum(1) for j in range(k)], axis=1), D


@pytest.mark.parametrize("metric", ["euclidean", "cosine", "manhattan", "canberra"])
def test_phase1_weights_and_gamma(metric):
    X, lab = _blobs(600, 4, 3, seed=5, sigma=2.0, shift=(metric == "canberra"))
    k, t = 3, 30.0
    smp = oracle.sample_pps(X, lab, k, metric, t=t, m0=6.0, seed=11, cid=2)
    W, D = _cluster_weights(X, lab, k, metric)
    sizes = np.bincount(lab, minlength=k)
    for j in range(k):
        members = np.flatnonzero(lab == j)
        f0 = np.flatnonzero(smp.in_f0 & (lab == j))
        assert len(f0) > 0
        # W of each initial-sample point is its full within-cluster sum (Eq. 4),
        # hence sum_{e in Cj} d(e, e_bar) / W(e_bar) = 1 (proof of Lemma 3).
        np.testing.assert_allclose(smp.w0[f0], W[f0, j], rtol=1e-12)
        ratio = D[np.ix_(members, f0)] / smp.w0[f0][None, :]
        np.testing.assert_allclose(ratio.sum(0), 1.0, rtol=1e-12)
        g = smp.gamma[members]
        # gamma is the larger of 1/|Cj| and the largest ratio (Algorithm 1)
        np.testing.assert_allclose(g, np.maximum(1.0 / sizes[j], ratio.max(1)), rtol=1e-12)
        assert (g >= 1.0 / sizes[j] - 1e-15).all()
        # sum of gamma bounded by 1 + |F0| (proof of Lemma 3)
        assert g.sum() <= 1.0 + len(f0) + 1e-9
        np.testing.assert_allclose(smp.p[members], np.minimum(1.0, t * g), rtol=1e-15)
    assert ((smp.p > 0) & (smp.p <= 1)).all()
    # the sample lists hold exactly the included elements, ascending per cluster
    for j in range(k):
        seg = smp.idx[smp.offsets[j]:smp.offsets[j + 1]]
        np.testing.assert_array_equal(seg, np.flatnonzero(smp.in_f & (lab == j)))
        np.testing.assert_array_equal(smp.ps[smp.offsets[j]:smp.offsets[j + 1]], smp.p[seg])


def test_small_clusters_taken_whole():
    X, lab = _blobs(200, 3, 4, seed=6)
    lab = lab.copy()
    sizes = np.bincount(lab)
    t = float(sizes.min())           # |Cj| <= t for the smallest cluster (Algorithm 1)
    smp = oracle.sample_pps(X, lab, 4, "euclidean", t=t, m0=5.0, seed=1)
    j = int(np.argmin(sizes))
    assert smp.in_f[lab == j].all()
    assert (smp.p[lab == j] == 1.0).all()
    assert not smp.in_f0[lab == j].any()


def test_f0_size_is_binomial():
    # |F0_j| ~ Bin(|Cj|, m0/|Cj|) (proof of Lemma 3)
    X, lab = _blobs(400, 2, 2, seed=7)
    sizes = np.bincount(lab)
    m0, R = 8.0, 400
    counts = np.zeros((R, 2))
    for r in range(R):
        smp = oracle.sample_pps(X, lab, 2, "euclidean", t=20.0, m0=m0, seed=1000 + r)
        counts[r] = [smp.in_f0[lab == j].sum() for j in range(2)]
    for j in range(2):
        q = m0 / sizes[j]
        mu, var = sizes[j] * q, sizes[j] * q * (1 - q)
        z = (counts[:, j].mean() - mu) / math.sqrt(var / R)
        assert abs(z) < 4.5


@pytest.mark.parametrize("k,delta", [(2, 0.01), (5, 0.2)])
def test_default_m0_is_two_ln_5k_over_delta(k, delta):
    # With m0 left to its default, Algorithm 1 draws the initial sample F0_j
    # with probability min(1, (2/|Cj|) ln(5k/delta)), so summed over the k
    # clusters E|F0| = sum_j |Cj| min(1, 2 ln(5k/delta)/|Cj|), with the binomial
    # variance.  A z-test over many seeds separates this from the MapReduce
    # round's ln(2k/delta) (z > 8 at these sizes), a dropped delta or factor 2.
    n = 200 * k
    X, lab = _blobs(n, 2, k, seed=20 + k)
    sizes = np.bincount(lab, minlength=k)
    t, R = 20.0, 300
    assert (sizes > t).all()          # every cluster draws an initial sample
    q = np.minimum(1.0, 2.0 * math.log(5.0 * k / delta) / sizes)
    mu, var = float((sizes * q).sum()), float((sizes * q * (1 - q)).sum())
    tot = np.array([oracle.sample_pps(X, lab, k, "euclidean", t=t, m0=None, delta=delta,
                                      seed=5000 + r).in_f0.sum() for r in range(R)])
    z = (tot.mean() - mu) / math.sqrt(var / R)
    assert abs(z) < 4.5, z
    # the alternative readings sit far outside that band
    for m_alt in (2.0 * math.log(2.0 * k / delta), 2.0 * math.log(5.0 * k),
                  math.log(5.0 * k / delta)):
        q_alt = np.minimum(1.0, m_alt / sizes)
        assert abs(float((sizes * q_alt).sum()) - mu) > 8 * math.sqrt(var / R)


def test_empty_initial_sample_gives_uniform_probabilities():
    # Clusters larger than t whose initial Poisson sample is empty (m0 tiny):
    # the maximum over F0_j ranges over no element, so gamma_e = 1/|Cj| (the
    # first term of Algorithm 1's maximum alone) and p_e = min(1, t/|Cj|) --
    # the probabilities of the uniform variant of Sec. 4.1.3, and the same draw.
    X, lab = _blobs(900, 3, 3, seed=12, sigma=2.0)
    k, t = 3, 30.0
    sizes = np.bincount(lab, minlength=k)
    assert (sizes > t).all()
    smp = oracle.sample_pps(X, lab, k, "manhattan", t=t, m0=1e-3, seed=6)
    assert not smp.in_f0.any()
    uni = oracle.sample_pps(X, lab, k, "manhattan", t=t, seed=6, uniform=True)
    for j in range(k):
        m = lab == j
        assert (smp.gamma[m] == 1.0 / sizes[j]).all()
        np.testing.assert_allclose(smp.p[m], t / sizes[j], rtol=2.0 ** -52, atol=0)
        np.testing.assert_allclose(uni.p[m], t / sizes[j], rtol=2.0 ** -52, atol=0)
    np.testing.assert_array_equal(smp.in_f, uni.in_f)
    # and the sample is the Poisson draw of those probabilities on stream 1
    np.testing.assert_array_equal(smp.in_f, oracle.poisson_draw(6, 1, 0, t / sizes[lab]))


def test_poisson_draw_frequency():
    probs = np.array([0.0, 0.05, 0.3, 0.5, 0.9, 1.0])
    R = 4000
    hits = np.zeros(len(probs))
    for r in range(R):
        hits += oracle.poisson_draw(r, 1, 0, probs)
    freq = hits / R
    assert freq[0] == 0.0 and freq[-1] == 1.0
    sd = np.sqrt(probs * (1 - probs) / R)
    assert (np.abs(freq[1:-1] - probs[1:-1]) <= 4.5 * sd[1:-1]).all()


# --------------------------------------------------------------- Phase 2

@pytest.mark.parametrize("metric", ["euclidean", "cosine", "manhattan", "canberra"])
def test_all_probabilities_one_gives_exact(metric):
    # |Cj| <= t for every j: F_j = C_j, p = 1, so Phase 2 is the definition.
    X, lab = _blobs(150, 4, 3, seed=8, sigma=2.0, shift=(metric == "canberra"))
    smp = oracle.sample_pps(X, lab, 3, metric, t=1e9, seed=2)
    assert smp.size == 150 and (smp.ps == 1.0).all()
    s_hat, a_hat, b_hat = oracle.estimate(X, lab, 3, metric, smp.offsets, smp.idx, smp.ps)
    s, a, b = oracle.exact(X, lab, 3, metric)
    np.testing.assert_allclose(s_hat, s, rtol=0, atol=1e-13)
    np.testing.assert_allclose(a_hat, a, rtol=1e-13)
    np.testing.assert_allclose(b_hat, b, rtol=1e-13)


def test_weight_estimator_is_unbiased():
    # E[W_hat_j(e)] = W_j(e) with the p's fixed (proof of Lemma 1), and the
    # variance of a Poisson-sampling Horvitz-Thompson sum is
    # sum d^2 (1 - p) / p.  Draws are independent Bernoulli(p) from numpy.
    X, lab = _blobs(240, 3, 3, seed=9, sigma=2.5)
    k = 3
    smp = oracle.sample_pps(X, lab, k, "euclidean", t=12.0, m0=5.0, seed=3)
    W, D = _cluster_weights(X, lab, k, "euclidean")
    rows = np.array([0, 17, 101, 200])
    rng = np.random.default_rng(0)
    R = 1500
    acc = np.zeros((len(rows), k))
    for _ in range(R):
        inc = rng.random(240) < smp.p
        off, idx, ps = oracle.build_sample(lab, k, inc, smp.p)
        _, _, _, Wh = oracle.estimate(X, lab, k, "euclidean", off, idx, ps, rows=rows,
                                      want_w=True)
        acc += Wh
    mean = acc / R
    for r, e in enumerate(rows):
        for j in range(k):
            mask = lab == j
            var = (D[e, mask] ** 2 * (1 - smp.p[mask]) / smp.p[mask]).sum()
            sd = math.sqrt(var / R) + 1e-12
            assert abs(mean[r, j] - W[e, j]) <= 4.5 * sd


def test_lemma2_bound_holds_for_realised_error():
    # Lemma 2: if every W_hat_j(e) has relative error <= eps < 1 then
    # |s_hat(e) - s(e)| <= 4 eps / (1 - eps).  Check it per element with that
    # element's realised eps.
    X, lab = _blobs(500, 4, 4, seed=10, sigma=3.0)
    k = 4
    smp = oracle.sample_pps(X, lab, k, "manhattan", t=25.0, m0=8.0, seed=4)
    s_hat, _, _, Wh = oracle.estimate(X, lab, k, "manhattan", smp.offsets, smp.idx, smp.ps,
                                      want_w=True)
    W, _ = _cluster_weights(X, lab, k, "manhattan")
    s, _, _ = oracle.exact(X, lab, k, "manhattan")
    eps = (np.abs(Wh - W) / W).max(1)
    ok = eps < 1
    assert ok.sum() > 400
    bound = 4 * eps[ok] / (1 - eps[ok])
    assert (np.abs(s_hat[ok] - s[ok]) <= bound + 1e-12).all()


def _theorem2_instance(m, L):
    """1-D instance of Theorem 2: two clusters of m points packed near 0 and
    near -1/m, each with one far outlier (R1 = L (R2+1) m/(m+1), R2 = m)."""
    r = 1e-3 / m
    c1 = np.linspace(-r, r, m)
    c2 = -1.0 / m + np.linspace(-r / 2, r / 2, m)
    R2 = float(m)
    R1 = L * (R2 + 1) * m / (m + 1)
    X = np.concatenate([c1, [R1], c2, [-R2]])[:, None]
    lab = np.array([0] * (m + 1) + [1] * (m + 1), dtype=np.int32)
    return X, lab


def test_theorem2_instance_pps_vs_uniform():
    m, L, t = 2000, 10.0, 40.0
    X, lab = _theorem2_instance(m, L)
    s, _, _ = oracle.exact(X, lab, 2, "euclidean")
    inner = np.arange(m)
    # Proposition 1: s(e_i) ~ (1 - L)/L
    assert np.abs(s[inner] - (1 - L) / L).max() < 0.01
    pps = oracle.sample_pps(X, lab, 2, "euclidean", t=t, m0=16.0, seed=5)
    assert pps.in_f[m] and pps.in_f[2 * m + 1]       # both outliers sampled
    s_pps, _, _ = oracle.estimate(X, lab, 2, "euclidean", pps.offsets, pps.idx, pps.ps,
                                  rows=inner)
    assert np.abs(s_pps - s[inner]).max() < 0.05      # PPS close to exact (~ -0.9)
    uni = oracle.sample_pps(X, lab, 2, "euclidean", t=t, seed=6, uniform=True)
    assert not uni.in_f[m]                            # outlier missed (prob 1 - t/(m+1))
    s_uni, _, _ = oracle.estimate(X, lab, 2, "euclidean", uni.offsets, uni.idx, uni.ps,
                                  rows=inner)
    assert s_uni.min() > 0.9                          # uniform sampling says ~ +1


def test_estimate_respects_row_subset_and_singletons():
    X, lab = _blobs(200, 3, 3, seed=12)
    lab = lab.copy(); lab[10] = 3
    smp = oracle.sample_pps(X, lab, 4, "canberra", t=20.0, m0=5.0, seed=7)
    s_all, _, _ = oracle.estimate(X, lab, 4, "canberra", smp.offsets, smp.idx, smp.ps)
    rows = np.array([10, 3, 199])
    s_sub, _, _ = oracle.estimate(X, lab, 4, "canberra", smp.offsets, smp.idx, smp.ps,
                                  rows=rows)
    np.testing.assert_array_equal(s_sub, s_all[rows])
    assert s_all[10] == 0.0
    assert (np.abs(s_all) <= 1).all()


# ---------------------------------------------------------------- global

def test_global_mean_is_exact_mean():
    rng = np.random.default_rng(0)
    v = rng.uniform(-1, 1, 100001)
    assert abs(oracle.mean(v) - math.fsum(v) / len(v)) <= 1e-16
    assert oracle.mean(np.array([1e16, 1.0, -1e16, 1.0])) == 0.5


def test_t_from_eps_lemma1():
    # Lemma 1: t = ceil((3c/eps^2) ln(5nk/delta)) with c = 18.
    assert oracle.t_from_eps(0.5, 0.01, 1000, 4) == math.ceil(216 * math.log(5 * 4000 / 0.01))


# ------------------------------------------------- cohesion and separation

@pytest.mark.parametrize("metric", ["euclidean", "cosine", "manhattan", "canberra"])
def test_cohesion_separation_are_mean_pair_distances(metric):
    # Coh is the mean distance over unordered same-cluster pairs, Sep the mean
    # over unordered cross-cluster pairs; scipy's pdist gives both by brute
    # force.  Exact W (all p = 1) must reproduce them through the estimator.
    from scipy.spatial.distance import pdist
    X, lab = _blobs(160, 5, 4, seed=21, sigma=2.0, shift=(metric == "canberra"))
    k = 4
    iu = np.triu_indices(X.shape[0], 1)
    dv = pdist(X, SCIPY[metric])
    same = lab[iu[0]] == lab[iu[1]]
    coh_ref, sep_ref = dv[same].mean(), dv[~same].mean()
    W, _ = _cluster_weights(X, lab, k, metric)
    coh, sep = oracle.cohsep(W, lab, k)
    assert coh == pytest.approx(coh_ref, rel=1e-12)
    assert sep == pytest.approx(sep_ref, rel=1e-12)
    smp = oracle.sample_pps(X, lab, k, metric, t=1e9, seed=1)
    _, _, _, Wh = oracle.estimate(X, lab, k, metric, smp.offsets, smp.idx, smp.ps, want_w=True)
    coh2, sep2 = oracle.cohsep(Wh, lab, k)
    assert coh2 == pytest.approx(coh_ref, rel=1e-12)
    assert sep2 == pytest.approx(sep_ref, rel=1e-12)


def test_cohesion_separation_two_clusters_and_singletons():
    # k = 2: Sep = sum_{e in C0} W_C1(e) / (|C0| |C1|).  Singleton clusters add
    # no same-cluster pairs; all-singleton clusterings have Coh = 0.
    X, lab = _blobs(50, 3, 2, seed=22)
    W, D = _cluster_weights(X, lab, 2, "euclidean")
    _, sep = oracle.cohsep(W, lab, 2)
    c0, c1 = lab == 0, lab == 1
    assert sep == pytest.approx(D[np.ix_(c0, c1)].sum() / (c0.sum() * c1.sum()), rel=1e-12)
    lab1 = np.arange(6, dtype=np.int32)
    W1, D1 = _cluster_weights(X[:6], lab1, 6, "euclidean")
    coh, sep = oracle.cohsep(W1, lab1, 6)
    assert coh == 0.0
    assert sep == pytest.approx(D1[np.triu_indices(6, 1)].mean(), rel=1e-12)


def test_cohesion_separation_error_bounded_by_weight_error():
    # Both numerators are positive combinations of the W_hat_j(e), so if every
    # W_hat_j(e) is within relative eps of W_j(e) the estimates are within eps
    # of Coh and Sep (the argument behind the appendix's theorem).
    X, lab = _blobs(900, 4, 5, seed=23, sigma=2.0)
    k = 5
    W, _ = _cluster_weights(X, lab, k, "euclidean")
    coh, sep = oracle.cohsep(W, lab, k)
    for seed in range(3):
        smp = oracle.sample_pps(X, lab, k, "euclidean", t=40.0, seed=seed)
        _, _, _, Wh = oracle.estimate(X, lab, k, "euclidean", smp.offsets, smp.idx, smp.ps,
                                      want_w=True)
        eps = np.max(np.abs(Wh - W) / W)
        ch, sh = oracle.cohsep(Wh, lab, k)
        assert abs(ch - coh) <= eps * coh * (1 + 1e-12)
        assert abs(sh - sep) <= eps * sep * (1 + 1e-12)


def _neighbour_brute(X, lab, k, metric):
    """b(e) and its cluster written out from Eq. 2 with plain loops: the mean
    distance to every other cluster, the smallest one, the lowest cluster
    index among equal means."""
    n = X.shape[0]
    nb = np.empty(n, dtype=np.int64)
    bv = np.empty(n)
    for e in range(n):
        best, arg = np.inf, -1
        for j in range(k):
            if j == lab[e]:
                continue
            members = [f for f in range(n) if lab[f] == j]
            m = sum(oracle.dist(metric, X[e], X[f]) for f in members) / len(members)
            if m < best:
                best, arg = m, j
        nb[e], bv[e] = arg, best
    return nb, bv


def test_figure1_neighbour_of_e14_gives_the_printed_value():
    # With the printed values' reading of e14 (-2.5, -3), b(e14) is its distance
    # to the singleton C4 = {e15}, 0.5, which with a(e14) gives the printed
    # s(e14) = -0.89 (Example 1 names C3, the reading of the drawn coordinate)
    X, lab, printed, _ = _figure1()
    s, a, b, nb = oracle.exact(X, lab, 4, "euclidean", want_nb=True)
    assert nb[13] == 3 and b[13] == 0.5
    assert round((b[13] - a[13]) / a[13], 2) == printed[13]
    want, bw = _neighbour_brute(X, lab, 4, "euclidean")
    np.testing.assert_array_equal(nb, want)
    np.testing.assert_allclose(b, bw, rtol=1e-14)


@pytest.mark.parametrize("metric", ["euclidean", "cosine", "manhattan", "canberra"])
def test_exact_neighbour_matches_brute_force(metric):
    X, lab = _blobs(60, 3, 4, seed=11, sigma=4.0, shift=(metric == "canberra"))
    s, a, b, nb = oracle.exact(X, lab, 4, metric, want_nb=True)
    want, bw = _neighbour_brute(X, lab, 4, metric)
    np.testing.assert_array_equal(nb, want)
    np.testing.assert_allclose(b, bw, rtol=1e-12)
    assert (nb != lab).all()


def test_neighbour_ties_take_the_lowest_cluster():
    # clusters 1 and 2 are mirror images about the y axis, so every point of
    # cluster 0 (on the axis) is at exactly equal mean distance from them
    X = np.array([[0.0, 0.0], [0.0, 1.0], [0.0, -1.5],
                  [4.0, 0.0], [5.0, 1.0], [6.0, -2.0],
                  [-4.0, 0.0], [-5.0, 1.0], [-6.0, -2.0]])
    lab = np.array([0, 0, 0, 1, 1, 1, 2, 2, 2], dtype=np.int32)
    for metric in ("euclidean", "manhattan"):
        _, _, b, nb = oracle.exact(X, lab, 3, metric, want_nb=True)
        assert (nb[:3] == 1).all()
        lab2 = np.array([0, 0, 0, 2, 2, 2, 1, 1, 1], dtype=np.int32)   # swap the names
        _, _, b2, nb2 = oracle.exact(X, lab2, 3, metric, want_nb=True)
        assert (nb2[:3] == 1).all() and np.array_equal(b[:3], b2[:3])


def test_estimate_neighbour_with_every_p_one_is_exact():
    # t >= max |Cj|: every p = 1, F_j = C_j, and Eq. 8 is Eq. 1-2
    X, lab = _blobs(80, 4, 5, seed=12, sigma=3.0)
    smp = oracle.sample_pps(X, lab, 5, "euclidean", t=1000.0, seed=1)
    assert (smp.p == 1.0).all()
    _, _, _, nb_e = oracle.estimate(X, lab, 5, "euclidean", smp.offsets, smp.idx, smp.ps,
                                    want_nb=True)
    _, _, _, nb_x = oracle.exact(X, lab, 5, "euclidean", want_nb=True)
    np.testing.assert_array_equal(nb_e, nb_x)
