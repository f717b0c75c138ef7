"""Batched Phase 2: many clusterings of one dataset in one persistent launch.

Each item's result must equal the single-clustering sweep (same arithmetic),
match the oracle on sampled rows within the FP32 bound, survive CUDA-graph
capture and replay, and agree across the autotuner's tile variants.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_01993_b300 import autotune, silh, synth

pytestmark = pytest.mark.gpu
S_TOL = 1e-5


def _dataset(n, d, seed, ks):
    X, _, _ = synth.gaussian_mixture(n, d, 16, seed=seed, sigma=1.5)
    labels = [synth.nearest_centre_labels(X, k, seed=seed + 10 * k) for k in ks]
    return X, labels


@pytest.fixture(scope="module")
def batch():
    ks = [2, 3, 5, 9, 17, 33]
    X, labels = _dataset(30000, 16, 40, ks)
    Xt = torch.from_numpy(X).cuda()
    items = []
    for c, (k, lab) in enumerate(zip(ks, labels)):
        lt = torch.from_numpy(lab).cuda()
        smp = silh.silh_sample_pps(Xt, lt, k, "euclidean", t=64.0, seed=5, clustering_id=c)
        items.append((lt, smp))
    return X, Xt, ks, labels, items


def test_batched_equals_single_sweeps(batch):
    X, Xt, ks, labels, items = batch
    outs = silh.silh_estimate_batched(Xt, items, "euclidean")
    for (lt, smp), k, out in zip(items, ks, outs):
        ref = silh.silh_estimate(Xt, lt, k, smp, "euclidean", prec="fp32")
        assert torch.equal(out, ref)


def test_batched_matches_oracle_on_sampled_rows(batch):
    X, Xt, ks, labels, items = batch
    outs = silh.silh_estimate_batched(Xt, items, "euclidean")
    Xh = X.astype(np.float64)
    rows = synth.seeded_rows(X.shape[0], 150, seed=3)
    for c in (0, 4, 5):
        os_ = oracle.sample_pps(Xh, labels[c], ks[c], "euclidean", t=64.0, seed=5, cid=c)
        s_o, _, _ = oracle.estimate(Xh, labels[c], ks[c], "euclidean", os_.offsets, os_.idx,
                                    os_.ps, rows=rows)
        got = outs[c][torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
        assert np.abs(got - s_o).max() <= S_TOL


@pytest.mark.parametrize("variant", range(silh.BATCH_VARIANTS))
def test_variants_agree(batch, variant):
    X, Xt, ks, labels, items = batch
    ref = silh.silh_estimate_batched(Xt, items, "euclidean", variant=-1)
    got = silh.silh_estimate_batched(Xt, items, "euclidean", variant=variant)
    for a, b in zip(got, ref):
        assert (a - b).abs().max().item() <= 1e-6


def test_graph_capture_and_replay(batch):
    X, Xt, ks, labels, items = batch
    outs = [torch.empty(X.shape[0], dtype=torch.float32, device="cuda") for _ in items]
    silh.silh_estimate_batched(Xt, items, "euclidean", outs=outs)      # warm-up off-graph
    torch.cuda.synchronize()
    ref = [o.clone() for o in outs]
    for o in outs:
        o.fill_(7.0)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        silh.silh_estimate_batched(Xt, items, "euclidean", outs=outs)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(outs, ref):
        assert torch.equal(a, b)
    for o in outs:
        o.fill_(7.0)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(outs, ref):
        assert torch.equal(a, b)


def test_autotuner_picks_a_variant(batch, tmp_path, monkeypatch):
    X, Xt, ks, labels, items = batch
    monkeypatch.setenv("SILH_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    v, times = autotune.tune_batched(Xt, items[:3], "euclidean", reps=1)
    assert 0 <= v < silh.BATCH_VARIANTS and len(times) == silh.BATCH_VARIANTS
    v2, _ = autotune.tune_batched(Xt, items[:3], "euclidean")        # cached
    assert v2 == v


@pytest.mark.parametrize("prec", ["3xtf32", "tf32"])
@pytest.mark.parametrize("metric", ["euclidean", "cosine"])
def test_tensor_core_tile_variants_equal_single_calls(batch, prec, metric):
    # the default tile shape of the batched tensor-core sweep (128 columns, one
    # accumulator per row tile) gives silh_estimate's results bit for bit; the
    # 64-column one (two accumulators) folds FP32 partial sums into FP64 every
    # 64 columns instead of 128, so it agrees to FP32 rounding
    X, Xt, ks, labels, items = batch
    want = [silh.silh_estimate(Xt, lt, k, smp, metric, prec=prec)
            for (lt, smp), k in zip(items, ks)]
    for v in (0, 1):
        got = silh.silh_estimate_batched(Xt, items, metric, variant=v, prec=prec)
        for a, b in zip(got, want):
            if v == 0:
                assert torch.equal(a, b), (metric, prec)
            else:
                assert (a - b).abs().max().item() <= 1e-6, (metric, prec)


def test_autotuner_times_the_tensor_core_variants(batch, tmp_path, monkeypatch):
    X, Xt, ks, labels, items = batch
    monkeypatch.setenv("SILH_AUTOTUNE_CACHE", str(tmp_path / "tune_tc.json"))
    v, times = autotune.tune_batched(Xt, items[:3], "euclidean", reps=1, prec="3xtf32")
    assert v in (0, 1) and sorted(times) == ["0", "1"]
    assert autotune.tune_batched(Xt, items[:3], "euclidean", prec="3xtf32")[0] == v


@pytest.mark.parametrize("metric", ["cosine", "manhattan", "canberra"])
def test_batched_other_metrics(metric):
    X, labels = _dataset(8000, 13, 41, [3, 7])
    if metric == "canberra":
        X = synth.abs_shift(X)
    Xt = torch.from_numpy(X).cuda()
    items = []
    for c, (k, lab) in enumerate(zip([3, 7], labels)):
        lt = torch.from_numpy(lab).cuda()
        items.append((lt, silh.silh_sample_pps(Xt, lt, k, metric, t=32.0, m0=8.0, seed=c)))
    outs = silh.silh_estimate_batched(Xt, items, metric)
    for (lt, smp), k, out in zip(items, [3, 7], outs):
        ref = silh.silh_estimate(Xt, lt, k, smp, metric, prec="fp32")
        assert torch.equal(out, ref)


# ---------------------------------------------------------------- tensor cores
# With prec tf32 / 3xtf32 / bf16 / bf16x3 (Euclidean or cosine, d <= 64) the
# batched call runs one persistent tensor-core sweep over every (clustering,
# row group); each clustering is swept exactly as silh_estimate sweeps it, so
# the results are equal bit for bit, and within the per-precision bound of the
# oracle.
TC_TOL = {"3xtf32": S_TOL, "tf32": 2e-3, "bf16x3": 2e-5, "bf16": 5e-3}
TC_PRECS = ["3xtf32", "tf32", "bf16x3", "bf16"]


def _items(Xt, ks, labels, metric, t=64.0):
    items = []
    for c, (k, lab) in enumerate(zip(ks, labels)):
        lt = torch.from_numpy(lab).cuda()
        items.append((lt, silh.silh_sample_pps(Xt, lt, k, metric, t=t, seed=5, clustering_id=c)))
    return items


@pytest.mark.parametrize("prec", TC_PRECS)
@pytest.mark.parametrize("metric", ["euclidean", "cosine"])
def test_batched_tensor_cores_equal_single_sweeps(batch, metric, prec):
    X, Xt, ks, labels, items = batch
    if metric != "euclidean":
        items = _items(Xt, ks, labels, metric)
    outs = silh.silh_estimate_batched(Xt, items, metric, prec=prec)
    for (lt, smp), k, out in zip(items, ks, outs):
        ref = silh.silh_estimate(Xt, lt, k, smp, metric, prec=prec)
        assert torch.equal(out, ref)


@pytest.mark.parametrize("prec", ["3xtf32", "bf16x3"])
@pytest.mark.parametrize("metric", ["euclidean", "cosine"])
def test_batched_tensor_cores_match_oracle(batch, metric, prec):
    X, Xt, ks, labels, items = batch
    items = _items(Xt, ks, labels, metric)
    outs = silh.silh_estimate_batched(Xt, items, metric, prec=prec)
    Xh = X.astype(np.float64)
    rows = synth.seeded_rows(X.shape[0], 150, seed=4)
    for c in (0, 3, 5):
        os_ = oracle.sample_pps(Xh, labels[c], ks[c], metric, t=64.0, seed=5, cid=c)
        s_o, _, _ = oracle.estimate(Xh, labels[c], ks[c], metric, os_.offsets, os_.idx,
                                    os_.ps, rows=rows)
        got = outs[c][torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
        assert np.abs(got - s_o).max() <= TC_TOL[prec]


@pytest.mark.parametrize("prec", ["3xtf32", "tf32", "bf16"])
def test_batched_tensor_cores_two_block_rows_bf16_data(prec):
    # d = 50: two 128-byte K blocks for TF32 operands (two row tiles per group);
    # BF16 storage; n = 7001 leaves a ragged last row group
    ks = [2, 6, 11]
    X, labels = _dataset(7001, 50, 42, ks)
    Xt = torch.from_numpy(X).cuda().to(torch.bfloat16)
    items = _items(Xt, ks, labels, "euclidean", t=48.0)
    outs = silh.silh_estimate_batched(Xt, items, "euclidean", prec=prec)
    for (lt, smp), k, out in zip(items, ks, outs):
        assert torch.equal(out, silh.silh_estimate(Xt, lt, k, smp, "euclidean", prec=prec))


def test_batched_tensor_cores_more_items_than_one_launch():
    # 300 clusterings: more than one launch's item table holds
    rng = np.random.default_rng(43)
    ks = [int(v) for v in rng.integers(2, 7, size=300)]
    X, _, _ = synth.gaussian_mixture(2500, 8, 6, seed=43, sigma=1.0)
    labels = [synth.nearest_centre_labels(X, k, seed=500 + i) for i, k in enumerate(ks)]
    Xt = torch.from_numpy(X).cuda()
    items = _items(Xt, ks, labels, "cosine", t=24.0)
    outs = silh.silh_estimate_batched(Xt, items, "cosine", prec="3xtf32")
    for (lt, smp), k, out in zip(items, ks, outs):
        assert torch.equal(out, silh.silh_estimate(Xt, lt, k, smp, "cosine", prec="3xtf32"))


def test_batched_tensor_cores_graph_capture_and_replay(batch):
    X, Xt, ks, labels, items = batch
    outs = [torch.empty(X.shape[0], dtype=torch.float32, device="cuda") for _ in items]
    silh.silh_estimate_batched(Xt, items, "euclidean", outs=outs, prec="3xtf32")
    torch.cuda.synchronize()
    ref = [o.clone() for o in outs]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        silh.silh_estimate_batched(Xt, items, "euclidean", outs=outs, prec="3xtf32")
    for _ in range(2):
        for o in outs:
            o.fill_(7.0)
        g.replay()
        torch.cuda.synchronize()
        for a, b in zip(outs, ref):
            assert torch.equal(a, b)


@pytest.mark.parametrize("d", [40, 100])
@pytest.mark.parametrize("metric", ["euclidean", "canberra"])
def test_batched_equals_single_wide_rows(d, metric):
    # rows padded to 64 and 128 elements: the default tile shape is the single
    # sweep's (64 columns per stage; 32 for Canberra at 128), so the results
    # are equal bit for bit
    X, _, _ = synth.gaussian_mixture(5000, d, 6, seed=d, sigma=1.5)
    if metric == "canberra":
        X = synth.abs_shift(X)
    Xt = torch.from_numpy(X).cuda()
    items, ks = [], [3, 7]
    for c, k in enumerate(ks):
        lt = torch.from_numpy(synth.nearest_centre_labels(X, k, seed=c)).cuda()
        items.append((lt, silh.silh_sample_pps(Xt, lt, k, metric, t=64.0, seed=c,
                                               clustering_id=c)))
    outs = silh.silh_estimate_batched(Xt, items, metric)
    for (lt, smp), k, out in zip(items, ks, outs):
        assert torch.equal(out, silh.silh_estimate(Xt, lt, k, smp, metric, prec="fp32"))
    # every tile shape launches at these widths and agrees to rounding
    for v in range(silh.BATCH_VARIANTS):
        got = silh.silh_estimate_batched(Xt, items, metric, variant=v)
        for a, b in zip(got, outs):
            assert (a - b).abs().max().item() <= 1e-6
