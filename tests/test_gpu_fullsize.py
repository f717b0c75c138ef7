"""Parity at the full workload sizes, in the launch configuration bench.py times.

The oracle runs Phase 1 in full (FP64, all n) so the sample sets are compared
element by element; Phase 2 and the exact silhouette are compared on seeded
row samples that the oracle evaluates one by one.  The global mean is checked
as a property that holds at any size (FP64 mean of the GPU's own s values).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_01993_b300 import silh, synth
from test_gpu_parity import S_TOL, _assert_close, _host_values, assert_same_sample

pytestmark = pytest.mark.gpu

LARGE = dict(n=1_000_000, d=32, k=32, t=256.0, delta=0.01, exact_rows=100_000, seed=1)


@pytest.fixture(scope="module")
def large():
    w = LARGE
    X, lab, _ = synth.large(seed=w["seed"], n=w["n"], d=w["d"], k=w["k"])
    rows_ex = synth.seeded_rows(w["n"], w["exact_rows"], seed=w["seed"] + 1000)
    return X, lab, rows_ex


PREC = {"euclidean": "3xtf32", "cosine": "3xtf32", "manhattan": "fp32", "canberra": "fp32"}


@pytest.mark.parametrize("metric", ["euclidean", "cosine", "manhattan", "canberra"])
def test_large_workload_sampled_parity(large, metric):
    """The launch configuration bench.py times (same precision per metric)."""
    w = LARGE
    X, lab, rows_ex = large
    if metric == "canberra":
        X = synth.abs_shift(X)
    k = w["k"]
    Xt = torch.from_numpy(X).cuda()
    lt = torch.from_numpy(lab).cuda()
    gs = silh.silh_sample_pps(Xt, lt, k, metric, t=w["t"], delta=w["delta"], seed=7,
                              clustering_id=1)
    s = silh.silh_estimate(Xt, lt, k, gs, metric, prec=PREC[metric])
    g = silh.silh_global(s).item()
    silh.silh_stream_status()
    Xh = X.astype(np.float64)
    os_ = oracle.sample_pps(Xh, lab, k, metric, t=w["t"], delta=w["delta"], seed=7, cid=1)
    ties = assert_same_sample(gs, os_, k, 7, 1, metric, lab)
    assert ties <= 2
    rows = synth.seeded_rows(w["n"], 300, seed=11)
    s_o, _, _ = oracle.estimate(Xh, lab, k, metric, os_.offsets, os_.idx, os_.ps, rows=rows)
    _assert_close(s[torch.from_numpy(rows).cuda()], s_o)
    s_h = s.cpu().numpy().astype(np.float64)
    assert np.isfinite(s_h).all() and (np.abs(s_h) <= 1).all()
    assert abs(g - s_h.mean()) <= 1e-9

    # exact silhouette of the 100k-row sub-dataset, checked on 200 of its rows
    Xs = np.ascontiguousarray(X[rows_ex])
    ls = np.ascontiguousarray(lab[rows_ex])
    se = silh.silh_exact(torch.from_numpy(Xs).cuda(), torch.from_numpy(ls).cuda(), k, metric,
                         prec=PREC[metric])
    r3 = synth.seeded_rows(len(rows_ex), 200, seed=12)
    se_o, _, _ = oracle.exact(Xs.astype(np.float64), ls, k, metric, rows=r3)
    _assert_close(se[torch.from_numpy(r3).cuda()], se_o)


def test_large_workload_cosine_collapsed(large):
    """The O(n k d) cosine path at n = 1M: sampled rows against the oracle, and
    every row against the per-pair tensor-core estimate on the same sample."""
    w = LARGE
    X, lab, _ = large
    k = w["k"]
    Xt = torch.from_numpy(X).cuda()
    lt = torch.from_numpy(lab).cuda()
    gs = silh.silh_sample_pps(Xt, lt, k, "cosine", t=w["t"], delta=w["delta"], seed=7,
                              clustering_id=1)
    sc = silh.silh_estimate_cosine_collapsed(Xt, lt, k, gs)
    sp = silh.silh_estimate(Xt, lt, k, gs, "cosine", prec="3xtf32")
    assert (sc - sp).abs().max().item() <= 2 * S_TOL
    Xh = X.astype(np.float64)
    os_ = oracle.sample_pps(Xh, lab, k, "cosine", t=w["t"], delta=w["delta"], seed=7, cid=1)
    assert_same_sample(gs, os_, k, 7, 1, "cosine", lab)
    rows = synth.seeded_rows(w["n"], 300, seed=11)
    s_o, _, _ = oracle.estimate(Xh, lab, k, "cosine", os_.offsets, os_.idx, os_.ps, rows=rows)
    _assert_close(sc[torch.from_numpy(rows).cuda()], s_o)


def test_precision_workload_bf16_sampled_parity():
    """n = 4M, d = 64, k = 64, 10% border points, data stored BF16; Euclidean."""
    X, lab, _ = synth.precision(seed=2)
    k, t = 64, 128.0
    Xt = torch.from_numpy(X).cuda().to(torch.bfloat16)
    del X
    lt = torch.from_numpy(lab).cuda()
    gs = silh.silh_sample_pps(Xt, lt, k, "euclidean", t=t, delta=0.01, seed=3)
    Xh = _host_values(Xt)
    os_ = oracle.sample_pps(Xh, lab, k, "euclidean", t=t, delta=0.01, seed=3)
    assert_same_sample(gs, os_, k, 3, 0)
    rows = synth.seeded_rows(lab.shape[0], 200, seed=13)
    s_o, _, _ = oracle.estimate(Xh, lab, k, "euclidean", os_.offsets, os_.idx, os_.ps, rows=rows)
    tol = {"fp32": S_TOL, "3xtf32": S_TOL, "bf16x3": 2e-5, "bf16": 5e-3}
    for prec in ("fp32", "3xtf32", "bf16x3", "bf16"):
        s = silh.silh_estimate(Xt, lt, k, gs, "euclidean", prec=prec,
                               rows=torch.from_numpy(rows).cuda())
        err = np.abs(s.cpu().numpy().astype(np.float64) - s_o).max()
        assert err <= tol[prec], (prec, err)
    assert S_TOL == 1e-5


def test_batching_workload_sampled_parity():
    """n = 500k, d = 16; clusterings with k in {2, 3, 17, 64, 257} (nearest random
    data-row centres) of the 256-clustering batching workload, t = 128, in one
    batched launch; each checked against the oracle on 100 seeded rows."""
    X = synth.batching(seed=3)
    Xt = torch.from_numpy(X).cuda()
    ks = [2, 3, 17, 64, 257]
    items, labs = [], []
    for k in ks:
        lt = synth.nearest_centre_labels_device(Xt, k, seed=1000 + k)
        labs.append(lt.cpu().numpy())
        items.append((lt, silh.silh_sample_pps(Xt, lt, k, "euclidean", t=128.0, seed=7,
                                               clustering_id=k - 2)))
    outs = silh.silh_estimate_batched(Xt, items, "euclidean")
    # the same launch on the tensor cores (split TF32): the data put many close
    # pairs in neighbouring clusters, so the direct FP32 recompute carries much
    # of the accuracy; held to the same bound
    outs_tc = silh.silh_estimate_batched(Xt, items, "euclidean", prec="3xtf32")
    Xh = X.astype(np.float64)
    rows = synth.seeded_rows(X.shape[0], 100, seed=21)
    rows_t = torch.from_numpy(rows).cuda()
    for k, lab, (lt, smp), out, out_tc in zip(ks, labs, items, outs, outs_tc):
        sizes = np.bincount(lab, minlength=k)
        assert sizes.min() >= 1
        os_ = oracle.sample_pps(Xh, lab, k, "euclidean", t=128.0, seed=7, cid=k - 2)
        assert_same_sample(smp, os_, k, 7, k - 2)
        s_o, _, _ = oracle.estimate(Xh, lab, k, "euclidean", os_.offsets, os_.idx, os_.ps,
                                    rows=rows)
        _assert_close(out[rows_t], s_o)
        _assert_close(out_tc[rows_t], s_o)


def test_serving_workload_largest_requests_sampled_parity():
    """The serving workload's 64 resident datasets; requests on its largest
    ones (n 0.74M-1.6M, d 64 and 128, FP32 and BF16 storage), one per metric,
    with k up to 100 nearest-centre clusters and t = 64, served concurrently by
    the continuous-batching server (FP32, the asynchronous chain).  Each
    request's sample set must equal the oracle's (up to the tie band), and its
    per-point s_hat must match the oracle's estimate on 100 seeded rows."""
    from paper_2607_01993_b300 import serve
    datasets, spec = synth.serving(seed=4)
    cases = [(9, "canberra", 64), (0, "euclidean", 100), (47, "cosine", 37), (49, "manhattan", 80)]
    reqs = []
    for i, (ds, metric, k) in enumerate(cases):
        lab = synth.nearest_centre_labels_device(datasets[ds].float(), k, seed=500 + i)
        reqs.append(serve.Request(dataset=ds, labels=lab, k=k, metric=metric, t=64.0,
                                  seed=900 + i, clustering_id=i, want_s=True))
    torch.cuda.synchronize()
    with serve.SilhServer(datasets, slots=4) as srv:
        res = [f.result(timeout=600) for f in [srv.submit(r) for r in reqs]]
    for i, ((ds, metric, k), req, r) in enumerate(zip(cases, reqs, res)):
        X = datasets[ds]
        n = X.shape[0]
        Xh = X.float().cpu().numpy().astype(np.float64)     # BF16 values exactly
        lab = req.labels.cpu().numpy()
        os_ = oracle.sample_pps(Xh, lab, k, metric, t=64.0, seed=900 + i, cid=i)
        gs = silh.silh_sample_pps(X, req.labels, k, metric, t=64.0, seed=900 + i,
                                  clustering_id=i)
        assert assert_same_sample(gs, os_, k, 900 + i, i, metric, lab) <= 2
        assert r.sample_size == gs.size
        rows = synth.seeded_rows(n, 100, seed=31 + i)
        s_o, _, _ = oracle.estimate(Xh, lab, k, metric, gs.offsets.cpu().numpy(),
                                    gs.idx[: gs.size].cpu().numpy().astype(np.int64),
                                    gs.p[: gs.size].cpu().numpy(), rows=rows)
        _assert_close(r.s_hat[torch.from_numpy(rows).cuda()], s_o)
        s_h = r.s_hat.cpu().numpy().astype(np.float64)
        assert abs(r.s_global - s_h.mean()) <= 1e-9
        assert spec[ds][0] == n
