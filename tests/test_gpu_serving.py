"""Continuous-batching server: results are the same alone and in the mix.

Requests over three device-resident datasets (FP32 and BF16, d in {8, 16, 64}),
mixed metrics and k, run (a) one at a time and (b) concurrently on four slots
with overlapping kernels; every global estimate and every per-point s_hat must
be bit-identical, also with high-priority streams for the small or the large
requests.  Admission by HBM footprint must cap concurrency, and one request is
checked against the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_01993_b300 import serve, silh, synth

pytestmark = pytest.mark.gpu
METRICS = ["euclidean", "cosine", "manhattan", "canberra"]


@pytest.fixture(scope="module")
def setup():
    specs = [(6000, 8, torch.float32, 51), (12000, 16, torch.bfloat16, 52), (9000, 64, torch.float32, 53)]
    host, dev = [], []
    for n, d, dt, seed in specs:
        X, _, _ = synth.gaussian_mixture(n, d, 8, seed=seed, sigma=1.5)
        X = synth.abs_shift(X)                # positive data: valid for every metric
        Xt = torch.from_numpy(X).cuda().to(dt)
        host.append(Xt.float().cpu().numpy().astype(np.float64))
        dev.append(Xt)
    rng = np.random.default_rng(7)
    reqs = []
    for i in range(16):
        ds = int(rng.integers(0, 3))
        k = int(rng.integers(2, 13))
        lab = synth.nearest_centre_labels(host[ds].astype(np.float32), k, seed=100 + i)
        reqs.append(dict(dataset=ds, labels=torch.from_numpy(lab).cuda(), k=k,
                         metric=METRICS[i % 4], t=48.0, seed=i, clustering_id=i, want_s=True))
    return host, dev, reqs


def _requests(reqs):
    return [serve.Request(**r) for r in reqs]


def test_same_result_alone_and_in_the_mix(setup):
    host, dev, reqs = setup
    alone = serve.run_one_at_a_time(dev, _requests(reqs))
    with serve.SilhServer(dev, slots=4, hbm_budget_bytes=1 << 40) as srv:
        futs = [srv.submit(r) for r in _requests(reqs)]
        mixed = [f.result(timeout=300) for f in futs]
        assert srv.peak_running >= 2                      # requests really overlapped
    for a, b in zip(alone, mixed):
        assert a.s_global == b.s_global
        assert a.sample_size == b.sample_size
        assert torch.equal(a.s_hat, b.s_hat)
    silh.silh_stream_status()


@pytest.mark.parametrize("priority", ["small", "large"])
def test_stream_priorities_leave_results_unchanged(setup, priority):
    # a mid-range threshold puts some requests on each kind of stream
    host, dev, reqs = setup
    alone = serve.run_one_at_a_time(dev, _requests(reqs))
    works = sorted(serve.request_work(dev[r["dataset"]].shape[0], dev[r["dataset"]].shape[1],
                                      r["k"], r["t"]) for r in reqs)
    with serve.SilhServer(dev, slots=4, hbm_budget_bytes=1 << 40, priority=priority,
                          big_work=works[len(works) // 2]) as srv:
        mixed = [f.result(timeout=300) for f in [srv.submit(r) for r in _requests(reqs)]]
    for a, b in zip(alone, mixed):
        assert a.s_global == b.s_global and a.sample_size == b.sample_size
        assert torch.equal(a.s_hat, b.s_hat)


def test_admission_by_footprint_caps_concurrency(setup):
    host, dev, reqs = setup
    # a budget of the smallest footprint: no two requests fit together (a request
    # larger than the whole budget is admitted only when nothing else runs)
    need = min(serve.footprint_bytes(dev[r["dataset"]].shape[0], dev[r["dataset"]].shape[1],
                                     r["k"], r["metric"], r["t"]) for r in reqs[:6])
    with serve.SilhServer(dev, slots=4, hbm_budget_bytes=need) as srv:
        futs = [srv.submit(r) for r in _requests(reqs[:6])]
        res = [f.result(timeout=300) for f in futs]
        assert srv.peak_running == 1                      # only one fits at a time
    assert all(np.isfinite(r.s_global) for r in res)


def test_served_request_matches_oracle(setup):
    host, dev, reqs = setup
    r = reqs[1]
    with serve.SilhServer(dev, slots=2) as srv:
        res = srv.submit(serve.Request(**r)).result(timeout=300)
    Xh = host[r["dataset"]]
    lab = r["labels"].cpu().numpy()
    os_ = oracle.sample_pps(Xh, lab, r["k"], r["metric"], t=r["t"], seed=r["seed"],
                            cid=r["clustering_id"])
    rows = synth.seeded_rows(Xh.shape[0], 200, seed=5)
    s_o, _, _ = oracle.estimate(Xh, lab, r["k"], r["metric"], os_.offsets, os_.idx, os_.ps,
                                rows=rows)
    got = res.s_hat[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    assert np.abs(got - s_o).max() <= 1e-5


def test_collapsed_cosine_server_matches_alone_and_oracle(setup):
    # cosine requests through the O(n k d) collapsed form: the same result alone
    # and in the mix, and within the FP32 bound of the oracle
    host, dev, reqs = setup
    cos = [dict(r, metric="cosine") for r in reqs[:6]]
    with serve.SilhServer(dev, slots=1, cosine="collapsed") as srv:
        alone = [srv.submit(serve.Request(**r)).result(timeout=300) for r in cos]
    with serve.SilhServer(dev, slots=4, cosine="collapsed") as srv:
        mixed = [f.result(timeout=300) for f in [srv.submit(serve.Request(**r)) for r in cos]]
    for a, b in zip(alone, mixed):
        assert a.s_global == b.s_global and torch.equal(a.s_hat, b.s_hat)
    r = cos[2]
    Xh = host[r["dataset"]]
    lab = r["labels"].cpu().numpy()
    os_ = oracle.sample_pps(Xh, lab, r["k"], "cosine", t=r["t"], seed=r["seed"],
                            cid=r["clustering_id"])
    rows = synth.seeded_rows(Xh.shape[0], 200, seed=6)
    s_o, _, _ = oracle.estimate(Xh, lab, r["k"], "cosine", os_.offsets, os_.idx, os_.ps,
                                rows=rows)
    got = mixed[2].s_hat[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    assert np.abs(got - s_o).max() <= 1e-5
