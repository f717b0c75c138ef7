"""The asynchronous request chain: silh_sample_pps_async + silh_estimate_async.

Phase 1 with every size kept on the device must give exactly the sample of the
synchronising silh_sample_pps (same kernels and arithmetic, planned on the
device), and Phase 2 reading |S| from the device exactly the estimate of
silh_estimate, for every metric, both precisions' paths, the uniform variant,
a row subset, FP32 and BF16 storage.  Errors surface in the device status word
with an empty sample that the next call can still consume in bounds.
"""
import numpy as np
import pytest
import torch

from paper_2607_01993_b300 import silh, synth

pytestmark = pytest.mark.gpu
METRICS = ["euclidean", "cosine", "manhattan", "canberra"]


def _data(n, d, k, seed, dtype=torch.float32, shift=False):
    X, lab, _ = synth.gaussian_mixture(n, d, k, seed=seed, sizes=synth.zipf_sizes(n, k),
                                       sigma_range=(0.5, 3.0))
    if shift:
        X = synth.abs_shift(X)
    return torch.from_numpy(X).cuda().to(dtype), torch.from_numpy(lab).cuda()


def _same_sample(a: silh.Sample, b: silh.Sample, size_b: int):
    assert torch.equal(a.sizes, b.sizes)
    assert torch.equal(a.offsets, b.offsets)
    assert torch.equal(a.idx[:size_b], b.idx[:size_b])
    assert torch.equal(a.p[:size_b], b.p[:size_b])


@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("case", ["multitile", "bf16_d50", "uniform"])
def test_async_chain_equals_synchronising_calls(metric, case):
    if case == "multitile":
        X, l = _data(40000, 32, 16, seed=61, shift=metric == "canberra")
        kw = dict(t=128.0, seed=4)
        k, prec = 16, "3xtf32"
    elif case == "bf16_d50":
        X, l = _data(23000, 50, 9, seed=62, dtype=torch.bfloat16, shift=metric == "canberra")
        kw = dict(t=64.0, m0=12.0, seed=5)
        k, prec = 9, "bf16x3"
    else:
        X, l = _data(30000, 13, 7, seed=63, shift=metric == "canberra")
        kw = dict(t=96.0, seed=6, uniform=True)
        k, prec = 7, "fp32"
    sync = silh.silh_sample_pps(X, l, k, metric, clustering_id=3, **kw)
    asmp, d_size, d_status = silh.silh_sample_pps_async(X, l, k, metric, clustering_id=3, **kw)
    torch.cuda.synchronize()
    assert int(d_status.item()) == 0
    assert int(d_size.item()) == sync.size
    _same_sample(asmp, sync, sync.size)
    for p in ("fp32", prec):
        want = silh.silh_estimate(X, l, k, sync, metric, prec=p, want_ab=True)
        got = silh.silh_estimate_async(X, l, k, asmp, d_size, metric, prec=p, want_ab=True)
        for g, w in zip(got, want):
            assert torch.equal(g, w), p
    rows = torch.arange(7, X.shape[0], 11, dtype=torch.int64, device="cuda")
    want = silh.silh_estimate(X, l, k, sync, metric, prec=prec, rows=rows)
    got = silh.silh_estimate_async(X, l, k, asmp, d_size, metric, prec=prec, rows=rows)
    assert torch.equal(got, want)


def test_async_capacity_and_invalid_clustering_give_status_and_empty_sample():
    X, l = _data(20000, 16, 6, seed=64)
    sync = silh.silh_sample_pps(X, l, 6, "euclidean", t=64.0, seed=7)
    # a capacity below |S|: SILH_ECAPACITY, |S| reported as 0, offsets all zero
    smp, d_size, d_status = silh.silh_sample_pps_async(X, l, 6, "euclidean", t=64.0, seed=7,
                                                       cap=sync.size - 1)
    torch.cuda.synchronize()
    assert int(d_status.item()) == silh.SILH_ECAPACITY
    assert int(d_size.item()) == 0
    assert int(smp.offsets.abs().sum().item()) == 0
    # the empty sample is still consumable: every W_hat is 0, so s_hat is 0
    for prec in ("fp32", "3xtf32"):
        s = silh.silh_estimate_async(X, l, 6, smp, d_size, "euclidean", prec=prec)
        silh.silh_stream_status()
        assert float(s.abs().max().item()) == 0.0
    # a label outside [0, k) and an empty cluster: SILH_EINVAL on the device
    for bad in ("label", "empty"):
        lb = l.clone()
        if bad == "label":
            lb[123] = 6
        else:
            lb[lb == 2] = 1
        smp, d_size, d_status = silh.silh_sample_pps_async(X, lb, 6, "manhattan", t=64.0, seed=8)
        s = silh.silh_estimate_async(X, lb if bad == "empty" else l, 6, smp, d_size, "manhattan")
        torch.cuda.synchronize()
        assert int(d_status.item()) == -1
        assert int(d_size.item()) == 0
        assert torch.isfinite(s).all()
    silh.silh_stream_status()


def test_async_chains_on_several_streams_match_one_at_a_time():
    X, l = _data(60000, 24, 12, seed=65)
    streams = [torch.cuda.Stream() for _ in range(4)]
    outs = []
    for i, st in enumerate(streams):
        with torch.cuda.stream(st):
            smp, d_size, _ = silh.silh_sample_pps_async(X, l, 12, METRICS[i], t=80.0, seed=20 + i,
                                                        stream=st)
            outs.append(silh.silh_estimate_async(X, l, 12, smp, d_size, METRICS[i],
                                                 prec="3xtf32", stream=st))
    torch.cuda.synchronize()
    for i, o in enumerate(outs):
        smp = silh.silh_sample_pps(X, l, 12, METRICS[i], t=80.0, seed=20 + i)
        assert torch.equal(o, silh.silh_estimate(X, l, 12, smp, METRICS[i], prec="3xtf32"))
