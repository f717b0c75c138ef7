"""The bounded-wait error path on the GPU.

Every wait of the tensor-core sweep gives up after a time limit and records the
failure, which silh_stream_status reports as SILH_ETIMEOUT.  Here a one-thread
kernel (no TMA, no MMA, no tensor memory) waits on an mbarrier that nothing ever
arrives on, with a 1 ms limit: the wait must run out, the status must read
SILH_ETIMEOUT once (and be cleared by reading it), and the context must stay
usable -- a Phase-2 estimate right after still matches the oracle.
"""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2607_01993_b300 import silh, synth

pytestmark = pytest.mark.gpu


def test_wait_that_completes_reports_ok():
    silh.silh_stream_status()                       # clear any earlier record
    silh.wait_selftest(arrive=True, timeout_ns=1_000_000)
    silh.silh_stream_status()                       # raises on a timeout record


def test_wait_that_never_completes_times_out_and_context_survives():
    silh.silh_stream_status()
    t0 = time.perf_counter()
    silh.wait_selftest(arrive=False, timeout_ns=1_000_000)
    with pytest.raises(silh.SilhError) as ei:
        silh.silh_stream_status()
    elapsed = time.perf_counter() - t0
    assert ei.value.status == -5                    # SILH_ETIMEOUT
    assert elapsed < 5.0                            # the 1 ms limit, not a hang
    silh.silh_stream_status()                       # the record was cleared
    # the context is still usable: one estimate against the oracle
    X, lab, _ = synth.tiny(seed=0)
    Xt, lt = torch.from_numpy(X).cuda(), torch.from_numpy(lab).cuda()
    smp = silh.silh_sample_pps(Xt, lt, 4, "euclidean", t=64.0, m0=16.0, seed=0)
    s = silh.silh_estimate(Xt, lt, 4, smp, "euclidean", prec="3xtf32")
    silh.silh_stream_status()
    Xh = X.astype(np.float64)
    ref = oracle.sample_pps(Xh, lab, 4, "euclidean", t=64.0, m0=16.0, seed=0)
    s_o, _, _ = oracle.estimate(Xh, lab, 4, "euclidean", ref.offsets, ref.idx, ref.ps)
    assert np.abs(s.cpu().numpy() - s_o).max() <= 1e-5


def test_wait_limit_is_validated():
    with pytest.raises(silh.SilhError) as ei:
        silh.wait_selftest(arrive=False, timeout_ns=0)
    assert ei.value.status == -1
    with pytest.raises(silh.SilhError):
        silh.wait_selftest(arrive=False, timeout_ns=5_000_000_000)
