"""Continuous-batching server for silhouette requests over device-resident data.

A request asks for the PPS silhouette estimate (Algorithm 1: Phase 1 + Phase 2
+ the global mean of Eq. 6) of one clustering of one of the server's resident
datasets, with its own k, metric, sample size t and seed.

Each admitted request runs as one asynchronous chain on its slot's CUDA stream:
silh_sample_pps_async (Phase 1, every size kept on the device), then
silh_estimate_async (Phase 2 reading |S| from the device), silh_global, and a
copy of (global mean, |S|, status) into pinned host memory, closed by an event.
Nothing in the chain waits for the device, so one scheduler thread keeps up to
`slots` requests in flight and their kernels overlap on the GPU.  The scheduler
loop admits the first queued request that fits (a free slot and an estimated
scratch footprint within the HBM budget left by the requests in flight; a
request larger than the whole budget runs alone), polls the in-flight events,
and completes the futures of finished requests with their latency from arrival.
A request whose device status reports a capacity overflow (the sample larger
than the capacity reserved for it, or initial samples beyond their planned
capacity: far below 1e-15 in probability) is redone with the synchronising
calls.  Results do not depend on what else is running: every step is
deterministic given the request's seed and inputs.
"""
from __future__ import annotations

import collections
import math
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import torch

from . import silh

SILH_ECAPACITY = -4


@dataclass
class Request:
    dataset: int                  # index into the server's datasets
    labels: torch.Tensor          # int32 CUDA, one label per row of the dataset
    k: int
    metric: str = "euclidean"
    t: float = 64.0
    seed: int = 0
    clustering_id: int = 0
    prec: str = "fp32"            # or "auto": split-TF32 tensor cores where eligible
    want_s: bool = False          # keep the per-point s_hat on the device
    arrival: float = field(default_factory=time.perf_counter)


@dataclass
class Result:
    s_global: float               # mean of s_hat (Eq. 6)
    sample_size: int
    latency_s: float
    s_hat: torch.Tensor | None = None


def resolve_prec(prec: str, metric: str, d: int) -> str:
    """"auto": split TF32 on the tensor cores for Euclidean / cosine with d <= 64,
    FP32 otherwise.  Requests default to FP32: on clusterings cut into Voronoi
    cells, whose close cross-cluster pairs the tensor-core sweep recomputes in
    FP32, the CUDA-core sweep is the faster of the two."""
    if prec != "auto":
        return prec
    return "3xtf32" if metric in ("euclidean", "cosine") and d <= 64 else "fp32"


def sample_capacity(n: int, k: int, t: float) -> int:
    """Columns reserved for a request's sample: min(n, 4 k t + 1024).  E|F_j| is
    at most t (1 + |F0_j|) and near t in practice; a larger sample is redone."""
    return int(min(n, math.ceil(4.0 * k * t) + 1024))


def footprint_bytes(n: int, d: int, k: int, metric: str, t: float) -> int:
    """Conservative device-memory estimate of one request in flight: Phase 1's
    scratch (flags, scans, order, the member x F0 distance matrices at their
    planned capacity), the sample at its capacity, Phase 2's operands (the
    tensor-core layout is the larger) and the per-point output."""
    m0 = 2.0 * math.log(5.0 * k / 0.01)
    cap = sample_capacity(n, k, t)
    phase1 = n * (4 * 3 + 8 * 5) + int(math.ceil(n * (m0 + 8 * math.sqrt(m0) + 16)) * 8)
    sample = cap * (4 + 8) + 16 * (k + 1)
    kd = 32 if d <= 32 else 64 if d <= 64 else 128
    cols = cap + 32 * k
    phase2 = n * (kd * 8 + 32) + cols * (kd * 16 + 16)
    return phase1 + sample + phase2 + 4 * n + (1 << 20)


class _Flight:
    """One admitted request: its stream slot, device buffers and completion event."""

    def __init__(self, req, fut, need, slot):
        self.req, self.fut, self.need, self.slot = req, fut, need, slot
        self.event = None
        self.s = self.smp = self.d_size = self.d_status = self.g = None
        self.host = None
        self.stream = None


def request_work(n: int, d: int, k: int, t: float) -> float:
    """Phase-2 work of a request in coordinate terms: n rows against its
    expected sample of min(n, k t) columns, d coordinates each."""
    return float(n) * min(float(n), k * t) * d


class SilhServer:
    """cosine="collapsed" runs cosine requests' Phase 2 in the O(n k d) form of
    silh_estimate_cosine_collapsed (the same estimate up to rounding; |ds| within
    the FP32 bound of the oracle) instead of the per-pair sweep.

    priority="large" launches requests whose request_work is at least big_work
    on high-priority streams (the GPU's block scheduler starts the pending
    thread blocks of higher-priority streams first); priority="small" puts the
    other requests there instead, which shortens the small requests' latency
    and lengthens the largest ones'; None (the default) gives every stream the
    same priority.  Results do not depend on the choice."""

    def __init__(self, datasets, slots: int = 4, hbm_budget_bytes: int | None = None,
                 cosine: str = "per_pair", priority: str | None = None,
                 big_work: float = 2e11):
        if cosine not in ("per_pair", "collapsed"):
            raise ValueError("cosine must be 'per_pair' or 'collapsed'")
        if priority not in (None, "large", "small"):
            raise ValueError("priority must be None, 'large' or 'small'")
        self.cosine = cosine
        self.priority = priority
        self.big_work = float(big_work)
        self.datasets = datasets                                   # list of 2-D CUDA tensors
        self.device = datasets[0].device
        self.slots = max(1, int(slots))
        if hbm_budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            hbm_budget_bytes = int(free * 0.5)
        self.budget = int(hbm_budget_bytes)
        self._queue = collections.deque()
        self._cv = threading.Condition()
        self._in_flight = 0
        self._running = 0
        self.peak_running = 0                                      # most requests seen at once
        self.redone = 0                                            # capacity overflows redone
        self._stop = False
        self.completed = []                                        # (request, result)
        self._streams = [torch.cuda.Stream(self.device) for _ in range(self.slots)]
        self._streams_hi = ([torch.cuda.Stream(self.device, priority=-1)
                             for _ in range(self.slots)] if priority else None)
        # pinned (global mean, |S|, status) per slot, written by the chain's last copies
        self._host = [torch.zeros(3, dtype=torch.float64).pin_memory() for _ in range(self.slots)]
        self._free_slots = list(range(self.slots))
        self._loop = threading.Thread(target=self._scheduler, daemon=True)
        self._loop.start()

    # ------------------------------------------------------------ client API
    def submit(self, req: Request) -> Future:
        fut = Future()
        X = self.datasets[req.dataset]
        need = footprint_bytes(X.shape[0], X.shape[1], req.k, req.metric, req.t)
        with self._cv:
            self._queue.append((req, fut, need))
            self._cv.notify_all()
        return fut

    def drain(self, timeout: float | None = None):
        end = None if timeout is None else time.perf_counter() + timeout
        with self._cv:
            while self._queue or self._running:
                left = None if end is None else end - time.perf_counter()
                if left is not None and left <= 0:
                    return False
                self._cv.wait(timeout=left if left is not None else 0.5)
        return True

    def close(self):
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        self._loop.join(timeout=60)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------ scheduler
    def _admit(self):
        """First queued request that fits (called with the lock held)."""
        if not self._free_slots:
            return None
        for i, (req, fut, need) in enumerate(self._queue):
            alone = self._running == 0
            if need <= self.budget - self._in_flight or alone:
                del self._queue[i]
                self._in_flight += need
                self._running += 1
                self.peak_running = max(self.peak_running, self._running)
                return _Flight(req, fut, need, self._free_slots.pop())
        return None

    def _stream_for(self, fl: _Flight):
        """The slot's stream, or its high-priority twin (see priority)."""
        if self.priority is None:
            return self._streams[fl.slot]
        n, d = self.datasets[fl.req.dataset].shape
        big = request_work(n, d, fl.req.k, fl.req.t) >= self.big_work
        hi = big if self.priority == "large" else not big
        return self._streams_hi[fl.slot] if hi else self._streams[fl.slot]

    def _launch(self, fl: _Flight):
        """Enqueue the request's whole chain on its slot stream (no host waits)."""
        req = fl.req
        X = self.datasets[req.dataset]
        n, d = X.shape
        stream = fl.stream = self._stream_for(fl)
        prec = resolve_prec(req.prec, req.metric, d)
        with torch.cuda.stream(stream):
            cap = sample_capacity(n, req.k, req.t)
            fl.smp, fl.d_size, fl.d_status = silh.silh_sample_pps_async(
                X, req.labels, req.k, req.metric, t=req.t, seed=req.seed,
                clustering_id=req.clustering_id, cap=cap, stream=stream)
            if req.metric == "cosine" and self.cosine == "collapsed":
                # the collapsed form reads the per-cluster lists through the
                # device offsets only; the host size just has to be consistent
                fl.smp.size = fl.smp.idx.shape[0]
                fl.s = silh.silh_estimate_cosine_collapsed(X, req.labels, req.k, fl.smp,
                                                           stream=stream)
            else:
                fl.s = silh.silh_estimate_async(X, req.labels, req.k, fl.smp, fl.d_size,
                                                req.metric, prec=prec, stream=stream)
            fl.g = silh.silh_global(fl.s, stream=stream)
            host = self._host[fl.slot]
            host[0:1].copy_(fl.g, non_blocking=True)
            host[1:2].copy_(fl.d_size, non_blocking=True)
            host[2:3].copy_(fl.d_status, non_blocking=True)
            fl.event = torch.cuda.Event()
            fl.event.record(stream)
        fl.host = host

    def _redo(self, fl: _Flight):
        """The synchronising path, for a request whose capacity overflowed."""
        req = fl.req
        X = self.datasets[req.dataset]
        stream = fl.stream
        prec = resolve_prec(req.prec, req.metric, X.shape[1])
        with torch.cuda.stream(stream):
            smp = silh.silh_sample_pps(X, req.labels, req.k, req.metric, t=req.t, seed=req.seed,
                                       clustering_id=req.clustering_id, stream=stream)
            if req.metric == "cosine" and self.cosine == "collapsed":
                s = silh.silh_estimate_cosine_collapsed(X, req.labels, req.k, smp, stream=stream)
            else:
                s = silh.silh_estimate(X, req.labels, req.k, smp, req.metric, prec=prec,
                                       stream=stream)
            g = silh.silh_global(s, stream=stream).item()
        return g, smp.size, s

    def _finish(self, fl: _Flight):
        status = int(fl.host[2].item())
        if status == SILH_ECAPACITY:
            self.redone += 1
            g, size, s = self._redo(fl)
        elif status != 0:
            raise silh.SilhError(status, "request failed on the device (invalid clustering)")
        else:
            g, size, s = float(fl.host[0].item()), int(fl.host[1].item()), fl.s
        done = time.perf_counter()
        return Result(g, size, done - fl.req.arrival, s if fl.req.want_s else None)

    def _scheduler(self):
        torch.cuda.set_device(self.device)
        flights = []
        while True:
            with self._cv:
                while True:
                    fl = self._admit()
                    if fl is None:
                        break
                    flights.append(fl)
                    try:
                        self._launch(fl)
                    except Exception as exc:           # invalid arguments: fail this request
                        flights.pop()
                        self._release(fl)
                        fl.fut.set_exception(exc)
                if self._stop and not flights:
                    return
                if not flights:
                    self._cv.wait(timeout=0.5)
                    continue
            still = []
            for fl in flights:
                if not fl.event.query():
                    still.append(fl)
                    continue
                try:
                    res = self._finish(fl)
                    self.completed.append((fl.req, res))
                    fl.fut.set_result(res)
                except Exception as exc:               # surfaced through the future
                    fl.fut.set_exception(exc)
                with self._cv:
                    self._release(fl)
            if len(still) == len(flights):
                time.sleep(20e-6)                      # nothing finished: poll again shortly
            flights = still

    def _release(self, fl: _Flight):
        """Return the flight's slot and memory budget (called with the lock held)."""
        self._in_flight -= fl.need
        self._running -= 1
        self._free_slots.append(fl.slot)
        self._cv.notify_all()


def run_one_at_a_time(datasets, requests, prec: str | None = None):
    """The same requests processed strictly one after another with the plain
    synchronising calls (the baseline).  prec None keeps each request's own
    precision rule; "fp32" is the plain FP32 path."""
    out = []
    for req in requests:
        X = datasets[req.dataset]
        p = resolve_prec(prec if prec is not None else req.prec, req.metric, X.shape[1])
        smp = silh.silh_sample_pps(X, req.labels, req.k, req.metric, t=req.t, seed=req.seed,
                                   clustering_id=req.clustering_id)
        s = silh.silh_estimate(X, req.labels, req.k, smp, req.metric, prec=p)
        g = silh.silh_global(s).item()
        out.append(Result(g, smp.size, time.perf_counter() - req.arrival,
                          s if req.want_s else None))
    return out
