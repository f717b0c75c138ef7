"""Continuous-batching server for silhouette requests over device-resident data.

A request asks for the PPS silhouette estimate (Algorithm 1: Phase 1 + Phase 2
+ the global mean of Eq. 6) of one clustering of one of the server's resident
datasets, with its own k, metric, sample size t and seed.  The server runs up to
`slots` requests at once, each on its own CUDA stream and host worker, so their
kernels overlap on the GPU.  A queued request is admitted as soon as a slot is
free and its estimated scratch footprint fits in the HBM budget left by the
requests in flight (first fitting request in arrival order; a request larger
than the whole budget runs alone).  Each completion records its latency from
arrival.  Results do not depend on what else is running: every step is
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


@dataclass
class Request:
    dataset: int                  # index into the server's datasets
    labels: torch.Tensor          # int32 CUDA, one label per row of the dataset
    k: int
    metric: str = "euclidean"
    t: float = 64.0
    seed: int = 0
    clustering_id: int = 0
    prec: str = "auto"            # "auto": split-TF32 tensor cores where eligible, else FP32
    want_s: bool = False          # keep the per-point s_hat on the device
    arrival: float = field(default_factory=time.perf_counter)


@dataclass
class Result:
    s_global: float               # mean of s_hat (Eq. 6)
    sample_size: int
    latency_s: float
    s_hat: torch.Tensor | None = None


def footprint_bytes(n: int, d: int, k: int, metric: str, t: float) -> int:
    """Conservative scratch estimate of one request (Phase 1 + Phase 2)."""
    m0 = 2.0 * math.log(5.0 * k / 0.01)
    phase1 = n * (4 * 3 + 8 * 3) + int(n * m0 * 8)          # flags, scans, order, D matrix
    sample = n * (4 + 8)                                       # idx + p at capacity n
    kd = 32 if d <= 32 else 64 if d <= 64 else 128
    cols = int(k * t * 4 + 32 * k)
    phase2 = n * (kd * 8 + 32) + cols * (kd * 16 + 16)        # tensor-core layout (upper bound)
    return phase1 + sample + phase2 + 4 * n + (1 << 20)


class SilhServer:
    def __init__(self, datasets, slots: int = 4, hbm_budget_bytes: int | None = None):
        self.datasets = datasets                                   # list of 2-D CUDA tensors
        self.slots = max(1, int(slots))
        if hbm_budget_bytes is None:
            free, _ = torch.cuda.mem_get_info()
            hbm_budget_bytes = int(free * 0.5)
        self.budget = int(hbm_budget_bytes)
        self._queue = collections.deque()
        self._cv = threading.Condition()
        self._in_flight = 0
        self._running = 0
        self.peak_running = 0                                      # most requests seen at once
        self._stop = False
        self.completed = []                                        # (request, result)
        self._workers = [threading.Thread(target=self._worker, args=(i,), daemon=True)
                         for i in range(self.slots)]
        self._streams = [torch.cuda.Stream() for _ in range(self.slots)]
        for w in self._workers:
            w.start()

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
        for w in self._workers:
            w.join(timeout=10)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -------------------------------------------------------------- workers
    def _admit(self):
        """First queued request that fits (called with the lock held)."""
        for i, (req, fut, need) in enumerate(self._queue):
            alone = self._running == 0
            if need <= self.budget - self._in_flight or alone:
                del self._queue[i]
                self._in_flight += need
                self._running += 1
                self.peak_running = max(self.peak_running, self._running)
                return req, fut, need
        return None

    def _worker(self, slot: int):
        stream = self._streams[slot]
        torch.cuda.set_device(self.datasets[0].device)
        while True:
            with self._cv:
                item = None
                while not self._stop:
                    item = self._admit()
                    if item is not None:
                        break
                    self._cv.wait(timeout=0.5)
                if item is None:
                    return
            req, fut, need = item
            try:
                res = self._run(req, stream)
                fut.set_result(res)
                self.completed.append((req, res))
            except Exception as exc:  # surfaced to the caller through the future
                fut.set_exception(exc)
            finally:
                with self._cv:
                    self._in_flight -= need
                    self._running -= 1
                    self._cv.notify_all()

    def _run(self, req: Request, stream) -> Result:
        X = self.datasets[req.dataset]
        prec = req.prec
        if prec == "auto":
            prec = "3xtf32" if req.metric in ("euclidean", "cosine") and X.shape[1] <= 64 else "fp32"
        with torch.cuda.stream(stream):
            smp = silh.silh_sample_pps(X, req.labels, req.k, req.metric, t=req.t, seed=req.seed,
                                       clustering_id=req.clustering_id, stream=stream)
            s = silh.silh_estimate(X, req.labels, req.k, smp, req.metric, prec=prec, stream=stream)
            g = silh.silh_global(s, stream=stream)
            gv = g.item()                                       # synchronises this stream
        done = time.perf_counter()
        return Result(gv, smp.size, done - req.arrival, s if req.want_s else None)


def run_one_at_a_time(datasets, requests):
    """The same requests processed strictly one after another (the baseline)."""
    srv = SilhServer(datasets, slots=1, hbm_budget_bytes=1 << 62)
    futs = [srv.submit(r) for r in requests]
    results = [f.result() for f in futs]
    srv.close()
    return results
