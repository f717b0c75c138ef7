"""Autotuner for the batched Phase-2 sweep.

The batched sweep has several tile shapes.  On CUDA cores (FP32): rows per
thread x columns staged per step, four variants.  On tensor cores (TF32 / split
TF32 / BF16 / split BF16, Euclidean and cosine, d <= 64): 128-column tiles with
one accumulator per row tile, or 64-column tiles with two (TF32 operands of
d <= 32).  The best one depends on the metric, the precision, the padded
dimension, the row count and the data (how many chunks need the close-pair
recompute), so it is chosen by timing every variant on the actual call with
CUDA events and cached (JSON) per (GPU, metric, precision, padded d, n bucket).
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

from . import silh

_DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json")
_lock = threading.Lock()


def _cache_path():
    return os.environ.get("SILH_AUTOTUNE_CACHE", _DEFAULT_CACHE)


def _key(X, metric, prec):
    d = X.shape[1]
    pad = 8 if d <= 8 else 16 if d <= 16 else 32 if d <= 32 else 64 if d <= 64 else 128
    nb = int(math.log2(max(2, X.shape[0])))
    return f"{torch.cuda.get_device_name(X.device)}|{metric}|{prec}|D{pad}|n2^{nb}"


TC_PRECS = ("tf32", "3xtf32", "bf16", "bf16x3")


def variants_for(X, metric, prec):
    """The distinct tile variants of silh_estimate_batched for this call shape."""
    d = X.shape[1]
    if prec in TC_PRECS and metric in ("euclidean", "cosine") and d <= 64:
        return [0, 1] if (d <= 32 and prec in ("tf32", "3xtf32")) else [0]
    return list(range(silh.BATCH_VARIANTS))


def _load():
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(table):
    path = _cache_path()
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune_batched(X, items, metric="euclidean", reps=2, force=False, prec="fp32"):
    """Best variant for this call shape (cached); returns (variant, {variant: ms})."""
    key = _key(X, metric, prec)
    with _lock:
        table = _load()
        if key in table and not force:
            return table[key]["variant"], table[key]["ms"]
    outs = [torch.empty(X.shape[0], dtype=torch.float32, device=X.device) for _ in items]
    times = {}
    for v in variants_for(X, metric, prec):
        silh.silh_estimate_batched(X, items, metric, variant=v, outs=outs, prec=prec)  # warm-up
        best = float("inf")
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            silh.silh_estimate_batched(X, items, metric, variant=v, outs=outs, prec=prec)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        times[str(v)] = best
    variant = int(min(times, key=times.get))
    with _lock:
        table = _load()
        table[key] = {"variant": variant, "ms": times}
        _store(table)
    return variant, times
