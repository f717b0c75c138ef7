"""Host-side logic of the continuous-batching server that needs no GPU: the
request-work estimate that sorts requests onto priority streams, the sample
capacity and footprint estimates admission uses, and argument checks made
before any device call."""
import math

import pytest
import torch

from paper_2607_01993_b300 import serve


def test_request_work_counts_rows_times_expected_columns_times_d():
    # n rows against min(n, k t) expected sample columns, d coordinates each
    assert serve.request_work(100_000, 64, 10, 64.0) == 100_000 * 640 * 64
    # a sample cannot exceed the dataset: k t above n is capped at n
    assert serve.request_work(5_000, 8, 100, 64.0) == 5_000 * 5_000 * 8


def test_sample_capacity_and_footprint_are_monotone():
    assert serve.sample_capacity(10_000, 4, 64.0) == min(10_000, math.ceil(4 * 4 * 64) + 1024)
    assert serve.sample_capacity(500, 50, 64.0) == 500
    small = serve.footprint_bytes(10_000, 16, 8, "euclidean", 64.0)
    assert serve.footprint_bytes(20_000, 16, 8, "euclidean", 64.0) > small
    assert serve.footprint_bytes(10_000, 128, 8, "euclidean", 64.0) > small


def test_server_rejects_unknown_options_before_touching_the_device():
    X = [torch.zeros(4, 2)]
    with pytest.raises(ValueError):
        serve.SilhServer(X, priority="medium")
    with pytest.raises(ValueError):
        serve.SilhServer(X, cosine="approximate")
