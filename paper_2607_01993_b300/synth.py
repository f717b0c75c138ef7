"""Seeded synthetic inputs shared by the GPU path's tests/benchmark and the oracle.

This module only draws data (numpy PCG64); it contains none of the silhouette
arithmetic.  The paper evaluates on UCI/SNAP datasets (Sec. 5.1, Table 2) that
are not available here; Gaussian mixtures with the paper's shapes (n up to
millions, d small, k clusters of uneven size) stand in for them.
"""
from __future__ import annotations

import numpy as np


def zipf_sizes(n: int, k: int, s: float = 1.1) -> np.ndarray:
    """Cluster sizes proportional to j^-s (j = 1..k), summing to n, each >= 1."""
    w = np.arange(1, k + 1, dtype=np.float64) ** (-s)
    raw = n * w / w.sum()
    sizes = np.maximum(np.floor(raw).astype(np.int64), 1)
    rem = n - int(sizes.sum())
    order = np.argsort(-(raw - np.floor(raw)), kind="stable")
    i = 0
    while rem != 0:
        j = order[i % k]
        if rem > 0:
            sizes[j] += 1; rem -= 1
        elif sizes[j] > 1:
            sizes[j] -= 1; rem += 1
        i += 1
    return sizes


def gaussian_mixture(n: int, d: int, k: int, *, seed: int, sizes=None, sigma=1.0,
                     sigma_range=None, box: float = 10.0, border_frac: float = 0.0,
                     shuffle: bool = True):
    """Isotropic Gaussian blobs; labels are the generating component.

    Centres are uniform in [-box, box]^d.  ``sigma_range=(lo, hi)`` draws one
    sigma per component uniformly.  ``border_frac`` of the points of each
    component are placed between their centre and the nearest other centre
    (x = c_j + lam (c_j' - c_j) + sigma N, lam ~ U[0.4, 0.6]), keeping label j.
    Returns (X float32 [n, d], labels int32 [n], centres float64 [k, d]).
    """
    rng = np.random.default_rng(seed)
    if sizes is None:
        sizes = np.full(k, n // k, dtype=np.int64)
        sizes[: n - int(sizes.sum())] += 1
    sizes = np.asarray(sizes, dtype=np.int64)
    assert sizes.sum() == n and (sizes > 0).all()
    centres = rng.uniform(-box, box, size=(k, d))
    if sigma_range is not None:
        sig = rng.uniform(sigma_range[0], sigma_range[1], size=k)
    else:
        sig = np.full(k, float(sigma))
    labels = np.repeat(np.arange(k, dtype=np.int32), sizes)
    X = np.empty((n, d), dtype=np.float32)
    if border_frac > 0:
        cc = ((centres[:, None, :] - centres[None, :, :]) ** 2).sum(-1)
        np.fill_diagonal(cc, np.inf)
        nearest = cc.argmin(1)
    start = 0
    for j in range(k):
        m = int(sizes[j])
        pts = centres[j] + sig[j] * rng.standard_normal((m, d))
        if border_frac > 0:
            nb = int(round(border_frac * m))
            lam = rng.uniform(0.4, 0.6, size=(nb, 1))
            pts[:nb] = (centres[j] + lam * (centres[nearest[j]] - centres[j])
                        + sig[j] * rng.standard_normal((nb, d)))
        X[start:start + m] = pts
        start += m
    if shuffle:
        perm = rng.permutation(n)
        X = X[perm]
        labels = labels[perm]
    return np.ascontiguousarray(X), np.ascontiguousarray(labels), centres


def abs_shift(X: np.ndarray) -> np.ndarray:
    """|x| + 1 elementwise: the strictly positive data the Canberra runs use."""
    return (np.abs(X) + 1.0).astype(X.dtype)


def nearest_centre_labels(X: np.ndarray, k: int, *, seed: int):
    """Labels from k distinct random data rows used as centres (no empty cluster)."""
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    cidx = rng.choice(n, size=k, replace=False)
    C = X[cidx].astype(np.float64)
    best = np.full(n, np.inf)
    lab = np.zeros(n, dtype=np.int32)
    for j in range(k):
        dj = ((X.astype(np.float64) - C[j]) ** 2).sum(1)
        upd = dj < best
        best[upd] = dj[upd]
        lab[upd] = j
    lab[cidx] = np.arange(k, dtype=np.int32)
    return lab


def nearest_centre_labels_device(Xt, k: int, *, seed: int, chunk: int = 1 << 18):
    """As nearest_centre_labels, on the device tensor Xt (torch), for large n."""
    import torch
    rng = np.random.default_rng(seed)
    n = Xt.shape[0]
    cidx = rng.choice(n, size=k, replace=False)
    C = Xt[torch.from_numpy(cidx).to(Xt.device)].double()
    lab = torch.empty(n, dtype=torch.int32, device=Xt.device)
    cn = (C * C).sum(1)
    for s0 in range(0, n, chunk):
        xb = Xt[s0:s0 + chunk].double()
        dist = (xb * xb).sum(1, keepdim=True) - 2.0 * xb @ C.T + cn[None, :]
        lab[s0:s0 + chunk] = dist.argmin(1).to(torch.int32)
    lab[torch.from_numpy(cidx).to(Xt.device)] = torch.arange(k, dtype=torch.int32, device=Xt.device)
    return lab


def gaussian_mixture_device(n: int, d: int, k: int, *, seed: int, device="cuda",
                            sigma_range=(0.5, 3.0), box: float = 10.0):
    """A Gaussian mixture drawn on the device from a seeded torch generator
    (for the many large resident datasets of the serving workload)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    centres = (torch.rand(k, d, generator=g, device=device) * 2 - 1) * box
    sig = torch.rand(k, generator=g, device=device) * (sigma_range[1] - sigma_range[0]) + sigma_range[0]
    comp = torch.randint(0, k, (n,), generator=g, device=device)
    X = centres[comp] + sig[comp, None] * torch.randn(n, d, generator=g, device=device)
    return X.float().contiguous()


def serving(seed: int = 4, ndatasets: int = 64, device="cuda"):
    """64 resident datasets: n log-uniform in [5k, 2M], d in {8, 16, 64, 128},
    stored FP32 or BF16; returns (list of tensors, list of (n, d, dtype))."""
    import torch
    rng = np.random.default_rng(seed)
    out, spec = [], []
    for i in range(ndatasets):
        n = int(round(np.exp(rng.uniform(np.log(5e3), np.log(2e6)))))
        d = int(rng.choice([8, 16, 64, 128]))
        dt = torch.bfloat16 if rng.random() < 0.5 else torch.float32
        X = gaussian_mixture_device(n, d, int(rng.integers(4, 33)), seed=seed * 1000 + i,
                                    device=device).to(dt)
        out.append(X)
        spec.append((n, d, str(dt).replace("torch.", "")))
    return out, spec


# ----------------------------------------------------------------- workloads

def tiny(seed: int = 0):
    """n=2000, d=8, k=4 equal isotropic blobs (sigma 1, centres in [-10,10]^8)."""
    return gaussian_mixture(2000, 8, 4, seed=seed, sigma=1.0)


def large(seed: int = 1, n: int = 1_000_000, d: int = 32, k: int = 32):
    """n=1M, d=32, k=32 Zipf(1.1) sizes, per-cluster sigma ~ U[0.5, 3]."""
    return gaussian_mixture(n, d, k, seed=seed, sizes=zipf_sizes(n, k, 1.1),
                            sigma_range=(0.5, 3.0))


def precision(seed: int = 2, n: int = 4_000_000, d: int = 64, k: int = 64):
    """n=4M, d=64, k=64 Zipf sizes, 10% of points on cluster borders."""
    return gaussian_mixture(n, d, k, seed=seed, sizes=zipf_sizes(n, k, 1.1),
                            sigma_range=(0.5, 3.0), border_frac=0.10)


def batching(seed: int = 3, n: int = 500_000, d: int = 16):
    """n=500k, d=16 data from a 16-component mixture; clusterings are made by
    nearest_centre_labels(_device) with k = 2..257 random data rows as centres."""
    X, _, _ = gaussian_mixture(n, d, 16, seed=seed, sigma_range=(0.5, 3.0))
    return X


def seeded_rows(n: int, m: int, *, seed: int) -> np.ndarray:
    """m distinct row indices drawn uniformly, ascending."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=m, replace=False)).astype(np.int64)
