"""Seeded synthetic cost matrices shaped like the paper's workloads.

This module holds no arithmetic of the assignment method itself: it only
draws points / vectors and turns them into integer cost matrices.  Both the
CUDA path and the CPU oracle are fed from here.

The paper's own datasets (Sec. 3.2: CircleSquare, NLP token embeddings,
MNIST pixels, CIFAR pixels) are not available; these generators stand in for
them with the same shapes and cost structure:

* ``grid_sqdist``   -- integer points uniform on a g x g grid, cost = squared
                       Euclidean distance (exact in int64, fits int32).  Used
                       for the n=256 (64x64 grid) and n=16384 (1024x1024
                       grid) single solves (CircleSquare-like, Table 1).
* ``shapes_sqdist`` -- 2-D points on circle / square / triangle boundaries in
                       [0,1]^2 plus N(0, 0.01^2) noise, cost =
                       round(1e4 * squared distance) in FP64 (CircleSquare).
* ``uniform_costs`` -- i.i.d. uniform integers in [0, 2^20).
* ``embedding_costs`` -- n + n unit-normalised 300-d Gaussian vectors, cost =
                       round(1e4 * Euclidean distance) in FP64 (NLP-like).
* ``pixel_sqdist``  -- random pixel positions (with replacement) on a 28 x 28
                       grid, cost = squared distance (MNIST-like, many ties).
* ``mnist_transport`` -- two images of distinct nonzero pixels with integer
                       intensities of equal totals (integer-supply transport).

Every generator takes an explicit integer seed (numpy PCG64); the batch and
serving streams derive per-instance seeds as ``base + index``.
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 20200503


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _sqdist_int(a: np.ndarray, b: np.ndarray, chunk: int = 2048) -> np.ndarray:
    """Exact squared distances between integer points (int64 math, int32 out)."""
    n, m = a.shape[0], b.shape[0]
    out = np.empty((n, m), np.int32)
    a = a.astype(np.int64)
    b = b.astype(np.int64)
    for s in range(0, n, chunk):
        d0 = a[s:s + chunk, None, 0] - b[None, :, 0]
        d1 = a[s:s + chunk, None, 1] - b[None, :, 1]
        out[s:s + chunk] = d0 * d0 + d1 * d1
    return out


def grid_sqdist(n: int, m: int | None = None, grid: int = 64, seed: int = BASE_SEED) -> np.ndarray:
    """n + m integer points uniform on a grid x grid lattice; C = squared distance."""
    m = n if m is None else m
    r = _rng(seed)
    a = r.integers(0, grid, size=(n, 2))
    b = r.integers(0, grid, size=(m, 2))
    return _sqdist_int(a, b)


def _boundary_points(shape: str, k: int, r: np.random.Generator) -> np.ndarray:
    t = r.random(k)
    if shape == "circle":
        ang = 2.0 * math.pi * t
        p = np.stack([0.5 + 0.5 * np.cos(ang), 0.5 + 0.5 * np.sin(ang)], 1)
    elif shape == "square":
        side = np.floor(t * 4.0)
        f = t * 4.0 - side
        lo, hi = 0.1, 0.9
        x = np.where(side == 0, lo + (hi - lo) * f, np.where(side == 1, hi, np.where(side == 2, hi - (hi - lo) * f, lo)))
        y = np.where(side == 0, lo, np.where(side == 1, lo + (hi - lo) * f, np.where(side == 2, hi, hi - (hi - lo) * f)))
        p = np.stack([x, y], 1)
    elif shape == "triangle":
        v = np.array([[0.5, 0.95], [0.05, 0.1], [0.95, 0.1]])
        e = np.roll(v, -1, axis=0) - v
        L = np.sqrt((e ** 2).sum(1))
        cum = np.concatenate([[0.0], np.cumsum(L)]) / L.sum()
        side = np.clip(np.searchsorted(cum, t, side="right") - 1, 0, 2)
        f = (t - cum[side]) / (cum[side + 1] - cum[side])
        p = v[side] + f[:, None] * e[side]
    else:
        raise ValueError(shape)
    return p + r.normal(0.0, 0.01, size=p.shape)


def shapes_sqdist(n: int, pair: str = "circle-square", seed: int = BASE_SEED,
                  scale: float = 1e4) -> np.ndarray:
    """Points on two shape boundaries; C = round(scale * squared distance), FP64."""
    r = _rng(seed)
    s0, s1 = pair.split("-")
    a = _boundary_points(s0, n, r)
    b = _boundary_points(s1, n, r)
    out = np.empty((n, n), np.int32)
    for s in range(0, n, 1024):
        d = a[s:s + 1024, None, :] - b[None, :, :]
        out[s:s + 1024] = np.rint(scale * (d * d).sum(-1)).astype(np.int32)
    return out


def uniform_costs(n: int, m: int | None = None, hi: int = 1 << 20, seed: int = BASE_SEED) -> np.ndarray:
    """C i.i.d. uniform integers in [0, hi)."""
    m = n if m is None else m
    return _rng(seed).integers(0, hi, size=(n, m), dtype=np.int32)


def embedding_costs(n: int, dim: int = 300, seed: int = BASE_SEED, scale: float = 1e4) -> np.ndarray:
    """n + n unit-normalised Gaussian vectors; C = round(scale * ||a - b||), FP64."""
    r = _rng(seed)
    a = r.standard_normal((n, dim))
    b = r.standard_normal((n, dim))
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b /= np.linalg.norm(b, axis=1, keepdims=True)
    d2 = (a * a).sum(1)[:, None] + (b * b).sum(1)[None, :] - 2.0 * (a @ b.T)
    return np.rint(scale * np.sqrt(np.maximum(d2, 0.0))).astype(np.int32)


def pixel_sqdist(n: int, m: int | None = None, side: int = 28, seed: int = BASE_SEED) -> np.ndarray:
    """Random pixel positions (with replacement) on a side x side image; C = squared distance."""
    m = n if m is None else m
    r = _rng(seed)
    pa = r.integers(0, side * side, size=n)
    pb = r.integers(0, side * side, size=m)
    a = np.stack([pa // side, pa % side], 1)
    b = np.stack([pb // side, pb % side], 1)
    return _sqdist_int(a, b)


def mnist_transport(n: int, m: int, total: int, side: int = 28, seed: int = BASE_SEED):
    """Two 'images' for integer-supply transport (MNIST-like, Table 1): n and
    m distinct nonzero pixels of a side x side grid, C = squared distance,
    and integer intensities (at least 1 per pixel) summing to `total` on both
    sides, drawn as uniform weights and rounded by largest remainder.
    Returns (C, supply, demand)."""
    r = _rng(seed)
    pa = r.choice(side * side, size=n, replace=False)
    pb = r.choice(side * side, size=m, replace=False)
    a = np.stack([pa // side, pa % side], 1)
    b = np.stack([pb // side, pb % side], 1)

    def weights(k):
        if total < k:
            raise ValueError("total must cover one unit per pixel")
        w = r.uniform(0.05, 1.0, size=k)
        x = (total - k) * w / w.sum()
        q = np.floor(x).astype(np.int64)
        rest = int(total - k - q.sum())
        q[np.argsort(q - x)[:rest]] += 1  # largest remainders first
        return (q + 1).astype(np.int32)

    return _sqdist_int(a, b), weights(n), weights(m)


# ---------------------------------------------------------------------------
# the five named workloads
# ---------------------------------------------------------------------------

def single_256(seed: int = BASE_SEED) -> np.ndarray:
    """n = m = 256, points uniform on a 64 x 64 grid, squared distance."""
    return grid_sqdist(256, 256, grid=64, seed=seed)


def single_4096(kind: str = "circle-square", seed: int = BASE_SEED) -> np.ndarray:
    """n = m = 4096: 'circle-square' / 'circle-triangle' shapes, or 'uniform'."""
    if kind == "uniform":
        return uniform_costs(4096, seed=seed)
    return shapes_sqdist(4096, pair=kind, seed=seed)


def batch_sizes(k: int, lo: int = 32, hi: int = 256, seed: int = BASE_SEED) -> np.ndarray:
    """Instance sizes n ~ U{lo..hi} for the multi-instance batch."""
    return _rng(seed).integers(lo, hi + 1, size=k)


def batch_embeddings(k: int = 4096, lo: int = 32, hi: int = 256, seed: int = BASE_SEED,
                     dim: int = 300) -> list[np.ndarray]:
    """k independent embedding-distance instances with n ~ U{lo..hi}."""
    sizes = batch_sizes(k, lo, hi, seed)
    return [embedding_costs(int(n), dim=dim, seed=seed + 1 + i) for i, n in enumerate(sizes)]


def served_requests(count: int, rate_per_s: float, lo: int = 16, hi: int = 2048,
                    seed: int = BASE_SEED) -> list[tuple[float, np.ndarray]]:
    """Open-loop Poisson stream: (arrival time in s, cost matrix) pairs with
    n log-uniform on [lo, hi] and MNIST-like pixel costs."""
    r = _rng(seed)
    gaps = r.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps) - gaps[0]
    sizes = np.exp(r.uniform(math.log(lo), math.log(hi + 1), size=count)).astype(np.int64)
    sizes = np.clip(sizes, lo, hi)
    return [(float(t[i]), pixel_sqdist(int(sizes[i]), seed=seed + 1 + i)) for i in range(count)]


def single_16384(seed: int = BASE_SEED) -> np.ndarray:
    """n = m = 16384, points uniform on a 1024 x 1024 grid, squared distance (1 GiB int32)."""
    return grid_sqdist(16384, 16384, grid=1024, seed=seed)
