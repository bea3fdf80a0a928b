"""Seeded synthetic inputs shared by the tests, the oracle checks and bench.py.

This module only draws and samples inputs (random mantissas, the manufactured
right-hand side, seeded smooth fields, instance sizes).  It holds none of the
method's arithmetic: no quantisation, no stencil, no multigrid step.
"""
from __future__ import annotations

import math

import numpy as np


def grid_n(levels_below: int) -> int:
    """Interior points per side n = 2^J - 1."""
    return (1 << levels_below) - 1


def manufactured_rhs(ndim: int, n: int) -> np.ndarray:
    """f = d pi^2 prod_i sin(pi x_i) for u = prod_i sin(pi x_i), shape (n,)*ndim, x fastest."""
    h = 1.0 / (n + 1)
    s = np.sin(np.pi * np.arange(1, n + 1) * h)
    u = s
    for _ in range(ndim - 1):
        u = np.multiply.outer(s, u)
    return (ndim * math.pi ** 2) * u


def random_mantissas(shape, w: int, seed: int, dist: str = "uniform") -> np.ndarray:
    """Mantissas in X_w = [-2^(w-1), 2^(w-1)-1] as int64.

    dist: "uniform" over X_w, "small" (a few bits used), "smooth" (a sampled
    low-frequency field scaled to the range, like a multigrid residual).
    """
    rng = np.random.default_rng(seed)
    lo, hi = -(1 << (w - 1)), (1 << (w - 1)) - 1
    if dist == "uniform":
        return rng.integers(lo, hi + 1, size=shape, dtype=np.int64)
    if dist == "small":
        k = max(1, w // 3)
        return rng.integers(-(1 << (k - 1)), 1 << (k - 1), size=shape, dtype=np.int64)
    if dist == "smooth":
        grids = np.meshgrid(*[np.linspace(0, 1, s) for s in shape], indexing="ij")
        f = np.zeros(shape)
        for _ in range(4):
            k = rng.integers(1, 4, size=len(shape))
            ph = rng.uniform(0, 2 * np.pi, size=len(shape))
            term = np.ones(shape)
            for g, kk, pp in zip(grids, k, ph):
                term = term * np.sin(np.pi * kk * g + pp)
            f += rng.uniform(-1, 1) * term
        f = f / max(np.abs(f).max(), 1e-300)
        m = np.floor(f * hi).astype(np.int64)
        return np.clip(m, lo, hi)
    raise ValueError(dist)


def random_exponent(seed: int, lo: int = -40, hi: int = 10) -> int:
    return int(np.random.default_rng(seed).integers(lo, hi + 1))


def batch_sizes(count: int = 256, seed: int = 3, sides=(127, 255, 511, 1023)) -> list:
    """Grid sides of a batch of independent instances, drawn uniformly from `sides`."""
    rng = np.random.default_rng(seed)
    return [int(v) for v in rng.choice(np.asarray(sides), size=count)]


def smoothed_random_rhs(n: int, seed: int, sweeps: int = 4) -> np.ndarray:
    """A seeded n x n right-hand side: uniform in [-1, 1], then `sweeps` passes of
    f <- f/2 + (W + E + S + N)/8 with zeros outside (rough but not white noise)."""
    f = np.random.default_rng(seed).uniform(-1.0, 1.0, size=(n, n))
    for _ in range(sweeps):
        p = np.pad(f, 1)
        f = 0.5 * f + 0.125 * (p[1:-1, :-2] + p[1:-1, 2:] + p[:-2, 1:-1] + p[2:, 1:-1])
    return f


def grf_nodes(n: int, seed: int = 1, modes: int = 64, kmax: int = 8, sigma: float = 1.0) -> np.ndarray:
    """Coefficient field k = exp(g) at the (n+2) x (n+2) grid nodes, boundary included
    (numpy order [y, x], node (i, j) at (i h, j h), h = 1/(n+1)).

    g is a seeded smooth Gaussian random field: sigma sqrt(2/modes) times the sum of
    `modes` terms cos(pi (kx x + ky y) + phi) with integer wave numbers kx, ky uniform in
    [-kmax, kmax] (not both zero) and phases uniform in [0, 2 pi).  The same (kx, ky, phi)
    for every n, so the coarse grids of a hierarchy sample the same field.
    """
    rng = np.random.default_rng(seed)
    kx, ky = [], []
    while len(kx) < modes:
        a, b = (int(v) for v in rng.integers(-kmax, kmax + 1, size=2))
        if a == 0 and b == 0:
            continue
        kx.append(a)
        ky.append(b)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=modes)
    t = np.arange(n + 2) / (n + 1)
    g = np.zeros((n + 2, n + 2))
    for m in range(modes):
        g += np.cos(np.pi * (kx[m] * t[None, :] + ky[m] * t[:, None]) + phi[m])
    return np.exp(sigma * math.sqrt(2.0 / modes) * g)
