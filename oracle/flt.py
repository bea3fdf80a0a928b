"""Float baselines (not in the paper): FP32 and BF16-storage / FP32-arithmetic
versions of the V-cycle ops and of the IR-V / FMG schedule of ``mg.BFPSolver``.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Every op is numpy float32 arithmetic (IEEE round to nearest, no fused
multiply-add) in the order the C ABI states for flt_jacobi, flt_residual,
flt_restrict and flt_prolong; BF16 storage keeps the upper 16 bits of a
float32 value, rounded to nearest-even.  The operator, weight and schedule are
those of the BFP solver (A' = D^-1 A_h in 2D, (h^2/8) A_h in 3D; the weight
quantised to w_omega bits by floor), so the three solvers differ only in the
number format of the V-cycle.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import bfp as B
from . import mg

F32, BF16 = 0, 1


def round_bf16(a) -> np.ndarray:
    """float32 -> BF16 (round to nearest, ties to even), returned as float32 values."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def store(a, dtype: int) -> np.ndarray:
    a = np.asarray(a, dtype=np.float32)
    return a if dtype == F32 else round_bf16(a)


def from_f64(x: np.ndarray, dtype: int) -> np.ndarray:
    """FP64 -> FP32 (round to nearest) [-> BF16]."""
    return store(np.asarray(x, dtype=np.float64).astype(np.float32), dtype)


def coefs(A: B.Stencil, om: B.Scalar):
    c = np.float32(A.center * 2.0 ** A.e)
    nb = np.float32(A.nbr * 2.0 ** A.e)
    w = np.float32(om.m * 2.0 ** om.e)
    assert float(c) == A.center * 2.0 ** A.e and float(w) == om.m * 2.0 ** om.e
    return c, nb, w


def _apply(A, y):
    nbs = mg.neighbours_f64(np.asarray(y, dtype=np.float32))   # W, E, S, N[, B, T], zero outside
    c, nb, _ = coefs(A, B.Scalar(0, 0))
    s = (nbs[0] + nbs[1]) + (nbs[2] + nbs[3])
    if y.ndim == 3:
        s = s + (nbs[4] + nbs[5])
    return c * y + nb * s


def jacobi(A: B.Stencil, om: B.Scalar, y, r, dtype: int) -> np.ndarray:
    """y + om (r - A'y) (y None: om r), float32 in the stated order, stored as dtype."""
    _, _, w = coefs(A, om)
    r = np.asarray(r, dtype=np.float32)
    if y is None:
        return store(w * r, dtype)
    y = np.asarray(y, dtype=np.float32)
    return store(y + w * (r - _apply(A, y)), dtype)


def residual(A: B.Stencil, y, r, dtype: int) -> np.ndarray:
    """r_v = A'y - r."""
    y = np.asarray(y, dtype=np.float32)
    return store(_apply(A, y) - np.asarray(r, dtype=np.float32), dtype)


def _fw_axis(f: np.ndarray, axis: int) -> np.ndarray:
    """(f[2I] + 2 f[2I+1]) + f[2I+2] along one axis."""
    n = f.shape[axis]
    m = (n - 1) // 2

    def sl(start):
        s = [slice(None)] * f.ndim
        s[axis] = slice(start, start + 2 * m, 2)
        return tuple(s)
    return (f[sl(0)] + np.float32(2.0) * f[sl(1)]) + f[sl(2)]


def restrict(rf, dtype: int) -> np.ndarray:
    """Full weighting: along x, then y [then z], times 2^-2 (2D) or 2^-4 (3D)."""
    f = np.asarray(rf, dtype=np.float32)
    nd = f.ndim
    for axis in range(nd - 1, -1, -1):        # x is the last numpy axis
        f = _fw_axis(f, axis)
    return store(np.float32(0.25 if nd == 2 else 0.0625) * f, dtype)


def _interp_axis(d: np.ndarray, axis: int) -> np.ndarray:
    """Fine index 2m+1 on coarse m; fine 2m between m-1 and m: 0.5 a + 0.5 b (zero outside)."""
    nc = d.shape[axis]
    pad = [(0, 0)] * d.ndim
    pad[axis] = (1, 1)
    dp = np.pad(d, pad)

    def take(idx):
        s = [slice(None)] * d.ndim
        s[axis] = idx
        return dp[tuple(s)]
    shape = list(d.shape)
    shape[axis] = 2 * nc + 1
    out = np.zeros(shape, dtype=np.float32)
    half = np.float32(0.5)
    for i in range(2 * nc + 1):
        s = [slice(None)] * d.ndim
        s[axis] = i
        if i % 2 == 1:
            out[tuple(s)] = take((i - 1) // 2 + 1)
        else:
            out[tuple(s)] = half * take(i // 2) + half * take(i // 2 + 1)
    return out


def prolong(d, y, fine_shape, dtype: int) -> np.ndarray:
    """y - P d (y given) or P d: interpolation along x, then y [then z]."""
    p = np.asarray(d, dtype=np.float32)
    for axis in range(p.ndim - 1, -1, -1):
        p = _interp_axis(p, axis)
    assert p.shape == tuple(fine_shape)
    if y is None:
        return store(p, dtype)
    return store(np.asarray(y, dtype=np.float32) - p, dtype)


@dataclass
class FloatSolver:
    """The IR-V / FMG schedule of mg.BFPSolver with float vectors (FP32 or BF16 storage)."""
    ndim: int
    n: int
    dtype: int = F32
    nu1: int = 2
    nu2: int = 2
    coarse_sweeps: int = 32
    omega: float = 0.8
    w_omega: int = 16
    n_fmg: int = 2

    def __post_init__(self):
        self.A = B.laplace_stencil(self.ndim)
        self.om = B.scalar_floor(mg.omega_scaled(self.ndim, self.omega), self.w_omega)
        sizes = []
        m = self.n
        while True:
            sizes.append(m)
            if m <= 3:
                break
            m = (m - 1) // 2
        self.sizes = sizes

    def vcycle(self, k: int, r: np.ndarray) -> np.ndarray:
        A, om, dt = self.A, self.om, self.dtype
        coarsest = k == len(self.sizes) - 1
        nu1 = self.coarse_sweeps if coarsest else self.nu1
        y = jacobi(A, om, None, r, dt)
        for _ in range(nu1 - 1):
            y = jacobi(A, om, y, r, dt)
        if coarsest:
            return y
        rv = residual(A, y, r, dt)
        rc = restrict(rv, dt)
        d = self.vcycle(k + 1, rc)
        y = prolong(d, y, r.shape, dt)
        for _ in range(self.nu2):
            y = jacobi(A, om, y, r, dt)
        return y

    def ir_step(self, k: int, b: np.ndarray, x: np.ndarray) -> np.ndarray:
        """FP64 residual (mg.residual_f64), rounded to FP32 [then BF16], float V-cycle, FP64 update."""
        r = from_f64(mg.residual_f64(b, x), self.dtype)
        y = self.vcycle(k, r)
        return x + y.astype(np.float64)

    def rhs_hierarchy(self, f: np.ndarray):
        bs = [mg.scaled_rhs(f)]
        for _ in self.sizes[1:]:
            bs.append(mg.restrict_f64(bs[-1]))
        return bs

    def fmg(self, f: np.ndarray) -> np.ndarray:
        bs = self.rhs_hierarchy(f)
        x = None
        for k in range(len(self.sizes) - 1, -1, -1):
            if x is None:
                x = np.zeros(bs[k].shape)
            else:
                xs = from_f64(x, self.dtype)
                x = prolong(xs, None, bs[k].shape, self.dtype).astype(np.float64)
            for _ in range(self.n_fmg):
                x = self.ir_step(k, bs[k], x)
        return x
