"""Multigrid reference: FP64 multigrid and the BFP V(2,2) / FMG / IR schedule.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Model problem (Sec. 5, eq. pde-poisson, discretised by finite differences as
the synthetic workloads require): -Laplace u = f on the unit square / cube,
zero Dirichlet boundary, n = 2^J - 1 interior points per side, h = 1/(n+1).

Scaling (Alg. solver-setup): the system is multiplied by h^2 / 2^p with 2^p
the smallest power of two >= 2d, giving A' (centre 2d / 2^p, neighbours
-1 / 2^p) and b' = (h^2 / 2^p) f.  In 2D this is exactly D^-1 A (D = I after
setup).  In 3D it keeps A' dyadic; the smoother weight absorbs 2^p / (2d).

V-cycle: the correction scheme of Alg. v-cycle with the paper's signs
(r_v = A y - r, y <- y - P d), generalised to nu1 pre- and nu2 post-sweeps
of damped Jacobi; FMG follows Alg. fmg with N IR-V steps per level; IR
follows Alg. ir with its residual and update in FP64 (r = b - A x, x <- x + y,
which is the paper's r = A x - b, x <- x - y with both signs flipped).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import bfp as B


# ---------------------------------------------------------------------------
# FP64 pieces with a fixed evaluation order (bit-reproducible)
# ---------------------------------------------------------------------------

def diag_coef(ndim: int) -> float:
    """Centre of A' = (h^2/2^p) A_h: 1 in 2D, 3/4 in 3D."""
    return (2.0 * ndim) / pscale(ndim)


def pscale(ndim: int) -> float:
    return 4.0 if ndim == 2 else 8.0


def nbr_coef(ndim: int) -> float:
    return -1.0 / pscale(ndim)


def omega_scaled(ndim: int, omega: float) -> float:
    """Jacobi weight for A': omega * 2^p / (2d)."""
    return omega * pscale(ndim) / (2.0 * ndim)


def neighbours_f64(x: np.ndarray) -> list:
    """The 2d neighbour arrays in the order W, E, S, N[, B, T], zero outside."""
    p = np.pad(x, 1)
    out = []
    for off in B.shifts(x.ndim):
        sl = tuple(slice(1 + o, p.shape[i] - 1 + o) for i, o in enumerate(off))
        out.append(p[sl])
    return out


def apply_f64(x: np.ndarray) -> np.ndarray:
    """A' x in FP64: s = ((W + E) + S) + N [+ B + T]; A'x = c*x + (nbr*s)."""
    nd = x.ndim
    nb = neighbours_f64(x)
    s = nb[0]
    for t in nb[1:]:
        s = s + t
    return diag_coef(nd) * x + nbr_coef(nd) * s


def residual_f64(b: np.ndarray, x: np.ndarray) -> np.ndarray:
    """IR residual r = b' - A' x (Alg. ir residual line, sign flipped)."""
    return b - apply_f64(x)


def restrict_f64(r: np.ndarray) -> np.ndarray:
    """Full weighting R~ in FP64, deltas in lexicographic order (outer axis first)."""
    import itertools
    nd = r.ndim
    cs = B.coarse_shape(r.shape)
    scale = 2.0 ** B.restrict_exponent(nd)
    acc = np.zeros(cs)
    for delta in itertools.product((-1, 0, 1), repeat=nd):
        wgt = 1
        sl = []
        for ax, dl in enumerate(delta):
            wgt *= 2 - abs(dl)
            sl.append(slice(1 + dl, 1 + dl + 2 * cs[ax], 2))
        acc = acc + (wgt * scale) * r[tuple(sl)]
    return acc


def prolong_f64(c: np.ndarray, fine_shape) -> np.ndarray:
    import itertools
    nd = c.ndim
    z = np.zeros(tuple(fine_shape))
    for delta in itertools.product((-1, 0, 1), repeat=nd):
        wgt = 1.0
        sl = []
        for ax, dl in enumerate(delta):
            wgt *= 1.0 if dl == 0 else 0.5
            sl.append(slice(1 + dl, 1 + dl + 2 * c.shape[ax], 2))
        z[tuple(sl)] += wgt * c
    return z


def energy_sq(e: np.ndarray) -> float:
    """e^T A' e (proportional to the discrete energy norm squared)."""
    return float(np.sum(e * apply_f64(e)))


# ---------------------------------------------------------------------------
# Manufactured problem (closed forms)
# ---------------------------------------------------------------------------

def grid_coords(n: int):
    h = 1.0 / (n + 1)
    return np.arange(1, n + 1) * h


def sin_product(ndim: int, n: int) -> np.ndarray:
    """u = prod sin(pi x_i) on the interior grid, shape (n,)*ndim (x fastest)."""
    s = np.sin(np.pi * grid_coords(n))
    u = s
    for _ in range(ndim - 1):
        u = np.multiply.outer(s, u)
    return u


def discrete_solution(ndim: int, n: int) -> np.ndarray:
    """u_h for f = d pi^2 u: u is an eigenvector of A_h with eigenvalue
    lambda_h = 4 d sin^2(pi h / 2) / h^2, so u_h = (d pi^2 / lambda_h) u."""
    h = 1.0 / (n + 1)
    lam = 4.0 * ndim * math.sin(math.pi * h / 2) ** 2 / h ** 2
    return (ndim * math.pi ** 2 / lam) * sin_product(ndim, n)


def scaled_rhs(f: np.ndarray) -> np.ndarray:
    """b' = (h^2 / 2^p) f (an exact power-of-two scaling)."""
    n = f.shape[0]
    h = 1.0 / (n + 1)
    return f * (h * h / pscale(f.ndim))


# ---------------------------------------------------------------------------
# FP64 V(nu1, nu2) multigrid (pins the BFP schedule's algebra)
# ---------------------------------------------------------------------------

def jacobi_f64(y: np.ndarray, r: np.ndarray, om: float) -> np.ndarray:
    return y + om * (r - apply_f64(y))


def vcycle_f64(r: np.ndarray, om: float, nu1=2, nu2=2, coarse_sweeps=32) -> np.ndarray:
    """FP64 V-cycle for A' y = r with the same schedule as the BFP one."""
    n = r.shape[0]
    if n <= 3:
        y = om * r
        for _ in range(coarse_sweeps - 1):
            y = jacobi_f64(y, r, om)
        return y
    y = om * r
    for _ in range(nu1 - 1):
        y = jacobi_f64(y, r, om)
    rv = apply_f64(y) - r
    rc = restrict_f64(rv)
    d = vcycle_f64(rc, om, nu1, nu2, coarse_sweeps)
    y = y - prolong_f64(d, r.shape)
    for _ in range(nu2):
        y = jacobi_f64(y, r, om)
    return y


# ---------------------------------------------------------------------------
# Chebyshev relaxation (Alg. cheby-nodes, Alg. v-cycle relaxation line)
# ---------------------------------------------------------------------------

L_EST = 5          # level on which the Chebyshev nodes are estimated (Sec. 4)
RHO_L5 = 1.995184726672197   # 1 + cos(pi/32) correctly rounded: rho_gen on level 5 without libm


def cheby_nodes(rho: float, eta: float) -> tuple[float, float]:
    """Alg. cheby-nodes: (c1, c2) of two Chebyshev steps targeting [eta rho, rho]."""
    alpha = 0.5 * (1.0 + eta) * rho
    c = 0.5 * (1.0 - eta) * rho
    beta = alpha - (c * c) / (2.0 * alpha)
    return 2.0 / beta, -1.0 / (alpha * beta)


def rho_gen(ndim: int, level: int = L_EST) -> float:
    """Largest eigenvalue of A x = lambda D x for the finite-difference Laplacian on level j
    (h = 2^-j): 1 + cos(pi h), the mode of highest frequency in every direction (the upper
    bound Alg. solver-setup asks for, taken exactly)."""
    del ndim
    return 1.0 + math.cos(math.pi * 2.0 ** -level)


def cheby_scaled(ndim: int, c1: float, c2: float) -> tuple[float, float]:
    """Coefficients for A' with diagonal d (1 in 2D, 3/4 in 3D): relaxing D^-1 A y = D^-1 r
    with (c1 I + c2 D^-1 A) is y = (c1 / d) r + (c2 / d^2) A' r."""
    d = diag_coef(ndim)
    return c1 / d, (c2 / d) / d


def cheby_f64(r: np.ndarray, c1: float, c2: float) -> np.ndarray:
    return c2 * apply_f64(r) + c1 * r


def vcycle10_f64(r: np.ndarray, c1: float, c2: float) -> np.ndarray:
    """FP64 V(1,0) of Alg. v-cycle with the Chebyshev relaxation (coarsest level: the
    relaxation alone); c1, c2 already scaled for A'."""
    y = cheby_f64(r, c1, c2)
    if r.shape[0] <= 3:
        return y
    d = vcycle10_f64(restrict_f64(apply_f64(y) - r), c1, c2)
    return y - prolong_f64(d, r.shape)


def vcycle10_rate(ndim: int, n: int, eta: float, iters: int = 40, seed: int = 0) -> float:
    """Asymptotic convergence factor of V(1,0) as a stationary iteration (power iteration on
    the error e <- e - V(A' e), unquantised coefficients)."""
    c1, c2 = cheby_scaled(ndim, *cheby_nodes(rho_gen(ndim), eta))
    e = np.random.default_rng(seed).standard_normal((n,) * ndim)
    e /= np.linalg.norm(e)
    rate = 0.0
    for i in range(iters):
        e = e - vcycle10_f64(apply_f64(e), c1, c2)
        nrm = float(np.linalg.norm(e))
        if i >= iters - 10:
            rate += math.log(nrm) / 10
        e /= nrm
    return math.exp(rate)


def eta_search(ndim: int, n: int = 31) -> float:
    """eta = i/100 (0 < i < 100) minimising the V(1,0) convergence factor on n^d points
    (Sec. 4: the targeted part of the spectrum is found empirically)."""
    rates = [(vcycle10_rate(ndim, n, i / 100.0), i) for i in range(1, 100)]
    return min(rates)[1] / 100.0


# ---------------------------------------------------------------------------
# BFP multigrid schedule
# ---------------------------------------------------------------------------

@dataclass
class BFPSolver:
    """Schedule of the BFP solver: widths, mode, sweeps and the quantised weight."""
    ndim: int
    n: int
    w: int = 16                      # one width for the input, working and inner widths (w_check = w = w_dot)
    mode: str = "qcomp"
    nu1: int = 2
    nu2: int = 2
    coarse_sweeps: int = 32
    omega: float = 0.8               # damped-Jacobi weight for A_h's diagonal
    w_omega: int = 16                # storage width of the weight (an input, w_check)
    n_fmg: int = 2                   # N of Alg. fmg
    w_step: int = 0                  # progressive precision: bits fewer per coarser level
    smoother: str = "jacobi"         # "jacobi": V(nu1, nu2) damped Jacobi; "cheby": the paper's V(1,0)
    eta: float = 0.15                # Chebyshev: targeted part [eta rho, rho] of the spectrum
    w_add_max: Optional[int] = None  # cap on every op's table w_add (Table tab:recomputation)
    ir_window: bool = True           # the IR residual's quantisation keeps Alg. qcomp's w_tmp window
    ir_window_bits: int = 32         # widest window kept (32-bit storage); a wider w_tmp recomputes
    stats: B.Stats = field(default_factory=B.Stats)

    def __post_init__(self):
        self.A = B.laplace_stencil(self.ndim)
        self.om = B.scalar_floor(omega_scaled(self.ndim, self.omega), self.w_omega)
        if self.smoother == "cheby":
            c1, c2 = cheby_scaled(self.ndim, *cheby_nodes(RHO_L5, self.eta))
            self.c1 = B.scalar_floor(c1, self.w_omega)
            self.c2 = B.scalar_floor(c2, self.w_omega)
            self.om_res = B.Scalar(self.c1.m, self.c1.e - 1)   # (2 c1 + 1)/4 = c1/2 + 1/4
        sizes = []
        m = self.n
        while True:
            sizes.append(m)
            if m <= 3:
                break
            m = (m - 1) // 2
        self.sizes = sizes
        self.ir_gamma = {}           # level -> mu* of that level's previous IR residual (its gamma)
        self.ir_counts = {}          # level -> [IR residual quantisations, of which recomputed]

    def width(self, k: int) -> int:
        """Inner width of level k (0 finest): w - k w_step, at least 2.  Progressive precision
        (Sec. 4, eq. width-bounds): the inner width w_dot_j = j m + q grows by m = 1 bit per finer
        level (never below 2 bits unless w is); every op of Alg. v-cycle on level j, the
        restriction to level j-1 included, outputs w_dot_j."""
        return max(self.w - k * self.w_step, min(self.w, 2))

    @property
    def q(self) -> B.Quant:
        return B.Quant(self.w, self.mode, w_add_max=self.w_add_max)

    def ql(self, k: int) -> B.Quant:
        return B.Quant(self.width(k), self.mode, w_add_max=self.w_add_max)

    def vcycle10(self, k: int, r: B.BFP) -> B.BFP:
        """Alg. v-cycle, V(1,0): y = qgemv(A, r, r, c2, c1); on levels above the coarsest the
        residual, restriction, coarse correction and interpolation follow (no post-smoothing)."""
        A, q, st = self.A, self.ql(k), self.stats
        y = B.cheby(A, self.c1, self.c2, r, q, st)
        if k == len(self.sizes) - 1:
            return y
        rv = B.residual(A, y, r, q, self.om_res, st)
        rc = B.restrict(rv, q, st)
        d = self.vcycle(k + 1, rc)
        return B.prolong(d, y, r.m.shape, q, st)

    def vcycle(self, k: int, r: B.BFP) -> B.BFP:
        if self.smoother == "cheby":
            return self.vcycle10(k, r)
        A, om, q, st = self.A, self.om, self.ql(k), self.stats
        if k == len(self.sizes) - 1:
            y = B.jacobi(A, om, None, r, q, st)
            for _ in range(self.coarse_sweeps - 1):
                y = B.jacobi(A, om, y, r, q, st)
            return y
        y = B.jacobi(A, om, None, r, q, st)
        for _ in range(self.nu1 - 1):
            y = B.jacobi(A, om, y, r, q, st)
        rv = B.residual(A, y, r, q, om, st)
        rc = B.restrict(rv, q, st)
        d = self.vcycle(k + 1, rc)
        y = B.prolong(d, y, r.m.shape, q, st)
        for _ in range(self.nu2):
            y = B.jacobi(A, om, y, r, q, st)
        return y

    def ir_quantize(self, k: int, r64: np.ndarray, first: bool = False) -> B.BFP:
        """quant(r) of Alg. ir on level k: the normalised floor quantisation of the FP64 residual
        (B.from_f64; Alg. qcomp's result does not depend on its window), plus the decision Alg. qcomp
        takes with the window of Table tab:estimates' IR residual rows.  gamma is the previous IR
        residual of the level: its window position msb(gamma_m) + e_gamma is taken as that residual's
        mu* (its exponent plus its width); w_add = 4 (i > 1), 5 for the first step on an FMG level,
        where gamma is the coarser level's last residual (the i = 1 row).  With no previous residual,
        or no window kept, the quantisation recomputes.  Overflow: mu_tmp < mu*; underflow:
        lambda_out < lambda_tmp (both in absolute exponents)."""
        w = self.width(k)
        r = B.from_f64(r64, w)
        mu = r.e + w
        w_add = 5 if first else 4
        if self.w_add_max is not None:
            w_add = min(w_add, self.w_add_max)
        w_tmp = w + w_add
        gam = self.ir_gamma.get(k)
        recomputed = True
        if self.ir_window and gam is not None and w_tmp <= self.ir_window_bits:
            overflow = gam < mu
            underflow = (mu - w) < (gam - w_tmp)
            recomputed = overflow or underflow
        cnt = self.ir_counts.setdefault(k, [0, 0])
        cnt[0] += 1
        cnt[1] += int(recomputed)
        self.ir_gamma[k] = mu
        return r

    def ir_totals(self, finest_only: bool = False) -> tuple[int, int]:
        """(IR residual quantisations, of which recomputed), over all levels or the finest."""
        ks = [0] if finest_only else list(self.ir_counts)
        return (sum(self.ir_counts.get(k, [0, 0])[0] for k in ks),
                sum(self.ir_counts.get(k, [0, 0])[1] for k in ks))

    def ir_step(self, k: int, b: np.ndarray, x: np.ndarray, trace: Optional[list] = None, first: bool = False):
        """One IR-V step (Alg. ir): FP64 residual, quantise (to the level's width), V-cycle, FP64 update."""
        r64 = residual_f64(b, x)
        r = self.ir_quantize(k, r64, first)
        y = self.vcycle(k, r)
        if trace is not None:
            trace.append((r, y))
        return x + B.to_f64(y)

    def ir_step_bfp(self, b: B.BFP, x: B.BFP) -> B.BFP:
        """One step of Alg. ir as printed, with x and b' held as BFP blocks (no FP64 pass):
        r = qgemv(A', x, b', 1, -1) at the inner width, y = V(r), x - y (qsub) at x's width
        (the working width).  Both results by Alg. qcomp: the IR residual always (the remark on
        skipping normalisation in IR-V, applied to every step), the update because x is the
        normalised working-precision iterate; the update's w_add is Table tab:estimates' IR
        correction row (0)."""
        r = B.residual(self.A, x, b, B.Quant(self.width(0), "qcomp"), self.om, self.stats)
        y = self.vcycle(0, r)
        return B.axpy(B.ONE, x, B.MINUS_ONE, y, B.Quant(x.w, "qcomp", 0), self.stats)

    def rhs_hierarchy(self, f: np.ndarray):
        bs = [scaled_rhs(f)]
        for _ in self.sizes[1:]:
            bs.append(restrict_f64(bs[-1]))
        return bs

    def fmg(self, f: np.ndarray, trace: Optional[list] = None) -> np.ndarray:
        """Alg. fmg: recurse to the coarsest level, interpolate at w (qspmv(P, x)), N IR-V steps."""
        bs = self.rhs_hierarchy(f)
        x = None
        self.ir_gamma = {}
        for k in range(len(self.sizes) - 1, -1, -1):
            if x is None:
                x = np.zeros(bs[k].shape)
            else:
                xq = B.from_f64(x, self.width(k + 1))
                xp = B.prolong(xq, None, bs[k].shape, self.ql(k), self.stats)
                x = B.to_f64(xp)
                self.ir_gamma[k] = self.ir_gamma.get(k + 1)     # gamma of the first step: the coarser residual
            for i in range(self.n_fmg):
                x = self.ir_step(k, bs[k], x, trace, first=(i == 0 and k < len(self.sizes) - 1))
        return x


def accuracy_ratio(ndim: int, x: np.ndarray) -> float:
    """||u - x||_L / ||u - u_h||_L (Sec. 5.1 acceptance test; <= 1.5 passes)."""
    n = x.shape[0]
    u = sin_product(ndim, n)
    uh = discrete_solution(ndim, n)
    return math.sqrt(energy_sq(u - x) / energy_sq(u - uh))
