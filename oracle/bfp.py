"""Exact block-floating-point (BFP) reference.  TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct CPU restatement of the BFP arithmetic of
Kohl, McCormick & Tamstorf, "Multigrid methods using Block Floating Point
Arithmetic" (arXiv:2307.00124).  Only ``tests/``, ``__graft_entry__.smoke``
and the CPU legs of ``bench.py`` may use it; the CUDA path shares no code
with it.

Conventions (each tied to the passage it follows)
-------------------------------------------------
* A BFP block is x = 2^e * m with integer mantissas m in X_w =
  [-2^(w-1), 2^(w-1)-1] and one shared exponent e (Sec. 2).
* ``msb(m)`` is the signed bit width min{v >= 1 : m in X_v}, so msb(0) = 1
  and msb(23) = 6, the value Fig. 2 gives for mu*.
* Truncation is the arithmetic right shift, i.e. floor (Sec. 2).
* An op first forms its exact result z* = 2^(e*) * Z with the App. B setup
  rules for e* and w* (Alg. espmv-setup, eaxpby-setup, egemv-setup), then
  quantises it:
    - qcomp (Alg. qcomp): the normalised floor quantisation to w_out bits;
      ``qcomp_def`` is that plain definition and ``qcomp_alg`` walks the
      algorithm's own steps (window from gamma and w_tmp, temporary,
      overflow / underflow, recompute) and must give the same mantissas;
    - nnqcomp (Alg. nnqcomp): window from gamma alone, floor shift, clamp
      to X_w_out.
* gamma and w_add follow Table tab:estimates; the damped-Jacobi rows are
  this library's reading (the paper's smoother is Chebyshev) and are marked
  as such below.

Arrays are numpy int64 when a static bound proves no overflow, else numpy
object arrays of Python ints (exact at any width).
"""
from __future__ import annotations

from dataclasses import dataclass
from fractions import Fraction
from typing import Optional

import numpy as np

INT64_SAFE_BITS = 62          # |values| < 2^62 keeps every +,- and <<1 exact


# ---------------------------------------------------------------------------
# Integer primitives (Sec. 2)
# ---------------------------------------------------------------------------

def msb(m: int) -> int:
    """Signed bit width of one integer: min{v >= 1 : m in X_v} (Sec. 2, Fig. 2)."""
    m = int(m)
    return (m if m >= 0 else -m - 1).bit_length() + 1


def bits_of(z) -> int:
    """Largest msb over an integer array (1 for an empty or all-zero array)."""
    if z.size == 0:
        return 1
    if z.dtype == object:
        hi, lo = max(z.flat), min(z.flat)
    else:
        hi, lo = int(z.max()), int(z.min())
    return max(msb(hi), msb(lo), 1)


def max_msb(z) -> int:
    """mu* of Alg. qcomp: max_i msb(z_i), starting from 1."""
    return bits_of(z)


def as_exact(z, bound_bits: int):
    """Return z as int64 when bound_bits fits, else as Python-int objects."""
    if bound_bits <= INT64_SAFE_BITS:
        return np.asarray(z).astype(np.int64)
    return to_object(z)


def to_object(z):
    z = np.asarray(z)
    if z.dtype == object:
        return z
    out = np.empty(z.shape, dtype=object)
    out.ravel()[:] = [int(v) for v in z.ravel()]
    return out


def _promote(z, need_bits: int):
    if z.dtype != object and need_bits > INT64_SAFE_BITS:
        return to_object(z)
    return z


def mul_c(z, c: int):
    """Exact z * c for an integer constant c."""
    z = _promote(np.asarray(z), bits_of(np.asarray(z)) + msb(c))
    return z * (int(c) if z.dtype == object else np.int64(c))


def add_exact(a, b):
    """Exact a + b of two integer arrays."""
    need = max(bits_of(a), bits_of(b)) + 1
    if a.dtype == object or b.dtype == object or need > INT64_SAFE_BITS:
        return to_object(a) + to_object(b)
    return a + b


def zpad(z):
    """Zero Dirichlet halo of width one (keeps Python ints for object arrays)."""
    if z.dtype != object:
        return np.pad(z, 1)
    out = np.empty(tuple(n + 2 for n in z.shape), dtype=object)
    out.fill(0)
    out[tuple(slice(1, -1) for _ in z.shape)] = z
    return out


def floor_shift(z, lam: int):
    """floor(z * 2^-lam): arithmetic right shift for lam >= 0, left shift else."""
    lam = int(lam)
    if lam >= 0:
        if z.dtype == object:
            return z >> lam
        return z >> min(lam, 63)
    k = -lam
    z = _promote(z, bits_of(z) + k)
    return z << k


def wrap(z, width: int):
    """decr(): keep the low ``width`` bits as a two's-complement integer (Sec. 2)."""
    half = 1 << (width - 1)
    mask = (1 << width) - 1
    if z.dtype != object and width <= INT64_SAFE_BITS and bits_of(z) <= INT64_SAFE_BITS - 1:
        return ((z + np.int64(half)) & np.int64(mask)) - np.int64(half)
    zo = to_object(z)
    return ((zo + half) & mask) - half


def clamp(z, width: int):
    """Saturate to X_width (Alg. nnqcomp, clamp step)."""
    lo, hi = -(1 << (width - 1)), (1 << (width - 1)) - 1
    if z.dtype == object:
        return np.minimum(np.maximum(z, lo), hi)
    return np.clip(z, lo, hi)


def clog2(m: int) -> int:
    """ceil(log2 m) for m >= 1."""
    return (int(m) - 1).bit_length()


# ---------------------------------------------------------------------------
# BFP blocks and scalars
# ---------------------------------------------------------------------------

@dataclass
class BFP:
    """One BFP block (Sec. 2): values 2^e * m, m in X_w."""
    m: np.ndarray
    e: int
    w: int

    def __post_init__(self):
        self.e = int(self.e)
        self.w = int(self.w)

    @property
    def norm_m(self) -> int:
        """max_i |m_i| (the mantissa of the exact max-norm)."""
        if self.m.size == 0:
            return 0
        return int(max(abs(int(self.m.max())), abs(int(self.m.min()))))

    def values(self):
        """Exact values as Fractions (small blocks only)."""
        return np.vectorize(lambda v: Fraction(int(v)) * Fraction(2) ** self.e,
                            otypes=[object])(self.m)

    def check(self):
        assert bits_of(self.m) <= self.w, "mantissa outside X_w"
        return self


@dataclass
class Scalar:
    """A BFP scalar alpha = 2^e * m (Sec. 2 with d = 1)."""
    m: int
    e: int

    @property
    def w(self) -> int:
        return msb(self.m)

    def value(self) -> Fraction:
        return Fraction(self.m) * Fraction(2) ** self.e


def scalar_floor(x: float | Fraction, w: int) -> Scalar:
    """quant(): normalised floor quantisation of one real to w bits.

    Alg. ir / v-cycle / fmg call quant() without fixing its rounding; this
    reading takes floor, the truncation Sec. 2 defines.
    """
    x = Fraction(x)
    if x == 0:
        return Scalar(0, 0)
    # smallest e with floor(x / 2^e) in X_w
    e = 0
    while True:
        m = (x / Fraction(2) ** e).__floor__()
        if msb(m) <= w:
            # try to lower e while it still fits
            while True:
                m2 = (x / Fraction(2) ** (e - 1)).__floor__()
                if msb(m2) <= w:
                    e -= 1
                    m = m2
                else:
                    return Scalar(int(m), e)
        e += 1


@dataclass
class Exact:
    """Exact result z* = 2^e * z with the App. B width w* (the setup-func output)."""
    z: np.ndarray
    e: int
    w: int


# ---------------------------------------------------------------------------
# Quantisation: qcomp (Alg. qcomp) and nnqcomp (Alg. nnqcomp)
# ---------------------------------------------------------------------------

def qcomp_def(ex: Exact, w_out: int) -> BFP:
    """Plain definition of the qcomp result: normalised floor quantisation.

    mu* = max_i msb(z*_i) (>= 1), lambda_out = mu* - w_out,
    e_out = e* + lambda_out, m_i = floor(z*_i / 2^lambda_out)
    (Alg. qcomp, the lines after the first parallel loop).
    """
    mu_star = max_msb(ex.z)
    lam_out = mu_star - w_out
    m = floor_shift(ex.z, lam_out)
    return BFP(as_exact(m, w_out), ex.e + lam_out, w_out)


def gamma_mu(gamma: tuple[int, int], e_star: int) -> int:
    """msb(m_gamma) + e_gamma - e*: the window MSB derived from gamma.

    gamma = (m, e) >= 0 as an exact dyadic.  gamma = 0 is read as the zero
    BFP scalar with exponent e*, so the term is msb(0) = 1 (the paper
    requires gamma > 0 and is silent on zero).
    """
    gm, ge = gamma
    if gm == 0:
        return 1
    return msb(gm) + ge - e_star


def qcomp_alg(ex: Exact, w_out: int, w_tmp: int, gamma: tuple[int, int]):
    """Alg. qcomp, step by step.  Returns (result, overflow, underflow).

    Window: mu_tmp = msb(gamma_m) + e_gamma - e*, lambda_tmp = mu_tmp - w_tmp;
    the temporary keeps decr(w* - w_tmp, z* >> lambda_tmp); after the first
    loop overflow = mu_tmp < mu*, underflow = lambda_out < lambda_tmp, and
    on either the result is recomputed from the exact values.
    """
    assert 0 < w_out <= w_tmp
    mu_tmp = gamma_mu(gamma, ex.e)
    lam_tmp = mu_tmp - w_tmp
    # first parallel loop: exact value, running max of its msb, windowed temporary
    mu_star = max_msb(ex.z)
    tmp = wrap(floor_shift(ex.z, lam_tmp), w_tmp)
    lam_out = mu_star - w_out
    e_out = ex.e + lam_out
    overflow = mu_tmp < mu_star
    underflow = lam_out < lam_tmp
    if overflow or underflow:
        m = wrap(floor_shift(ex.z, lam_out), w_out)        # recompute from exact values
    else:
        m = wrap(floor_shift(tmp, lam_out - lam_tmp), w_tmp)  # narrow the temporary
        m = wrap(m, w_out)
    return BFP(as_exact(m, w_out), e_out, w_out), bool(overflow), bool(underflow)


def nnqcomp(ex: Exact, w_out: int, gamma: tuple[int, int]):
    """Alg. nnqcomp: window from gamma, floor shift, saturate.  Returns (result, n_saturated)."""
    mu_out = gamma_mu(gamma, ex.e)
    lam_out = mu_out - w_out
    t = floor_shift(ex.z, lam_out)
    c = clamp(t, w_out)
    nsat = int(np.count_nonzero(c != t))
    return BFP(as_exact(c, w_out), ex.e + lam_out, w_out), nsat


# ---------------------------------------------------------------------------
# Exact dyadic helpers for gamma
# ---------------------------------------------------------------------------

def dy_add(a: tuple[int, int], b: tuple[int, int]) -> tuple[int, int]:
    (am, ae), (bm, be) = a, b
    if am == 0:
        return (bm, be)
    if bm == 0:
        return (am, ae)
    e = min(ae, be)
    return ((am << (ae - e)) + (bm << (be - e)), e)


def dy_mul(a: tuple[int, int], b: tuple[int, int]) -> tuple[int, int]:
    return (a[0] * b[0], a[1] + b[1])


def norm(x: BFP) -> tuple[int, int]:
    """Exact ||x||_inf = max|m| * 2^e."""
    return (x.norm_m, x.e)


def sabs(s: Scalar) -> tuple[int, int]:
    return (abs(s.m), s.e)


# ---------------------------------------------------------------------------
# Operators of the 2D / 3D model problem (setup S with a dyadic diagonal)
# ---------------------------------------------------------------------------

@dataclass
class Stencil:
    """Constant-coefficient star stencil stored as one BFP block.

    2D: A' = (h^2/4) A_h = D^-1 A_h, centre 1 (m=4), neighbours -1/4 (m=-1),
        e = -2: exactly the operator Alg. solver-setup produces (D = I).
    3D: A' = (h^2/8) A_h, centre 3/4 (m=6), neighbours -1/8 (m=-1), e = -3.
        Setup S would give the non-dyadic -1/6; this reading keeps the
        operator exact and moves the factor 8/6 into the smoother weight.
    """
    ndim: int
    center: int
    nbr: int
    e: int

    @property
    def w(self) -> int:
        return max(msb(self.center), msb(self.nbr))

    @property
    def m_A(self) -> int:
        return 2 * self.ndim + 1

    @property
    def norm_inf(self) -> tuple[int, int]:
        return (abs(self.center) + 2 * self.ndim * abs(self.nbr), self.e)


def laplace_stencil(ndim: int) -> Stencil:
    if ndim == 2:
        return Stencil(2, 4, -1, -2)
    if ndim == 3:
        return Stencil(3, 6, -1, -3)
    raise ValueError(ndim)


def shifts(ndim):
    """Neighbour offsets in the fixed order W, E, S, N[, B, T] (x fastest)."""
    out = []
    for ax in range(ndim):           # ax 0 = x (last numpy axis)
        for s in (-1, +1):
            off = [0] * ndim
            off[ndim - 1 - ax] = s
            out.append(tuple(off))
    return out


def neighbour_sum(x):
    """Sum over the 2*ndim axis neighbours with zero Dirichlet halo (exact ints)."""
    nd = x.ndim
    x = _promote(x, bits_of(x) + 3)
    p = zpad(x)
    acc = None
    for off in shifts(nd):
        sl = tuple(slice(1 + o, p.shape[i] - 1 + o) for i, o in enumerate(off))
        acc = p[sl].copy() if acc is None else acc + p[sl]
    return acc


def espmv_stencil(A: Stencil, x: BFP) -> Exact:
    """Alg. espmv-setup / espmv-row for the star stencil.

    w* = w_A + w_x + ceil(log2 m_A), e* = e_A + e_x; row i sums the exact
    integer products A_ij * x_j over the nonzeros of row i.
    """
    w_star = A.w + x.w + clog2(A.m_A)
    xm = as_exact(x.m, w_star)
    z = add_exact(mul_c(xm, A.center), mul_c(neighbour_sum(xm), A.nbr))
    return Exact(z, A.e + x.e, w_star)


def eaxpby(alpha: Scalar, a: Exact | BFP, beta: Scalar, b: Exact | BFP) -> Exact:
    """Alg. eaxpby-setup / eaxpby-row: exact alpha*a + beta*b.

    Widths w_alpha + w_a and w_beta + w_b, exponents e_alpha + e_a and
    e_beta + e_b; the term with the larger exponent is sign-extended and
    left-shifted by |d|; w* = max(...) + 1, e* = min(e_a*, e_b*).
    """
    am, ae, aw = (a.z, a.e, a.w) if isinstance(a, Exact) else (a.m, a.e, a.w)
    bm, be, bw = (b.z, b.e, b.w) if isinstance(b, Exact) else (b.m, b.e, b.w)
    wa, wb = alpha.w + aw, beta.w + bw
    ea, eb = alpha.e + ae, beta.e + be
    d = ea - eb
    if d < 0:
        w_star = max(wa, wb + abs(d)) + 1
    else:
        w_star = max(wb, wa + abs(d)) + 1
    A = mul_c(np.asarray(am), alpha.m)
    B = mul_c(np.asarray(bm), beta.m)
    if d < 0:
        B = floor_shift(B, d)        # left shift by |d|
    else:
        A = floor_shift(A, -d)
    return Exact(add_exact(A, B), min(ea, eb), w_star)


def egemv(A: Stencil, x: BFP, y: BFP, alpha: Scalar, beta: Scalar) -> Exact:
    """Alg. egemv-setup / egemv-row: exact alpha*A*x + beta*y via espmv and eaxpby."""
    g = espmv_stencil(A, x)
    return eaxpby(alpha, g, beta, y)


def jacobi_operator(A: Stencil, omega: Scalar) -> Stencil:
    """S = I - omega*A as one BFP block with exponent e_S = min(0, e_omega + e_A)."""
    e_s = min(0, omega.e + A.e)
    k = omega.e + A.e - e_s
    c = (1 << (0 - e_s)) - (omega.m * A.center << k)
    n = -(omega.m * A.nbr << k)
    return Stencil(A.ndim, c, n, e_s)


ONE = Scalar(1, 0)
MINUS_ONE = Scalar(-1, 0)


# --- grid transfers (2D bilinear / 3D trilinear P, full-weighting R~) -------

def _p1(delta: int) -> int:
    """1D interpolation mantissa at exponent -1: 2 for the coinciding node, 1 for a neighbour."""
    return {0: 2, -1: 1, 1: 1}.get(delta, 0)


def coarse_shape(fine_shape):
    return tuple((n - 1) // 2 for n in fine_shape)


def prolong_exponent(ndim: int) -> int:
    return -ndim


def prolong_norm(ndim: int) -> tuple[int, int]:
    """||P||_inf: every fine row sums to 1."""
    return (1 << ndim, -ndim)


def restrict_exponent(ndim: int) -> int:
    """R~ = D_c^-1 R_FW D_f: P^T in 2D (e = -2), P^T / 2 in 3D (e = -4)."""
    return -2 if ndim == 2 else -4


def restrict_norm(ndim: int) -> tuple[int, int]:
    return (4 ** ndim, restrict_exponent(ndim))


def espmv_restrict(r: BFP) -> Exact:
    """Exact R~ r_v: coarse node J collects fine nodes 2J+1+delta, weights prod(2-|delta|).

    m_R = 3^d nonzeros per row, w_R = msb(2^d), w* = w_R + w_r + ceil(log2 m_R).
    """
    nd = r.m.ndim
    m_R = 3 ** nd
    w_R = msb(2 ** nd)
    w_star = w_R + r.w + clog2(m_R)
    f = as_exact(r.m, w_star)
    cs = coarse_shape(f.shape)
    z = as_exact(np.zeros(cs, dtype=np.int64), w_star)
    import itertools
    for delta in itertools.product((-1, 0, 1), repeat=nd):
        wgt = 1
        sl = []
        for ax, dl in enumerate(delta):
            wgt *= 2 - abs(dl)
            start = 1 + dl
            sl.append(slice(start, start + 2 * cs[ax] - 1 + 1, 2))
        z = add_exact(z, mul_c(f[tuple(sl)], wgt))
    return Exact(z, restrict_exponent(nd) + r.e, w_star)


def espmv_prolong(d: BFP, fine_shape) -> Exact:
    """Exact P d: fine node i gets sum over coarse I of prod_ax p1(i_ax - (2 I_ax + 1)).

    Mantissas in {2^d, ..., 1} at e = -d (2D: 4, 2, 1 at e=-2); m_P = 2^d,
    w* = w_P + w_d + ceil(log2 m_P).
    """
    nd = d.m.ndim
    m_P = 2 ** nd
    w_P = msb(2 ** nd)
    w_star = w_P + d.w + clog2(m_P)
    c = as_exact(d.m, w_star)
    assert tuple(coarse_shape(fine_shape)) == tuple(c.shape)
    z = as_exact(np.zeros(tuple(fine_shape), dtype=np.int64), w_star)
    import itertools
    # coarse node I sits at fine index 2I+1; it contributes to 2I, 2I+1, 2I+2
    for delta in itertools.product((-1, 0, 1), repeat=nd):
        wgt = 1
        sl = []
        for ax, dl in enumerate(delta):
            wgt *= _p1(dl)
            start = 1 + dl
            sl.append(slice(start, start + 2 * c.shape[ax] - 1 + 1, 2))
        z[tuple(sl)] = z[tuple(sl)] + c * wgt
    return Exact(z, prolong_exponent(nd) + d.e, w_star)


# ---------------------------------------------------------------------------
# gamma rules (Table tab:estimates; Jacobi rows are this library's reading)
# ---------------------------------------------------------------------------

W_ADD = {
    "jacobi": 2,       # Table tab:estimates, V relaxation row
    "cheby": 2,        # V relaxation row (the paper's Chebyshev step)
    "residual": 4,     # V residual row
    "restrict": 6,     # V restriction row
    "correct": 1,      # V correction row
    "interp": 0,       # FMG prolongation row
    "apply": 2,        # "w_add = 2 for all operations" (Sec. 5.3 closing remark)
    "axpy": 2,
    "normalize": 2,
}


def gamma_jacobi(A: Stencil, omega: Scalar, y: Optional[BFP], r: BFP):
    """||S||_inf ||y|| + |omega| ||r||, S = I - omega A (relaxation row read for Jacobi)."""
    g = dy_mul(sabs(omega), norm(r))
    if y is not None:
        S = jacobi_operator(A, omega)
        g = dy_add(dy_mul(S.norm_inf, norm(y)), g)
    return g


def gamma_residual(A: Stencil, omega: Scalar, y: BFP, r: BFP):
    """1/4 (2 c1 + 1) ||r|| with c1 = 2 omega (V residual row; two Jacobi sweeps from 0
    equal one Chebyshev step with c1 = 2 omega, c2 = -omega^2)."""
    del A, y
    # (2*(2 omega) + 1) / 4 = omega + 1/4
    coef = dy_add(sabs(omega), (1, -2))
    return dy_mul(coef, norm(r))


def gamma_restrict(rv: BFP):
    return dy_mul(restrict_norm(rv.m.ndim), norm(rv))


def gamma_correct(y: Optional[BFP], d: BFP):
    g = dy_mul(prolong_norm(d.m.ndim), norm(d))
    if y is not None:
        g = dy_add(norm(y), g)
    return g


def gamma_apply(A: Stencil, x: BFP):
    return dy_mul(A.norm_inf, norm(x))


def gamma_axpy(alpha: Scalar, x: BFP, beta: Scalar, y: BFP):
    return dy_add(dy_mul(sabs(alpha), norm(x)), dy_mul(sabs(beta), norm(y)))


# ---------------------------------------------------------------------------
# Ops mirroring the C ABI
# ---------------------------------------------------------------------------

@dataclass
class Quant:
    """Quantisation request: result width, mode, extra temporary bits, optional gamma."""
    w_out: int
    mode: str = "qcomp"           # "qcomp" | "nnqcomp"
    w_add: Optional[int] = None   # None -> Table tab:estimates value of the op
    gamma: Optional[tuple[int, int]] = None   # None -> rule of the op
    w_add_max: Optional[int] = None   # cap on the table value (Table tab:recomputation's experiment)


@dataclass
class Stats:
    calls: int = 0
    recomputed: int = 0
    overflow: int = 0
    underflow: int = 0
    saturated: int = 0

    def add(self, other: "Stats"):
        for k in ("calls", "recomputed", "overflow", "underflow", "saturated"):
            setattr(self, k, getattr(self, k) + getattr(other, k))


def quantize(ex: Exact, q: Quant, op: str, gamma_rule, stats: Optional[Stats] = None) -> BFP:
    g = q.gamma if q.gamma is not None else gamma_rule
    st = Stats(calls=1)
    if q.mode == "qcomp":
        w_add = W_ADD[op] if q.w_add is None else q.w_add
        if q.w_add is None and q.w_add_max is not None:
            w_add = min(w_add, q.w_add_max)
        out, ovf, unf = qcomp_alg(ex, q.w_out, q.w_out + max(w_add, 0), g)
        ref = qcomp_def(ex, q.w_out)
        assert out.e == ref.e and np.array_equal(to_object(out.m), to_object(ref.m))
        st.overflow, st.underflow, st.recomputed = int(ovf), int(unf), int(ovf or unf)
    elif q.mode == "nnqcomp":
        out, nsat = nnqcomp(ex, q.w_out, g)
        st.saturated = nsat
    else:
        raise ValueError(q.mode)
    if stats is not None:
        stats.add(st)
    return out


def normalize(x: BFP, q: Quant, stats=None) -> BFP:
    """Re-quantise a block to q.w_out bits (exact z* = x)."""
    return quantize(Exact(x.m, x.e, x.w), q, "normalize", norm(x), stats)


def stencil_apply(A: Stencil, x: BFP, q: Quant, stats=None) -> BFP:
    """qspmv: z = A x (Alg. espmv + qcomp / nnqcomp)."""
    return quantize(espmv_stencil(A, x), q, "apply", gamma_apply(A, x), stats)


def residual(A: Stencil, y: BFP, r: BFP, q: Quant, omega: Scalar, stats=None) -> BFP:
    """r_v = A y - r (Alg. v-cycle residual line: qgemv with alpha = 1, beta = -1)."""
    ex = egemv(A, y, r, ONE, MINUS_ONE)
    return quantize(ex, q, "residual", gamma_residual(A, omega, y, r), stats)


def jacobi(A: Stencil, omega: Scalar, y: Optional[BFP], r: BFP, q: Quant, stats=None) -> BFP:
    """Damped Jacobi y' = y + omega (r - A y) = S y + omega r, S = I - omega A.

    Computed as egemv(S, y, r, 1, omega); with y = None (zero initial guess)
    the exact result is omega * r (e* = e_omega + e_r).
    """
    if y is None:
        ex = Exact(mul_c(as_exact(r.m, omega.w + r.w), omega.m), omega.e + r.e, omega.w + r.w)
    else:
        S = jacobi_operator(A, omega)
        ex = egemv(S, y, r, ONE, omega)
    return quantize(ex, q, "jacobi", gamma_jacobi(A, omega, y, r), stats)


def cheby(A: Stencil, c1: Scalar, c2: Scalar, r: BFP, q: Quant, stats=None) -> BFP:
    """Alg. v-cycle relaxation line from y = 0: y = qgemv(A, r, r, c2, c1) = c2 A r + c1 r
    (two Chebyshev steps in one qgemv); gamma = c1 ||r|| (Table tab:estimates relaxation row)."""
    return quantize(egemv(A, r, r, c2, c1), q, "cheby", dy_mul(sabs(c1), norm(r)), stats)


def restrict(rv: BFP, q: Quant, stats=None) -> BFP:
    """r_c = R~ r_v (Alg. v-cycle restriction line: qspmv with R)."""
    return quantize(espmv_restrict(rv), q, "restrict", gamma_restrict(rv), stats)


def prolong(d: BFP, y: Optional[BFP], fine_shape, q: Quant, stats=None) -> BFP:
    """y' = y - P d (Alg. v-cycle correction: qgemv(P, d, y, -1, 1)); y = None gives P d
    (Alg. fmg interpolation: qspmv(P, x))."""
    pd = espmv_prolong(d, fine_shape)
    if y is None:
        return quantize(pd, q, "interp", gamma_correct(None, d), stats)
    ex = eaxpby(MINUS_ONE, pd, ONE, y)
    return quantize(ex, q, "correct", gamma_correct(y, d), stats)


def axpy(alpha: Scalar, x: BFP, beta: Scalar, y: BFP, q: Quant, stats=None) -> BFP:
    """z = alpha x + beta y (Alg. eaxpby + qcomp / nnqcomp)."""
    return quantize(eaxpby(alpha, x, beta, y), q, "axpy", gamma_axpy(alpha, x, beta, y), stats)


def dot(x: BFP, y: BFP, w_out: int) -> Scalar:
    """Exact sum_i x_i y_i, then normalised to w_out bits (Sec. 2 remark on BFP dot
    products: one accumulator of w_x + w_y + ceil(log2 n) bits, one final shift)."""
    n = x.m.size
    w_star = x.w + y.w + clog2(max(n, 1))
    s = int(np.sum(to_object(x.m.ravel()) * to_object(y.m.ravel()))) if n else 0
    ex = Exact(np.array([s], dtype=object), x.e + y.e, w_star)
    out = qcomp_def(ex, w_out)
    return Scalar(int(out.m[0]), out.e)


F64_E_STAR = -1074   # every finite double is an integer multiple of 2^-1074


def f64_split(x: np.ndarray):
    """Exact integer significand and exponent: x = M * 2^E (zeros get M = 0, E = -1074)."""
    x = np.asarray(x, dtype=np.float64)
    if not np.all(np.isfinite(x)):
        raise ValueError("non-finite input")
    fm, fe = np.frexp(x)
    M = (fm * 2.0 ** 53).astype(np.int64)       # exact: |fm| in [0.5, 1) times 2^53
    E = fe.astype(np.int64) - 53
    E = np.where(M == 0, F64_E_STAR, E)
    return M, E


def from_f64(x: np.ndarray, w_out: int) -> BFP:
    """Floor-quantise doubles to a normalised BFP block of w_out bits.

    The doubles are one exact BFP block with e* = -1074; the result is
    qcomp_def of it: e_out = max_i (msb(M_i) + E_i) - w_out and
    m_i = floor(x_i / 2^e_out) (quant() read as floor, Alg. ir).
    """
    M, E = f64_split(x)
    v = np.where(M < 0, -M - 1, M)
    mb = np.zeros(M.shape, dtype=np.int64)
    # exact bit length of each |significand| < 2^53
    t = v.copy()
    for k in (32, 16, 8, 4, 2, 1):
        big = t >= (1 << k)
        mb = mb + np.where(big, k, 0)
        t = np.where(big, t >> k, t)
    mb = mb + (t > 0)
    msb_i = mb + 1
    mv = np.where(M == 0, F64_E_STAR + 1, msb_i + E)
    mu_abs = int(mv.max()) if mv.size else F64_E_STAR + 1
    mu_abs = max(mu_abs, F64_E_STAR + 1)
    e_out = mu_abs - w_out
    sh = E - e_out                      # left shift when >= 0
    left = np.where(sh >= 0, sh, 0)
    right = np.minimum(np.where(sh < 0, -sh, 0), 63)
    m = np.where(sh >= 0, M << left, M >> right)
    return BFP(m.astype(np.int64), e_out, w_out)


def to_f64(x: BFP) -> np.ndarray:
    """m * 2^e as doubles (exact whenever the value is representable, e.g. w <= 53)."""
    return np.ldexp(np.asarray(x.m, dtype=np.float64), x.e)
