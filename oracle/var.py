"""Variable-coefficient 2D operator -div(k grad u) = f in BFP and FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

A variable-coefficient workload beside the model problem (not in the paper, whose
experiments use constant-coefficient FE problems): 5-point finite differences
on n = 2^J - 1 interior points per side with zero Dirichlet boundary, face
coefficients the harmonic means of k at the two nodes they join.  The
readings below are this library's; each is stated where it is used.

* Scaling.  The system is multiplied by h^2 (A' = h^2 A_h, b' = h^2 f, an
  exact power of two): A' has the face coefficients k_f themselves and the
  centre c = k_W + k_E + k_S + k_N on every level.  Folding D^-1 into the
  operator as setup S does for constant coefficients would make every
  neighbour coefficient -k_f / c non-dyadic, and their floor quantisation
  makes the row sums negative (the 3D constant case shows how that breaks
  definiteness); here the quantised operator keeps zero row sums.
* Storage.  The four per-point face arrays W, E, S, N are one BFP block:
  mantissas floor(k_f / 2^e_k) in X_16 with one exponent e_k (the largest
  face gets 15 significant bits); the centre is their exact integer sum.
* Smoother.  Damped Jacobi with the diagonal, y' = y + Q (r - A' y), Q =
  diag(q_i 2^e_q), q_i = floor(omega_m 2^s / c_i) (exact integer division) with
  the weight omega of the constant 2D case; then ||I - Q A'||_inf = 1 exactly
  (diagonal 1 - q_i c_i >= 0, off-diagonals summing to q_i c_i).
* gamma (Table tab:estimates read for this operator): Jacobi ||y|| +
  ||q||_inf ||r|| (the relaxation row with ||S|| = 1), zero guess
  ||q||_inf ||r||, residual (omega + 1/4) ||r|| (the V residual row as in the
  constant case), A' x: ||A'||_inf ||x|| with ||A'||_inf = max_i 2 c_i.
* Coarse levels: k injected to the coarse nodes, faces rediscretised; R~ and P
  are those of the constant 2D case (with A' = h^2 A_h on every level the
  coarse right-hand side is P^T times the fine one).
* FP64 IR residual: r = b' - (c64 x - (((k_W x_W + k_E x_E) + k_S x_S) + k_N x_N))
  with the unquantised FP64 faces, c64 = ((k_W + k_E) + k_S) + k_N, every
  product and sum correctly rounded in this order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import bfp as B
from . import mg

W_K = 16          # face-coefficient mantissa width of the V-cycle's operator (int16)
W_IR = 26         # face width of the finest operator in the BFP IR residual (Alg. ir quantises A to
                  # the input width): A'x within the 62-bit group bound for x up to 32 bits


def harmonic(a, b):
    """Harmonic mean of two node values, ((2 a) b) / (a + b) in FP64 (symmetric in a, b)."""
    return ((2.0 * a) * b) / (a + b)


def face_arrays(K: np.ndarray):
    """Per-point face coefficients (W, E, S, N) from node values K of shape (n+2, n+2)
    (boundary nodes included, numpy order [y, x])."""
    c = K[1:-1, 1:-1]
    return (harmonic(K[1:-1, :-2], c), harmonic(c, K[1:-1, 2:]),
            harmonic(K[:-2, 1:-1], c), harmonic(c, K[2:, 1:-1]))


def quantize_faces(faces, w: int = W_K):
    """Floor quantisation of the four face arrays as one BFP block: e_k such that the
    largest face has mantissa in [2^(w-2), 2^(w-1)), m = floor(k / 2^e_k)."""
    M = max(float(np.max(f)) for f in faces)
    _, fe = math.frexp(M)               # M = fm 2^fe, fm in [0.5, 1)
    e_k = fe - (w - 1)
    ms = [np.floor(np.ldexp(f, -e_k)).astype(np.int64) for f in faces]
    return ms, e_k


def smoother_weights(c: np.ndarray, e_k: int, om: B.Scalar, w: int = W_K):
    """q_i = floor(omega_m 2^s / c_i) with the largest s for which max q fits X_w;
    q_i 2^e_q ~ omega / (c_i 2^e_k) with e_q = e_omega - e_k - s."""
    wm = int(om.m)
    lim = (1 << (w - 1)) * int(c.min())        # max q <= 2^(w-1) - 1  <=>  omega_m 2^s < lim

    def fits(sv: int) -> bool:
        return (wm << sv) < lim if sv >= 0 else wm < (lim << -sv)

    s = lim.bit_length() - wm.bit_length()
    while not fits(s):
        s -= 1
    while fits(s + 1):
        s += 1

    # exact integer floor division (omega_m 2^s < 2^15 c_min < 2^33: int64 is exact)
    c64 = np.asarray(c, dtype=np.int64)
    q = (np.int64(wm << s) // c64) if s >= 0 else (np.int64(wm) // (c64 << np.int64(-s)))
    return q.astype(np.int64), int(om.e) - e_k - s


@dataclass
class VarOp:
    """One level's operator: face mantissas (W, E, S, N) at e_k, centre c = their sum,
    smoother weights q at e_q, and the unquantised FP64 faces for the IR residual."""
    kw: np.ndarray
    ke: np.ndarray
    ks: np.ndarray
    kn: np.ndarray
    e_k: int
    q: np.ndarray
    e_q: int
    f64: tuple
    c64: np.ndarray
    c: np.ndarray = field(init=False)

    def __post_init__(self):
        self.c = self.kw + self.ke + self.ks + self.kn

    @property
    def a_norm(self) -> tuple[int, int]:
        """||A'||_inf = max_i 2 c_i (row i: centre c_i, faces summing to c_i)."""
        return (2 * int(self.c.max()), self.e_k)

    @property
    def q_norm(self) -> tuple[int, int]:
        return (int(self.q.max()), self.e_q)


def make_level(K: np.ndarray, om: B.Scalar) -> VarOp:
    faces = face_arrays(K)
    (kw, ke, ks, kn), e_k = quantize_faces(faces)
    c = kw + ke + ks + kn
    q, e_q = smoother_weights(c, e_k, om)
    fw, fe, fs, fn = faces
    c64 = ((fw + fe) + fs) + fn
    return VarOp(kw, ke, ks, kn, e_k, q, e_q, faces, c64)


def make_ir_level(K: np.ndarray, om: B.Scalar, w: int = W_IR) -> VarOp:
    """The finest operator for the IR residual with BFP x and b: the same faces floor-quantised
    to w bits as one block (no smoother weights: apply / residual only)."""
    faces = face_arrays(K)
    (kw, ke, ks, kn), e_k = quantize_faces(faces, w)
    fw, fe, fs, fn = faces
    zero = np.zeros_like(kw)
    return VarOp(kw, ke, ks, kn, e_k, zero, 0, faces, ((fw + fe) + fs) + fn)


def coarse_nodes(K: np.ndarray) -> np.ndarray:
    """Injection of the node values: coarse node c sits on fine node 2c (boundary included)."""
    return K[::2, ::2]


# ---------------------------------------------------------------------------
# BFP ops (exact result, then the quantisation of oracle.bfp)
# ---------------------------------------------------------------------------

def _nbrs(m):
    p = B.zpad(np.asarray(m))
    return p[1:-1, :-2], p[1:-1, 2:], p[:-2, 1:-1], p[2:, 1:-1]


def apply_exact(op: VarOp, x: B.BFP) -> B.Exact:
    """Exact A' x = c x - (k_W x_W + k_E x_E + k_S x_S + k_N x_N) at e_k + e_x."""
    xo = B.to_object(x.m)
    W, E, S, N = _nbrs(xo)
    z = B.to_object(op.c) * xo - (B.to_object(op.kw) * W + B.to_object(op.ke) * E +
                                  B.to_object(op.ks) * S + B.to_object(op.kn) * N)
    return B.Exact(z, op.e_k + x.e, B.bits_of(z))


def gamma_jacobi(op: VarOp, y: Optional[B.BFP], r: B.BFP):
    g = B.dy_mul(op.q_norm, B.norm(r))
    if y is not None:
        g = B.dy_add(B.norm(y), g)
    return g


def apply(op: VarOp, x: B.BFP, q: B.Quant, stats=None) -> B.BFP:
    return B.quantize(apply_exact(op, x), q, "apply", B.dy_mul(op.a_norm, B.norm(x)), stats)


def residual(op: VarOp, y: B.BFP, r: B.BFP, q: B.Quant, om: B.Scalar, stats=None) -> B.BFP:
    """r_v = A' y - r (the paper's sign, as for constant coefficients)."""
    ex = B.eaxpby(B.ONE, apply_exact(op, y), B.MINUS_ONE, r)
    return B.quantize(ex, q, "residual", B.dy_mul(B.dy_add(B.sabs(om), (1, -2)), B.norm(r)), stats)


def jacobi(op: VarOp, y: Optional[B.BFP], r: B.BFP, q: B.Quant, stats=None) -> B.BFP:
    """y' = y + Q (r - A' y) exactly (y = None: Q r), then quantised."""
    qo, ro = B.to_object(op.q), B.to_object(r.m)
    if y is None:
        z = qo * ro
        ex = B.Exact(z, op.e_q + r.e, B.bits_of(z))
    else:
        ay = apply_exact(op, y)
        E = min(y.e, op.e_q + r.e, op.e_q + ay.e)
        z = ((B.to_object(y.m) << (y.e - E)) + ((qo * ro) << (op.e_q + r.e - E)) -
             ((qo * ay.z) << (op.e_q + ay.e - E)))
        ex = B.Exact(z, E, B.bits_of(z))
    return B.quantize(ex, q, "jacobi", gamma_jacobi(op, y, r), stats)


# ---------------------------------------------------------------------------
# FP64 pieces (fixed order)
# ---------------------------------------------------------------------------

def apply_f64(op: VarOp, x: np.ndarray) -> np.ndarray:
    fw, fe, fs, fn = op.f64
    W, E, S, N = _nbrs(x)
    s = ((fw * W + fe * E) + fs * S) + fn * N
    return op.c64 * x - s


def residual_f64(op: VarOp, b: np.ndarray, x: np.ndarray) -> np.ndarray:
    return b - apply_f64(op, x)


def scaled_rhs(f: np.ndarray) -> np.ndarray:
    """b' = h^2 f (exact power-of-two scaling)."""
    h = 1.0 / (f.shape[0] + 1)
    return f * (h * h)


# ---------------------------------------------------------------------------
# Solver: the schedule of oracle.mg.BFPSolver with the variable operator
# ---------------------------------------------------------------------------

@dataclass
class VarSolver:
    K: np.ndarray                    # node values of k, shape (n+2, n+2)
    w: int = 16
    mode: str = "qcomp"
    nu1: int = 2
    nu2: int = 2
    coarse_sweeps: int = 32
    omega: float = 0.8
    w_omega: int = 16
    n_fmg: int = 2
    w_step: int = 0                  # progressive precision (as mg.BFPSolver)
    w_ir: int = W_IR                 # face width of the BFP IR residual's operator
    stats: B.Stats = field(default_factory=B.Stats)

    def __post_init__(self):
        self.om = B.scalar_floor(self.omega, self.w_omega)
        self.n = self.K.shape[0] - 2
        self.ops, self.sizes = [], []
        K, m = self.K, self.n
        while True:
            self.ops.append(make_level(K, self.om))
            self.sizes.append(m)
            if m <= 3:
                break
            K, m = coarse_nodes(K), (m - 1) // 2

    def width(self, k: int) -> int:
        return max(self.w - k * self.w_step, min(self.w, 2))

    @property
    def q(self) -> B.Quant:
        return B.Quant(self.w, self.mode)

    def ql(self, k: int) -> B.Quant:
        return B.Quant(self.width(k), self.mode)

    def vcycle(self, k: int, r: B.BFP) -> B.BFP:
        op, q, st = self.ops[k], self.ql(k), self.stats
        coarsest = k == len(self.sizes) - 1
        y = jacobi(op, None, r, q, st)
        for _ in range((self.coarse_sweeps if coarsest else self.nu1) - 1):
            y = jacobi(op, y, r, q, st)
        if coarsest:
            return y
        rv = residual(op, y, r, q, self.om, st)
        rc = B.restrict(rv, q, st)
        d = self.vcycle(k + 1, rc)
        y = B.prolong(d, y, r.m.shape, q, st)
        for _ in range(self.nu2):
            y = jacobi(op, y, r, q, st)
        return y

    def ir_step(self, k: int, b: np.ndarray, x: np.ndarray) -> np.ndarray:
        r = B.from_f64(residual_f64(self.ops[k], b, x), self.width(k))
        return x + B.to_f64(self.vcycle(k, r))

    def ir_step_bfp(self, b: B.BFP, x: B.BFP) -> B.BFP:
        """mg.BFPSolver.ir_step_bfp with the finest variable operator; the residual's operator
        has W_IR-bit faces (Alg. ir: A quantised to the input width), the V-cycle's W_K-bit."""
        if not hasattr(self, "op_ir"):
            self.op_ir = make_ir_level(self.K, self.om, self.w_ir)
        r = residual(self.op_ir, x, b, B.Quant(self.width(0), "qcomp"), self.om, self.stats)
        y = self.vcycle(0, r)
        return B.axpy(B.ONE, x, B.MINUS_ONE, y, B.Quant(x.w, "qcomp", 0), self.stats)

    def rhs_hierarchy(self, f: np.ndarray):
        bs = [scaled_rhs(f)]
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
                xp = B.prolong(B.from_f64(x, self.width(k + 1)), None, bs[k].shape, self.ql(k), self.stats)
                x = B.to_f64(xp)
            for _ in range(self.n_fmg):
                x = self.ir_step(k, bs[k], x)
        return x


# ---------------------------------------------------------------------------
# Discrete solutions and the accuracy test (u unknown)
# ---------------------------------------------------------------------------

def sparse_matrix(op: VarOp):
    """A' (FP64 faces) as a scipy CSR matrix, unknowns in row-major [y, x] order."""
    import scipy.sparse as sp
    n = op.c64.shape[0]
    idx = np.arange(n * n).reshape(n, n)
    fw, fe, fs, fn = op.f64
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [op.c64.ravel()]
    for coef, di, dj in ((fw, 0, -1), (fe, 0, 1), (fs, -1, 0), (fn, 1, 0)):
        jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        ok = (ii + dj >= 0) & (ii + dj < n) & (jj + di >= 0) & (jj + di < n)
        rows.append(idx[ok])
        cols.append(idx[(jj + di)[ok], (ii + dj)[ok]])
        vals.append(-coef[ok])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n * n, n * n))


def discrete_solution(op: VarOp, b: np.ndarray) -> np.ndarray:
    import scipy.sparse.linalg as spla
    return spla.spsolve(sparse_matrix(op).tocsc(), b.ravel()).reshape(b.shape)


def energy(op: VarOp, e: np.ndarray) -> float:
    return math.sqrt(max(float(np.sum(e * apply_f64(op, e))), 0.0))


def accuracy_ok(op: VarOp, x: np.ndarray, uh: np.ndarray, uh_coarse: np.ndarray) -> tuple[bool, float]:
    """||u_h - x||_A <= 0.5 ||u_h - P u_2h||_A (the sufficient test for an unknown u);
    returns (passed, ratio of the two norms)."""
    disc = energy(op, uh - mg.prolong_f64(uh_coarse, uh.shape))
    alg = energy(op, uh - x)
    return alg <= 0.5 * disc, alg / disc
