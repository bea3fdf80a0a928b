"""Pins of the variable-coefficient oracle (oracle/var.py) against things other than itself:
the constant-coefficient oracle (k = 1), exact rational arithmetic on tiny grids,
the quantisation bounds, symmetry / definiteness of the operator, and the
accuracy test against a sparse direct solve."""
from fractions import Fraction

import numpy as np
import pytest

from bfp_inputs import grf_nodes, manufactured_rhs, random_mantissas, smoothed_random_rhs
from oracle import bfp as B
from oracle import mg
from oracle import var as V

OM = B.scalar_floor(0.8, 16)


def test_unit_coefficients_equal_the_constant_operator():
    """k = 1: faces 1, A'_var = 4 A'_const exactly, q c = omega exactly."""
    op = V.make_level(np.ones((17, 17)), OM)
    assert op.kw.max() == op.kw.min() == 1 << 14 and op.e_k == -14
    assert np.all(op.q * op.c * 2.0 ** (op.e_q + op.e_k) == float(OM.value()))
    A = B.laplace_stencil(2)
    x = B.BFP(random_mantissas((15, 15), 16, 1), -7, 16)
    for mode in ("qcomp", "nnqcomp"):
        q = B.Quant(16, mode)
        zv, zc = V.apply(op, x, q), B.stencil_apply(A, x, q)
        assert np.array_equal(zv.m, zc.m) and zv.e == zc.e + 2
        # jacobi with r scaled by 4 (the var system is the constant one times 4)
        r = B.BFP(random_mantissas((15, 15), 16, 2, "smooth"), -9, 16)
        r4 = B.BFP(r.m, r.e + 2, 16)
        for y in (None, x):
            jv, jc = V.jacobi(op, y, r4, q), B.jacobi(A, OM, y, r, q)
            assert np.array_equal(jv.m, jc.m) and jv.e == jc.e
        rv, rc = V.residual(op, x, r4, q, OM), B.residual(A, x, r, q, OM)
        assert np.array_equal(rv.m, rc.m) and rv.e == rc.e + 2


@pytest.mark.parametrize("mode", ["qcomp", "nnqcomp"])
def test_unit_coefficients_fmg_equals_constant_solver(mode):
    """The whole FMG + IR solve with k = 1 is the constant solver's, bit for bit
    (the FP64 residual is 4x the constant one exactly: power-of-two scalings)."""
    n = 31
    f = manufactured_rhs(2, n)
    sv = V.VarSolver(np.ones((n + 2, n + 2)), w=16, mode=mode)
    sc = mg.BFPSolver(2, n, w=16, mode=mode)
    xv, xc = sv.fmg(f), sc.fmg(f)
    assert np.array_equal(xv, xc)
    b = sv.rhs_hierarchy(f)[0]
    assert np.array_equal(V.residual_f64(sv.ops[0], b, xv), 4.0 * mg.residual_f64(sc.rhs_hierarchy(f)[0], xc))


def _frac(m, e):
    return Fraction(int(m)) * Fraction(2) ** int(e)


def test_exact_ops_by_rationals():
    """apply / jacobi exact results against Fraction arithmetic on a 4x3 grid."""
    K = grf_nodes(4, seed=5)[:5, :6]           # (ny + 2) x (nx + 2) with ny = 3, nx = 4
    op = V.make_level(K, OM)
    ny, nx = op.c.shape
    y = B.BFP(random_mantissas((ny, nx), 12, 3), -5, 12)
    r = B.BFP(random_mantissas((ny, nx), 12, 4), 3, 12)

    def Y(i, j):
        return _frac(y.m[j, i], y.e) if 0 <= i < nx and 0 <= j < ny else Fraction(0)

    def Ay(i, j):
        kf = [_frac(a[j, i], op.e_k) for a in (op.kw, op.ke, op.ks, op.kn)]
        return sum(kf) * Y(i, j) - (kf[0] * Y(i - 1, j) + kf[1] * Y(i + 1, j) + kf[2] * Y(i, j - 1) +
                                    kf[3] * Y(i, j + 1))
    ex = V.apply_exact(op, y)
    for j in range(ny):
        for i in range(nx):
            assert _frac(ex.z[j, i], ex.e) == Ay(i, j)
    # jacobi: y + q (r - A'y), through the quantiser's exact input
    for j in range(ny):
        for i in range(nx):
            want = Y(i, j) + _frac(op.q[j, i], op.e_q) * (_frac(r.m[j, i], r.e) - Ay(i, j))
            qd = B.Quant(12, "qcomp")
            got = V.jacobi(op, y, r, qd)
            # quantised output is the floor of the exact value at the output exponent
            assert _frac(got.m[j, i], got.e) <= want < _frac(got.m[j, i] + 1, got.e)


def test_quantisation_bounds_and_weights():
    K = grf_nodes(63, seed=1)
    op = V.make_level(K, OM)
    faces = V.face_arrays(K)
    for m, f in zip((op.kw, op.ke, op.ks, op.kn), faces):
        err = f - np.ldexp(m.astype(np.float64), op.e_k)
        assert np.all(err >= 0) and np.all(err < 2.0 ** op.e_k)
    assert (1 << 14) <= max(int(a.max()) for a in (op.kw, op.ke, op.ks, op.kn)) < (1 << 15)
    # smoother weights: floor of omega / c, largest scale that fits 16 bits
    qc = op.q.astype(object) * op.c.astype(object)
    lim = Fraction(int(OM.m)) * Fraction(2) ** (OM.e - op.e_q - op.e_k)
    assert all(Fraction(v) <= lim for v in qc.ravel())
    assert all(lim - Fraction(v) < Fraction(int(c)) for v, c in zip(qc.ravel(), op.c.ravel()))
    assert int(op.q.max()) < (1 << 15) and 2 * int(op.q.max()) >= (1 << 14)


def test_operator_symmetric_and_definite():
    K = grf_nodes(15, seed=7)
    op = V.make_level(K, OM)
    assert np.array_equal(op.ke[:, :-1], op.kw[:, 1:]) and np.array_equal(op.kn[:-1, :], op.ks[1:, :])
    ones = B.BFP(np.ones((15, 15), dtype=np.int64), 0, 2)
    z = V.apply_exact(op, ones).z
    inner = np.asarray(z[1:-1, 1:-1], dtype=np.int64)
    assert np.all(inner == 0)                            # zero row sums away from the boundary
    M = V.sparse_matrix(op).toarray()
    assert np.allclose(M, M.T, rtol=0, atol=0)
    assert np.linalg.eigvalsh(M).min() > 0


def test_fp64_residual_order_and_scaling():
    n = 15
    K = grf_nodes(n, seed=9)
    op = V.make_level(K, OM)
    x = np.random.default_rng(1).standard_normal((n, n))
    b = V.scaled_rhs(smoothed_random_rhs(n, 2))
    r = V.residual_f64(op, b, x)
    # the same sequence written out point by point
    fw, fe, fs, fn = op.f64
    for j in (0, 7, 14):
        for i in (0, 3, 14):
            def X(a, c):
                return x[c, a] if 0 <= a < n and 0 <= c < n else 0.0
            s = ((fw[j, i] * X(i - 1, j) + fe[j, i] * X(i + 1, j)) + fs[j, i] * X(i, j - 1)) + fn[j, i] * X(i, j + 1)
            c64 = ((fw[j, i] + fe[j, i]) + fs[j, i]) + fn[j, i]
            assert r[j, i] == b[j, i] - (c64 * x[j, i] - s)
    # solution of A' u = b' solves the unscaled system A_h u = f
    uh = V.discrete_solution(op, b)
    assert np.abs(V.residual_f64(op, b, uh)).max() < 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("w", [16, 24])
def test_fmg_ir_reaches_accuracy(w):
    """FMG + IR-V steps on a variable field reach ||u_h - x|| <= 0.5 ||u_h - P u_2h||."""
    n = 63
    K = grf_nodes(n, seed=1)
    f = smoothed_random_rhs(n, 2)
    s = V.VarSolver(K, w=w, mode="nnqcomp")
    bs = s.rhs_hierarchy(f)
    uh = V.discrete_solution(s.ops[0], bs[0])
    u2h = V.discrete_solution(s.ops[1], bs[1])
    x = s.fmg(f)
    for _ in range(2):
        x = s.ir_step(0, bs[0], x)
    ok, ratio = V.accuracy_ok(s.ops[0], x, uh, u2h)
    assert ok, ratio
    # IR keeps converging to the FP64 discrete solution (rediscretised coarse operators on a
    # rough k contract ~0.5 per IR-V step here; k = 1 gives ~0.15)
    e0 = V.energy(s.ops[0], uh - x)
    for _ in range(6):
        x = s.ir_step(0, bs[0], x)
    assert V.energy(s.ops[0], uh - x) <= 0.6 ** 6 * e0


def test_bfp_ir_fixed_point_and_convergence():
    """Alg. ir with BFP x and b on the variable operator: b = A'x exactly leaves x unchanged;
    from x = 0 the iteration follows the FP64-residual IR (same V-cycle) towards the discrete
    solution of A'u = b' (sparse direct solve) until a floor set by the width of the residual's
    operator (Alg. ir quantises A to the input width): 10 more face bits (26 vs 16) lower the
    floor by about 2^10."""
    n = 31
    K = grf_nodes(n, seed=4)
    s = V.VarSolver(K, w=16, mode="nnqcomp")
    x = B.normalize(B.BFP(random_mantissas((n, n), 12, 8), -20, 12), B.Quant(12, "qcomp"))
    ex = V.apply_exact(V.make_ir_level(K, s.om), x)
    b = B.BFP(np.asarray(ex.z, dtype=np.int64), ex.e, 40)
    xn = s.ir_step_bfp(b, x)
    assert xn.e == x.e and np.array_equal(xn.m, x.m)
    f = smoothed_random_rhs(n, 5)
    op = s.ops[0]
    bp = s.rhs_hierarchy(f)[0]
    uh = V.discrete_solution(op, bp)
    eu = V.energy(op, uh)
    floors = {}
    for w_ir in (26, 16):
        sv = V.VarSolver(K, w=16, mode="nnqcomp", w_ir=w_ir)
        bq = B.from_f64(bp, 32)
        x, xf = B.BFP(np.zeros((n, n), dtype=np.int64), 0, 32), np.zeros((n, n))
        errs, errf = [], []
        for _ in range(30):
            x, xf = sv.ir_step_bfp(bq, x), sv.ir_step(0, bp, xf)
            errs.append(V.energy(op, B.to_f64(x) - uh) / eu)
            errf.append(V.energy(op, xf - uh) / eu)
        floors[w_ir] = errs[-1]
        assert errs[-1] <= 1.1 * min(errs[-5:])                      # settled
        for e, g in zip(errs, errf):
            assert e <= 1.05 * g + 2 * errs[-1]
    assert floors[26] < 5e-6
    assert 2 ** 8 <= floors[16] / floors[26] <= 2 ** 12, floors
