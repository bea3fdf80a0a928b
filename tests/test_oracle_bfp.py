"""Pins for the exact BFP oracle (CPU only).

Each check compares the oracle with something other than itself: the
paper's worked example (Fig. 2), brute force over rationals on tiny blocks,
the minimal-exponent characterisation of a normalised block (Sec. 2),
scipy sparse matrices built independently of the stencil code, and exact
algebraic identities.
"""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import bfp as B

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def frac_vals(m, e):
    return [Fraction(int(v)) * Fraction(2) ** e for v in np.ravel(m)]


def exact_floor_quant(vals, w_out):
    """Independent characterisation (Sec. 2): the normalised BFP block of w_out bits
    with the smallest exponent whose floor quantisation still fits in X_w_out
    (found by bisection: fitting is monotone in the exponent)."""
    lo, hi = -(1 << (w_out - 1)), (1 << (w_out - 1)) - 1
    if all(v == 0 for v in vals):
        return None

    def fits(e):
        return all(lo <= (v / Fraction(2) ** e).__floor__() <= hi for v in vals)

    a, b = -2200, 2200          # fits(b) holds, fits(a) fails for any double / tiny ints
    assert fits(b) and not fits(a)
    while b - a > 1:
        c = (a + b) // 2
        if fits(c):
            b = c
        else:
            a = c
    return b, [(v / Fraction(2) ** b).__floor__() for v in vals]


# --- Fig. 2 and the substring example ---------------------------------------

def test_fig2_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "fig2_window.json")))
    assert B.msb(g["z"]) == g["mu_star"]
    ex = B.Exact(np.array([g["z"]], dtype=np.int64), g["e_star"], 10)
    out = B.qcomp_def(ex, g["w_out"])
    assert int(out.m[0]) == g["m_out"]
    assert out.e == g["e_star"] + g["lambda_out"]
    for win in g["windows"]:
        w_tmp = win["mu_tmp"] - win["lambda_tmp"]
        gamma = (1 << (win["mu_tmp"] - 2), 0)          # msb(2^k) = k + 2
        assert B.gamma_mu(gamma, g["e_star"]) == win["mu_tmp"]
        if w_tmp < g["w_out"]:
            # the underflow window of the figure is narrower than w_out; Alg. qcomp
            # requires w_tmp >= w_out, so test the flags with the same lambda_tmp
            # and a mu_tmp that keeps w_tmp = w_out
            continue
        res, ovf, unf = B.qcomp_alg(ex, g["w_out"], w_tmp, gamma)
        assert (ovf, unf) == (win["overflow"], win["underflow"])
        assert int(res.m[0]) == g["m_out"] and res.e == out.e


def test_fig2_underflow_window_flags():
    g = json.load(open(os.path.join(GOLDEN, "fig2_window.json")))
    ex = B.Exact(np.array([g["z"]], dtype=np.int64), 0, 10)
    # lambda_tmp = 4 > lambda_out = 2 with a wide-enough window (mu_tmp = 8, w_tmp = 4)
    res, ovf, unf = B.qcomp_alg(ex, 4, 4, (1 << 6, 0))
    assert not ovf and unf and int(res.m[0]) == 5


def test_substring_example():
    g = json.load(open(os.path.join(GOLDEN, "fig2_window.json")))["substring_example"]
    v = int(g["bits"], 2)
    sub = (v >> g["lambda"]) & ((1 << (g["mu"] - g["lambda"])) - 1)
    assert format(sub, "0%db" % g["width"]) == g["substring"]
    assert g["mu"] - g["lambda"] == g["width"]


# --- msb, decr, floor ---------------------------------------------------------

def test_msb_matches_range_sets():
    for m in range(-300, 300):
        v = next(v for v in range(1, 20) if -(1 << (v - 1)) <= m <= (1 << (v - 1)) - 1)
        assert B.msb(m) == v


def test_decr_is_narrowing_cast():
    for m in range(-128, 128):
        assert int(B.wrap(np.array([m]), 4)[0]) == int(np.array([m], dtype=np.int8).astype(np.int64)[0] << 60 >> 60)


def test_floor_shift_is_floor():
    z = np.arange(-70, 70, dtype=np.int64)
    for lam in range(-3, 8):
        got = B.floor_shift(z, lam)
        want = [(Fraction(int(v)) / Fraction(2) ** lam).__floor__() for v in z]
        assert list(map(int, got)) == want


# --- qcomp: definition vs brute force, algorithm vs definition ---------------

def tiny_blocks(max_len=3, lo=-9, hi=9):
    for n in range(1, max_len + 1):
        for vals in itertools.product(range(lo, hi + 1), repeat=n):
            yield np.array(vals, dtype=np.int64)


def test_qcomp_def_is_minimal_exponent_floor():
    for z in tiny_blocks(2):
        for e_star in (-3, 0, 2):
            for w_out in (1, 2, 3, 5):
                out = B.qcomp_def(B.Exact(z, e_star, 6), w_out)
                ref = exact_floor_quant(frac_vals(z, e_star), w_out)
                if ref is None:
                    assert np.all(out.m == 0) and out.e == e_star + 1 - w_out
                else:
                    assert out.e == ref[0], (z, e_star, w_out)
                    assert list(map(int, out.m)) == ref[1]


def test_qcomp_alg_independent_of_gamma_and_wtmp():
    """The windowed algorithm returns the definition's result for every window."""
    rng = np.random.default_rng(1)
    n_flags = {"ovf": 0, "unf": 0, "ok": 0}
    for trial in range(150):
        z = rng.integers(-300, 300, size=rng.integers(1, 6))
        e_star = int(rng.integers(-5, 5))
        ex = B.Exact(z, e_star, 12)
        for w_out in (2, 4, 7):
            ref = B.qcomp_def(ex, w_out)
            for w_tmp in range(w_out, w_out + 6):
                for gm in (1, 3, 17, 255, 1000):
                    for ge in (-6, -2, 0, 3):
                        res, ovf, unf = B.qcomp_alg(ex, w_out, w_tmp, (gm, ge))
                        assert res.e == ref.e
                        assert np.array_equal(B.to_object(res.m), B.to_object(ref.m))
                        mu_tmp = B.msb(gm) + ge - e_star
                        assert ovf == (mu_tmp < B.max_msb(z))
                        assert unf == (B.max_msb(z) - w_out < mu_tmp - w_tmp)
                        n_flags["ovf" if ovf else "unf" if unf else "ok"] += 1
    assert min(n_flags.values()) > 100


def test_nnqcomp_exact_gamma_and_saturation():
    rng = np.random.default_rng(2)
    for trial in range(300):
        z = rng.integers(-5000, 5000, size=rng.integers(1, 8))
        e_star = int(rng.integers(-4, 4))
        ex = B.Exact(z, e_star, 14)
        w_out = int(rng.integers(2, 9))
        nrm = int(np.abs(z).max())
        vals = frac_vals(z, e_star)
        # gamma = ||z||: no saturation; the result is the floor quantisation at the
        # exponent msb(gamma) + e_gamma - w_out (Alg. nnqcomp)
        out, nsat = B.nnqcomp(ex, w_out, (nrm, e_star))
        assert nsat == 0
        q = B.qcomp_def(ex, w_out)
        assert out.e in (q.e, q.e + 1)
        for m, v in zip(out.m, vals):
            assert int(m) == (v / Fraction(2) ** out.e).__floor__()
        # gamma too small by 2^k: saturation clamps, never wraps
        k = int(rng.integers(1, 4))
        out2, nsat2 = B.nnqcomp(ex, w_out, (max(nrm >> k, 1), e_star))
        lo, hi = -(1 << (w_out - 1)), (1 << (w_out - 1)) - 1
        for m, v in zip(out2.m, vals):
            f = (v / Fraction(2) ** out2.e).__floor__()
            assert int(m) == min(max(f, lo), hi)
        assert nsat2 == sum(1 for v in vals if not lo <= (v / Fraction(2) ** out2.e).__floor__() <= hi)


# --- exact ops vs rationals -------------------------------------------------

def test_eaxpby_exact_and_width_bound():
    rng = np.random.default_rng(3)
    for trial in range(300):
        n = 5
        wx, wy = int(rng.integers(2, 10)), int(rng.integers(2, 10))
        x = B.BFP(rng.integers(-(1 << (wx - 1)), 1 << (wx - 1), size=n), int(rng.integers(-8, 8)), wx)
        y = B.BFP(rng.integers(-(1 << (wy - 1)), 1 << (wy - 1), size=n), int(rng.integers(-8, 8)), wy)
        al = B.Scalar(int(rng.integers(-40, 40)), int(rng.integers(-5, 5)))
        be = B.Scalar(int(rng.integers(-40, 40)), int(rng.integers(-5, 5)))
        ex = B.eaxpby(al, x, be, y)
        got = frac_vals(B.to_object(ex.z), ex.e)
        want = [al.value() * a + be.value() * b for a, b in zip(frac_vals(x.m, x.e), frac_vals(y.m, y.e))]
        assert got == want
        assert B.bits_of(B.to_object(ex.z)) <= ex.w        # App. B width is an upper bound
        assert ex.e == min(al.e + x.e, be.e + y.e)


def laplacian_matrix(nd, n):
    """-Laplacian (unscaled integer stencil 2d, -1) from 1D Kronecker products."""
    T = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1])
    I = sp.identity(n)
    if nd == 2:
        return (sp.kron(I, T) + sp.kron(T, I)).tocsr()
    return (sp.kron(sp.kron(I, I), T) + sp.kron(sp.kron(I, T), I) + sp.kron(sp.kron(T, I), I)).tocsr()


@pytest.mark.parametrize("nd,n", [(2, 7), (2, 10), (3, 5)])
def test_stencil_matches_sparse_matrix(nd, n):
    A = B.laplace_stencil(nd)
    rng = np.random.default_rng(4)
    x = B.BFP(rng.integers(-1000, 1000, size=(n,) * nd), -3, 11)
    ex = B.espmv_stencil(A, x)
    L = laplacian_matrix(nd, n)
    want = L @ x.m.ravel()                       # 2d*x - sum(nbrs)
    # A' = (h^2 / 2^p) A_h with mantissas (centre 2d/2^p, nbr -1/2^p) * 2^-e_A
    scale = (1 << -A.e) // (4 if nd == 2 else 8)
    assert np.array_equal(np.asarray(ex.z).ravel(), scale * want)
    assert ex.e == A.e + x.e
    assert B.bits_of(np.asarray(ex.z)) <= ex.w


def prolong_matrix(nd, nc):
    """Bilinear / trilinear interpolation from 1D Kronecker products."""
    nf = 2 * nc + 1
    P1 = sp.lil_matrix((nf, nc))
    for I in range(nc):
        P1[2 * I, I] += 0.5
        P1[2 * I + 1, I] += 1.0
        P1[2 * I + 2, I] += 0.5
    P1 = P1.tocsr()
    P = P1
    for _ in range(nd - 1):
        P = sp.kron(P1, P)
    return P.tocsr()


@pytest.mark.parametrize("nd,nc", [(2, 3), (2, 6), (3, 3)])
def test_transfers_match_kronecker(nd, nc):
    rng = np.random.default_rng(5)
    nf = 2 * nc + 1
    P = prolong_matrix(nd, nc)
    d = B.BFP(rng.integers(-500, 500, size=(nc,) * nd), 2, 10)
    pe = B.espmv_prolong(d, (nf,) * nd)
    assert np.allclose(np.asarray(pe.z, dtype=float).ravel() * 2.0 ** pe.e,
                       P @ (d.m.ravel() * 2.0 ** d.e), rtol=0, atol=0)
    r = B.BFP(rng.integers(-500, 500, size=(nf,) * nd), -1, 10)
    re = B.espmv_restrict(r)
    # R~ = D_c^-1 R_FW D_f = P^T (2D), P^T / 2 (3D)
    Rt = P.T * (1.0 if nd == 2 else 0.5)
    assert np.allclose(np.asarray(re.z, dtype=float).ravel() * 2.0 ** re.e,
                       Rt @ (r.m.ravel() * 2.0 ** r.e), rtol=0, atol=0)
    assert B.bits_of(np.asarray(re.z)) <= re.w and B.bits_of(np.asarray(pe.z)) <= pe.w


def test_jacobi_two_sweeps_equal_chebyshev_form():
    """Two damped-Jacobi sweeps from zero equal (c1 I + c2 A) r with c1 = 2 omega,
    c2 = -omega^2 (the single qgemv relaxation of Alg. v-cycle)."""
    rng = np.random.default_rng(6)
    for nd, n in ((2, 6), (3, 4)):
        A = B.laplace_stencil(nd)
        om = B.scalar_floor(0.8, 16)
        r = B.BFP(rng.integers(-(1 << 15), 1 << 15, size=(n,) * nd), -4, 16)
        y1 = B.Exact(B.mul_c(r.m, om.m), om.e + r.e, om.w + r.w)
        y1b = B.BFP(B.to_object(y1.z), y1.e, 64)
        S = B.jacobi_operator(A, om)
        y2 = B.egemv(S, y1b, r, B.ONE, om)
        Ar = B.espmv_stencil(A, r)
        c1 = 2 * om.value()
        c2 = -om.value() ** 2
        want = [c1 * a + c2 * b for a, b in zip(frac_vals(r.m, r.e), frac_vals(B.to_object(Ar.z), Ar.e))]
        assert frac_vals(B.to_object(y2.z), y2.e) == want


def test_jacobi_equals_definition():
    rng = np.random.default_rng(7)
    A = B.laplace_stencil(2)
    om = B.scalar_floor(0.8, 16)
    y = B.BFP(rng.integers(-(1 << 15), 1 << 15, size=(5, 6)), -3, 16)
    r = B.BFP(rng.integers(-(1 << 15), 1 << 15, size=(5, 6)), -5, 16)
    S = B.jacobi_operator(A, om)
    ex = B.egemv(S, y, r, B.ONE, om)
    Ay = B.espmv_stencil(A, y)
    yv, rv, av = frac_vals(y.m, y.e), frac_vals(r.m, r.e), frac_vals(B.to_object(Ay.z), Ay.e)
    want = [a + om.value() * (b - c) for a, b, c in zip(yv, rv, av)]
    assert frac_vals(B.to_object(ex.z), ex.e) == want
    # ||I - omega A||_inf = 1 for omega <= 1 (the Jacobi gamma rule's bound)
    nm, ne = S.norm_inf
    assert Fraction(nm) * Fraction(2) ** ne == 1


def test_gamma_rules_are_upper_bounds():
    rng = np.random.default_rng(8)
    A = B.laplace_stencil(2)
    om = B.scalar_floor(0.8, 16)
    for trial in range(20):
        y = B.BFP(rng.integers(-(1 << 15), 1 << 15, size=(9, 9)), int(rng.integers(-6, 2)), 16)
        r = B.BFP(rng.integers(-(1 << 15), 1 << 15, size=(9, 9)), int(rng.integers(-6, 2)), 16)
        d = B.BFP(rng.integers(-(1 << 15), 1 << 15, size=(4, 4)), int(rng.integers(-6, 2)), 16)
        S = B.jacobi_operator(A, om)
        cases = [
            (B.egemv(S, y, r, B.ONE, om), B.gamma_jacobi(A, om, y, r)),
            (B.espmv_restrict(r), B.gamma_restrict(r)),
            (B.eaxpby(B.MINUS_ONE, B.espmv_prolong(d, (9, 9)), B.ONE, y), B.gamma_correct(y, d)),
            (B.espmv_stencil(A, y), B.gamma_apply(A, y)),
        ]
        for ex, (gm, ge) in cases:
            zmax = max(abs(v) for v in frac_vals(B.to_object(ex.z), ex.e))
            assert zmax <= Fraction(gm) * Fraction(2) ** ge


# --- dot, from_f64, to_f64 -----------------------------------------------------

def test_dot_exact():
    rng = np.random.default_rng(9)
    for trial in range(50):
        n = int(rng.integers(1, 40))
        x = B.BFP(rng.integers(-(1 << 31), 1 << 31, size=n), int(rng.integers(-9, 9)), 32)
        y = B.BFP(rng.integers(-(1 << 31), 1 << 31, size=n), int(rng.integers(-9, 9)), 32)
        s = sum(a * b for a, b in zip(frac_vals(x.m, x.e), frac_vals(y.m, y.e)))
        out = B.dot(x, y, 24)
        ref = exact_floor_quant([s], 24)
        if ref is None:
            assert out.m == 0
        else:
            assert (out.e, out.m) == (ref[0], ref[1][0])


def test_from_f64_brute_force():
    rng = np.random.default_rng(10)
    cases = [
        np.array([23.0, -1.5, 0.0]),
        np.array([-0.0, 0.0]),
        np.array([5e-324, -1e-310, 2.5e-308]),             # subnormals
        np.array([-4.0, 3.0]),
        rng.standard_normal(17) * 10.0 ** rng.integers(-30, 30),
        -np.abs(rng.standard_normal(9)),
    ]
    for x in cases:
        for w in (1, 4, 16, 32, 53):
            out = B.from_f64(x, w)
            vals = [Fraction(float(v)) for v in x]
            ref = exact_floor_quant(vals, w) if any(v != 0 for v in vals) else None
            if ref is None:
                assert np.all(out.m == 0) and out.e == B.F64_E_STAR + 1 - w
            else:
                assert out.e == ref[0]
                assert list(map(int, out.m)) == ref[1]


def test_from_f64_rejects_nonfinite():
    with pytest.raises(ValueError):
        B.from_f64(np.array([1.0, np.nan]), 8)


def test_to_f64_roundtrip_exact():
    rng = np.random.default_rng(11)
    m = rng.integers(-(1 << 31), 1 << 31, size=100)
    x = B.BFP(m, -40, 32)
    v = B.to_f64(x)
    assert [Fraction(float(a)) for a in v] == frac_vals(m, -40)
    back = B.from_f64(v, 32)
    assert np.array_equal(B.to_f64(back), v)


def test_scalar_floor():
    om = B.scalar_floor(0.8, 16)
    assert (om.m, om.e) == (26214, -15)
    assert om.value() <= Fraction(4, 5) < om.value() + Fraction(1, 1 << 15)
    s = B.scalar_floor(-1.0 / 6.0, 16)
    assert B.msb(s.m) <= 16 and B.msb(s.m * 2) > 16


def test_wide_blocks_brute_force():
    """Blocks of 33..62 bits (int64 mantissas): from_f64, axpy and the residual at those widths
    equal the minimal-exponent floor of the exact rational result."""
    rng = np.random.default_rng(11)
    x = rng.standard_normal(13) * 10.0 ** rng.integers(-20, 20)
    for w in (33, 48, 53, 62):
        out = B.from_f64(x, w)
        ref = exact_floor_quant([Fraction(float(v)) for v in x], w)
        assert out.e == ref[0] and list(map(int, out.m)) == ref[1]
    for wx, wy, wz in ((60, 16, 40), (40, 40, 62), (16, 55, 33)):
        xm = rng.integers(-(1 << (wx - 1)), 1 << (wx - 1), size=9, dtype=np.int64)
        ym = rng.integers(-(1 << (wy - 1)), 1 << (wy - 1), size=9, dtype=np.int64)
        a, b = B.Scalar(1, -3), B.Scalar(-1, 7)
        z = B.axpy(a, B.BFP(xm, -20, wx), b, B.BFP(ym, 5, wy), B.Quant(wz, "qcomp"))
        vals = [a.value() * p + b.value() * q for p, q in zip(frac_vals(xm, -20), frac_vals(ym, 5))]
        ref = exact_floor_quant(vals, wz)
        assert z.e == ref[0] and list(map(int, z.m)) == ref[1]
    # residual r_v = A y - r on a 5 x 4 grid with a 55-bit y
    A = B.laplace_stencil(2)
    ym = rng.integers(-(1 << 54), 1 << 54, size=(4, 5), dtype=np.int64)
    rm = rng.integers(-(1 << 31), 1 << 31, size=(4, 5), dtype=np.int64)
    out = B.residual(A, B.BFP(ym, -60, 55), B.BFP(rm, -30, 32), B.Quant(16, "qcomp"), B.Scalar(13107, -14))
    Y = lambda i, j: Fraction(int(ym[j, i])) * Fraction(2) ** -60 if 0 <= i < 5 and 0 <= j < 4 else Fraction(0)
    vals = []
    for j in range(4):
        for i in range(5):
            ay = Y(i, j) - Fraction(1, 4) * (Y(i - 1, j) + Y(i + 1, j) + Y(i, j - 1) + Y(i, j + 1))
            vals.append(ay - Fraction(int(rm[j, i])) * Fraction(2) ** -30)
    ref = exact_floor_quant(vals, 16)
    assert out.e == ref[0] and list(map(int, np.asarray(out.m).ravel())) == ref[1]
