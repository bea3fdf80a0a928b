"""Parity of every BFP op (CUDA path through the C ABI) with the exact oracle.

Bit-exact: mantissas, exponent, the max-norm word, and the qcomp
overflow / underflow / recompute and nnqcomp saturation counters.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2307_00124_gb300 as bfp  # noqa: E402
from bfp_inputs import random_mantissas  # noqa: E402
from oracle import bfp as B  # noqa: E402

pytestmark = pytest.mark.gpu


def dev_vec(m, e, w, junk_seed=None):
    v = bfp.BFPVector.from_mantissas(m, e, w)
    if junk_seed is not None and v.ld > m.shape[-1]:
        # garbage in the padding columns must be ignored by every op
        g = torch.randint(-(1 << (min(w, 16) - 1)), 1 << (min(w, 16) - 1), v.mant[:, m.shape[-1]:].shape,
                          generator=torch.Generator().manual_seed(junk_seed)).to(v.mant.dtype)
        v.mant[:, m.shape[-1]:] = g.cuda()
    return v


def out_vec(shape, w):
    v = bfp.BFPVector(shape, w)
    v.mant.fill_(7)          # stale contents must be overwritten
    v.meta.fill_(123)
    return v


def stats_tensor():
    return torch.zeros(8, dtype=torch.uint64 if hasattr(torch, "uint64") else torch.int64, device="cuda")


def read_stats(t):
    h = t.cpu().numpy().astype(np.int64)
    return dict(calls=int(h[0]), recomputed=int(h[1]), overflow=int(h[2]), underflow=int(h[3]),
                saturated=int(h[4]))


def check(out, ref: B.BFP, st=None, ref_st: B.Stats = None):
    torch.cuda.synchronize()
    got = out.mantissas()
    want = np.asarray(ref.m).astype(np.int64)
    assert got.shape == want.shape
    bad = np.argwhere(got != want)
    assert bad.size == 0, "first mismatch at %s: got %d want %d (e %d vs %d)" % (
        tuple(bad[0]), got[tuple(bad[0])], want[tuple(bad[0])], out.exponent, ref.e)
    assert out.exponent == ref.e
    assert out.norm_m == ref.norm_m
    assert np.all(out.padding() == 0)
    if st is not None:
        s = read_stats(st)
        assert s["calls"] == ref_st.calls
        assert (s["recomputed"], s["overflow"], s["underflow"], s["saturated"]) == (
            ref_st.recomputed, ref_st.overflow, ref_st.underflow, ref_st.saturated), (s, ref_st)


def oq(w_out, mode, gamma=None, w_add=None):
    return B.Quant(w_out, "qcomp" if mode == bfp.QCOMP else "nnqcomp", w_add, gamma)


def gq(w_out, mode, gamma=None, w_add=-1, tmp=None):
    return bfp.q(w_out, mode, w_add, gamma, tmp)


MODES = [bfp.QCOMP, bfp.NNQCOMP]
WIDTHS = [4, 8, 12, 16, 24, 32]


# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(1000,), (37, 53), (5, 7, 9), (1, 1), (0,)])
@pytest.mark.parametrize("w_in,w_out", [(16, 8), (8, 16), (32, 12), (12, 32), (24, 24), (4, 4)])
@pytest.mark.parametrize("mode", MODES)
def test_normalize(shape, w_in, w_out, mode):
    seed = hash((shape, w_in, w_out, mode)) % 1000
    m = random_mantissas(shape, w_in, seed)
    x = dev_vec(m, -7, w_in, junk_seed=seed)
    z = out_vec(shape, w_out)
    st = stats_tensor()
    tmp = torch.zeros((z.rows, z.ld), dtype=torch.int32, device="cuda")
    bfp.bfp_normalize(x, z, gq(w_out, mode, tmp=tmp), st)
    rs = B.Stats()
    ref = B.normalize(B.BFP(m, -7, w_in), oq(w_out, mode), rs)
    check(z, ref, st, rs)


@pytest.mark.parametrize("ea,eb", [(0, 0), (-3, 5), (40, -30), (100, 0), (-7, 200), (0, -70)])
@pytest.mark.parametrize("w", [8, 16, 32])
@pytest.mark.parametrize("mode", MODES)
def test_axpy(ea, eb, w, mode):
    rng = np.random.default_rng(abs(ea * 31 + eb) + w)
    shape = (13, 29)
    xm = random_mantissas(shape, w, 1)
    ym = random_mantissas(shape, w, 2)
    a = B.Scalar(int(rng.integers(-(1 << 14), 1 << 14)), ea)
    b = B.Scalar(int(rng.integers(-(1 << 14), 1 << 14)), eb)
    x, y = dev_vec(xm, -3, w, 5), dev_vec(ym, 2, w, 6)
    z = out_vec(shape, w)
    st = stats_tensor()
    bfp.bfp_axpy(bfp.scalar(a.m, a.e), x, bfp.scalar(b.m, b.e), y, z, gq(w, mode), st)
    rs = B.Stats()
    ref = B.axpy(a, B.BFP(xm, -3, w), b, B.BFP(ym, 2, w), oq(w, mode), rs)
    check(z, ref, st, rs)


def test_axpy_zero_top_group_far_exponent():
    """x = 0 with an exponent 150 above y: the guarded combine must fall back to y exactly."""
    shape = (9, 16)
    xm = np.zeros(shape, dtype=np.int64)
    ym = random_mantissas(shape, 16, 3)
    for mode in MODES:
        x, y = dev_vec(xm, 150, 16), dev_vec(ym, 0, 16)
        z = out_vec(shape, 16)
        st = stats_tensor()
        bfp.bfp_axpy(bfp.scalar(3, 0), x, bfp.scalar(-5, 0), y, z, gq(16, mode), st)
        rs = B.Stats()
        ref = B.axpy(B.Scalar(3, 0), B.BFP(xm, 150, 16), B.Scalar(-5, 0), B.BFP(ym, 0, 16), oq(16, mode), rs)
        check(z, ref, st, rs)


# ---------------------------------------------------------------------------

def lap(nd, w_omega=16):
    A = bfp.bfp_laplace_stencil(nd, 0.8 if nd == 2 else 6 / 7, w_omega)
    OA = B.Stencil(nd, A.center, A.nbr, A.e)
    om = B.Scalar(A.omega.m, A.omega.e)
    return A, OA, om


def test_laplace_stencil_matches_oracle():
    from oracle import mg
    for nd in (2, 3):
        A, OA, om = lap(nd)
        assert OA == B.laplace_stencil(nd)
        ref = B.scalar_floor(mg.omega_scaled(nd, 0.8 if nd == 2 else 6 / 7), 16)
        assert (om.m, om.e) == (ref.m, ref.e)


# 3D: several strips of rows per plane, two column chunks, ragged tails in x and y
STAR_SHAPES = [(37, 45), (1, 1), (2, 3), (63, 63), (70, 300), (5, 6, 7), (3, 3, 3), (9, 70, 300), (3, 260, 17)]


@pytest.mark.parametrize("shape", STAR_SHAPES)
@pytest.mark.parametrize("w", WIDTHS)
@pytest.mark.parametrize("mode", MODES)
def test_stencil_apply(shape, w, mode):
    nd = len(shape)
    A, OA, om = lap(nd)
    xm = random_mantissas(shape, w, w + len(shape))
    x = dev_vec(xm, -4, w, junk_seed=1)
    z = out_vec(shape, w)
    st = stats_tensor()
    bfp.bfp_stencil_apply(A, x, z, gq(w, mode), st)
    rs = B.Stats()
    ref = B.stencil_apply(OA, B.BFP(xm, -4, w), oq(w, mode), rs)
    check(z, ref, st, rs)


@pytest.mark.parametrize("shape", STAR_SHAPES)
@pytest.mark.parametrize("w", WIDTHS)
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("ey,er", [(-5, -3), (10, -60), (-90, 20)])
def test_residual(shape, w, mode, ey, er):
    nd = len(shape)
    A, OA, om = lap(nd)
    ym = random_mantissas(shape, w, 11, "smooth")
    rm = random_mantissas(shape, w, 12)
    y, r = dev_vec(ym, ey, w, 2), dev_vec(rm, er, w, 3)
    rv = out_vec(shape, w)
    st = stats_tensor()
    bfp.bfp_residual(A, y, r, rv, gq(w, mode), st)
    rs = B.Stats()
    ref = B.residual(OA, B.BFP(ym, ey, w), B.BFP(rm, er, w), oq(w, mode), om, rs)
    check(rv, ref, st, rs)


@pytest.mark.parametrize("shape", STAR_SHAPES)
@pytest.mark.parametrize("w", WIDTHS)
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("zero_guess", [False, True])
def test_jacobi(shape, w, mode, zero_guess):
    nd = len(shape)
    A, OA, om = lap(nd)
    ym = random_mantissas(shape, w, 21)
    rm = random_mantissas(shape, w, 22, "smooth")
    y, r = dev_vec(ym, -9, w, 4), dev_vec(rm, -8, w, 5)
    yo = out_vec(shape, w)
    st = stats_tensor()
    bfp.bfp_jacobi(A, None if zero_guess else y, r, yo, gq(w, mode), st)
    rs = B.Stats()
    ref = B.jacobi(OA, om, None if zero_guess else B.BFP(ym, -9, w), B.BFP(rm, -8, w), oq(w, mode), rs)
    check(yo, ref, st, rs)


# coarse shapes; (70, 300) and the 3D ones span several strips of rows and column chunks of the fine grid
TRANSFER_SHAPES = [(1, 1), (3, 3), (20, 33), (70, 300), (2, 2, 2), (4, 3, 5), (5, 40, 140), (3, 70, 9), (0, 0),
                   (0, 0, 0)]


@pytest.mark.parametrize("nc", TRANSFER_SHAPES)
@pytest.mark.parametrize("w", [8, 16, 24, 27, 32])   # int32 fine mantissas of <= 27 bits take the staged kernel
@pytest.mark.parametrize("mode", MODES)
def test_restrict(nc, w, mode):
    nf = tuple(2 * c + 1 for c in nc)
    fm = random_mantissas(nf, w, 31)
    f = dev_vec(fm, 3, w, 6)
    c = out_vec(nc, w)
    st = stats_tensor()
    bfp.bfp_restrict(f, c, gq(w, mode), st)
    rs = B.Stats()
    ref = B.restrict(B.BFP(fm, 3, w), oq(w, mode), rs)
    check(c, ref, st, rs)


@pytest.mark.parametrize("nc", TRANSFER_SHAPES)
@pytest.mark.parametrize("w", [8, 16, 24, 29, 32])   # int32 coarse mantissas of <= 29 bits take the staged kernel
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("correct", [True, False])
def test_prolong(nc, w, mode, correct):
    nf = tuple(2 * c + 1 for c in nc)
    dm = random_mantissas(nc, w, 41)
    ym = random_mantissas(nf, w, 42)
    d, y = dev_vec(dm, -2, w, 7), dev_vec(ym, -1, w, 8)
    out = out_vec(nf, w)
    st = stats_tensor()
    bfp.bfp_prolong(d, y if correct else None, out, gq(w, mode), st)
    rs = B.Stats()
    ref = B.prolong(B.BFP(dm, -2, w), B.BFP(ym, -1, w) if correct else None, nf, oq(w, mode), rs)
    check(out, ref, st, rs)


# ---- forced windows and saturation ---------------------------------------------

@pytest.mark.parametrize("gshift", [-12, -3, 0, 2, 9])
@pytest.mark.parametrize("w_add", [0, 2, 6])
@pytest.mark.parametrize("shape", [(33, 40), (6, 33, 270)])
def test_qcomp_forced_overflow_underflow(gshift, w_add, shape):
    """A gamma too small forces overflow, too large forces underflow; the result never changes."""
    A, OA, om = lap(len(shape))
    ym = random_mantissas(shape, 16, 51)
    rm = random_mantissas(shape, 16, 52)
    gamma = (1, 10 + gshift)
    for use_tmp in (False, True):
        y, r = dev_vec(ym, 0, 16), dev_vec(rm, 0, 16)
        yo = out_vec(shape, 16)
        tmp = torch.zeros((yo.rows, yo.ld), dtype=torch.int32, device="cuda") if use_tmp else None
        st = stats_tensor()
        bfp.bfp_jacobi(A, y, r, yo, gq(16, bfp.QCOMP, gamma, w_add, tmp), st)
        rs = B.Stats()
        ref = B.jacobi(OA, om, B.BFP(ym, 0, 16), B.BFP(rm, 0, 16), B.Quant(16, "qcomp", w_add, gamma), rs)
        check(yo, ref, st, rs)


@pytest.mark.parametrize("gshift", [-20, -4, -1, 0, 3])
@pytest.mark.parametrize("shape", [(31, 31), (7, 31, 290)])
def test_nnqcomp_saturation(gshift, shape):
    A, OA, om = lap(len(shape))
    ym = random_mantissas(shape, 16, 61)
    rm = random_mantissas(shape, 16, 62)
    gamma = (1, 14 + gshift)
    y, r = dev_vec(ym, 0, 16), dev_vec(rm, 0, 16)
    rv = out_vec(shape, 12)
    st = stats_tensor()
    bfp.bfp_residual(A, y, r, rv, gq(12, bfp.NNQCOMP, gamma), st)
    rs = B.Stats()
    ref = B.residual(OA, B.BFP(ym, 0, 16), B.BFP(rm, 0, 16), B.Quant(12, "nnqcomp", None, gamma), om, rs)
    check(rv, ref, st, rs)


@pytest.mark.parametrize("mode", MODES)
def test_zero_vectors(mode):
    shape = (17, 19)
    A, OA, om = lap(2)
    zm = np.zeros(shape, dtype=np.int64)
    for op in ("apply", "jacobi", "residual"):
        x, r = dev_vec(zm, 5, 16), dev_vec(zm, -3, 16)
        out = out_vec(shape, 16)
        st = stats_tensor()
        rs = B.Stats()
        if op == "apply":
            bfp.bfp_stencil_apply(A, x, out, gq(16, mode), st)
            ref = B.stencil_apply(OA, B.BFP(zm, 5, 16), oq(16, mode), rs)
        elif op == "jacobi":
            bfp.bfp_jacobi(A, x, r, out, gq(16, mode), st)
            ref = B.jacobi(OA, om, B.BFP(zm, 5, 16), B.BFP(zm, -3, 16), oq(16, mode), rs)
        else:
            bfp.bfp_residual(A, x, r, out, gq(16, mode), st)
            ref = B.residual(OA, B.BFP(zm, 5, 16), B.BFP(zm, -3, 16), oq(16, mode), om, rs)
        check(out, ref, st, rs)


# ---- dot and FP64 conversion -----------------------------------------------------

@pytest.mark.parametrize("w", [4, 16, 32])
@pytest.mark.parametrize("n", [1, 777, 100000])
def test_dot(w, n):
    xm = random_mantissas((n,), w, 71)
    ym = random_mantissas((n,), w, 72)
    x, y = dev_vec(xm, -5, w, 9), dev_vec(ym, 7, w, 10)
    out = torch.zeros(8, dtype=torch.int64, device="cuda")
    for w_out in (8, 31, 62):
        bfp.bfp_dot(x, y, w_out, out)
        ref = B.dot(B.BFP(xm, -5, w), B.BFP(ym, 7, w), w_out)
        h = out.cpu().numpy()
        assert (int(h[0]), int(h[1])) == (ref.m, ref.e)


@pytest.mark.parametrize("w", [1, 4, 16, 24, 32])
def test_from_to_f64(w):
    rng = np.random.default_rng(w)
    cases = [rng.standard_normal((21, 30)) * 1e-3,
             np.zeros((4, 9)),
             np.array([[5e-324, -1e-310, 2.5e-308, 0.0, -0.0, 1e300, -3.0, 23.0]]),
             -np.abs(rng.standard_normal((3, 4, 17)))]
    for xv in cases:
        xt = torch.from_numpy(np.ascontiguousarray(xv)).cuda()
        out = out_vec(xv.shape, w)
        bfp.bfp_from_f64(xt, out)
        ref = B.from_f64(xv, w)
        check(out, ref)
        back = torch.empty_like(xt)
        bfp.bfp_to_f64(out, back)
        torch.cuda.synchronize()
        assert np.array_equal(back.cpu().numpy(), B.to_f64(ref))


def test_from_f64_nonfinite_flag():
    xt = torch.tensor([[1.0, float("nan"), 2.0]], dtype=torch.float64, device="cuda")
    out = out_vec((1, 3), 16)
    bfp.bfp_from_f64(xt, out)
    torch.cuda.synchronize()
    assert int(out.meta[3].item()) & 1


# ---- argument errors are synchronous --------------------------------------------

def test_shape_and_alias_errors():
    A, _, _ = lap(2)
    x = bfp.BFPVector((8, 8), 16)
    z = bfp.BFPVector((8, 9), 16)
    with pytest.raises(bfp.BFPError):
        bfp.bfp_stencil_apply(A, x, z, gq(16, bfp.QCOMP))
    with pytest.raises(bfp.BFPError):
        bfp.bfp_stencil_apply(A, x, x, gq(16, bfp.QCOMP))
    with pytest.raises(bfp.BFPError):
        bfp.bfp_stencil_apply(A, x, bfp.BFPVector((8, 8), 16), gq(12, bfp.QCOMP))


# ---- full-size workload, sampled ----------------------------------------------------

@pytest.mark.parametrize("mode", MODES)
def test_full_size_jacobi_and_residual_4095(mode):
    """The 4095^2 finest level at w = 16 (the launch shape the bench times), compared in full."""
    n = 4095
    A, OA, om = lap(2)
    ym = random_mantissas((n, n), 16, 81, "smooth") // 3 + random_mantissas((n, n), 16, 83) // 5
    rm = random_mantissas((n, n), 16, 82)
    y, r = dev_vec(ym, -20, 16), dev_vec(rm, -19, 16)
    yo = out_vec((n, n), 16)
    bfp.bfp_jacobi(A, y, r, yo, gq(16, mode))
    ref = B.jacobi(OA, om, B.BFP(ym, -20, 16), B.BFP(rm, -19, 16), oq(16, mode))
    check(yo, ref)
    rv = out_vec((n, n), 16)
    bfp.bfp_residual(A, y, r, rv, gq(16, mode))
    ref = B.residual(OA, B.BFP(ym, -20, 16), B.BFP(rm, -19, 16), oq(16, mode), om)
    check(rv, ref)


# ---- int64 mantissas (33 <= w <= 62): normalise, from / to FP64, axpy, residual ----

WIDE = [(40, 16), (16, 48), (62, 62), (48, 33), (33, 40), (24, 56)]


@pytest.mark.parametrize("shape", [(37, 53), (5, 7, 9), (1000,)])
@pytest.mark.parametrize("w_in,w_out", WIDE)
@pytest.mark.parametrize("mode", MODES)
def test_wide_normalize(shape, w_in, w_out, mode):
    seed = hash((shape, w_in, w_out, mode)) % 1000
    m = random_mantissas(shape, w_in, seed)
    x = dev_vec(m, -7, w_in)
    z = out_vec(shape, w_out)
    st = stats_tensor()
    bfp.bfp_normalize(x, z, gq(w_out, mode), st)
    rs = B.Stats()
    check(z, B.normalize(B.BFP(m, -7, w_in), oq(w_out, mode), rs), st, rs)


@pytest.mark.parametrize("w", [33, 40, 53, 62])
def test_wide_from_to_f64(w):
    rng = np.random.default_rng(w)
    x = rng.standard_normal((19, 45)) * np.exp(rng.uniform(-30, 30, (19, 45)))
    xt = torch.from_numpy(x).cuda()
    z = out_vec((19, 45), w)
    bfp.bfp_from_f64(xt, z)
    check(z, B.from_f64(x, w))
    back = torch.empty_like(xt)
    bfp.bfp_to_f64(z, back)
    torch.cuda.synchronize()
    assert np.array_equal(back.cpu().numpy(), B.to_f64(B.from_f64(x, w)))


@pytest.mark.parametrize("wx,wy,wz", [(40, 16, 40), (60, 32, 16), (16, 16, 48), (48, 48, 48), (32, 60, 24)])
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("ea,eb", [(0, 0), (-3, 25), (40, -30)])
def test_wide_axpy(wx, wy, wz, mode, ea, eb):
    seed = hash((wx, wy, wz, mode, ea, eb)) % 1000
    xm = random_mantissas((21, 70), wx, seed)
    ym = random_mantissas((21, 70), wy, seed + 1)
    a, b = B.Scalar(1 if wx > 58 else 3, ea), B.Scalar(-1, eb)   # msb(a) + w_x <= 62
    x, y = dev_vec(xm, -3, wx), dev_vec(ym, 2, wy)
    z = out_vec((21, 70), wz)
    st = stats_tensor()
    rs = B.Stats()
    ref = B.axpy(a, B.BFP(xm, -3, wx), b, B.BFP(ym, 2, wy), oq(wz, mode), rs)
    bfp.bfp_axpy(bfp.scalar(a.m, a.e), x, bfp.scalar(b.m, b.e), y, z, gq(wz, mode), st)
    check(z, ref, st, rs)


@pytest.mark.parametrize("shape", [(37, 45), (63, 63), (5, 6, 7), (3, 260, 17)])
@pytest.mark.parametrize("wy,wr", [(40, 40), (55, 32), (48, 16), (16, 32), (24, 44)])
@pytest.mark.parametrize("mode", MODES)
def test_wide_residual(shape, wy, wr, mode):
    nd = len(shape)
    A = bfp.bfp_laplace_stencil(nd, 0.8 if nd == 2 else 6 / 7, 16)
    seed = hash((shape, wy, wr, mode)) % 1000
    ym = random_mantissas(shape, wy, seed, "smooth")
    rm = random_mantissas(shape, wr, seed + 1)
    y, r = dev_vec(ym, -40, wy), dev_vec(rm, -20, wr)
    z = out_vec(shape, 16)
    st = stats_tensor()
    rs = B.Stats()
    As = B.laplace_stencil(nd)
    om = B.Scalar(A.omega.m, A.omega.e)
    ref = B.residual(As, B.BFP(ym, -40, wy), B.BFP(rm, -20, wr), oq(16, mode), om, rs)
    bfp.bfp_residual(A, y, r, z, gq(16, mode), st)
    check(z, ref, st, rs)


def test_wide_rejected_elsewhere():
    A = bfp.bfp_laplace_stencil(2, 0.8, 16)
    x = bfp.BFPVector((15, 15), 40)
    z = bfp.BFPVector((15, 15), 16)
    with pytest.raises(bfp.BFPError):
        bfp.bfp_stencil_apply(A, x, z, gq(16, bfp.QCOMP))
    with pytest.raises(bfp.BFPError):
        bfp.bfp_jacobi(A, None, x, z, gq(16, bfp.QCOMP))
    y = bfp.BFPVector((15, 15), 56)     # A y would pass 62 bits: 4 + 56 + 3
    with pytest.raises(bfp.BFPError):
        bfp.bfp_residual(A, y, z, bfp.BFPVector((15, 15), 16), gq(16, bfp.QCOMP))
    x62 = bfp.BFPVector((15, 15), 62)   # 3 x would pass 62 bits
    with pytest.raises(bfp.BFPError):
        bfp.bfp_axpy(bfp.scalar(3, 0), x62, bfp.scalar(1, 0), z, bfp.BFPVector((15, 15), 40), gq(40, bfp.QCOMP))


# ---- mixed int16 / int32 operands (progressive widths across the 16-bit boundary) ----

@pytest.mark.parametrize("shape", [(37, 45), (63, 63), (5, 6, 7), (3, 260, 17)])
@pytest.mark.parametrize("wy,wr,wo", [(16, 24, 16), (24, 12, 24), (17, 16, 17), (12, 32, 12)])
@pytest.mark.parametrize("mode", MODES)
def test_mixed_jacobi(shape, wy, wr, wo, mode):
    nd = len(shape)
    omega = 0.8 if nd == 2 else 6 / 7
    A = bfp.bfp_laplace_stencil(nd, omega, 16)
    om = B.Scalar(A.omega.m, A.omega.e)
    seed = hash((shape, wy, wr, wo, mode)) % 1000
    ym = random_mantissas(shape, wy, seed, "smooth")
    rm = random_mantissas(shape, wr, seed + 1)
    y, r = dev_vec(ym, -9, wy, seed), dev_vec(rm, -12, wr, seed + 2)
    z = out_vec(shape, wo)
    st = stats_tensor()
    bfp.bfp_jacobi(A, y, r, z, gq(wo, mode), st)
    rs = B.Stats()
    check(z, B.jacobi(B.laplace_stencil(nd), om, B.BFP(ym, -9, wy), B.BFP(rm, -12, wr), oq(wo, mode), rs), st, rs)


@pytest.mark.parametrize("cshape", [(15, 15), (31, 7), (3, 7, 5)])
@pytest.mark.parametrize("wd,wy", [(12, 24), (24, 16), (16, 17)])
@pytest.mark.parametrize("mode", MODES)
def test_mixed_prolong(cshape, wd, wy, mode):
    fshape = tuple(2 * c + 1 for c in cshape)
    seed = hash((cshape, wd, wy, mode)) % 1000
    dm = random_mantissas(cshape, wd, seed, "smooth")
    ym = random_mantissas(fshape, wy, seed + 1, "smooth")
    d, y = dev_vec(dm, -14, wd, seed), dev_vec(ym, -13, wy, seed + 3)
    z = out_vec(fshape, wy)
    st = stats_tensor()
    bfp.bfp_prolong(d, y, z, gq(wy, mode), st)
    rs = B.Stats()
    check(z, B.prolong(B.BFP(dm, -14, wd), B.BFP(ym, -13, wy), fshape, oq(wy, mode), rs), st, rs)
