"""The paper's V(1,0) with the Chebyshev relaxation on the GPU against the oracle, bit for bit:
bfp_cheby (two Chebyshev steps in one qgemv) on 2D / 3D shapes and widths, the V(1,0) cycle
(global levels, the on-chip coarse cycle, progressive widths), FMG + IR; argument checks."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2307_00124_gb300 as bfp  # noqa: E402
from bfp_inputs import manufactured_rhs, random_mantissas  # noqa: E402
from oracle import bfp as B  # noqa: E402
from oracle import mg  # noqa: E402

from test_gpu_ops import check, dev_vec, gq, oq, out_vec, stats_tensor  # noqa: E402

pytestmark = pytest.mark.gpu


def mstr(mode):
    return "qcomp" if mode == bfp.QCOMP else "nnqcomp"


SHAPES = [(63, 63), (9, 300), (260, 17), (1, 1), (0, 0), (15, 15, 15), (5, 9, 300), (3, 260, 17)]
COEFS = [None, ((3, -1), (-12345, -15)), ((1, 0), (-1, -2))]   # None: the solver's c1, c2


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("w_in,w_out", [(16, 16), (8, 12), (24, 16), (32, 32), (12, 24)])
@pytest.mark.parametrize("mode", [bfp.QCOMP, bfp.NNQCOMP])
@pytest.mark.parametrize("coef", range(len(COEFS)))
def test_cheby_op_bit_exact(shape, w_in, w_out, mode, coef):
    nd = len(shape)
    A = bfp.bfp_laplace_stencil(nd, 0.8 if nd == 2 else 6 / 7, 16)
    if COEFS[coef] is None:
        s = mg.BFPSolver(nd, 7, smoother="cheby")
        c1, c2 = s.c1, s.c2
    else:
        c1, c2 = B.Scalar(*COEFS[coef][0]), B.Scalar(*COEFS[coef][1])
    seed = hash((shape, w_in, w_out, mode, coef)) % 1000
    m = random_mantissas(shape, w_in, seed, "smooth" if seed % 2 and np.prod(shape) > 0 else "uniform")
    r = dev_vec(m, -11, w_in, junk_seed=seed)
    z = out_vec(shape, w_out)
    st = stats_tensor()
    bfp.bfp_cheby(A, bfp.scalar(int(c1.m), int(c1.e)), bfp.scalar(int(c2.m), int(c2.e)), r, z, gq(w_out, mode), st)
    rs = B.Stats()
    ref = B.cheby(B.laplace_stencil(nd), c1, c2, B.BFP(m, -11, w_in), oq(w_out, mode), rs)
    check(z, ref, st, rs)


def make(nd, n, w, mode, onchip=1, w_step=0, use_graph=1):
    o = bfp.bfp_solver_opts_default(nd, n, w)
    o.mode = mode
    o.coarse_onchip = onchip
    o.w_step = w_step
    o.use_graph = use_graph
    o.smoother = bfp.SMOOTH_CHEBY
    h = bfp.Hierarchy(o)
    s = mg.BFPSolver(nd, n, w=w, mode=mstr(mode), omega=o.omega, w_omega=o.w_omega, w_step=w_step,
                     smoother="cheby", eta=o.cheby_eta)
    return h, s


@pytest.mark.parametrize("nd,n", [(2, 63), (2, 255), (2, 31), (3, 15), (3, 31)])
@pytest.mark.parametrize("w", [8, 16, 32])
@pytest.mark.parametrize("mode", [bfp.QCOMP, bfp.NNQCOMP])
@pytest.mark.parametrize("onchip", [1, 63, 15, 0])
def test_vcycle10_bit_exact(nd, n, w, mode, onchip):
    h, s = make(nd, n, w, mode, onchip)
    rm = random_mantissas((n,) * nd, w, 5, "smooth")
    r = bfp.BFPVector.from_mantissas(rm, -30, w)
    y = bfp.BFPVector((n,) * nd, w)
    h.reset_stats()
    h.vcycle(r, y)
    ref = s.vcycle(0, B.BFP(rm, -30, w))
    torch.cuda.synchronize()
    assert y.exponent == ref.e
    assert np.array_equal(y.mantissas(), np.asarray(ref.m).astype(np.int64))
    st = h.stats()
    assert (st["calls"], st["recomputed"], st["saturated"]) == (s.stats.calls, s.stats.recomputed,
                                                               s.stats.saturated)
    h.close()


@pytest.mark.parametrize("nd,n,w,w_step", [(2, 63, 16, 0), (2, 127, 12, 1), (2, 255, 16, 1), (3, 15, 16, 0),
                                           (2, 63, 24, 0)])
@pytest.mark.parametrize("mode", [bfp.QCOMP, bfp.NNQCOMP])
def test_fmg_and_ir_bit_exact(nd, n, w, w_step, mode):
    h, s = make(nd, n, w, mode, w_step=w_step)
    f = manufactured_rhs(nd, n)
    ft = torch.from_numpy(f).cuda()
    xt = torch.zeros_like(ft)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        h.fmg(ft, xt)
    stream.synchronize()
    xr = s.fmg(f)
    assert np.array_equal(xt.cpu().numpy(), xr)
    b = s.rhs_hierarchy(f)[0]
    for it in range(3):
        with torch.cuda.stream(stream):
            h.ir_iterate(ft, xt, 1)
        stream.synchronize()
        xr = s.ir_step(0, b, xr)
        assert np.array_equal(xt.cpu().numpy(), xr), it
    h.close()


def test_bfp_ir_with_cheby_bit_exact():
    """The all-BFP IR on a V(1,0) hierarchy."""
    n = 63
    h, s = make(2, n, 16, bfp.NNQCOMP)
    f = manufactured_rhs(2, n)
    b_ref = B.from_f64(s.rhs_hierarchy(f)[0], 32)
    x_ref = B.from_f64(0.5 * mg.discrete_solution(2, n), 32)
    b = bfp.BFPVector.from_mantissas(np.asarray(b_ref.m, dtype=np.int64), b_ref.e, 32)
    x = bfp.BFPVector.from_mantissas(np.asarray(x_ref.m, dtype=np.int64), x_ref.e, 32)
    h.ir_iterate_bfp(b, x, 3)
    torch.cuda.synchronize()
    for _ in range(3):
        x_ref = s.ir_step_bfp(b_ref, x_ref)
    assert x.exponent == x_ref.e and np.array_equal(x.mantissas(), np.asarray(x_ref.m, dtype=np.int64))
    h.close()


def test_argument_checks():
    o = bfp.bfp_solver_opts_default(2, 63, 16)
    o.smoother = bfp.SMOOTH_CHEBY
    for field, value in (("arith", bfp.ARITH_FP32), ("cheby_eta", 0.0), ("cheby_eta", 1.0), ("smoother", 2)):
        oo = bfp.bfp_solver_opts_default(2, 63, 16)
        oo.smoother = bfp.SMOOTH_CHEBY
        setattr(oo, field, value)
        with pytest.raises(bfp.BFPError):
            bfp.Hierarchy(oo)
    with pytest.raises(bfp.BFPError):
        bfp.Hierarchy(o, k_nodes=np.ones((65, 65)))
    # a T = c1 I + c2 A whose coefficients pass 31 bits
    A = bfp.bfp_laplace_stencil(2, 0.8, 16)
    r = bfp.BFPVector((15, 15), 16)
    z = bfp.BFPVector((15, 15), 16)
    with pytest.raises(bfp.BFPError):
        bfp.bfp_cheby(A, bfp.scalar(1, 30), bfp.scalar(-1, -30), r, z, gq(16, bfp.QCOMP))
