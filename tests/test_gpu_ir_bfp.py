"""IR with the iterate x and the right-hand side b' held as BFP blocks (bfp_ir_iterate_bfp:
Alg. ir with the qgemv residual and the qsub update, no FP64 pass) against
oracle.mg / oracle.var ir_step_bfp, bit for bit: constant coefficients in 2D and 3D
(x up to 55 bits in int64 storage, b of any storage), variable coefficients (the
26-bit residual operator included), direct and graph launches, odd and even step
counts."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2307_00124_gb300 as bfp  # noqa: E402
from bfp_inputs import grf_nodes, manufactured_rhs, random_mantissas, smoothed_random_rhs  # noqa: E402
from oracle import bfp as B  # noqa: E402
from oracle import mg  # noqa: E402
from oracle import var as V  # noqa: E402

pytestmark = pytest.mark.gpu


def mstr(mode):
    return "qcomp" if mode == bfp.QCOMP else "nnqcomp"


def run_and_compare(h, s, b_ref, x_ref, wx, wb, steps, stream):
    b = bfp.BFPVector.from_mantissas(np.asarray(b_ref.m, dtype=np.int64), b_ref.e, wb)
    x = bfp.BFPVector.from_mantissas(np.asarray(x_ref.m, dtype=np.int64), x_ref.e, wx)
    h.reset_stats()
    s.stats = B.Stats()
    for k in steps:
        if stream is None:
            h.ir_iterate_bfp(b, x, k)
        else:
            with torch.cuda.stream(stream):
                h.ir_iterate_bfp(b, x, k)
            stream.synchronize()
        torch.cuda.synchronize()
        for _ in range(k):
            x_ref = s.ir_step_bfp(b_ref, x_ref)
        assert x.exponent == x_ref.e, k
        assert np.array_equal(x.mantissas(), np.asarray(x_ref.m, dtype=np.int64)), k
        assert np.all(x.padding() == 0)
    st = h.stats()
    assert (st["calls"], st["recomputed"], st["saturated"]) == (s.stats.calls, s.stats.recomputed,
                                                               s.stats.saturated)
    return x_ref


@pytest.mark.parametrize("nd,n,w", [(2, 63, 16), (2, 127, 12), (2, 31, 24), (3, 15, 16)])
@pytest.mark.parametrize("wx,wb", [(32, 32), (24, 28), (16, 16), (40, 40), (48, 32), (55, 16)])
@pytest.mark.parametrize("mode", [bfp.QCOMP, bfp.NNQCOMP])
@pytest.mark.parametrize("graph", [0, 1])
def test_constant_bit_exact(nd, n, w, wx, wb, mode, graph):
    o = bfp.bfp_solver_opts_default(nd, n, w)
    o.mode = mode
    o.use_graph = graph
    h = bfp.Hierarchy(o)
    s = mg.BFPSolver(nd, n, w=w, mode=mstr(mode), omega=o.omega, w_omega=o.w_omega)
    f = manufactured_rhs(nd, n)
    bp = s.rhs_hierarchy(f)[0]
    assert np.array_equal(h.rhs_scale() * f, bp)
    b_ref = B.from_f64(bp, wb)
    x0 = B.from_f64(0.75 * mg.discrete_solution(nd, n), wx)
    stream = torch.cuda.Stream() if graph else None
    run_and_compare(h, s, b_ref, x0, wx, wb, (1, 2, 3), stream)
    # from x = 0 (exponent 0, all mantissas 0)
    z = B.BFP(np.zeros((n,) * nd, dtype=np.int64), 0, wx)
    run_and_compare(h, s, b_ref, z, wx, wb, (2, 1), stream)
    h.close()


def read_faces(ptr, n, ld, w):
    """An n x n int16 / int32 device array (row pitch ld) read back exactly (bfp_to_f64, e = 0)."""
    meta = torch.zeros(8, dtype=torch.int64, device="cuda")
    v = bfp.bfp_vec()
    v.mant, v.meta, v.w, v.ndim = ptr, meta.data_ptr(), w, 2
    v.n[0], v.n[1], v.n[2], v.ld = n, n, 1, ld
    out = torch.empty((n, n), dtype=torch.float64, device="cuda")
    assert bfp._lib.bfp_to_f64(C.byref(v), C.c_void_p(out.data_ptr()), None) == 0
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.int64)


@pytest.mark.parametrize("n", [63, 127])
def test_var_ir_operator_matches_oracle(n):
    K = grf_nodes(n, seed=2)
    o = bfp.bfp_solver_opts_default(2, n, 16)
    h = bfp.Hierarchy(o, k_nodes=K)
    A = h.var_ir_operator()
    s = V.VarSolver(K)
    op = V.make_ir_level(K, s.om)
    assert A.k_storage == 32 and A.q is None
    assert (A.e_k, A.a_norm) == (op.e_k, op.a_norm[0])
    assert (1 << 24) <= max(int(a.max()) for a in (op.kw, op.ke, op.ks, op.kn)) < (1 << 25)
    for ptr, want in zip(list(A.k), (op.kw, op.ke, op.ks, op.kn)):
        assert np.array_equal(read_faces(ptr, n, A.ld, 32), want)
    h.close()


@pytest.mark.parametrize("wy", [8, 16, 24, 32])
@pytest.mark.parametrize("mode", [bfp.QCOMP, bfp.NNQCOMP])
def test_var_wide_faces_ops_bit_exact(wy, mode):
    """bfp_var_apply / bfp_var_residual with int32 faces against the oracle ops."""
    n = 63
    K = grf_nodes(n, seed=3)
    h = bfp.Hierarchy(bfp.bfp_solver_opts_default(2, n, 16), k_nodes=K)
    A = h.var_ir_operator()
    op = V.make_ir_level(K, V.VarSolver(K).om)
    om = B.scalar_floor(0.8, 16)
    ym = random_mantissas((n, n), wy, 31, "smooth")
    rm = random_mantissas((n, n), wy, 32)
    wo = 16
    for ey, er in ((-5, 20), (-30, -40)):
        y = bfp.BFPVector.from_mantissas(ym, ey, wy)
        r = bfp.BFPVector.from_mantissas(rm, er, wy)
        z = bfp.BFPVector((n, n), wo)
        rs = B.Stats()
        bfp.bfp_var_apply(A, y, z, bfp.q(wo, mode))
        torch.cuda.synchronize()
        ref = V.apply(op, B.BFP(ym, ey, wy), B.Quant(wo, mstr(mode)), rs)
        assert z.exponent == ref.e and np.array_equal(z.mantissas(), np.asarray(ref.m, dtype=np.int64))
        bfp.bfp_var_residual(A, y, r, z, bfp.q(wo, mode))
        torch.cuda.synchronize()
        ref = V.residual(op, B.BFP(ym, ey, wy), B.BFP(rm, er, wy), B.Quant(wo, mstr(mode)), om, rs)
        assert z.exponent == ref.e and np.array_equal(z.mantissas(), np.asarray(ref.m, dtype=np.int64))
    # Jacobi needs the int16 faces and the weights
    with pytest.raises(bfp.BFPError):
        bfp.bfp_var_jacobi(A, None, r, z, bfp.q(wo, mode))
    h.close()


@pytest.mark.parametrize("n,w", [(63, 16), (31, 24), (127, 12)])
@pytest.mark.parametrize("wx,wb", [(32, 32), (24, 24)])
@pytest.mark.parametrize("mode", [bfp.QCOMP, bfp.NNQCOMP])
@pytest.mark.parametrize("graph", [0, 1])
def test_var_bit_exact(n, w, wx, wb, mode, graph):
    K = grf_nodes(n, seed=5)
    o = bfp.bfp_solver_opts_default(2, n, w)
    o.mode = mode
    o.use_graph = graph
    h = bfp.Hierarchy(o, k_nodes=K)
    s = V.VarSolver(K, w=w, mode=mstr(mode))
    f = smoothed_random_rhs(n, 3)
    bp = s.rhs_hierarchy(f)[0]
    assert np.array_equal(h.rhs_scale() * f, bp)
    b_ref = B.from_f64(bp, wb)
    x0 = B.from_f64(s.fmg(f), wx)
    stream = torch.cuda.Stream() if graph else None
    run_and_compare(h, s, b_ref, x0, wx, wb, (1, 2, 3), stream)
    h.close()


def test_argument_checks():
    n = 31
    o = bfp.bfp_solver_opts_default(2, n, 16)
    h = bfp.Hierarchy(o)
    b = bfp.BFPVector((n, n), 32)
    xs = bfp.BFPVector((15, 15), 32)
    with pytest.raises(bfp.BFPError):
        h.ir_iterate_bfp(b, xs, 1)           # not the finest shape
    with pytest.raises(bfp.BFPError):
        h.ir_iterate_bfp(b, b, 1)            # aliasing
    h.ir_iterate_bfp(b, bfp.BFPVector((n, n), 32), 0)   # k = 0: nothing to do
    with pytest.raises(bfp.BFPError):
        h.ir_iterate_bfp(b, bfp.BFPVector((n, n), 56), 1)   # A'x past 62 bits
    o.arith = bfp.ARITH_FP32
    hf = bfp.Hierarchy(o)
    with pytest.raises(bfp.BFPError):
        hf.ir_iterate_bfp(b, bfp.BFPVector((n, n), 32), 1)
    hf.close()
    h.close()
