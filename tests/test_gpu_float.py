"""Float baselines on the GPU (FP32 and BF16 storage): every op, the V-cycle and
whole FMG / IR-V solves bit for bit against oracle/flt.py, and the per-sweep
error against FP64 within 1e-5 (FP32) / 1e-2 (BF16)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2307_00124_gb300 as bfp  # noqa: E402
from bfp_inputs import manufactured_rhs  # noqa: E402
from oracle import bfp as B  # noqa: E402
from oracle import flt  # noqa: E402
from oracle import mg  # noqa: E402

pytestmark = pytest.mark.gpu

DT = {flt.F32: bfp.F32, flt.BF16: bfp.BF16}


def stencil(nd):
    return bfp.bfp_laplace_stencil(nd, 0.8 if nd == 2 else 6.0 / 7.0, 16)


def om_of(nd):
    return B.scalar_floor(mg.omega_scaled(nd, 0.8 if nd == 2 else 6.0 / 7.0), 16)


def vec(a, dt):
    return bfp.FltVector.from_array(flt.store(a, dt), DT[dt])


def data(shape, seed, dt):
    rng = np.random.default_rng(seed)
    return flt.store(rng.standard_normal(shape) * 2.0 ** rng.integers(-3, 3), dt)


SHAPES = [(2, (63, 63)), (2, (31, 45)), (2, (255, 255)), (2, (129, 517)), (3, (15, 15, 15)), (3, (7, 9, 13))]


@pytest.mark.parametrize("dt", [flt.F32, flt.BF16])
@pytest.mark.parametrize("nd,shape", SHAPES)
def test_stencil_ops_bit_exact(dt, nd, shape):
    A = stencil(nd)
    Ao, om = B.laplace_stencil(nd), om_of(nd)
    y, r = data(shape, 1, dt), data(shape, 2, dt)
    yv, rv = vec(y, dt), vec(r, dt)
    out = bfp.FltVector(shape, DT[dt])
    out.data.fill_(7)
    bfp.flt_jacobi(A, yv, rv, out)
    assert np.array_equal(out.values(), flt.jacobi(Ao, om, y, r, dt))
    assert np.all(out.padding() == 0)
    bfp.flt_jacobi(A, None, rv, out)
    assert np.array_equal(out.values(), flt.jacobi(Ao, om, None, r, dt))
    bfp.flt_residual(A, yv, rv, out)
    assert np.array_equal(out.values(), flt.residual(Ao, y, r, dt))


@pytest.mark.parametrize("dt", [flt.F32, flt.BF16])
@pytest.mark.parametrize("nd,n", [(2, 63), (2, 255), (2, 1023), (3, 15), (3, 31)])
def test_transfers_bit_exact(dt, nd, n):
    shape = (n,) * nd
    cs = B.coarse_shape(shape)
    f, y, c = data(shape, 3, dt), data(shape, 4, dt), data(cs, 5, dt)
    out_c = bfp.FltVector(cs, DT[dt])
    bfp.flt_restrict(vec(f, dt), out_c)
    assert np.array_equal(out_c.values(), flt.restrict(f, dt))
    out = bfp.FltVector(shape, DT[dt])
    bfp.flt_prolong(vec(c, dt), vec(y, dt), out)
    assert np.array_equal(out.values(), flt.prolong(c, y, shape, dt))
    bfp.flt_prolong(vec(c, dt), None, out)
    assert np.array_equal(out.values(), flt.prolong(c, None, shape, dt))
    assert np.all(out.padding() == 0)


@pytest.mark.parametrize("dt,tol", [(flt.F32, 1e-5), (flt.BF16, 1e-2)])
@pytest.mark.parametrize("nd,n", [(2, 4095), (3, 63)])
def test_sweep_error_against_fp64(dt, tol, nd, n):
    """Per-sweep error of the GPU float Jacobi at full size against the FP64 sweep."""
    shape = (n,) * nd
    rng = np.random.default_rng(11)
    y = flt.store(mg.sin_product(nd, n) + 0.05 * rng.standard_normal(shape), dt)
    r = flt.store(1e-3 * rng.standard_normal(shape), dt)
    out = bfp.FltVector(shape, DT[dt])
    bfp.flt_jacobi(stencil(nd), vec(y, dt), vec(r, dt), out)
    om = om_of(nd)
    ref = mg.jacobi_f64(y.astype(np.float64), r.astype(np.float64), om.m * 2.0 ** om.e)
    got = out.values().astype(np.float64)
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()


def make(nd, n, dt, **kw):
    o = bfp.bfp_solver_opts_default(nd, n, 16)
    o.arith = bfp.ARITH_FP32 if dt == flt.F32 else bfp.ARITH_BF16
    for k, v in kw.items():
        setattr(o, k, v)
    h = bfp.Hierarchy(o)
    s = flt.FloatSolver(nd, n, dtype=dt, omega=o.omega, w_omega=o.w_omega)
    return h, s


@pytest.mark.parametrize("dt", [flt.F32, flt.BF16])
@pytest.mark.parametrize("nd,n", [(2, 63), (2, 255), (3, 15)])
def test_vcycle_bit_exact(dt, nd, n):
    h, s = make(nd, n, dt)
    shape = (n,) * nd
    r = data(shape, 9, dt)
    y = bfp.FltVector(shape, DT[dt])
    h.vcycle(vec(r, dt), y)
    torch.cuda.synchronize()
    assert np.array_equal(y.values(), s.vcycle(0, r))


@pytest.mark.parametrize("dt", [flt.F32, flt.BF16])
@pytest.mark.parametrize("nd,n", [(2, 63), (2, 127), (3, 15)])
def test_fmg_and_ir_bit_exact(dt, nd, n):
    h, s = make(nd, n, dt)
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
    if nd == 2 and dt == flt.F32:
        assert mg.accuracy_ratio(nd, xt.cpu().numpy()) <= 1.5


def test_float_hierarchy_rejects_bfp_calls():
    h, _ = make(2, 63, flt.F32)
    r = bfp.BFPVector((63, 63), 16)
    y = bfp.BFPVector((63, 63), 16)
    with pytest.raises(bfp.BFPError):
        h.vcycle(r, y)
