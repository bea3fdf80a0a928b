"""Pins for the float-baseline oracle (CPU only): BF16 rounding against torch's
conversion, the float ops against the FP64 multigrid pieces (exactly on
small-integer data, within the per-sweep tolerances otherwise), and the float
IR-V / FMG schedule against discretisation accuracy."""
import numpy as np
import pytest

from bfp_inputs import manufactured_rhs
from oracle import bfp as B
from oracle import flt
from oracle import mg

torch = pytest.importorskip("torch")


def test_round_bf16_matches_torch():
    rng = np.random.default_rng(0)
    a = (rng.standard_normal(20000) * np.exp2(rng.integers(-40, 40, 20000))).astype(np.float32)
    # ties: the low 16 bits exactly 0x8000, with even and odd upper halves
    ties = (np.arange(1, 2001, dtype=np.uint32) << 16 | 0x8000).view(np.float32)
    for x in (a, ties, -ties):
        ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
        assert np.array_equal(flt.round_bf16(x), ref)


def _om(nd):
    return B.scalar_floor(mg.omega_scaled(nd, 0.8 if nd == 2 else 6.0 / 7.0), 16)


@pytest.mark.parametrize("nd,n", [(2, 15), (3, 7)])
def test_float_ops_exact_on_small_integers(nd, n):
    """With small integer data every FP32 operation is exact, so the float ops equal
    the FP64 definitions (mg) exactly: this pins operands, signs and weights."""
    rng = np.random.default_rng(nd)
    shape = (n,) * nd
    A = B.laplace_stencil(nd)
    om = _om(nd)
    w = om.m * 2.0 ** om.e
    y = rng.integers(-64, 64, size=shape).astype(np.float64)
    r = rng.integers(-64, 64, size=shape).astype(np.float64)
    assert np.array_equal(flt.jacobi(A, om, y, r, flt.F32), mg.jacobi_f64(y, r, w))
    assert np.array_equal(flt.jacobi(A, om, None, r, flt.F32), w * r)
    assert np.array_equal(flt.residual(A, y, r, flt.F32), mg.apply_f64(y) - r)
    assert np.array_equal(flt.restrict(y, flt.F32), mg.restrict_f64(y))
    c = rng.integers(-64, 64, size=B.coarse_shape(shape)).astype(np.float64)
    assert np.array_equal(flt.prolong(c, None, shape, flt.F32), mg.prolong_f64(c, shape))
    assert np.array_equal(flt.prolong(c, y, shape, flt.F32), y - mg.prolong_f64(c, shape))


@pytest.mark.parametrize("dtype,tol", [(flt.F32, 1e-5), (flt.BF16, 1e-2)])
@pytest.mark.parametrize("nd,n", [(2, 63), (3, 15)])
def test_float_sweep_error_against_fp64(dtype, tol, nd, n):
    """One Jacobi sweep (and one V-cycle residual) in the float format against FP64 on the same
    (representable) inputs: relative max-norm error within the stated per-sweep tolerance."""
    rng = np.random.default_rng(5)
    shape = (n,) * nd
    A = B.laplace_stencil(nd)
    om = _om(nd)
    w = om.m * 2.0 ** om.e
    y = flt.store(mg.sin_product(nd, n) + 0.1 * rng.standard_normal(shape), dtype).astype(np.float64)
    r = flt.store(0.01 * rng.standard_normal(shape), dtype).astype(np.float64)
    ref = mg.jacobi_f64(y, r, w)
    got = flt.jacobi(A, om, y, r, dtype).astype(np.float64)
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    ref = mg.apply_f64(y) - r
    got = flt.residual(A, y, r, dtype).astype(np.float64)
    assert np.abs(got - ref).max() <= tol * np.abs(y).max()


@pytest.mark.parametrize("dtype", [flt.F32, flt.BF16])
def test_float_fmg_reaches_discretisation_accuracy(dtype):
    n = 63
    s = flt.FloatSolver(2, n, dtype=dtype)
    f = manufactured_rhs(2, n)
    x = s.fmg(f)
    b = s.rhs_hierarchy(f)[0]
    for _ in range(2 if dtype == flt.F32 else 6):
        x = s.ir_step(0, b, x)
    assert mg.accuracy_ratio(2, x) <= 1.5
