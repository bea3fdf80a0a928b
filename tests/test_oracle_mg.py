"""Pins for the multigrid oracle (CPU only): closed forms, O(h^2), local Fourier
analysis of damped Jacobi, dense-eigensolve V-cycle factors (Sec. 5.2
conv-rate-v-cycle), and the BFP schedule against the FP64 one."""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from bfp_inputs import manufactured_rhs
from oracle import bfp as B
from oracle import mg

from test_oracle_bfp import laplacian_matrix, prolong_matrix


@pytest.mark.parametrize("nd,n", [(2, 31), (2, 63), (3, 15)])
def test_discrete_solution_closed_form(nd, n):
    f = manufactured_rhs(nd, n)
    b = mg.scaled_rhs(f)
    uh = mg.discrete_solution(nd, n)
    r = mg.residual_f64(b, uh)
    assert np.abs(r).max() <= 1e-12 * np.abs(b).max()
    # same check with an independently built sparse matrix A_h = L / h^2
    h = 1.0 / (n + 1)
    L = laplacian_matrix(nd, n) / h ** 2
    assert np.allclose(L @ uh.ravel(), f.ravel(), rtol=1e-11, atol=1e-9)


@pytest.mark.parametrize("nd", [2, 3])
def test_discretisation_error_is_second_order(nd):
    errs = []
    ns = (15, 31, 63) if nd == 3 else (63, 127, 255)
    for n in ns:
        u = mg.sin_product(nd, n)
        uh = mg.discrete_solution(nd, n)
        errs.append(np.abs(u - uh).max())
    for a, b in zip(errs, errs[1:]):
        assert 3.9 < a / b < 4.1
    # closed form |1 - d pi^2 / lambda_h| ~ pi^2 h^2 / 12 for the finest grid
    h = 1.0 / (ns[-1] + 1)
    assert abs(errs[-1] / (math.pi ** 2 * h ** 2 / 12) - 1) < 1e-3


def eigenmode(nd, n, ks):
    h = 1.0 / (n + 1)
    x = np.arange(1, n + 1) * h
    m = np.sin(np.pi * ks[0] * x)
    for k in ks[1:]:
        m = np.multiply.outer(np.sin(np.pi * k * x), m)
    lam = sum(1 - math.cos(math.pi * k * h) for k in ks) * 2.0 / mg.pscale(nd)
    return m, lam


@pytest.mark.parametrize("nd,omega,mu", [(2, 0.8, 3 / 5), (3, 6 / 7, 5 / 7)])
def test_jacobi_smoothing_factor_lfa(nd, omega, mu):
    """Damped Jacobi on A': each sine mode is an eigenvector; the worst high-frequency
    amplification matches the LFA closed form max(|1-2w|, |1-w/d|)."""
    n = 15 if nd == 2 else 7
    om = mg.omega_scaled(nd, omega)
    worst = 0.0
    import itertools
    for ks in itertools.product(range(1, n + 1), repeat=nd):
        m, lam = eigenmode(nd, n, ks)
        assert np.allclose(mg.apply_f64(m), lam * m, atol=1e-12)
        y = mg.jacobi_f64(m, np.zeros_like(m), om)
        amp = 1 - om * lam
        assert np.allclose(y, amp * m, atol=1e-12)
        if max(ks) > (n + 1) // 2:
            worst = max(worst, abs(amp))
    assert worst <= mu + 1e-12
    assert worst > mu - 0.15
    assert abs(mu - max(abs(1 - 2 * omega), abs(1 - omega / nd))) < 1e-12


def vcycle_matrix(nd, n, omega):
    """Error propagation V = I - Vcycle(A') applied to canonical basis vectors."""
    N = n ** nd
    om = mg.omega_scaled(nd, omega)
    V = np.zeros((N, N))
    for i in range(N):
        e = np.zeros(N)
        e[i] = 1.0
        e = e.reshape((n,) * nd)
        y = mg.vcycle_f64(mg.apply_f64(e), om)
        V[:, i] = (e - y).ravel()
    return V


def test_vcycle_energy_factor_dense_eigensolve():
    """rho_v = ||V||_A from V^T A V x = lambda A x (Sec. 5.2), mesh independent,
    and close to the asymptotic rate seen by iterating."""
    rhos = []
    for n in (7, 15):
        h = 1.0 / (n + 1)
        A = (laplacian_matrix(2, n) / 4.0).toarray()
        V = vcycle_matrix(2, n, 0.8)
        lam = sla.eigh(V.T @ A @ V, A, eigvals_only=True)
        rhos.append(math.sqrt(lam.max()))
    assert all(0.05 < r < 0.25 for r in rhos), rhos
    assert abs(rhos[0] - rhos[1]) < 0.05
    rng = np.random.default_rng(0)
    n = 63
    x = rng.standard_normal((n, n))
    b = np.zeros((n, n))
    om = mg.omega_scaled(2, 0.8)
    e0 = math.sqrt(mg.energy_sq(x))
    for _ in range(12):
        x = x + mg.vcycle_f64(mg.residual_f64(b, x), om)
        e1 = math.sqrt(mg.energy_sq(x))
        fac, e0 = e1 / e0, e1
    assert fac <= rhos[1] + 0.02


def test_fp64_restriction_matches_matrix():
    for nd, nc in ((2, 5), (3, 3)):
        rng = np.random.default_rng(1)
        nf = 2 * nc + 1
        r = rng.standard_normal((nf,) * nd)
        P = prolong_matrix(nd, nc)
        Rt = P.T * (1.0 if nd == 2 else 0.5)
        assert np.allclose(mg.restrict_f64(r).ravel(), Rt @ r.ravel(), atol=1e-14)
        c = rng.standard_normal((nc,) * nd)
        assert np.allclose(mg.prolong_f64(c, (nf,) * nd).ravel(), P @ c.ravel(), atol=1e-14)


@pytest.mark.parametrize("nd,n", [(2, 31), (3, 15)])
def test_bfp_vcycle_tracks_fp64_vcycle_at_32_bits(nd, n):
    """The BFP schedule at w = 32 equals the FP64 V-cycle up to quantisation."""
    omega = 0.8 if nd == 2 else 6 / 7
    s = mg.BFPSolver(nd, n, w=32, w_omega=32, omega=omega, mode="qcomp")
    rng = np.random.default_rng(2)
    r64 = rng.standard_normal((n,) * nd)
    r = B.from_f64(r64, 32)
    y = B.to_f64(s.vcycle(0, r))
    y64 = mg.vcycle_f64(B.to_f64(r), float(s.om.value()))
    assert np.abs(y - y64).max() <= 1e-7 * np.abs(y64).max()


@pytest.mark.parametrize("mode", ["qcomp", "nnqcomp"])
def test_bfp_fmg_reaches_discretisation_accuracy(mode):
    """Sec. 5.1 acceptance ||u - x||_L / ||u - u_h||_L <= 1.5 after FMG at w = 16 (63^2)."""
    f = manufactured_rhs(2, 63)
    s = mg.BFPSolver(2, 63, w=16, mode=mode)
    x = s.fmg(f)
    assert mg.accuracy_ratio(2, x) <= 1.5
    if mode == "nnqcomp":
        assert s.stats.recomputed == 0


def test_bfp_ir_converges_to_discrete_solution():
    f = manufactured_rhs(2, 63)
    s = mg.BFPSolver(2, 63, w=16, mode="qcomp")
    b = s.rhs_hierarchy(f)[0]
    x = np.zeros_like(b)
    uh = mg.discrete_solution(2, 63)
    errs = []
    for _ in range(10):
        x = s.ir_step(0, b, x)
        errs.append(math.sqrt(mg.energy_sq(x - uh)))
    facs = [b_ / a_ for a_, b_ in zip(errs, errs[1:])]
    assert max(facs[:6]) < 0.3
    assert errs[-1] < 1e-8 * math.sqrt(mg.energy_sq(uh))


def test_progressive_precision_widths():
    """Progressive precision (inner width w_dot_j = j + q: one bit fewer per coarser level, Sec. 4 eq.
    width-bounds): level widths follow w - k, never below 2; the smallest finest width with which
    FMG + 1 IR-V step reaches the accuracy test is within one bit of the uniform-width one, and it
    grows by 1 to 3 bits per halving of h (second-order accuracy: about 2 bits)."""
    s = mg.BFPSolver(2, 255, w=9, w_step=1)
    assert [s.width(k) for k in range(len(s.sizes))] == [9, 8, 7, 6, 5, 4, 3]
    assert mg.BFPSolver(2, 63, w=1).width(4) == 1
    prog, uni = [], []
    for n in (63, 127, 255):
        f = manufactured_rhs(2, n)
        for step, out in ((1, prog), (0, uni)):
            for w in range(6, 20):
                sv = mg.BFPSolver(2, n, w=w, mode="nnqcomp", w_step=step)
                x = sv.ir_step(0, sv.rhs_hierarchy(f)[0], sv.fmg(f))
                if mg.accuracy_ratio(2, x) <= 1.5:
                    out.append(w)
                    break
    assert len(prog) == len(uni) == 3, (prog, uni)
    for p, u in zip(prog, uni):
        assert p <= u + 1
    for a, b in zip(prog, prog[1:]):
        assert 1 <= b - a <= 3


def _exact_rhs(A, x):
    """b = A' x exactly, as a BFP block (the IR residual of x is then exactly 0)."""
    ex = B.espmv_stencil(A, x)
    z = np.asarray(ex.z, dtype=np.int64)
    return B.BFP(z, ex.e, 32)


@pytest.mark.parametrize("mode", ["qcomp", "nnqcomp"])
def test_bfp_ir_fixed_point(mode):
    """Alg. ir with BFP x and b: when b = A' x exactly the residual is 0, V(0) = 0 and the
    update returns x itself (a dropped b term or a wrong scale moves x)."""
    s = mg.BFPSolver(2, 31, w=16, mode=mode)
    x = B.normalize(B.BFP(np.asarray(np.random.default_rng(3).integers(-2**23, 2**23, (31, 31))), -40, 24),
                    B.Quant(24, "qcomp"))
    xn = s.ir_step_bfp(_exact_rhs(s.A, x), x)
    assert xn.e == x.e and np.array_equal(xn.m, x.m)
    # b lowered at one point by 2^12 of its units (above x's ulp after A'^-1): x moves down
    # there, most at that point (A'^-1 has positive entries, largest on the diagonal)
    b = _exact_rhs(s.A, x)
    b.m[7, 9] -= 1 << 12
    d = s.ir_step_bfp(b, x).m - x.m
    assert d.max() <= 0 and d.min() < 0 and d[7, 9] == d.min()


def _bfp_ir_errors(s, b, x, uh, steps):
    eu = math.sqrt(mg.energy_sq(uh))
    out = []
    for _ in range(steps):
        x = s.ir_step_bfp(b, x)
        out.append(math.sqrt(mg.energy_sq(B.to_f64(x) - uh)) / eu)
    return x, out


def test_bfp_ir_converges_to_the_width_floor():
    """From x = 0, Alg. ir with BFP x, b (w_b = max(32, w_x), inner w = 16) contracts like the
    FP64-residual IR (V-cycle factor ~0.11 here) down to a floor set by x's width: the
    floor at w_x = 28 is 2^4 times the one at 32 and the one at 40 is 2^-8 times it (within a
    factor 2)."""
    n = 63
    f = manufactured_rhs(2, n)
    uh = mg.discrete_solution(2, n)
    floors = {}
    for wx in (32, 28, 40):
        s = mg.BFPSolver(2, n, w=16, mode="qcomp")
        b = B.from_f64(s.rhs_hierarchy(f)[0], max(32, wx))   # b finer than x: x sets the floor
        x0 = B.BFP(np.zeros((n, n), dtype=np.int64), 0, wx)
        x, errs = _bfp_ir_errors(s, b, x0, uh, 12)
        assert x.w == wx
        facs = [e1 / e0 for e0, e1 in zip(errs, errs[1:6])]
        assert max(facs) < 0.15, facs
        floors[wx] = errs[-1]
        assert errs[-1] <= 1.1 * min(errs[-4:])           # settled
    assert floors[32] < 3e-8
    assert 8 <= floors[28] / floors[32] <= 32, floors
    assert 2 ** 7 <= floors[32] / floors[40] <= 2 ** 9, floors        # int64 iterate (w > 32)


def _f64_block(x):
    """The doubles as one exact BFP block z* 2^-1074 (Python integers; every double is an
    integer multiple of 2^-1074)."""
    M, E = B.f64_split(x)
    z = np.empty(x.shape, dtype=object)
    z.ravel()[:] = [int(m) << int(e - B.F64_E_STAR) for m, e in zip(M.ravel(), E.ravel())]
    return B.Exact(z, B.F64_E_STAR, 2100)


def test_ir_window_model_matches_alg_qcomp():
    """The IR residual's quantisation (ir_quantize: from_f64 plus the window decision) against
    Alg. qcomp run step by step on the exact FP64 block, for windows around the residual's own mu*
    and both IR residual rows of Table tab:estimates (w_add 4, and 5 for an FMG level's first step):
    the same result, and a recomputation exactly when Alg. qcomp overflows or underflows."""
    rng = np.random.default_rng(11)
    s = mg.BFPSolver(2, 7, w=16, mode="qcomp")
    seen = set()
    for trial in range(6):
        r64 = rng.standard_normal((7, 7)) * 10.0 ** int(rng.integers(-12, 3))
        if trial == 5:
            r64[:] = 0.0                                   # all-zero residual: mu* at e* + 1
        ex = _f64_block(r64)
        ref = B.from_f64(r64, 16)
        mu = ref.e + 16
        for first in (False, True):
            w_tmp = 16 + (5 if first else 4)
            for gam in range(mu - 8, mu + 9):
                s.ir_gamma, s.ir_counts = {0: gam}, {}
                got = s.ir_quantize(0, r64, first)
                out, ovf, unf = B.qcomp_alg(ex, 16, w_tmp, (1, gam - 2))   # msb(1) + (gam - 2) = gam
                assert got.e == out.e == ref.e
                assert np.array_equal(np.asarray(got.m, dtype=object), np.asarray(out.m, dtype=object))
                assert s.ir_counts[0] == [1, int(ovf or unf)]
                assert s.ir_gamma[0] == mu                   # the next residual's gamma
                seen.add((ovf, unf))
    assert seen == {(False, False), (True, False), (False, True)}


def test_ir_window_model_recomputes_without_a_window():
    r64 = np.linspace(-1.0, 2.0, 49).reshape(7, 7) * 1e-6
    mu = B.from_f64(r64, 16).e + 16
    for kw in ({"ir_window": False}, {"ir_window_bits": 19}, {}):
        s = mg.BFPSolver(2, 7, w=16, mode="qcomp", **kw)
        if kw:
            s.ir_gamma = {0: mu}                            # a perfect gamma, but no window kept
        s.ir_quantize(0, r64)                               # (no gamma at all in the last case)
        assert s.ir_counts[0] == [1, 1]
    s = mg.BFPSolver(2, 7, w=16, mode="qcomp", w_add_max=0)
    s.ir_gamma = {0: mu + 1}                                 # w_add capped at 0: lambda_out < lambda_tmp
    s.ir_quantize(0, r64)
    assert s.ir_counts[0] == [1, 1]
    s = mg.BFPSolver(2, 7, w=16, mode="qcomp")
    s.ir_gamma = {0: mu + 1}
    s.ir_quantize(0, r64)
    assert s.ir_counts[0] == [1, 0]
