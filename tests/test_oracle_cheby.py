"""Pins of the Chebyshev V(1,0) oracle (Alg. cheby-nodes, the relaxation line of Alg. v-cycle,
Alg. solver-setup's eigenvalue bound) against the Chebyshev polynomials, sparse eigensolves,
exact rational arithmetic, dense V-cycle matrices and the FP64 cycle."""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from numpy.polynomial import chebyshev as npcheb

from bfp_inputs import manufactured_rhs, random_mantissas
from oracle import bfp as B
from oracle import mg

from test_oracle_bfp import laplacian_matrix


@pytest.mark.parametrize("rho,eta", [(2.0, 0.15), (1.99, 0.3), (1.5, 0.05), (mg.RHO_L5, 0.9)])
def test_cheby_nodes_is_the_scaled_chebyshev_polynomial(rho, eta):
    """1 - lam (c1 + c2 lam) = T_2((alpha - lam)/c) / T_2(alpha/c) on [eta rho, rho] (two steps of
    Chebyshev iteration from zero), so |p| <= 1/T_2(alpha/c) there and p(0) = 1."""
    c1, c2 = mg.cheby_nodes(rho, eta)
    alpha, c = 0.5 * (1 + eta) * rho, 0.5 * (1 - eta) * rho
    lam = np.linspace(0.0, rho, 41)
    p = 1.0 - lam * (c1 + c2 * lam)
    t2 = npcheb.chebval((alpha - lam) / c, [0, 0, 1]) / npcheb.chebval(alpha / c, [0, 0, 1])
    assert np.allclose(p, t2, rtol=0, atol=1e-12)
    band = lam >= eta * rho
    assert np.abs(p[band]).max() <= 1.0 / npcheb.chebval(alpha / c, [0, 0, 1]) + 1e-12
    assert c1 > 0 > c2


def test_rho_is_the_level5_generalised_eigenvalue():
    """rho: the largest eigenvalue of A x = lambda D x on level 5 (h = 1/32), 2D and 3D."""
    assert abs(mg.RHO_L5 - (1.0 + math.cos(math.pi / 32))) <= 2.3e-16
    for nd in (2, 3):
        L = laplacian_matrix(nd, 31) / (2.0 * nd)      # D^-1 A (D = diag 2d)
        lam = spla.eigsh(L, k=1, which="LA", return_eigenvectors=False)[0]
        assert abs(lam - mg.RHO_L5) < 1e-9
        assert mg.rho_gen(nd) == pytest.approx(mg.RHO_L5, abs=1e-15)


@pytest.mark.parametrize("nd", [2, 3])
def test_scaled_coefficients_relax_the_scaled_system(nd):
    """For A' with diagonal d, (c1/d) r + (c2/d^2) A' r equals (c1 I + c2 D^-1 A)(D^-1 r) with
    D^-1 A = A'/d: the relaxation of D^-1 A y = D^-1 r that Alg. solver-setup prescribes."""
    n = 7
    c1, c2 = mg.cheby_nodes(mg.RHO_L5, 0.15)
    s1, s2 = mg.cheby_scaled(nd, c1, c2)
    d = mg.diag_coef(nd)
    r = np.random.default_rng(1).standard_normal((n,) * nd)
    y = mg.cheby_f64(r, s1, s2)
    Dinv_A = laplacian_matrix(nd, n) / (2.0 * nd)
    want = c1 * (r.ravel() / d) + c2 * (Dinv_A @ (r.ravel() / d))
    assert np.allclose(y.ravel(), want, rtol=1e-13, atol=1e-13)


def test_cheby_op_exact_by_rationals():
    """B.cheby: floor of c2 A r + c1 r at the qcomp exponent, checked element by element."""
    s = mg.BFPSolver(2, 7, w=12, smoother="cheby")
    r = B.BFP(random_mantissas((5, 6), 12, 3), -9, 12)
    y = B.cheby(s.A, s.c1, s.c2, r, B.Quant(12, "qcomp"))
    c1 = Fraction(int(s.c1.m)) * Fraction(2) ** int(s.c1.e)
    c2 = Fraction(int(s.c2.m)) * Fraction(2) ** int(s.c2.e)
    R = lambda i, j: Fraction(int(r.m[j, i])) * Fraction(2) ** r.e if 0 <= i < 6 and 0 <= j < 5 else Fraction(0)
    for j in range(5):
        for i in range(6):
            ar = R(i, j) - Fraction(1, 4) * (R(i - 1, j) + R(i + 1, j) + R(i, j - 1) + R(i, j + 1))
            z = c2 * ar + c1 * R(i, j)
            lo = Fraction(int(y.m[j, i])) * Fraction(2) ** y.e
            assert lo <= z < lo + Fraction(2) ** y.e
    assert np.abs(y.m).max() >= 1 << 10          # normalised


def vcycle10_matrix(nd, n, eta):
    c1, c2 = mg.cheby_scaled(nd, *mg.cheby_nodes(mg.RHO_L5, eta))
    N = n ** nd
    V = np.zeros((N, N))
    for i in range(N):
        e = np.zeros(N)
        e[i] = 1.0
        e = e.reshape((n,) * nd)
        V[:, i] = (e - mg.vcycle10_f64(mg.apply_f64(e), c1, c2)).ravel()
    return V


def test_vcycle10_rate_matches_dense_spectral_radius_and_eta_is_interior():
    """vcycle10_rate (power iteration) against the spectral radius of the dense V(1,0) error
    propagation matrix; the rate at the default eta = 0.15 (the search's minimum on level 5) is below
    those at 0.05 and 0.5, and the search on 15^2 lands next to it."""
    for eta in (0.15, 0.5):
        V = vcycle10_matrix(2, 15, eta)
        rad = np.abs(np.linalg.eigvals(V)).max()
        assert abs(mg.vcycle10_rate(2, 15, eta, iters=80) - rad) < 0.01 * rad
    r = {eta: mg.vcycle10_rate(2, 31, eta) for eta in (0.05, 0.15, 0.5)}
    assert r[0.15] < r[0.05] and r[0.15] < r[0.5] and 0.3 < r[0.15] < 0.45, r
    assert abs(mg.eta_search(2, 15) - 0.15) <= 0.03


@pytest.mark.parametrize("nd,n", [(2, 31), (3, 15)])
def test_bfp_vcycle10_tracks_fp64_at_32_bits(nd, n):
    s = mg.BFPSolver(nd, n, w=32, w_omega=32, mode="qcomp", smoother="cheby")
    r64 = np.random.default_rng(2).standard_normal((n,) * nd)
    r = B.from_f64(r64, 32)
    y = B.to_f64(s.vcycle(0, r))
    y64 = mg.vcycle10_f64(B.to_f64(r), float(s.c1.value()), float(s.c2.value()))
    assert np.abs(y - y64).max() <= 1e-7 * np.abs(y64).max()


@pytest.mark.parametrize("mode", ["qcomp", "nnqcomp"])
def test_bfp_fmg_cheby_reaches_discretisation_accuracy(mode):
    """FMG with V(1,0) and the Chebyshev relaxation at w = 16 on 63^2: the accuracy ratio falls
    with N (IR-V steps per level) and reaches the test by N = 6; IR-V(1,0) contracts at ~0.37 per
    step, the FP64 V(1,0) factor.  (With bilinear FMG interpolation the energy error after
    interpolation is O(h) against an O(h^2) discretisation error at the nodes, so N grows slowly with
    the grid in this finite-difference setting.)"""
    f = manufactured_rhs(2, 63)
    ratios = []
    for N in (2, 4, 6):
        s = mg.BFPSolver(2, 63, w=16, mode=mode, smoother="cheby", n_fmg=N)
        ratios.append(mg.accuracy_ratio(2, s.fmg(f)))
    assert ratios[0] > ratios[1] > ratios[2] and ratios[2] <= 1.5, ratios
    b = s.rhs_hierarchy(f)[0]
    uh = mg.discrete_solution(2, 63)
    x = np.zeros_like(b)
    e = [math.sqrt(mg.energy_sq(uh))]
    for _ in range(5):
        x = s.ir_step(0, b, x)
        e.append(math.sqrt(mg.energy_sq(x - uh)))
    facs = [b_ / a_ for a_, b_ in zip(e, e[1:])]
    assert max(facs) < 0.42 and min(facs) > 0.3, facs
