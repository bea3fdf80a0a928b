"""Whole-solve parity of the CUDA multigrid (V-cycle, IR, FMG) with the oracle schedule."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2307_00124_gb300 as bfp  # noqa: E402
from bfp_inputs import manufactured_rhs, random_mantissas  # noqa: E402
from oracle import bfp as B  # noqa: E402
from oracle import mg  # noqa: E402

pytestmark = pytest.mark.gpu


def make(nd, n, w, mode, use_tmp=1, use_graph=1, coarse_onchip=1, w_step=0):
    o = bfp.bfp_solver_opts_default(nd, n, w)
    o.mode = mode
    o.use_tmp = use_tmp
    o.use_graph = use_graph
    o.coarse_onchip = coarse_onchip
    o.w_step = w_step
    h = bfp.Hierarchy(o)
    s = mg.BFPSolver(nd, n, w=w, mode="qcomp" if mode == bfp.QCOMP else "nnqcomp",
                     omega=o.omega, w_omega=o.w_omega, w_step=w_step, ir_window=bool(use_tmp))
    return h, s


def ir_counters_match(h, s):
    """The IR residual counters (quantisations, recomputations) equal the oracle's window model,
    over all levels and on the finest level."""
    st, fin = h.stats(), h.finest_stats()
    assert (st["ir_residuals"], st["ir_recomputed"]) == s.ir_totals()
    assert (fin["ir_residuals"], fin["ir_recomputed"]) == s.ir_totals(finest_only=True)


@pytest.mark.parametrize("nd,n", [(2, 63), (2, 31), (2, 255), (3, 15)])
@pytest.mark.parametrize("w", [8, 16, 32])
@pytest.mark.parametrize("mode", [bfp.QCOMP, bfp.NNQCOMP])
@pytest.mark.parametrize("onchip", [1, 63, 15, 0])
def test_vcycle_bit_exact(nd, n, w, mode, onchip):
    h, s = make(nd, n, w, mode, coarse_onchip=onchip)
    rm = random_mantissas((n,) * nd, w, 5, "smooth")
    r = bfp.BFPVector.from_mantissas(rm, -30, w)
    y = bfp.BFPVector((n,) * nd, w)
    h.vcycle(r, y)
    ref = s.vcycle(0, B.BFP(rm, -30, w))
    torch.cuda.synchronize()
    assert y.exponent == ref.e
    assert np.array_equal(y.mantissas(), np.asarray(ref.m).astype(np.int64))
    st = h.stats()
    assert st["calls"] == s.stats.calls
    assert (st["recomputed"], st["saturated"]) == (s.stats.recomputed, s.stats.saturated)


@pytest.mark.parametrize("nd,n,w", [(2, 63, 16), (2, 63, 8), (2, 127, 24), (3, 15, 16)])
@pytest.mark.parametrize("mode", [bfp.QCOMP, bfp.NNQCOMP])
def test_fmg_and_ir_bit_exact(nd, n, w, mode):
    """C1: FMG then IR-V steps; the FP64 iterate must match the oracle bit for bit."""
    h, s = make(nd, n, w, mode)
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
    ir_counters_match(h, s)
    if nd == 2 and w >= 16:
        assert mg.accuracy_ratio(nd, xt.cpu().numpy()) <= 1.5


def test_ir_solve_reaches_tolerance():
    h, s = make(2, 255, 16, bfp.QCOMP)
    f = manufactured_rhs(2, 255)
    ft = torch.from_numpy(f).cuda()
    xt = torch.zeros_like(ft)
    # the FP64 residual of A' x has a rounding floor near 5e-12 relative to ||b'|| at h = 1/256
    rep = h.ir_solve(ft, xt, max_iter=30, tol=1e-10)
    assert rep.converged and rep.iterations <= 12
    assert rep.res_inf <= 1e-10 * rep.res0_inf
    uh = mg.discrete_solution(2, 255)
    x = xt.cpu().numpy()
    assert np.abs(x - uh).max() <= 1e-6 * np.abs(uh).max()
    assert mg.accuracy_ratio(2, x) <= 1.001


def test_graph_and_direct_ir_agree():
    hg, _ = make(2, 127, 16, bfp.NNQCOMP, use_graph=1)
    hd, _ = make(2, 127, 16, bfp.NNQCOMP, use_graph=0)
    f = torch.from_numpy(manufactured_rhs(2, 127)).cuda()
    xg, xd = torch.zeros_like(f), torch.zeros_like(f)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        hg.ir_iterate(f, xg, 4)
        hd.ir_iterate(f, xd, 4)
    st.synchronize()
    assert torch.equal(xg, xd)


@pytest.mark.parametrize("nd,n", [(2, 127), (2, 63), (3, 31), (3, 15)])
def test_ir_residual_window_and_padding(nd, n):
    """bfp_ir_residual equals quant(b' - A'x) of the oracle; the qcomp window (gamma =
    previous residual norm) is used from the second call on; padding is zeroed."""
    h, s = make(nd, n, 16, bfp.QCOMP)
    f = manufactured_rhs(nd, n)
    b = s.rhs_hierarchy(f)[0]
    rng = np.random.default_rng(n)
    ft = torch.from_numpy(f).cuda()
    shape = (n,) * nd
    r = bfp.BFPVector(shape, 16)
    x = rng.standard_normal(shape) * 1e-3
    for it in range(4):
        if it == 3:
            x = x * 1e6          # far larger residual: the window overflows, pass 2 recomputes
        xt = torch.from_numpy(x).cuda()
        r.mant.fill_(-5)
        h.ir_residual(ft, xt, r)
        ref = s.ir_quantize(0, mg.residual_f64(b, x))
        torch.cuda.synchronize()
        assert r.exponent == ref.e
        assert np.array_equal(r.mantissas(), ref.m)
        assert np.all(r.padding() == 0)
        x = x + 1e-9 * rng.standard_normal(shape)
    st = h.stats()
    assert st["ir_residuals"] == 4
    assert st["ir_recomputed"] == 2       # the first call (no gamma yet) and the overflowing one
    ir_counters_match(h, s)


@pytest.mark.parametrize("nd,n,w,onchip,step", [(2, 63, 16, 63, 1), (2, 63, 16, 0, 1), (2, 127, 12, 63, 1),
                                                (2, 255, 14, 15, 1), (3, 15, 16, 0, 1),
                                                # wider than 16 bits: int32 fine levels, int16 coarse ones
                                                (2, 63, 20, 63, 1), (2, 127, 24, 63, 2), (2, 255, 32, 15, 3),
                                                (2, 63, 32, 63, 1), (3, 15, 24, 0, 4), (3, 31, 20, 0, 2)])
@pytest.mark.parametrize("mode", [bfp.QCOMP, bfp.NNQCOMP])
def test_progressive_precision_bit_exact(nd, n, w, onchip, step, mode):
    """Level k's ops at w - k w_step bits (the restriction at the finer level's width; storage per
    width, so a level where the width crosses 16 bits mixes int32 and int16 operands); V-cycle,
    FMG and IR steps against the oracle bit for bit, counters included."""
    h, s = make(nd, n, w, mode, coarse_onchip=onchip, w_step=step)
    rm = random_mantissas((n,) * nd, w, 5, "smooth")
    r = bfp.BFPVector.from_mantissas(rm, -18, w)
    y = bfp.BFPVector((n,) * nd, w)
    h.reset_stats()
    h.vcycle(r, y)
    torch.cuda.synchronize()
    ref = s.vcycle(0, B.BFP(rm, -18, w))
    assert y.exponent == ref.e and np.array_equal(y.mantissas(), ref.m)
    st = h.stats()
    assert (st["calls"], st["saturated"]) == (s.stats.calls, s.stats.saturated)
    f = manufactured_rhs(nd, n)
    ft = torch.from_numpy(f).cuda()
    xt = torch.zeros_like(ft)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        h.fmg(ft, xt)
        h.ir_iterate(ft, xt, 2)
    stream.synchronize()
    xr = s.fmg(f)
    b = s.rhs_hierarchy(f)[0]
    for _ in range(2):
        xr = s.ir_step(0, b, xr)
    assert np.array_equal(xt.cpu().numpy(), xr)


def test_progressive_precision_rejects_float_and_wide_variable():
    o = bfp.bfp_solver_opts_default(2, 63, 16)
    o.w_step, o.arith = 1, bfp.ARITH_FP32
    with pytest.raises(bfp.BFPError):
        bfp.Hierarchy(o)
    o = bfp.bfp_solver_opts_default(2, 63, 24)
    o.w_step = 1
    with pytest.raises(bfp.BFPError):
        bfp.Hierarchy(o, k_nodes=np.ones((65, 65)))
    bfp.Hierarchy(bfp.bfp_solver_opts_default(2, 63, 24)).close()


@pytest.mark.parametrize("cap", [0, 2, 4])
@pytest.mark.parametrize("smoother", ["jacobi", "cheby"])
@pytest.mark.parametrize("onchip", [63, 0])
def test_w_add_cap_matches_oracle_counts(cap, smoother, onchip):
    """opts.w_add_max (Table tab:recomputation's experiment): results stay bit-exact (qcomp), and
    the recomputation counters equal the oracle's with the same cap; the finest level's counters
    hold its own ops only."""
    n, w = 127, 16
    o = bfp.bfp_solver_opts_default(2, n, w)
    o.mode = bfp.QCOMP
    o.w_add_max = cap
    o.coarse_onchip = onchip
    o.smoother = bfp.SMOOTH_CHEBY if smoother == "cheby" else bfp.SMOOTH_JACOBI
    h = bfp.Hierarchy(o)
    s = mg.BFPSolver(2, n, w=w, mode="qcomp", omega=o.omega, w_omega=o.w_omega, smoother=smoother,
                     w_add_max=cap)
    rm = random_mantissas((n, n), w, 9, "smooth")
    r = bfp.BFPVector.from_mantissas(rm, -25, w)
    y = bfp.BFPVector((n, n), w)
    h.reset_stats()
    h.vcycle(r, y)
    ref = s.vcycle(0, B.BFP(rm, -25, w))
    torch.cuda.synchronize()
    assert y.exponent == ref.e and np.array_equal(y.mantissas(), np.asarray(ref.m).astype(np.int64))
    st, fin = h.stats(), h.finest_stats()
    assert (st["calls"], st["recomputed"], st["overflow"], st["underflow"]) == (
        s.stats.calls, s.stats.recomputed, s.stats.overflow, s.stats.underflow)
    assert fin["calls"] == (4 if smoother == "cheby" else 7)      # the finest level's own ops
    assert fin["recomputed"] <= st["recomputed"]
    h.close()


def _policy_oracle(s, b, x, steps):
    """The stall fallback of ir_solve restated: before step i, if the residual norm is above half
    the one two steps back, step i and every later step run the V-cycle with qcomp."""
    hist, fb = [-1.0, -1.0], -1
    for it in range(steps):
        rn = float(np.abs(mg.residual_f64(b, x)).max())
        if fb < 0 and hist[1] >= 0 and rn > 0.5 * hist[1]:
            fb = it
        hist = [rn, hist[0]]
        mode = s.mode
        if fb >= 0:
            s.mode = "qcomp"
        x = s.ir_step(0, b, x)
        s.mode = mode
    return x, fb


@pytest.mark.parametrize("w", [8, 6])
def test_ir_solve_stall_fallback_matches_oracle(w):
    """IR-V from zero under nnqcomp first raises the residual (the paper's remark on skipping
    normalisation); the fallback switches the V-cycle to qcomp at the same step as the restated
    policy, and the iterate matches it bit for bit."""
    n, steps = 63, 8
    h, s = make(2, n, w, bfp.NNQCOMP, coarse_onchip=0)
    f = manufactured_rhs(2, n)
    ft = torch.from_numpy(f).cuda()
    xt = torch.zeros_like(ft)
    rep = h.ir_solve(ft, xt, max_iter=steps, tol=0.0, fmg_start=False, stall_fallback=True)
    torch.cuda.synchronize()
    b = s.rhs_hierarchy(f)[0]
    xr, fb = _policy_oracle(s, b, np.zeros_like(b), steps)
    assert rep.fallback_at == fb and fb >= 0
    assert np.array_equal(xt.cpu().numpy(), xr)
    # without the fallback the solve keeps nnqcomp
    xt.zero_()
    rep = h.ir_solve(ft, xt, max_iter=steps, tol=0.0, fmg_start=False)
    assert rep.fallback_at == -1


@pytest.mark.parametrize("mode", [bfp.NNQCOMP, bfp.QCOMP])
def test_benchmarked_ir_steps_4095(mode):
    """The benchmarked workload itself (2D Poisson 4095^2, w = 16, the library's default schedule:
    graph-replayed IR-V(2,2) steps, on-chip coarse cycle from 63 down): two IR-V steps from x = 0
    equal the oracle's FP64 iterate bit for bit (FP64 residual and update, every level's ops, the
    4095 -> 2047 transfers); the next IR residual on its own (the full 4095^2 grid, window from the
    previous residual) equals the oracle's quantisation; the V-cycle and IR counters equal the
    oracle's."""
    n = 4095
    o = bfp.bfp_solver_opts_default(2, n, 16)
    o.mode = mode
    h = bfp.Hierarchy(o)
    s = mg.BFPSolver(2, n, w=16, mode="qcomp" if mode == bfp.QCOMP else "nnqcomp", omega=o.omega,
                     w_omega=o.w_omega)
    f = manufactured_rhs(2, n)
    b = s.rhs_hierarchy(f)[0]
    ft = torch.from_numpy(f).cuda()
    xt = torch.zeros_like(ft)
    stream = torch.cuda.Stream()
    xr = np.zeros_like(f)
    for it in range(2):
        with torch.cuda.stream(stream):
            h.ir_iterate(ft, xt, 1)
        stream.synchronize()
        xr = s.ir_step(0, b, xr)
        assert np.array_equal(xt.cpu().numpy(), xr), it
    st = h.stats()
    assert (st["calls"], st["recomputed"], st["saturated"]) == (s.stats.calls, s.stats.recomputed,
                                                                 s.stats.saturated)
    ir_counters_match(h, s)
    r = bfp.BFPVector((n, n), 16)
    r.mant.fill_(-5)
    h.ir_residual(ft, xt, r)
    ref = s.ir_quantize(0, mg.residual_f64(b, xr))
    torch.cuda.synchronize()
    assert r.exponent == ref.e
    assert np.array_equal(r.mantissas(), ref.m)
    assert np.all(r.padding() == 0)
    ir_counters_match(h, s)
    h.close()


def test_ir_step_3d_255_bit_exact():
    """3D at 255^3 (16.6 M DOF, 7 levels, the seven-point kernels' 3D grids over many planes and
    strips): one IR-V(2,2) step from x = 0 with the default schedule equals the oracle's FP64 iterate
    bit for bit, with the op and IR counters."""
    n = 255
    o = bfp.bfp_solver_opts_default(3, n, 16)
    o.mode = bfp.NNQCOMP
    h = bfp.Hierarchy(o)
    s = mg.BFPSolver(3, n, w=16, mode="nnqcomp", omega=o.omega, w_omega=o.w_omega)
    f = manufactured_rhs(3, n)
    ft = torch.from_numpy(f).cuda()
    xt = torch.zeros_like(ft)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        h.ir_iterate(ft, xt, 1)
    stream.synchronize()
    xr = s.ir_step(0, s.rhs_hierarchy(f)[0], np.zeros_like(f))
    assert np.array_equal(xt.cpu().numpy(), xr)
    st = h.stats()
    assert (st["calls"], st["saturated"]) == (s.stats.calls, s.stats.saturated)
    ir_counters_match(h, s)
    h.close()


@pytest.mark.parametrize("mode", [bfp.NNQCOMP, bfp.QCOMP])
def test_ir_resume_from_saved_iterate(mode):
    """Checkpoint and resume: the whole state of the IR solve is the FP64 iterate.  FMG + 3 IR-V steps,
    x saved to host memory and the hierarchy destroyed; a new hierarchy loads x and runs 3 more steps.
    The result equals FMG + 6 steps in one run bit for bit (the IR residual is quantised by Alg. qcomp,
    whose result does not depend on the window the previous residual set)."""
    n = 127
    f = torch.from_numpy(manufactured_rhs(2, n)).cuda()
    stream = torch.cuda.Stream()
    h, _ = make(2, n, 16, mode)
    x = torch.zeros_like(f)
    with torch.cuda.stream(stream):
        h.fmg(f, x)
        h.ir_iterate(f, x, 6)
    stream.synchronize()
    h.close()
    h1, _ = make(2, n, 16, mode)
    y = torch.zeros_like(f)
    with torch.cuda.stream(stream):
        h1.fmg(f, y)
        h1.ir_iterate(f, y, 3)
    stream.synchronize()
    saved = y.cpu().numpy().copy()                      # the checkpoint
    h1.close()
    h2, _ = make(2, n, 16, mode)
    z = torch.from_numpy(saved).cuda()
    with torch.cuda.stream(stream):
        h2.ir_iterate(f, z, 3)
    stream.synchronize()
    assert torch.equal(z, x)
    h2.close()
