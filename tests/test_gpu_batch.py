"""Batched solves: every instance of one graph launch equals the same work done
through a single hierarchy (FMG + IR-V steps), bit for bit, for mixed sizes,
widths, modes and schedules; per-instance times are reported."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2307_00124_gb300 as bfp  # noqa: E402
from bfp_inputs import batch_sizes, smoothed_random_rhs  # noqa: E402
from oracle import mg  # noqa: E402

pytestmark = pytest.mark.gpu


def opts(n, w, mode, tile_rows=0, coarse_onchip=63):
    o = bfp.bfp_solver_opts_default(2, n, w)
    o.mode, o.tile_rows, o.coarse_onchip = mode, tile_rows, coarse_onchip
    return o


def test_batch_matches_single_solves():
    spec = [(63, 16, bfp.NNQCOMP, 0, 63), (127, 16, bfp.QCOMP, 4, 31), (31, 8, bfp.NNQCOMP, 2, 0),
            (255, 16, bfp.NNQCOMP, 8, 127), (63, 24, bfp.QCOMP, 0, 15), (15, 16, bfp.NNQCOMP, 0, 63)]
    olist = [opts(*s) for s in spec]
    ks = [2, 1, 3, 2, 0, 1]
    fs = [torch.from_numpy(smoothed_random_rhs(s[0], 100 + i)).cuda() for i, s in enumerate(spec)]
    xs = [torch.zeros_like(f) for f in fs]
    stream = torch.cuda.Stream()
    b = bfp.Batch(olist)
    for rep in range(2):                       # the second launch replays the captured graph
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            b.solve(fs, xs, ks, fmg=True)
        t = b.times()
        assert all(v > 0 for v in t)
        for i, (o, k) in enumerate(zip(olist, ks)):
            h = bfp.Hierarchy(o)
            xr = torch.zeros_like(fs[i])
            with torch.cuda.stream(stream):
                h.fmg(fs[i], xr)
                h.ir_iterate(fs[i], xr, k)
            stream.synchronize()
            assert torch.equal(xs[i], xr), (rep, i)
            h.close()
    # one instance alone, as its own launch
    x1 = torch.zeros_like(fs[1])
    with torch.cuda.stream(stream):
        b.solve_one(1, fs[1], x1, ks[1], fmg=True)
    stream.synchronize()
    assert torch.equal(x1, xs[1])
    b.close()


def test_batch_instances_reach_tolerance():
    sides = batch_sizes(8, seed=3, sides=(31, 63, 127))
    fs = [torch.from_numpy(smoothed_random_rhs(n, 1000 + i)).cuda() for i, n in enumerate(sides)]
    xs = [torch.zeros_like(f) for f in fs]
    b = bfp.Batch([opts(n, 16, bfp.NNQCOMP) for n in sides])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.solve(fs, xs, [8] * len(sides), fmg=True)
    stream.synchronize()
    for n, f, x in zip(sides, fs, xs):
        bb = mg.scaled_rhs(f.cpu().numpy())
        r = mg.residual_f64(bb, x.cpu().numpy())
        assert np.abs(r).max() <= 1e-8 * np.abs(bb).max()   # about 7x per IR-V step from ~7e-3 after FMG
    b.close()


def test_batch_with_chebyshev_and_progressive_instances():
    """Instances with the paper's V(1,0) (Chebyshev relaxation), progressive widths and a w_add cap
    beside damped-Jacobi ones: each equals its single-hierarchy solve, bit for bit."""
    spec = [(63, 16, bfp.NNQCOMP, 0, 63), (127, 16, bfp.QCOMP, 0, 0), (255, 12, bfp.NNQCOMP, 0, 63)]
    olist = [opts(*s) for s in spec]
    olist[0].smoother = bfp.SMOOTH_CHEBY
    olist[1].smoother = bfp.SMOOTH_CHEBY
    olist[1].w_add_max = 2
    olist[2].w_step = 1
    ks = [3, 2, 1]
    fs = [torch.from_numpy(smoothed_random_rhs(s[0], 200 + i)).cuda() for i, s in enumerate(spec)]
    xs = [torch.zeros_like(f) for f in fs]
    stream = torch.cuda.Stream()
    b = bfp.Batch(olist)
    with torch.cuda.stream(stream):
        b.solve(fs, xs, ks, fmg=True)
    stream.synchronize()
    for i, (o, k) in enumerate(zip(olist, ks)):
        h = bfp.Hierarchy(o)
        xr = torch.zeros_like(fs[i])
        with torch.cuda.stream(stream):
            h.fmg(fs[i], xr)
            h.ir_iterate(fs[i], xr, k)
        stream.synchronize()
        assert torch.equal(xs[i], xr), i
        h.close()
    b.close()


def test_batch_instances_equal_the_oracle():
    """Every instance of one batched launch (mixed sides, widths, modes, strip rows and first on-chip
    levels) equals the oracle's FMG + K IR-V steps for that instance, bit for bit."""
    from oracle import mg as M
    spec = [(255, 16, bfp.NNQCOMP, 8, 127), (127, 16, bfp.QCOMP, 4, 31), (63, 8, bfp.NNQCOMP, 2, 0),
            (31, 16, bfp.QCOMP, 0, 63), (127, 12, bfp.NNQCOMP, 2, 15), (63, 24, bfp.QCOMP, 0, 15)]
    olist = [opts(*sp) for sp in spec]
    ks = [2, 1, 3, 2, 1, 0]
    fh = [smoothed_random_rhs(sp[0], 300 + i) for i, sp in enumerate(spec)]
    fs = [torch.from_numpy(f).cuda() for f in fh]
    xs = [torch.zeros_like(f) for f in fs]
    stream = torch.cuda.Stream()
    b = bfp.Batch(olist)
    with torch.cuda.stream(stream):
        b.solve(fs, xs, ks, fmg=True)
    stream.synchronize()
    for i, (sp, o, k) in enumerate(zip(spec, olist, ks)):
        s = M.BFPSolver(2, sp[0], w=sp[1], mode="qcomp" if sp[2] == bfp.QCOMP else "nnqcomp",
                        omega=o.omega, w_omega=o.w_omega)
        xr = s.fmg(fh[i])
        bb = s.rhs_hierarchy(fh[i])[0]
        for _ in range(k):
            xr = s.ir_step(0, bb, xr)
        assert np.array_equal(xs[i].cpu().numpy(), xr), i
    b.close()


def test_batch_groups_merge_and_equal_the_oracle():
    """Instances with equal options run as one group: each op of the shared schedule is one launch
    over the group's instances still running (different step counts end at different points).
    Every instance equals the oracle's FMG + K IR-V steps bit for bit, and the per-instance end
    times are ordered by step count within a group."""
    from oracle import mg as M
    spec = [(63, 16, bfp.NNQCOMP, 0, 63)] * 3 + [(127, 16, bfp.QCOMP, 4, 31)] * 3 + [(255, 12, bfp.NNQCOMP, 8, 127)] * 2
    ks = [1, 3, 2, 0, 2, 1, 2, 1]
    olist = [opts(*sp) for sp in spec]
    fh = [smoothed_random_rhs(sp[0], 400 + i) for i, sp in enumerate(spec)]
    fs = [torch.from_numpy(f).cuda() for f in fh]
    xs = [torch.zeros_like(f) for f in fs]
    stream = torch.cuda.Stream()
    b = bfp.Batch(olist)
    for rep in range(2):                       # capture, then replay of the captured graph
        for x in xs:
            x.zero_()
        with torch.cuda.stream(stream):
            b.solve(fs, xs, ks, fmg=True)
        stream.synchronize()
        assert b.info() == (3, 0)
        t = b.times()
        assert t[1] >= t[2] >= t[0] and t[4] >= t[5] >= t[3] and t[6] >= t[7]
        for i, (sp, o, k) in enumerate(zip(spec, olist, ks)):
            s = M.BFPSolver(2, sp[0], w=sp[1], mode="qcomp" if sp[2] == bfp.QCOMP else "nnqcomp",
                            omega=o.omega, w_omega=o.w_omega)
            xr = s.fmg(fh[i])
            bb = s.rhs_hierarchy(fh[i])[0]
            for _ in range(k):
                xr = s.ir_step(0, bb, xr)
            assert np.array_equal(xs[i].cpu().numpy(), xr), (rep, i)
    b.close()


@pytest.mark.parametrize("w_wide,info", [(32, (1, 2)), (24, (2, 0))])
def test_batch_without_batched_form_runs_separately(w_wide, info):
    """A group whose schedule has ops without a batched form (int32 mantissas above 30 bits, w = 32,
    which the staged kernels do not take) runs its instances on branches of their own; at w = 24 the
    staged int32 kernels have batched forms and the group merges.  Either way the results equal the
    single-hierarchy solves."""
    spec = [(63, w_wide, bfp.NNQCOMP, 0, 63)] * 2 + [(63, 16, bfp.NNQCOMP, 0, 63)] * 2
    olist = [opts(*sp) for sp in spec]
    fs = [torch.from_numpy(smoothed_random_rhs(sp[0], 500 + i)).cuda() for i, sp in enumerate(spec)]
    xs = [torch.zeros_like(f) for f in fs]
    stream = torch.cuda.Stream()
    b = bfp.Batch(olist)
    with torch.cuda.stream(stream):
        b.solve(fs, xs, [2, 2, 2, 2], fmg=True)
    stream.synchronize()
    assert b.info() == info
    for i, o in enumerate(olist):
        h = bfp.Hierarchy(o)
        xr = torch.zeros_like(fs[i])
        with torch.cuda.stream(stream):
            h.fmg(fs[i], xr)
            h.ir_iterate(fs[i], xr, 2)
        stream.synchronize()
        assert torch.equal(xs[i], xr), i
        h.close()
    b.close()
