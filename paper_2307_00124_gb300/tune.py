"""Autotuner for the solver's launch schedule.

For each grid side it times candidate (tile_rows, coarse_onchip) pairs -- the
rows per warp strip of the row-walking kernels and the first level of the
on-chip coarse V-cycle -- and keeps the fastest.  ``tune`` times
graph-replayed IR-V steps of one hierarchy; ``tune_batch`` times the side's
group the way a batched solve runs it (every op one launch over the group's
instances), FMG plus IR-V steps of up to ``max_group`` instances of that
side.  Timing uses CUDA events on the solver's stream after a warm-up run.
"""
from __future__ import annotations

import numpy as np

from . import ARITH_BFP, NNQCOMP, Batch, Hierarchy, bfp_solver_opts_default


def opts_for(n: int, w: int = 16, mode: int = NNQCOMP, tile_rows: int = 0, coarse_onchip: int = 63,
             arith: int = ARITH_BFP):
    o = bfp_solver_opts_default(2, n, w)
    o.mode = mode
    o.tile_rows = tile_rows
    o.coarse_onchip = coarse_onchip
    o.arith = arith
    return o


def _rhs(torch, n):
    h_ = 1.0 / (n + 1)
    s1 = np.sin(np.pi * np.arange(1, n + 1) * h_)
    return torch.from_numpy(2 * np.pi ** 2 * np.outer(s1, s1)).cuda()


def tune(sides, w: int = 16, mode: int = NNQCOMP, rows=(0, 4, 8, 16), onchip=(0, 31, 63, 127), steps: int = 4,
         warmup: int = 2) -> dict:
    """{n: {"tile_rows", "coarse_onchip", "ms_per_step"}} for each distinct side n (2D), one hierarchy each."""
    import torch
    stream = torch.cuda.Stream()
    best = {}
    for n in sorted(set(int(s) for s in sides)):
        f = _rhs(torch, n)
        for tr in rows:
            for oc in onchip:
                h = Hierarchy(opts_for(n, w, mode, tr, oc))
                x = torch.zeros_like(f)
                with torch.cuda.stream(stream):
                    h.ir_iterate(f, x, warmup)
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    h.ir_iterate(f, x, steps)
                    b.record(stream)
                stream.synchronize()
                ms = a.elapsed_time(b) / steps
                h.close()
                if n not in best or ms < best[n]["ms_per_step"]:
                    best[n] = {"tile_rows": int(tr), "coarse_onchip": int(oc), "ms_per_step": float(ms)}
    return best


def tune_batch(sides, w: int = 16, mode: int = NNQCOMP, rows=(0, 4, 8, 16), onchip=(31, 63, 127),
               ir_steps: int = 2, max_group: int = 16, reps: int = 2) -> dict:
    """{n: {"tile_rows", "coarse_onchip", "ms", "instances"}}: for each distinct side, the candidate
    whose merged group (min(count of that side, max_group) instances, FMG + ir_steps IR-V steps in one
    batched launch) finishes first."""
    import torch
    stream = torch.cuda.Stream()
    counts = {}
    for s in sides:
        counts[int(s)] = counts.get(int(s), 0) + 1
    best = {}
    for n in sorted(counts):
        g = min(counts[n], max_group)
        fs = [_rhs(torch, n) for _ in range(g)]
        xs = [torch.zeros_like(f) for f in fs]
        for tr in rows:
            for oc in onchip:
                b = Batch([opts_for(n, w, mode, tr, oc) for _ in range(g)])
                times = []
                for rep in range(reps + 1):
                    with torch.cuda.stream(stream):
                        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        a.record(stream)
                        b.solve(fs, xs, [ir_steps] * g, fmg=True, stream=stream)
                        e.record(stream)
                    stream.synchronize()
                    if rep:
                        times.append(a.elapsed_time(e))
                b.close()
                ms = min(times)
                if n not in best or ms < best[n]["ms"]:
                    best[n] = {"tile_rows": int(tr), "coarse_onchip": int(oc), "ms": float(ms), "instances": g}
    return best
