"""Autotuner for the solver's launch schedule.

For each grid side it times graph-replayed IR-V steps over candidate
(tile_rows, coarse_onchip) pairs -- the rows per warp strip of the
row-walking kernels and the first level of the on-chip coarse V-cycle -- and
keeps the fastest.  Timing uses CUDA events on the solver's stream after
warm-up steps.
"""
from __future__ import annotations

import numpy as np

from . import ARITH_BFP, NNQCOMP, Hierarchy, bfp_solver_opts_default


def opts_for(n: int, w: int = 16, mode: int = NNQCOMP, tile_rows: int = 0, coarse_onchip: int = 63,
             arith: int = ARITH_BFP):
    o = bfp_solver_opts_default(2, n, w)
    o.mode = mode
    o.tile_rows = tile_rows
    o.coarse_onchip = coarse_onchip
    o.arith = arith
    return o


def tune(sides, w: int = 16, mode: int = NNQCOMP, rows=(0, 4, 8, 16), onchip=(0, 31, 63, 127), steps: int = 4,
         warmup: int = 2) -> dict:
    """{n: {"tile_rows", "coarse_onchip", "ms_per_step"}} for each distinct side n (2D)."""
    import torch
    stream = torch.cuda.Stream()
    best = {}
    for n in sorted(set(int(s) for s in sides)):
        h_ = 1.0 / (n + 1)
        s1 = np.sin(np.pi * np.arange(1, n + 1) * h_)
        f = torch.from_numpy(2 * np.pi ** 2 * np.outer(s1, s1)).cuda()
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
