#!/usr/bin/env python
"""Benchmark: BFP IR-V steps on the 2D Poisson workload (4095^2 interior points, w = 16).

One step is one iteration of FP64 iterative refinement with a BFP V(2,2)
inner cycle (Alg. ir / v-cycle): FP64 residual r = b' - A'x and its
normalised BFP quantisation, the V-cycle over 11 levels (damped Jacobi,
residual, full-weighting restriction, bilinear correction), and the FP64
update.  Metric: fine-grid DOF x V-cycles per second (GDOF/s), whole job.

Prints ONE JSON line on rank 0.  ``--impl reference`` times the CPU oracle
instead (the exact reference this library is checked against).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

UNIT = "GDOF/s"
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the timed Jacobi kernel version at 4095^2
# from one ncu capture (None until this kernel version has been captured)
JACOBI_TRAFFIC = None


def metric_name(nd, n, w):
    """The metric as run: BFP V-cycle GDOF/s of IR-V steps on the configured grid and width."""
    grid = ("%d^2" % n) if nd == 2 else ("%d^3" % n)
    return "BFP V-cycle GDOF/s (IR-V steps, %dD Poisson %s, w=%d)" % (nd, grid, w)


def levels_of(n):
    out = []
    while n >= 3:
        out.append(n)
        n = (n - 1) // 2
    return out


# Algorithmic bytes per DOF of each op on int16 mantissas (each operand read once, each result
# written once; FP64 x, f are 8 bytes): the V(2,2) schedule of one level is the zero-guess sweep
# (r in, y out), a sweep (y, r in, y out), the residual (y, r in, r_v out), the restriction (fine r_v
# in, coarse out: 2 + 2/2^d), the correction (coarse d in, y in, y out) and two sweeps.
OP_BYTES = {"jacobi0": 4.0, "jacobi": 6.0, "residual": 6.0, "ir_residual": 18.0, "ir_update": 18.0}


def step_bytes(nd, n, mb=2):
    """Algorithmic bytes of one IR-V(2,2) step: every level's V(2,2) ops plus the FP64 IR residual
    (x, f in; BFP r out) and update (x, y in; x out)."""
    total = 0.0
    for m in levels_of(n):
        dof = m ** nd
        cdof = ((m - 1) // 2) ** nd
        lvl = (2 * mb) + 3 * (3 * mb) + (3 * mb)            # zero-guess, three sweeps, residual
        lvl_dof = lvl * dof
        lvl_dof += mb * dof + mb * cdof                      # restriction
        lvl_dof += mb * cdof + 2 * mb * dof                  # correction
        total += lvl_dof
    dof = n ** nd
    total += (16 + mb) * dof + (16 + mb) * dof
    return total


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--mode", default="nnqcomp", choices=["nnqcomp", "qcomp"])
    p.add_argument("--n", type=int, default=4095)
    p.add_argument("--nd", type=int, default=2, choices=[2, 3], help="dimension of the --op problem")
    p.add_argument("--var", action="store_true", help="--op on the variable-coefficient 2D problem")
    p.add_argument("--onchip", type=int, default=None,
                   help="opts.coarse_onchip of the timed hierarchy (default: the library's)")
    p.add_argument("--smoother", default="jacobi", choices=["jacobi", "cheby"],
                   help="--op: the hierarchy's relaxation (cheby: the paper's V(1,0))")
    p.add_argument("--w", type=int, default=16)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-compare", action="store_true", help="skip the float baselines and time to accuracy")
    p.add_argument("--batch", type=int, default=0, help="run the batched-solve measurement with this many instances")
    p.add_argument("--op", default=None, choices=[None, "jacobi", "residual", "restrict", "prolong", "ir_residual",
                                                  "ir_update", "step", "vcycle"],
                   help="run one finest-level op --reps times and exit (profiling driver)")
    p.add_argument("--reps", type=int, default=3)
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.proc:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(t, device):
    """The slowest rank's time (replicas: the job ends with its last rank); t itself at one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def replica_value(ws, units_per_rank, steps, t):
    """Whole-job throughput: the units every rank processed over the slowest rank's time (G/s)."""
    return ws * units_per_rank * steps / t / 1e9


class OracleRun:
    """The CPU oracle (oracle/mg.py, numpy exact integers and FP64) stepping the same workload: IR-V
    steps from x = 0, continuing from the previous iterate like the GPU run."""

    def __init__(self, n, w, mode, nd=2):
        from bfp_inputs import manufactured_rhs
        from oracle import mg
        import numpy as np
        self.s = mg.BFPSolver(nd, n, w=w, mode=mode)
        self.b = self.s.rhs_hierarchy(manufactured_rhs(nd, n))[0]
        self.x = np.zeros_like(self.b)

    def step(self):
        """One IR-V step; returns (wall seconds, process CPU seconds)."""
        w0, c0 = time.perf_counter(), time.process_time()
        self.x = self.s.ir_step(0, self.b, self.x)
        return time.perf_counter() - w0, time.process_time() - c0


def cores_used(wall, cpu):
    """Host cores the timed oracle kept busy: process CPU time over wall time (numpy's elementwise
    kernels run on one thread; no threaded BLAS is on this path)."""
    return max(1, int(round(cpu / wall))) if wall > 0 else 1


def run_reference(args):
    ws, rank, _ = dist_init(args)
    if rank != 0:
        return
    # the oracle on the host cores, on the same workload as the GPU arm: each step is one IR-V step
    # of the 4095^2 (or --n) problem
    n = args.n
    o = OracleRun(n, args.w, args.mode)
    wall, cpu = 0.0, 0.0
    for i in range(args.warmup + args.steps):
        tw, tc = o.step()
        if i >= args.warmup:
            wall += tw
            cpu += tc
    dof = n * n
    value = dof * args.steps / wall / 1e9
    line = {
        "impl": "reference", "metric": metric_name(2, n, args.w), "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int16+f64",
        "data": "synthetic", "config": {"workload": "2D Poisson 5-point, %dx%d interior, FP64 IR with BFP V(2,2) "
                                                    "damped Jacobi omega=4/5, w=%d, %s" % (n, n, args.w, args.mode),
                                        "sample": "the full %d^2 grid: one oracle IR-V step per step" % n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores_used(wall, cpu), "kind": "oracle",
                         "sample": "%d IR-V steps of the %d^2 workload after %d untimed" % (args.steps, n,
                                                                                           args.warmup)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _energy_gpu(torch, e):
    """e^T A_h e / h^(d-2)-free form: sum over points of e (2d e - sum of neighbours), zero boundary
    (the discrete energy norm squared up to the common factor h^(d-2))."""
    nd = e.dim()
    p = torch.nn.functional.pad(e, (1, 1) * nd)
    inner = tuple(slice(1, -1) for _ in range(nd))
    ae = (2.0 * nd) * e
    for ax in range(nd):
        for d in (-1, 1):
            sl = list(inner)
            sl[ax] = slice(1 + d, p.shape[ax] - 1 + d)
            ae = ae - p[tuple(sl)]
    return float((e * ae).sum())


def discrete_solution_gpu(torch, nd, n, device):
    """u = prod sin(pi x_i) and the closed-form discrete solution u_h = (d pi^2 / lambda_h) u
    (u is an eigenvector of A_h, lambda_h = 4 d sin^2(pi h / 2) / h^2)."""
    import math
    h = 1.0 / (n + 1)
    s = torch.sin(math.pi * torch.arange(1, n + 1, dtype=torch.float64, device=device) * h)
    u = s
    for _ in range(nd - 1):
        u = u.unsqueeze(0) * s.reshape((n,) + (1,) * u.dim())
    lam = 4.0 * nd * math.sin(math.pi * h / 2) ** 2 / h ** 2
    return u, (nd * math.pi ** 2 / lam) * u


def accuracy_ratio_gpu(torch, x, n):
    """||u - x||_L / ||u - u_h||_L in the discrete energy norm (e^T A_h e)^(1/2), u = prod sin(pi x_i)
    and u_h its closed-form discrete solution (measurement only, outside every timed region)."""
    import math
    u, uh = discrete_solution_gpu(torch, x.dim(), n, x.device)
    return math.sqrt(_energy_gpu(torch, u - x) / _energy_gpu(torch, u - uh))


def error_vs_discrete(torch, x, n):
    """||x - u_h||_A / ||u_h||_A: the solver's error against the exact discrete solution (the
    solution an FP64 multigrid converges to), relative, in the energy norm."""
    import math
    _, uh = discrete_solution_gpu(torch, x.dim(), n, x.device)
    return math.sqrt(_energy_gpu(torch, x - uh) / _energy_gpu(torch, uh))


def var_compare(bfp, torch, stream, n=2047, steps=10):
    """The variable-coefficient workload (-div(k grad u) = f on 2047^2, k = exp(GRF seed 1), RHS seed 2
    smoothed): IR-V step throughput, and time to discretisation accuracy at w = 16 and w = 24 (FMG + K IR-V
    steps, K the smallest with ||u_h - x||_A <= 0.5 ||u_h - P u_2h||_A; u_h, u_2h from FMG + 100 IR-V steps at
    w = 24, qcomp).  The energy norms are measurement only, outside every timed region."""
    import math
    import numpy as np
    from bfp_inputs import grf_nodes, smoothed_random_rhs
    K = grf_nodes(n, seed=1)
    f_host = smoothed_random_rhs(n, 2)
    f = torch.from_numpy(f_host).cuda()
    Kt = torch.from_numpy(K).cuda()

    def faces(Kn):
        def hm(a, b):
            return ((2.0 * a) * b) / (a + b)
        c = Kn[1:-1, 1:-1]
        return hm(Kn[1:-1, :-2], c), hm(c, Kn[1:-1, 2:]), hm(Kn[:-2, 1:-1], c), hm(c, Kn[2:, 1:-1])
    fw, fe, fs, fn = faces(Kt)

    def energy(e):
        p = torch.nn.functional.pad(e, (1, 1, 1, 1))
        ae = (fw + fe + fs + fn) * e - (fw * p[1:-1, :-2] + fe * p[1:-1, 2:] + fs * p[:-2, 1:-1] + fn * p[2:, 1:-1])
        return math.sqrt(max(float((e * ae).sum()), 0.0))

    def hier(nn, w, mode, Kn):
        o = bfp.bfp_solver_opts_default(2, nn, w)
        o.mode = mode
        return bfp.Hierarchy(o, k_nodes=Kn)

    # reference discrete solutions on the grid and on the next coarser one
    nc = (n - 1) // 2
    bprime = torch.from_numpy(f_host * (1.0 / (n + 1)) ** 2).cuda()
    bc = torch.zeros((nc, nc), dtype=torch.float64, device="cuda")
    for dj in (-1, 0, 1):                                   # b'_2h = R~ b'_h (full weighting, P^T)
        for di in (-1, 0, 1):
            wgt = (2 - abs(dj)) * (2 - abs(di)) * 0.25
            bc += wgt * bprime[1 + dj:1 + dj + 2 * nc:2, 1 + di:1 + di + 2 * nc:2]
    fc = bc / (1.0 / (nc + 1)) ** 2
    href, hc = hier(n, 24, bfp.QCOMP, K), hier(nc, 24, bfp.QCOMP, K[::2, ::2])
    uh, uc = torch.zeros_like(f), torch.zeros_like(fc)
    with torch.cuda.stream(stream):
        href.fmg(f, uh)
        href.ir_iterate(f, uh, 100)
        hc.fmg(fc, uc)
        hc.ir_iterate(fc, uc, 100)
    stream.synchronize()
    href.close()
    hc.close()
    # bilinear P u_2h: fine index 2I+1 on coarse I, fine 2I halfway between I-1 and I (zero outside)
    pc = torch.nn.functional.pad(uc, (1, 1, 1, 1))
    tx = torch.zeros((nc + 2, n), dtype=torch.float64, device="cuda")
    tx[:, 1::2] = pc[:, 1:-1]
    tx[:, 0::2] = 0.5 * (pc[:, :-1] + pc[:, 1:])
    pu = torch.zeros_like(f)
    pu[1::2, :] = tx[1:-1, :]
    pu[0::2, :] = 0.5 * (tx[:-1, :] + tx[1:, :])
    disc = energy(uh - pu)
    out = {"workload": "-div(k grad u) = f, 2047^2, k = exp(GRF, 64 modes, |k_x|,|k_y| <= 8, sigma 1, seed 1), "
                       "RHS uniform seed 2 smoothed, nnqcomp, FMG + IR-V"}
    for w in (16, 24):
        h = hier(n, w, bfp.NNQCOMP, K)
        x = torch.zeros_like(f)
        with torch.cuda.stream(stream):
            h.ir_iterate(f, x, 3)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.ir_iterate(f, x, steps)
            b.record(stream)
        stream.synchronize()
        ms = a.elapsed_time(b) / steps
        x.zero_()
        with torch.cuda.stream(stream):
            h.fmg(f, x)
        stream.synchronize()
        k, ratio = 0, energy(uh - x) / disc
        while ratio > 0.5 and k < 40:
            with torch.cuda.stream(stream):
                h.ir_iterate(f, x, 1)
            stream.synchronize()
            k += 1
            ratio = energy(uh - x) / disc
        times = []
        for _ in range(3):
            x.zero_()
            with torch.cuda.stream(stream):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                h.fmg(f, x)
                if k:
                    h.ir_iterate(f, x, k)
                b.record(stream)
            stream.synchronize()
            times.append(a.elapsed_time(b))
        out["w%d" % w] = {"ir_step_ms": ms, "GDOF/s": n * n / ms / 1e6, "ir_steps_after_fmg": k,
                          "error_ratio": ratio, "reached": bool(ratio <= 0.5), "time_to_accuracy_ms": min(times)}
        h.close()
    return out


def width_sweep(bfp, torch, args, f, stream, steps=10):
    """The 4095^2 workload at mantissa widths 4 ... 32 (int16 storage up to 16, int32 above): IR-V step
    throughput, and the accuracy ratio after FMG and after one more IR-V step, for nnqcomp (FMG's saturation /
    truncation heuristic) and qcomp (renormalising ops); plus progressive precision (w = 16, 24, 32 on the finest
    level, one bit fewer per coarser level; int32 fine levels and int16 coarse ones above 16 bits)."""
    n = args.n
    dof = n * n
    out = []
    cases = [(w, m, 0) for w in (4, 8, 12, 16, 24, 32) for m in ("nnqcomp", "qcomp")] + \
        [(16, "nnqcomp", 1), (24, "nnqcomp", 1), (32, "nnqcomp", 1)]
    for w, m, step in cases:
        o = bfp.bfp_solver_opts_default(2, n, w)
        o.mode = bfp.NNQCOMP if m == "nnqcomp" else bfp.QCOMP
        o.w_step = step
        try:
            h = bfp.Hierarchy(o)
        except bfp.BFPError as exc:   # a configuration the library refuses is reported, not fatal
            out.append({"w": w, "mode": m, "w_step": step, "error": str(exc)})
            continue
        x = torch.zeros_like(f)
        with torch.cuda.stream(stream):
            h.ir_iterate(f, x, 3)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.ir_iterate(f, x, steps)
            b.record(stream)
        stream.synchronize()
        ms = a.elapsed_time(b) / steps
        x.zero_()
        with torch.cuda.stream(stream):
            h.fmg(f, x)
        stream.synchronize()
        r0 = accuracy_ratio_gpu(torch, x, n)
        with torch.cuda.stream(stream):
            h.ir_iterate(f, x, 1)
        stream.synchronize()
        r1 = accuracy_ratio_gpu(torch, x, n)
        out.append({"w": w, "mode": m, "w_step": step, "ir_step_ms": ms, "GDOF/s": dof / ms / 1e6,
                    "ratio_after_fmg": r0, "ratio_after_fmg_plus_1": r1})
        h.close()
    return out


def bfp_ir_compare(bfp, torch, args, stream, sizes=(1023, 2047, 4095), widths=(32, 40), steps=10):
    """IR with BFP x and b' (bfp_ir_iterate_bfp: qgemv residual at the inner width, V-cycle, qsub at x's
    width w_x; b' quantised to w_x bits, int64 storage above 32) beside the FP64-residual IR on the same
    hierarchy, per grid size: ms per IR-V step, and IR-V steps and ms from x = 0 to the accuracy ratio <= 1.5
    (at most 30 steps).  The floor quantisation of the iterate leaves an energy-norm error of about
    0.26 ulp / h, above the discretisation error at h = 1/4096 for w_x = 32."""
    from bfp_inputs import manufactured_rhs
    out = []
    for n in sizes:
        f = torch.from_numpy(manufactured_rhs(2, n)).cuda()
        o = bfp.bfp_solver_opts_default(2, n, args.w)
        o.mode = bfp.NNQCOMP if args.mode == "nnqcomp" else bfp.QCOMP
        h = bfp.Hierarchy(o)
        bp = f * h.rhs_scale()
        xd = torch.zeros_like(f)
        with torch.cuda.stream(stream):
            h.ir_iterate(f, xd, 4)
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.ir_iterate(f, xd, steps)
            c.record(stream)
        stream.synchronize()
        fp64_ms = a.elapsed_time(c) / steps

        def to_accuracy(step, reset, read):
            k, ratio, best = 0, float("inf"), float("inf")
            reset()
            while ratio > 1.5 and k < 30:
                with torch.cuda.stream(stream):
                    step(1)
                    read()
                stream.synchronize()
                k += 1
                ratio = accuracy_ratio_gpu(torch, xd, n)
                best = min(best, ratio)
            times = []
            for _ in range(3):
                reset()
                with torch.cuda.stream(stream):
                    a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    step(k)
                    c.record(stream)
                stream.synchronize()
                times.append(a.elapsed_time(c))
            return {"ir_steps": k, "ms": min(times), "accuracy_ratio": ratio, "best_ratio": best,
                    "reached": bool(ratio <= 1.5)}

        fp64 = to_accuracy(lambda k: h.ir_iterate(f, xd, k), lambda: xd.zero_(), lambda: None)
        for wx in widths:
            b = bfp.BFPVector((n, n), wx)
            x = bfp.BFPVector((n, n), wx)
            with torch.cuda.stream(stream):
                bfp.bfp_from_f64(bp, b, stream)
                h.ir_iterate_bfp(b, x, 4)
                a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                h.ir_iterate_bfp(b, x, steps)
                c.record(stream)
            stream.synchronize()

            def reset():
                x.mant.zero_()
                x.meta.zero_()
                xd.zero_()
            row = {"n": n, "w_inner": args.w, "w_x": wx, "w_b": wx, "mode": args.mode,
                   "bfp_ir_step_ms": a.elapsed_time(c) / steps, "fp64_ir_step_ms": fp64_ms,
                   "bfp_from_zero": to_accuracy(lambda k: h.ir_iterate_bfp(b, x, k), reset,
                                                lambda: bfp.bfp_to_f64(x, xd, stream)),
                   "fp64_from_zero": fp64}
            out.append(row)
        h.close()
    return out


def recompute_table(bfp, torch, args, f, stream):
    """The analogue of Table tab:recomputation on this workload: qcomp calls that recomputed (the
    w_tmp window from gamma overflowed or underflowed) during one BFP-FMG (N = 2) on the finest level,
    with w_tmp = w_out + min(w_add*, w_add_max), for w_add_max in {inf, 4, 2, 0}; the damped-Jacobi
    V(2,2) and the paper's Chebyshev V(1,0).  Counts cover the V-cycle ops, the FMG interpolation and
    the IR residual (FP64, quantised by qcomp with the previous residual as gamma)."""
    n = args.n
    rows = []
    for smoother in ("jacobi", "cheby"):
        for cap in (-1, 4, 2, 0):
            o = bfp.bfp_solver_opts_default(2, n, args.w)
            o.mode = bfp.QCOMP
            o.w_add_max = cap
            o.smoother = bfp.SMOOTH_CHEBY if smoother == "cheby" else bfp.SMOOTH_JACOBI
            h = bfp.Hierarchy(o)
            x = torch.zeros_like(f)
            h.reset_stats(stream)
            with torch.cuda.stream(stream):
                h.fmg(f, x)
            stream.synchronize()
            fin, tot = h.finest_stats(stream), h.stats(stream)
            rows.append({"smoother": smoother, "w_add_max": None if cap < 0 else cap,
                         "finest": {"recomputed": fin["recomputed"] + fin["ir_recomputed"],
                                    "qcomp_calls": fin["calls"] + fin["ir_residuals"],
                                    "ir_residual_recomputed": fin["ir_recomputed"]},
                         "all_levels": {"recomputed": tot["recomputed"] + tot["ir_recomputed"],
                                        "qcomp_calls": tot["calls"] + tot["ir_residuals"]}})
            h.close()
    return rows


def c1_time_to_accuracy(bfp, torch, stream, w=16, n=63):
    """The small 2D configuration (63^2, w = 16, V(2,2), 5 levels): FMG + K IR-V steps, K the smallest
    with accuracy ratio <= 1.5, timed on the GPU (one graph per IR step; best of 20) and by the CPU
    oracle (same schedule, same result bit for bit; one host thread)."""
    import numpy as np
    from bfp_inputs import manufactured_rhs
    from oracle import mg
    fh = manufactured_rhs(2, n)
    f = torch.from_numpy(fh).cuda()
    o = bfp.bfp_solver_opts_default(2, n, w)
    o.mode = bfp.NNQCOMP
    h = bfp.Hierarchy(o)
    x = torch.zeros_like(f)
    with torch.cuda.stream(stream):
        h.fmg(f, x)
    stream.synchronize()
    k, ratio = 0, accuracy_ratio_gpu(torch, x, n)
    while ratio > 1.5 and k < 20:
        with torch.cuda.stream(stream):
            h.ir_iterate(f, x, 1)
        stream.synchronize()
        k += 1
        ratio = accuracy_ratio_gpu(torch, x, n)
    times = []
    for _ in range(20):
        x.zero_()
        with torch.cuda.stream(stream):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.fmg(f, x)
            if k:
                h.ir_iterate(f, x, k)
            b.record(stream)
        stream.synchronize()
        times.append(a.elapsed_time(b))
    h.close()
    s = mg.BFPSolver(2, n, w=w, mode="nnqcomp", omega=o.omega, w_omega=o.w_omega)
    t0 = time.perf_counter()
    xr = s.fmg(fh)
    bb = s.rhs_hierarchy(fh)[0]
    for _ in range(k):
        xr = s.ir_step(0, bb, xr)
    t_cpu = time.perf_counter() - t0
    return {"workload": "2D Poisson 63^2, w=%d, nnqcomp, V(2,2), 5 levels" % w, "ir_steps_after_fmg": k,
            "accuracy_ratio": ratio, "gpu_ms": min(times), "oracle_ms": 1e3 * t_cpu, "oracle_cores": 1,
            "bit_exact_with_oracle": bool(np.array_equal(x.cpu().numpy(), xr))}


def solver_compare(bfp, torch, args, f, stream, hbfp):
    """Float baselines beside the BFP solver on the same workload: GDOF/s of IR-V steps, and time to
    discretisation accuracy (FMG + K IR-V steps, K the smallest with accuracy ratio <= 1.5)."""
    n, nd = args.n, args.nd
    dof = n ** nd
    out, tta = {}, {}
    for name, arith in (("bfp", bfp.ARITH_BFP), ("fp32", bfp.ARITH_FP32), ("bf16", bfp.ARITH_BF16),
                        ("bfp_cheby_v10", bfp.ARITH_BFP)):
        if name == "bfp":
            h = hbfp
        else:
            o = bfp.bfp_solver_opts_default(nd, n, args.w)
            o.arith = arith
            if name == "bfp_cheby_v10":      # the paper's V(1,0) with two Chebyshev steps per relaxation
                o.smoother = bfp.SMOOTH_CHEBY
                o.mode = bfp.NNQCOMP if args.mode == "nnqcomp" else bfp.QCOMP
            h = bfp.Hierarchy(o)
        x = torch.zeros_like(f)
        if name != "bfp":
            with torch.cuda.stream(stream):
                h.ir_iterate(f, x, 3)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                h.ir_iterate(f, x, args.steps)
                b.record(stream)
            stream.synchronize()
            t = a.elapsed_time(b) / 1e3
            out[name] = {"value": dof * args.steps / t / 1e9, "unit": "GDOF/s", "ms_per_step": 1e3 * t / args.steps}
        # K: IR-V steps after FMG until the accuracy ratio is <= 1.5 (at most 20; 40 for V(1,0))
        x.zero_()
        with torch.cuda.stream(stream):
            h.fmg(f, x)
        stream.synchronize()
        k, ratio = 0, accuracy_ratio_gpu(torch, x, n)
        while ratio > 1.5 and k < (40 if name == "bfp_cheby_v10" else 20):
            with torch.cuda.stream(stream):
                h.ir_iterate(f, x, 1)
            stream.synchronize()
            k += 1
            ratio = accuracy_ratio_gpu(torch, x, n)
        times = []
        for _ in range(3):
            x.zero_()
            with torch.cuda.stream(stream):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                h.fmg(f, x)
                if k:
                    h.ir_iterate(f, x, k)
                b.record(stream)
            stream.synchronize()
            times.append(a.elapsed_time(b))
        tta[name] = {"ms": min(times), "ir_steps_after_fmg": k, "accuracy_ratio": ratio,
                     "reached": bool(ratio <= 1.5), "error_vs_discrete_solution": error_vs_discrete(torch, x, n)}
        if h is not hbfp:
            h.close()
    return out, tta


def e2e_run(bfp, torch, o, h, f_host, stream, ws, dof, k2):
    """IR-V steps of two independent problems, alternating, through the public API with pinned host
    buffers: every step copies its f and x to the device, runs one IR-V step and copies x back.  Each
    problem has its own hierarchy and stream, so one problem's copies overlap the other's step (both
    directions of the host link in use).  Also the link's own copy rate, one direction at a time."""
    h2 = bfp.Hierarchy(o)
    hs = [h, h2]
    streams = [stream, torch.cuda.Stream()]
    fh = [torch.from_numpy(f_host).pin_memory(), torch.from_numpy(f_host * 0.5).pin_memory()]
    xh = [torch.zeros_like(fh[0]).pin_memory(), torch.zeros_like(fh[0]).pin_memory()]
    fd = [torch.empty(f_host.shape, dtype=torch.float64, device="cuda") for _ in range(2)]
    xd = [torch.empty_like(fd[0]) for _ in range(2)]

    def step(i):
        p, st = i % 2, streams[i % 2]
        with torch.cuda.stream(st):
            fd[p].copy_(fh[p], non_blocking=True)
            xd[p].copy_(xh[p], non_blocking=True)
            hs[p].ir_iterate(fd[p], xd[p], 1)
            xh[p].copy_(xd[p], non_blocking=True)

    for i in range(4):                    # warm-up (the second hierarchy captures its graph)
        step(i)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(streams[0])
    streams[1].wait_event(a)
    for i in range(k2):
        step(i)
    streams[0].wait_stream(streams[1])
    b.record(streams[0])
    torch.cuda.synchronize()
    te = a.elapsed_time(b) / 1e3

    def copy_rate(dst, src):
        with torch.cuda.stream(stream):
            dst.copy_(src, non_blocking=True)
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            for _ in range(3):
                dst.copy_(src, non_blocking=True)
            c1.record(stream)
        stream.synchronize()
        return 3 * src.numel() * src.element_size() / (c0.elapsed_time(c1) / 1e3) / 1e9

    link = {"h2d_GBps": copy_rate(fd[0], fh[0]), "d2h_GBps": copy_rate(xh[0], xd[0])}
    h2.close()
    return {"value": ws * dof * k2 / te / 1e9, "unit": UNIT, "h2d_bytes_per_step": 2 * 8 * dof,
            "d2h_bytes_per_step": 8 * dof, "ms_per_step": 1e3 * te / k2, "steps": k2,
            "schedule": "two independent problems alternating on two streams (copies of one overlap the "
                        "other's IR-V step)", "link": link}


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_init(args)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2307_00124_gb300 as bfp
    from bfp_inputs import manufactured_rhs

    nd, n, w = args.nd, args.n, args.w
    mode = bfp.NNQCOMP if args.mode == "nnqcomp" else bfp.QCOMP
    o = bfp.bfp_solver_opts_default(nd, n, w)
    o.mode = mode
    if args.onchip is not None:
        o.coarse_onchip = args.onchip
    h = bfp.Hierarchy(o)
    f_host = manufactured_rhs(nd, n)
    f = torch.from_numpy(f_host).cuda()
    x = torch.zeros_like(f)
    stream = torch.cuda.Stream()
    dof = n ** nd

    # warm-up (the first call captures one IR step into a CUDA graph)
    l0 = bfp.bfp_kernel_launches()
    with torch.cuda.stream(stream):
        h.ir_iterate(f, x, 1)
    stream.synchronize()
    launches_per_step = bfp.bfp_kernel_launches() - l0
    with torch.cuda.stream(stream):
        h.ir_iterate(f, x, max(args.warmup - 1, 0))
    stream.synchronize()

    # timed region: inputs (4 x 134 MB of FP64 plus 33 MB BFP levels) exceed the 129 MB L2
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        h.ir_iterate(f, x, args.steps)
        e1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    clocks = clk.stop()
    t = e0.elapsed_time(e1) / 1e3
    h.reset_stats()
    with torch.cuda.stream(stream):
        h.ir_iterate(f, x, 2)
    stream.synchronize()
    op_stats = h.stats()
    t = max_over_ranks(t, "cuda")
    value = replica_value(ws, dof, args.steps, t)

    h_levels = levels_of(n)
    # roofline: the finest-level kernels timed alone with CUDA events on their stream; each op rotates
    # over three buffer sets so that its inputs are not in L2 when it runs (3 x 100 MB at 4095^2)
    hbm, peak_kind = peaks()
    A = bfp.bfp_laplace_stencil(nd, o.omega, o.w_omega)
    rng = np.random.default_rng(0)
    ym = rng.integers(-(1 << 12), 1 << 12, size=(n,) * nd)
    nsets = 3 if nd == 2 else 1                 # a 3D vector alone exceeds L2
    sets = []
    for i in range(nsets):
        sets.append((bfp.BFPVector.from_mantissas(np.roll(ym, i), -20, w),
                     bfp.BFPVector.from_mantissas(np.roll(ym[::-1], i).copy(), -19, w),
                     bfp.BFPVector((n,) * nd, w)))
    q = bfp.q(w, mode)
    reps = 30
    kern = {}

    def timeit(fn, bufs=None):
        bufs = sets if bufs is None else bufs
        with torch.cuda.stream(stream):
            for i in range(3):
                fn(bufs[i % nsets])
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for i in range(reps):
                fn(bufs[i % nsets])
            b.record(stream)
        stream.synchronize()
        return a.elapsed_time(b) / 1e3 / reps

    mb = 2 if w <= 16 else 4
    scale = mb / 2.0
    kern["jacobi"] = (timeit(lambda v: bfp.bfp_jacobi(A, v[0], v[1], v[2], q, stream=stream)),
                      OP_BYTES["jacobi"] * scale * dof)
    kern["jacobi0"] = (timeit(lambda v: bfp.bfp_jacobi(A, None, v[1], v[2], q, stream=stream)),
                       OP_BYTES["jacobi0"] * scale * dof)
    kern["residual"] = (timeit(lambda v: bfp.bfp_residual(A, v[0], v[1], v[2], q, stream=stream)),
                        OP_BYTES["residual"] * scale * dof)
    kern["ir_residual"] = (timeit(lambda v: h.ir_residual(f, x, v[2], stream=stream)), (16 + mb) * dof)
    kern["ir_update"] = (timeit(lambda v: bfp.bfp_ir_update(x, v[0], stream=stream)), (16 + mb) * dof)
    # context for the sweep's fraction: torch's elementwise int16 add over arrays of the sweep's shape
    # moves the same bytes (two reads, one write) with no stencil, timed the same way
    tsets = [tuple(torch.randint(-4096, 4096, (n, sets[0][2].ld), dtype=torch.int16, device="cuda")
                   for _ in range(3)) for _ in range(nsets)] if nd == 2 else None
    t_add = timeit(lambda v: torch.add(v[0], v[1], out=v[2]), tsets) if nd == 2 else None
    sets_ld = sets[0][2].ld
    del sets, tsets
    kern_out = {k: {"ms": 1e3 * v[0], "algorithmic_bytes": v[1], "GBps": v[1] / v[0] / 1e9,
                    "frac": v[1] / v[0] / 1e9 / hbm} for k, v in kern.items()}
    # the dominant kernel by share of the step's device time (ncu launch list): the finest-level
    # damped-Jacobi sweep; traffic = dram bytes read + written per launch from one ncu capture of
    # this kernel version, None when not captured
    dom = "jacobi"
    sb = step_bytes(nd, n, mb)
    roof = {"bound": "hbm", "kernel": dom, "achieved": kern_out[dom]["GBps"], "peak": hbm, "unit": "GB/s",
            "frac": kern_out[dom]["GBps"] / hbm, "peak_kind": peak_kind,
            "traffic": JACOBI_TRAFFIC if (nd, n, w) == (2, 4095, 16) else None,
            "timing": "CUDA events over %d launches alone on the op's stream, inputs rotated over %d buffer "
                      "sets (larger than L2)" % (reps, nsets),
            "context": None if t_add is None else {
                "what": "torch int16 add (two reads, one write) of arrays of the sweep's shape, timed the same way",
                "GBps": 3 * 2 * n * sets_ld / t_add / 1e9, "frac": 3 * 2 * n * sets_ld / t_add / 1e9 / hbm},
            "step": {"algorithmic_bytes": sb, "ms": 1e3 * t / args.steps,
                     "achieved": sb / (t / args.steps) / 1e9, "frac": sb / (t / args.steps) / 1e9 / hbm}}

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        e2e = e2e_run(bfp, torch, o, h, f_host, stream, ws, dof, max(4, args.steps // 2))

    floats, tta, var, sweep, irb, rtab, c1 = None, None, None, None, None, None, None
    if rank == 0 and not args.no_compare:
        floats, tta = solver_compare(bfp, torch, args, f, stream, h)
        sweep = width_sweep(bfp, torch, args, f, stream) if nd == 2 else None
        var = var_compare(bfp, torch, stream) if nd == 2 else None
        irb = bfp_ir_compare(bfp, torch, args, stream) if nd == 2 else None
        rtab = recompute_table(bfp, torch, args, f, stream) if nd == 2 else None
        c1 = c1_time_to_accuracy(bfp, torch, stream)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        try:
            ns = n if nd == 2 else min(n, 255)     # 3D: a 255^3 grid of the same problem (per-DOF rate)
            orc = OracleRun(ns, w, args.mode, nd)
            nst, wall, cpu_s = 0, 0.0, 0.0
            while nst < 3 and wall < 20.0:         # a bounded sample: up to 3 IR-V steps, ~10-20 s
                tw, tc = orc.step()
                nst, wall, cpu_s = nst + 1, wall + tw, cpu_s + tc
            cpu = {"value": ns ** nd * nst / wall / 1e9, "unit": UNIT, "cores": cores_used(wall, cpu_s),
                   "kind": "oracle", "sample": "%d IR-V steps of the %s problem from x = 0 (numpy "
                                               "exact-integer oracle, %.1f s)%s" % (
                                                   nst, "x".join([str(ns)] * nd), wall,
                                                   "" if ns == n else "; GDOF/s per DOF of that grid")}
        except Exception as exc:  # the oracle is a reported baseline, never the product path
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": "failed: %s" % exc}

    if rank == 0:
        line = {
            "metric": metric_name(nd, n, w), "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int16+f64" if w <= 16 else "int32+f64",
            "data": "synthetic",
            "config": {"workload": ("2D Poisson 5-point, %dx%d interior, FP64 IR with BFP V(2,2) damped Jacobi "
                                    "omega=4/5, %d levels, w=%d, %s" % (n, n, len(h_levels), w, args.mode)) if nd == 2
                       else ("3D Poisson 7-point, %dx%dx%d interior, FP64 IR with BFP V(2,2) damped Jacobi "
                             "omega=6/7, %d levels, w=%d, %s" % (n, n, n, len(h_levels), w, args.mode)),
                       "l2": "inputs larger than L2 (x, f: %d MB each)" % (8 * dof // 10 ** 6),
                       "parallelism": "replicas" if ws > 1
                       else "single GPU"},
            "roofline": roof, "kernels": kern_out, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": int(launches_per_step * args.steps),
            "op_stats_2_steps": op_stats,
            "float_baselines": floats, "time_to_accuracy": tta, "width_sweep": sweep,
            "variable_coefficients": var, "bfp_ir": irb, "recomputations": rtab, "c1_small": c1,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    h.close()


def run_batch(args):
    """Independent instances of uneven sizes (sides drawn from {127, 255, 511, 1023}), each solved by FMG
    + K_i IR-V steps, K_i the smallest step count that brings ||b' - A'x||_inf <= 1e-8 ||b'||_inf;
    all instances in one graph launch, against one launch per instance.  Schedules come from the
    autotuner (per side: rows per warp strip, first on-chip coarse level)."""
    import math
    import time as _time
    import torch
    import paper_2307_00124_gb300 as bfp
    from paper_2307_00124_gb300.tune import opts_for, tune_batch
    from bfp_inputs import batch_sizes, smoothed_random_rhs

    mode = bfp.NNQCOMP if args.mode == "nnqcomp" else bfp.QCOMP
    count = args.batch
    sides = batch_sizes(count, seed=3)
    t0 = _time.perf_counter()
    tuned = tune_batch(sides, w=args.w, mode=mode)
    t_tune = _time.perf_counter() - t0
    olist = [opts_for(n, args.w, mode, tuned[n]["tile_rows"], tuned[n]["coarse_onchip"]) for n in sides]
    b = bfp.Batch(olist)
    fs = [torch.from_numpy(smoothed_random_rhs(n, 1000 + i)).cuda() for i, n in enumerate(sides)]
    xs = [torch.zeros_like(f) for f in fs]
    stream = torch.cuda.Stream()
    tol = 1e-8

    def relres(f, x, n):
        h = 1.0 / (n + 1)
        bb = f * (h * h / 4.0)
        p = torch.nn.functional.pad(x, (1, 1, 1, 1))
        r = bb - (x - 0.25 * (p[1:-1, :-2] + p[1:-1, 2:] + p[:-2, 1:-1] + p[2:, 1:-1]))
        return float(r.abs().max() / bb.abs().max())

    K = [None] * count
    for k in range(0, 31):
        for x in xs:
            x.zero_()
        with torch.cuda.stream(stream):
            b.solve(fs, xs, [k] * count, fmg=True)
        stream.synchronize()
        for i in range(count):
            if K[i] is None and relres(fs[i], xs[i], sides[i]) <= tol:
                K[i] = k
        if all(v is not None for v in K):
            break
    K = [30 if v is None else v for v in K]
    dof = sum(n * n for n in sides)

    def pct(v, q):
        v = sorted(v)
        return v[min(len(v) - 1, int(math.ceil(q * len(v))) - 1)]

    best, inst = None, None
    t1 = _time.perf_counter()
    for rep in range(4):
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            b.solve(fs, xs, K, fmg=True)
            e.record(stream)
        stream.synchronize()
        ms = a.elapsed_time(e)
        if rep == 0:
            t_capture = _time.perf_counter() - t1
        elif best is None or ms < best:
            best, inst = ms, b.times()
    groups, separate = b.info()
    seq_ms = []
    for i in range(count):
        xs[i].zero_()
        with torch.cuda.stream(stream):
            b.solve_one(i, fs[i], xs[i], K[i], fmg=True)       # capture and warm-up
        stream.synchronize()
        xs[i].zero_()
        with torch.cuda.stream(stream):
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            b.solve_one(i, fs[i], xs[i], K[i], fmg=True)
            e.record(stream)
        stream.synchronize()
        seq_ms.append(a.elapsed_time(e))
    seq_total = sum(seq_ms)
    done = [relres(fs[i], xs[i], sides[i]) <= tol for i in range(count)]
    # fine-grid DOF x V-cycles of the whole batch: K_i IR-V steps on the finest grid plus FMG's
    # n_fmg IR-V steps on every level (each weighted by that level's DOF)
    cyc = 0
    for n, k in zip(sides, K):
        m, fmg_dof = n, 0
        while m >= 3:
            fmg_dof += 2 * m * m
            m = (m - 1) // 2
        cyc += k * n * n + fmg_dof
    line = {
        "metric": "batched BFP solves: aggregate GDOF/s (FMG + IR-V to 1e-8 relative residual)",
        "value": dof / (best / 1e3) / 1e9, "unit": "GDOF/s", "n_gpus": 1, "higher_is_better": True,
        "dtype": "int16+f64", "data": "synthetic",
        "config": {"workload": "%d 2D Poisson instances, sides from {127,255,511,1023} (rng seed 3), smoothed "
                               "uniform right-hand sides (seeds 1000+i), w=%d, %s" % (count, args.w, args.mode),
                   "dof": dof},
        "batched": {"ms": best, "p50_ms": pct(inst, 0.5), "p99_ms": pct(inst, 0.99), "capture_s": t_capture,
                    "dof_vcycles_per_s": cyc / (best / 1e3) / 1e9, "merged_groups": groups,
                    "instances_on_own_branches": separate},
        "one_launch_per_instance": {"ms": seq_total, "p50_ms": pct(seq_ms, 0.5), "p99_ms": pct(seq_ms, 0.99),
                                    "value": dof / (seq_total / 1e3) / 1e9},
        "speedup": seq_total / best,
        "ir_steps_after_fmg": {"min": min(K), "max": max(K), "mean": sum(K) / count},
        "reached_tolerance": sum(done), "tuned": {str(k): v for k, v in tuned.items()}, "tune_s": t_tune,
    }
    print(json.dumps(line), flush=True)
    b.close()


def run_op(args):
    """Runs one op of the finest level --reps times (the launch configuration the step uses)."""
    import numpy as np
    import torch
    import paper_2307_00124_gb300 as bfp
    from bfp_inputs import manufactured_rhs
    nd, n, w = args.nd, args.n, args.w
    mode = bfp.NNQCOMP if args.mode == "nnqcomp" else bfp.QCOMP
    o = bfp.bfp_solver_opts_default(nd, n, w)
    o.mode = mode
    if args.smoother == "cheby":
        o.smoother = bfp.SMOOTH_CHEBY
    if args.var:
        from bfp_inputs import grf_nodes
        h = bfp.Hierarchy(o, k_nodes=grf_nodes(n, seed=1))
    else:
        h = bfp.Hierarchy(o)
    f = torch.from_numpy(manufactured_rhs(nd, n)).cuda()
    x = torch.zeros_like(f)
    A = bfp.bfp_laplace_stencil(nd, o.omega, o.w_omega)
    rng = np.random.default_rng(0)
    ym = rng.integers(-(1 << 12), 1 << 12, size=(n,) * nd, dtype=np.int32)
    y = bfp.BFPVector.from_mantissas(ym, -20, w)
    r = bfp.BFPVector.from_mantissas(ym[::-1].copy(), -19, w)
    yo = bfp.BFPVector((n,) * nd, w)
    nc = (n - 1) // 2
    yc = bfp.BFPVector((nc,) * nd, w)
    d = bfp.BFPVector.from_mantissas(ym[(slice(0, nc),) * nd].copy(), -18, w)
    q = bfp.q(w, mode)
    ops = {
        "jacobi": lambda: bfp.bfp_jacobi(A, y, r, yo, q),
        "residual": lambda: bfp.bfp_residual(A, y, r, yo, q),
        "restrict": lambda: bfp.bfp_restrict(y, yc, q),
        "prolong": lambda: bfp.bfp_prolong(d, y, yo, q),
        "ir_residual": lambda: h.ir_residual(f, x, yo),
        "ir_update": lambda: bfp.bfp_ir_update(x, y),
        "step": lambda: h.ir_iterate(f, x, 1),
        "vcycle": lambda: h.vcycle(r, yo),
    }
    if args.op == "step":
        for _ in range(5):      # reach the steady state (windows and exponents of a converging solve)
            ops["step"]()
    for _ in range(args.reps):
        ops[args.op]()
    torch.cuda.synchronize()
    print(json.dumps({"op": args.op, "reps": args.reps, "nd": nd, "n": n, "w": w, "mode": args.mode}))
    h.close()


def main():
    args = parse()
    if args.op:
        run_op(args)
        return
    if args.batch:
        run_batch(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
