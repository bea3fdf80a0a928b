"""The C-ABI library loads and exports every function include/bfp/bfp.h declares;
host-only helpers agree with the oracle; argument errors are synchronous (CPU)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bfp", "bfp.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\([^;{]*\)\s*;", txt, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    import paper_2307_00124_gb300 as bfp
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(bfp._lib, n), n
    # and the binding covers them all
    assert set(names) <= set(bfp.exported_symbols())
    out = subprocess.run(["nm", "-D", "--defined-only", bfp.LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert set(names) <= exported


def test_scalar_from_double_matches_oracle():
    import paper_2307_00124_gb300 as bfp
    from oracle import bfp as B
    rng = np.random.default_rng(0)
    vals = [0.8, 6 / 7 * 8 / 6, -1 / 6, 1.0, -1.0, 3.0, -4.0, 0.5, 1e-300, -7.3e12, 5e-324]
    vals += list(rng.standard_normal(200) * 10.0 ** rng.integers(-20, 20, 200))
    for v in vals:
        for w in (1, 2, 5, 16, 31, 32):
            s = bfp.bfp_scalar_from_double(v, w)
            r = B.scalar_floor(v, w)
            assert (s.m, s.e) == (r.m, r.e) or (r.m == 0 and s.m == 0), (v, w, s.m, s.e, r)


def test_pitch_and_status_strings():
    import paper_2307_00124_gb300 as bfp
    assert [bfp.pitch(n) for n in (0, 1, 8, 9, 4095)] == [8, 8, 8, 16, 4096]
    for code in range(-7, 1):
        assert bfp._lib.bfp_status_str(code)


def test_argument_errors_return_before_any_device_call():
    import paper_2307_00124_gb300 as bfp
    v = bfp.bfp_vec()
    v.mant, v.meta, v.w, v.ndim = 16, 16, 63, 2          # w = 63 is invalid
    v.n[0], v.n[1], v.n[2], v.ld = 8, 8, 1, 8
    q = bfp.q(16)
    assert bfp._lib.bfp_normalize(C.byref(v), C.byref(v), C.byref(q), None, None) == -1
    v.w = 16
    v.ld = 7                                              # ld % 8 != 0
    assert bfp._lib.bfp_normalize(C.byref(v), C.byref(v), C.byref(q), None, None) == -2
    A = bfp.bfp_laplace_stencil(2, 0.8)
    assert (A.center, A.nbr, A.e, A.omega.m, A.omega.e) == (4, -1, -2, 26214, -15)
    o = bfp.bfp_solver_opts()
    assert bfp._lib.bfp_solver_opts_default(4, 63, 16, C.byref(o)) == -1
    h = C.c_void_p()
    assert bfp._lib.bfp_solver_opts_default(2, 63, 16, C.byref(o)) == 0
    o.n = 62                                              # not 2^J - 1
    assert bfp._lib.bfp_hierarchy_create(C.byref(o), C.byref(h)) == -2
    # defaults of the options added with the paper's variants
    assert bfp._lib.bfp_solver_opts_default(2, 63, 16, C.byref(o)) == 0
    assert (o.smoother, o.cheby_eta, o.w_add_max, o.w_step) == (0, 0.15, -1, 0)
    for field, value in (("smoother", 2), ("w_add_max", 40), ("w_step", -1)):
        oo = bfp.bfp_solver_opts()
        bfp._lib.bfp_solver_opts_default(2, 63, 16, C.byref(oo))
        setattr(oo, field, value)
        assert bfp._lib.bfp_hierarchy_create(C.byref(oo), C.byref(h)) == -1, field
    oo = bfp.bfp_solver_opts()
    bfp._lib.bfp_solver_opts_default(2, 63, 16, C.byref(oo))
    oo.smoother, oo.cheby_eta = 1, 1.0                    # eta outside (0, 1)
    assert bfp._lib.bfp_hierarchy_create(C.byref(oo), C.byref(h)) == -1
    oo.cheby_eta, oo.arith = 0.15, 1                      # Chebyshev V(1,0) is BFP only
    assert bfp._lib.bfp_hierarchy_create(C.byref(oo), C.byref(h)) == -1
    # null hierarchies and bad vectors of the newer entry points
    d = C.c_double()
    st = (C.c_uint64 * 8)()
    vs = bfp.bfp_varstencil()
    assert bfp._lib.bfp_hierarchy_rhs_scale(None, C.byref(d)) == -1
    assert bfp._lib.bfp_hierarchy_read_finest_stats(None, st, None) == -1
    assert bfp._lib.bfp_hierarchy_var_ir_operator(None, C.byref(vs)) == -1
    v.w, v.ld = 16, 8
    assert bfp._lib.bfp_ir_iterate_bfp(None, C.byref(v), C.byref(v), 1, None) == -1
    v.w = 63
    assert bfp._lib.bfp_cheby(C.byref(A), bfp.scalar(1, 0), bfp.scalar(-1, -2), C.byref(v), C.byref(v),
                              C.byref(q), None, None) == -1


STRUCTS = ["bfp_vec", "bfp_scalar", "bfp_q", "bfp_stats", "bfp_stencil", "bfp_varstencil", "bfp_solver_opts",
           "flt_vec", "bfp_ir_opts", "bfp_ir_report"]


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct the binding mirrors has the header's size and field offsets (gcc on the header)."""
    import paper_2307_00124_gb300 as bfp
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bfp/bfp.h"', "int main(void) {"]
    for name in STRUCTS:
        cls = getattr(bfp, name)
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for fld, _ in cls._fields_:
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, fld, name, fld))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(ln.rsplit(" ", 1) for ln in out if ln)
    for name in STRUCTS:
        cls = getattr(bfp, name)
        assert int(got[name + " size"]) == C.sizeof(cls), name
        for fld, _ in cls._fields_:
            assert int(got["%s.%s" % (name, fld)]) == getattr(cls, fld).offset, (name, fld)
