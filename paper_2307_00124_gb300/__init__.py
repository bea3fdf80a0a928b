"""Python binding of the GB300 BFP multigrid library (C ABI in include/bfp/bfp.h).

Argument marshalling only: every step of the computation runs in the CUDA
library ``lib/libbfpmg.so``.  PyTorch supplies device memory and streams.
Importing this package without the built library raises ImportError; build
it with ``python -m paper_2307_00124_gb300.build`` (or
``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libbfpmg.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libbfpmg.so is not built (%s); run paper_2307_00124_gb300/build.py" % LIB_PATH)
_lib = C.CDLL(LIB_PATH)

META_WORDS = 8
QCOMP, NNQCOMP = 0, 1
ARITH_BFP, ARITH_FP32, ARITH_BF16 = 0, 1, 2
SMOOTH_JACOBI, SMOOTH_CHEBY = 0, 1
F32, BF16 = 0, 1

STATUS = {0: "BFP_OK", -1: "BFP_ERR_ARG", -2: "BFP_ERR_SHAPE", -3: "BFP_ERR_WIDTH", -4: "BFP_ERR_CUDA",
          -5: "BFP_ERR_NONFINITE", -6: "BFP_ERR_TIMEOUT", -7: "BFP_ERR_NOCONV", -8: "BFP_ERR_CAPACITY"}


class BFPError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.bfp_status_str(status).decode()
        super().__init__("%s: %s (%s)" % (where, STATUS.get(status, status), msg))


# ---- ctypes mirrors of the C structs ----------------------------------------

class bfp_vec(C.Structure):
    _fields_ = [("mant", C.c_void_p), ("meta", C.c_void_p), ("w", C.c_int32), ("ndim", C.c_int32),
                ("n", C.c_int64 * 3), ("ld", C.c_int64)]


class bfp_scalar(C.Structure):
    _fields_ = [("m", C.c_int64), ("e", C.c_int64)]


class bfp_q(C.Structure):
    _fields_ = [("w_out", C.c_int32), ("w_add", C.c_int32), ("mode", C.c_int32), ("has_gamma", C.c_int32),
                ("gamma", bfp_scalar), ("tmp", C.c_void_p)]


class bfp_stats(C.Structure):
    _fields_ = [("counters", C.c_void_p)]


class bfp_stencil(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("reserved", C.c_int32), ("center", C.c_int64), ("nbr", C.c_int64),
                ("e", C.c_int64), ("omega", bfp_scalar)]


class bfp_varstencil(C.Structure):
    _fields_ = [("n", C.c_int64 * 2), ("ld", C.c_int64), ("k", C.c_void_p * 4), ("e_k", C.c_int64),
                ("q", C.c_void_p), ("e_q", C.c_int64), ("a_norm", C.c_int64), ("q_norm", C.c_int64),
                ("omega", bfp_scalar), ("k_storage", C.c_int32), ("reserved", C.c_int32)]


class bfp_solver_opts(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("w", C.c_int32), ("n", C.c_int64), ("mode", C.c_int32),
                ("nu1", C.c_int32), ("nu2", C.c_int32), ("coarse_sweeps", C.c_int32), ("n_fmg", C.c_int32),
                ("omega", C.c_double), ("w_omega", C.c_int32), ("use_tmp", C.c_int32),
                ("use_graph", C.c_int32), ("coarse_onchip", C.c_int32), ("arith", C.c_int32),
                ("tile_rows", C.c_int32), ("w_step", C.c_int32), ("smoother", C.c_int32),
                ("cheby_eta", C.c_double), ("w_add_max", C.c_int32)]


class flt_vec(C.Structure):
    _fields_ = [("data", C.c_void_p), ("dtype", C.c_int32), ("ndim", C.c_int32), ("n", C.c_int64 * 3),
                ("ld", C.c_int64)]


class bfp_ir_opts(C.Structure):
    _fields_ = [("max_iter", C.c_int32), ("fmg_start", C.c_int32), ("tol", C.c_double),
                ("stall_fallback", C.c_int32), ("reserved", C.c_int32)]


class bfp_ir_report(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("res_inf", C.c_double),
                ("res0_inf", C.c_double), ("fallback_at", C.c_int32), ("reserved", C.c_int32)]


P = C.POINTER
_sig = {
    "bfp_status_str": (C.c_char_p, [C.c_int32]),
    "bfp_version": (C.c_int32, []),
    "bfp_pitch": (C.c_int64, [C.c_int64]),
    "bfp_kernel_launches": (C.c_int64, []),
    "bfp_scalar_from_double": (C.c_int32, [C.c_double, C.c_int32, P(bfp_scalar)]),
    "bfp_laplace_stencil": (C.c_int32, [C.c_int32, C.c_double, C.c_int32, P(bfp_stencil)]),
    "bfp_normalize": (C.c_int32, [P(bfp_vec), P(bfp_vec), P(bfp_q), P(bfp_stats), C.c_void_p]),
    "bfp_from_f64": (C.c_int32, [C.c_void_p, P(bfp_vec), C.c_void_p]),
    "bfp_to_f64": (C.c_int32, [P(bfp_vec), C.c_void_p, C.c_void_p]),
    "bfp_block_norm": (C.c_int32, [P(bfp_vec), C.c_void_p]),
    "bfp_axpy": (C.c_int32, [bfp_scalar, P(bfp_vec), bfp_scalar, P(bfp_vec), P(bfp_vec), P(bfp_q),
                             P(bfp_stats), C.c_void_p]),
    "bfp_dot": (C.c_int32, [P(bfp_vec), P(bfp_vec), C.c_int32, C.c_void_p, C.c_void_p]),
    "bfp_stencil_apply": (C.c_int32, [P(bfp_stencil), P(bfp_vec), P(bfp_vec), P(bfp_q), P(bfp_stats),
                                      C.c_void_p]),
    "bfp_residual": (C.c_int32, [P(bfp_stencil), P(bfp_vec), P(bfp_vec), P(bfp_vec), P(bfp_q),
                                 P(bfp_stats), C.c_void_p]),
    "bfp_jacobi": (C.c_int32, [P(bfp_stencil), P(bfp_vec), P(bfp_vec), P(bfp_vec), P(bfp_q), P(bfp_stats),
                               C.c_void_p]),
    "bfp_restrict": (C.c_int32, [P(bfp_vec), P(bfp_vec), P(bfp_q), P(bfp_stats), C.c_void_p]),
    "bfp_prolong": (C.c_int32, [P(bfp_vec), P(bfp_vec), P(bfp_vec), P(bfp_q), P(bfp_stats), C.c_void_p]),
    "bfp_noalloc_window_capacity": (C.c_int64, []),
    "bfp_jacobi_noalloc": (C.c_int32, [P(bfp_stencil), P(bfp_vec), P(bfp_vec), P(bfp_vec), P(bfp_q),
                                       P(bfp_stats), C.c_void_p]),
    "bfp_solver_opts_default": (C.c_int32, [C.c_int32, C.c_int64, C.c_int32, P(bfp_solver_opts)]),
    "bfp_hierarchy_create": (C.c_int32, [P(bfp_solver_opts), P(C.c_void_p)]),
    "bfp_hierarchy_create_var": (C.c_int32, [P(bfp_solver_opts), C.c_void_p, P(C.c_void_p)]),
    "bfp_hierarchy_var_level": (C.c_int32, [C.c_void_p, C.c_int32, P(bfp_varstencil)]),
    "bfp_hierarchy_var_ir_operator": (C.c_int32, [C.c_void_p, P(bfp_varstencil)]),
    "bfp_cheby": (C.c_int32, [P(bfp_stencil), bfp_scalar, bfp_scalar, P(bfp_vec), P(bfp_vec), P(bfp_q),
                              P(bfp_stats), C.c_void_p]),
    "bfp_var_apply": (C.c_int32, [P(bfp_varstencil), P(bfp_vec), P(bfp_vec), P(bfp_q), P(bfp_stats), C.c_void_p]),
    "bfp_var_residual": (C.c_int32, [P(bfp_varstencil), P(bfp_vec), P(bfp_vec), P(bfp_vec), P(bfp_q),
                                     P(bfp_stats), C.c_void_p]),
    "bfp_var_jacobi": (C.c_int32, [P(bfp_varstencil), P(bfp_vec), P(bfp_vec), P(bfp_vec), P(bfp_q),
                                   P(bfp_stats), C.c_void_p]),
    "bfp_hierarchy_destroy": (None, [C.c_void_p]),
    "bfp_hierarchy_read_stats": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "bfp_hierarchy_reset_stats": (C.c_int32, [C.c_void_p, C.c_void_p]),
    "bfp_hierarchy_read_finest_stats": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "bfp_vcycle": (C.c_int32, [C.c_void_p, P(bfp_vec), P(bfp_vec), C.c_void_p]),
    "bfp_ir_iterate": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "bfp_ir_iterate_bfp": (C.c_int32, [C.c_void_p, P(bfp_vec), P(bfp_vec), C.c_int32, C.c_void_p]),
    "bfp_hierarchy_rhs_scale": (C.c_int32, [C.c_void_p, P(C.c_double)]),
    "bfp_fmg": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "bfp_ir_residual": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, P(bfp_vec), C.c_void_p]),
    "bfp_ir_update": (C.c_int32, [C.c_void_p, P(bfp_vec), C.c_void_p]),
    "ir_solve": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, P(bfp_ir_opts), P(bfp_ir_report),
                             C.c_void_p]),
    "flt_jacobi": (C.c_int32, [P(bfp_stencil), P(flt_vec), P(flt_vec), P(flt_vec), C.c_void_p]),
    "flt_residual": (C.c_int32, [P(bfp_stencil), P(flt_vec), P(flt_vec), P(flt_vec), C.c_void_p]),
    "flt_restrict": (C.c_int32, [P(flt_vec), P(flt_vec), C.c_void_p]),
    "flt_prolong": (C.c_int32, [P(flt_vec), P(flt_vec), P(flt_vec), C.c_void_p]),
    "flt_vcycle": (C.c_int32, [C.c_void_p, P(flt_vec), P(flt_vec), C.c_void_p]),
    "bfp_batch_create": (C.c_int32, [P(bfp_solver_opts), C.c_int32, P(C.c_void_p)]),
    "bfp_batch_solve": (C.c_int32, [C.c_void_p, P(C.c_void_p), P(C.c_void_p), P(C.c_int32), C.c_int32,
                                    C.c_void_p]),
    "bfp_batch_times": (C.c_int32, [C.c_void_p, P(C.c_float)]),
    "bfp_batch_solve_one": (C.c_int32, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                        C.c_void_p]),
    "bfp_batch_info": (C.c_int32, [C.c_void_p, P(C.c_int32), P(C.c_int32)]),
    "bfp_batch_destroy": (None, [C.c_void_p]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def _check(rc: int, where: str):
    if rc != 0:
        raise BFPError(rc, where)


def _stream(stream):
    import torch
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def bfp_kernel_launches() -> int:
    return int(_lib.bfp_kernel_launches())


def pitch(n0: int) -> int:
    return int(_lib.bfp_pitch(n0))


# ---- BFP vectors backed by torch device memory --------------------------------

class BFPVector:
    """A BFP block in device memory: mantissas (rows x ld, int16 / int32 / int64 for w <= 16 / 32 / 62)
    + meta (int64[8]).

    ``shape`` is the numpy-order logical shape ((n,), (ny, nx) or (nz, ny, nx)).
    """

    def __init__(self, shape, w: int, device="cuda", mant=None, meta=None):
        import torch
        self.shape = tuple(int(s) for s in shape)
        self.w = int(w)
        nx = self.shape[-1]
        self.ld = pitch(nx)
        self.rows = int(np.prod(self.shape[:-1])) if len(self.shape) > 1 else 1
        dt = torch.int16 if self.w <= 16 else (torch.int32 if self.w <= 32 else torch.int64)
        # at least one row of storage: the C ABI wants a non-null mantissa pointer, also for an empty grid
        self.mant = mant if mant is not None else torch.zeros((max(self.rows, 1), self.ld), dtype=dt, device=device)
        self.meta = meta if meta is not None else torch.zeros(META_WORDS, dtype=torch.int64, device=device)

    @property
    def ndim(self):
        return len(self.shape)

    def struct(self) -> bfp_vec:
        v = bfp_vec()
        v.mant = self.mant.data_ptr()
        v.meta = self.meta.data_ptr()
        v.w = self.w
        v.ndim = self.ndim
        n = list(reversed(self.shape)) + [1] * (3 - self.ndim)
        for i in range(3):
            v.n[i] = n[i]
        v.ld = self.ld
        return v

    @classmethod
    def from_mantissas(cls, m: np.ndarray, e: int, w: int, device="cuda"):
        import torch
        m = np.asarray(m, dtype=np.int64)
        v = cls(m.shape, w, device)
        host = np.zeros(tuple(v.mant.shape), dtype=np.int16 if w <= 16 else (np.int32 if w <= 32 else np.int64))
        host[: v.rows, : m.shape[-1]] = m.reshape(v.rows, m.shape[-1])
        v.mant.copy_(torch.from_numpy(host))
        meta = np.zeros(META_WORDS, dtype=np.int64)
        meta[0] = e
        v.meta.copy_(torch.from_numpy(meta))
        bfp_block_norm(v)                       # the norm word, by the library
        return v

    def mantissas(self) -> np.ndarray:
        h = self.mant.cpu().numpy().astype(np.int64)
        return h[: self.rows, : self.shape[-1]].reshape(self.shape)

    def padding(self) -> np.ndarray:
        return self.mant.cpu().numpy()[: self.rows, self.shape[-1]:]

    @property
    def exponent(self) -> int:
        return int(self.meta[0].item())

    @property
    def norm_m(self) -> int:
        return int(self.meta[1].item())


class FltVector:
    """A float-baseline vector in device memory: FP32 or BF16 (as int16 bit patterns), rows x ld.

    ``shape`` is the numpy-order logical shape ((ny, nx) or (nz, ny, nx)).
    """

    def __init__(self, shape, dtype: int = F32, device="cuda", data=None):
        import torch
        self.shape = tuple(int(s) for s in shape)
        self.dtype = int(dtype)
        self.ld = pitch(self.shape[-1])
        self.rows = int(np.prod(self.shape[:-1]))
        td = torch.float32 if self.dtype == F32 else torch.int16
        self.data = data if data is not None else torch.zeros((self.rows, self.ld), dtype=td, device=device)

    @property
    def ndim(self):
        return len(self.shape)

    def struct(self) -> flt_vec:
        v = flt_vec()
        v.data = self.data.data_ptr()
        v.dtype = self.dtype
        v.ndim = self.ndim
        n = list(reversed(self.shape)) + [1] * (3 - self.ndim)
        for i in range(3):
            v.n[i] = n[i]
        v.ld = self.ld
        return v

    @classmethod
    def from_array(cls, a: np.ndarray, dtype: int = F32, device="cuda"):
        """a: float32 values (BF16: float32 values whose low 16 bits are zero)."""
        import torch
        a = np.asarray(a, dtype=np.float32)
        v = cls(a.shape, dtype, device)
        host = np.zeros((v.rows, v.ld), dtype=np.float32)
        host[:, : a.shape[-1]] = a.reshape(v.rows, a.shape[-1])
        if dtype == F32:
            v.data.copy_(torch.from_numpy(host))
        else:
            bits = host.view(np.uint32) >> 16
            v.data.copy_(torch.from_numpy(bits.astype(np.uint16).view(np.int16)))
        return v

    def values(self) -> np.ndarray:
        """float32 values of the logical shape."""
        h = self.data.cpu().numpy()
        if self.dtype == BF16:
            h = (h.view(np.uint16).astype(np.uint32) << 16).view(np.float32)
        return h[:, : self.shape[-1]].reshape(self.shape)

    def padding(self) -> np.ndarray:
        h = self.data.cpu().numpy()
        return h[:, self.shape[-1]:]


def q(w_out: int, mode: int = QCOMP, w_add: int = -1, gamma=None, tmp=None) -> bfp_q:
    r = bfp_q()
    r.w_out = w_out
    r.w_add = w_add
    r.mode = mode
    r.has_gamma = 0 if gamma is None else 1
    if gamma is not None:
        r.gamma.m, r.gamma.e = int(gamma[0]), int(gamma[1])
    r.tmp = None if tmp is None else tmp.data_ptr()
    return r


def stats_of(counters) -> bfp_stats:
    s = bfp_stats()
    s.counters = counters.data_ptr()
    return s


def _st(stats):
    return None if stats is None else C.byref(stats_of(stats) if not isinstance(stats, bfp_stats) else stats)


def scalar(m: int, e: int) -> bfp_scalar:
    s = bfp_scalar()
    s.m, s.e = int(m), int(e)
    return s


def bfp_scalar_from_double(x: float, w: int) -> bfp_scalar:
    s = bfp_scalar()
    _check(_lib.bfp_scalar_from_double(float(x), int(w), C.byref(s)), "bfp_scalar_from_double")
    return s


def bfp_laplace_stencil(ndim: int, omega: float, w_omega: int = 16) -> bfp_stencil:
    A = bfp_stencil()
    _check(_lib.bfp_laplace_stencil(ndim, float(omega), w_omega, C.byref(A)), "bfp_laplace_stencil")
    return A


# ---- ops (same names as the C ABI) ---------------------------------------------

def bfp_normalize(x, out, qq, stats=None, stream=None):
    _check(_lib.bfp_normalize(C.byref(x.struct()), C.byref(out.struct()), C.byref(qq), _st(stats),
                              _stream(stream)), "bfp_normalize")


def bfp_from_f64(x, out, stream=None):
    assert x.is_cuda and x.dtype.is_floating_point and x.is_contiguous()
    _check(_lib.bfp_from_f64(C.c_void_p(x.data_ptr()), C.byref(out.struct()), _stream(stream)), "bfp_from_f64")


def bfp_to_f64(x, out, stream=None):
    assert out.is_cuda and out.is_contiguous()
    _check(_lib.bfp_to_f64(C.byref(x.struct()), C.c_void_p(out.data_ptr()), _stream(stream)), "bfp_to_f64")


def bfp_block_norm(x, stream=None):
    _check(_lib.bfp_block_norm(C.byref(x.struct()), _stream(stream)), "bfp_block_norm")


def bfp_axpy(a, x, b, y, z, qq, stats=None, stream=None):
    _check(_lib.bfp_axpy(a, C.byref(x.struct()), b, C.byref(y.struct()), C.byref(z.struct()), C.byref(qq),
                         _st(stats), _stream(stream)), "bfp_axpy")


def bfp_dot(x, y, w_out, out, stream=None):
    _check(_lib.bfp_dot(C.byref(x.struct()), C.byref(y.struct()), int(w_out), C.c_void_p(out.data_ptr()),
                        _stream(stream)), "bfp_dot")


def bfp_stencil_apply(A, x, z, qq, stats=None, stream=None):
    _check(_lib.bfp_stencil_apply(C.byref(A), C.byref(x.struct()), C.byref(z.struct()), C.byref(qq),
                                  _st(stats), _stream(stream)), "bfp_stencil_apply")


def bfp_residual(A, y, r, rv, qq, stats=None, stream=None):
    _check(_lib.bfp_residual(C.byref(A), C.byref(y.struct()), C.byref(r.struct()), C.byref(rv.struct()),
                             C.byref(qq), _st(stats), _stream(stream)), "bfp_residual")


def bfp_cheby(A, c1, c2, r, y_out, qq, stats=None, stream=None):
    _check(_lib.bfp_cheby(C.byref(A), c1, c2, C.byref(r.struct()), C.byref(y_out.struct()), C.byref(qq),
                          _st(stats), _stream(stream)), "bfp_cheby")


def bfp_jacobi(A, y, r, y_out, qq, stats=None, stream=None):
    yp = None if y is None else C.byref(y.struct())
    _check(_lib.bfp_jacobi(C.byref(A), yp, C.byref(r.struct()), C.byref(y_out.struct()), C.byref(qq),
                           _st(stats), _stream(stream)), "bfp_jacobi")


def bfp_var_apply(A, x, z, qq, stats=None, stream=None):
    _check(_lib.bfp_var_apply(C.byref(A), C.byref(x.struct()), C.byref(z.struct()), C.byref(qq), _st(stats),
                              _stream(stream)), "bfp_var_apply")


def bfp_var_residual(A, y, r, rv, qq, stats=None, stream=None):
    _check(_lib.bfp_var_residual(C.byref(A), C.byref(y.struct()), C.byref(r.struct()), C.byref(rv.struct()),
                                 C.byref(qq), _st(stats), _stream(stream)), "bfp_var_residual")


def bfp_var_jacobi(A, y, r, y_out, qq, stats=None, stream=None):
    yp = None if y is None else C.byref(y.struct())
    _check(_lib.bfp_var_jacobi(C.byref(A), yp, C.byref(r.struct()), C.byref(y_out.struct()), C.byref(qq),
                               _st(stats), _stream(stream)), "bfp_var_jacobi")


def bfp_jacobi_noalloc(A, y, r, y_out, qq, stats=None, stream=None):
    """bfp_jacobi whose qcomp window lives in the library's static device array (no allocation)."""
    yp = None if y is None else C.byref(y.struct())
    _check(_lib.bfp_jacobi_noalloc(C.byref(A), yp, C.byref(r.struct()), C.byref(y_out.struct()), C.byref(qq),
                                   _st(stats), _stream(stream)), "bfp_jacobi_noalloc")


def bfp_noalloc_window_capacity() -> int:
    return int(_lib.bfp_noalloc_window_capacity())


def bfp_restrict(rf, rc, qq, stats=None, stream=None):
    _check(_lib.bfp_restrict(C.byref(rf.struct()), C.byref(rc.struct()), C.byref(qq), _st(stats),
                             _stream(stream)), "bfp_restrict")


def bfp_prolong(d, y, y_out, qq, stats=None, stream=None):
    yp = None if y is None else C.byref(y.struct())
    _check(_lib.bfp_prolong(C.byref(d.struct()), yp, C.byref(y_out.struct()), C.byref(qq), _st(stats),
                            _stream(stream)), "bfp_prolong")


# ---- float baselines (not in the paper) ----------------------------------------------

def flt_jacobi(A, y, r, out, stream=None):
    yp = None if y is None else C.byref(y.struct())
    _check(_lib.flt_jacobi(C.byref(A), yp, C.byref(r.struct()), C.byref(out.struct()), _stream(stream)),
           "flt_jacobi")


def flt_residual(A, y, r, out, stream=None):
    _check(_lib.flt_residual(C.byref(A), C.byref(y.struct()), C.byref(r.struct()), C.byref(out.struct()),
                             _stream(stream)), "flt_residual")


def flt_restrict(rf, rc, stream=None):
    _check(_lib.flt_restrict(C.byref(rf.struct()), C.byref(rc.struct()), _stream(stream)), "flt_restrict")


def flt_prolong(d, y, out, stream=None):
    yp = None if y is None else C.byref(y.struct())
    _check(_lib.flt_prolong(C.byref(d.struct()), yp, C.byref(out.struct()), _stream(stream)), "flt_prolong")


# ---- multigrid ---------------------------------------------------------------------

def bfp_solver_opts_default(ndim: int, n: int, w: int) -> bfp_solver_opts:
    o = bfp_solver_opts()
    _check(_lib.bfp_solver_opts_default(ndim, n, w, C.byref(o)), "bfp_solver_opts_default")
    return o


class Hierarchy:
    """Owns a bfp_hierarchy (level buffers, captured graphs) on the current device."""

    def __init__(self, opts: bfp_solver_opts, k_nodes=None):
        """k_nodes: None (the constant-coefficient model problem) or the (n+2) x (n+2) node
        values of k for -div(k grad u) = f (2D, host float64, [y, x], boundary included)."""
        self.opts = opts
        h = C.c_void_p()
        if k_nodes is None:
            _check(_lib.bfp_hierarchy_create(C.byref(opts), C.byref(h)), "bfp_hierarchy_create")
        else:
            k = np.ascontiguousarray(k_nodes, dtype=np.float64)
            if k.shape != (opts.n + 2, opts.n + 2):
                raise ValueError("k_nodes must have shape (n+2, n+2)")
            _check(_lib.bfp_hierarchy_create_var(C.byref(opts), k.ctypes.data_as(C.c_void_p), C.byref(h)),
                   "bfp_hierarchy_create_var")
        self.h = h

    def var_level(self, level: int = 0) -> bfp_varstencil:
        """The variable-coefficient operator of a level (arrays owned by the hierarchy)."""
        out = bfp_varstencil()
        _check(_lib.bfp_hierarchy_var_level(self.h, level, C.byref(out)), "bfp_hierarchy_var_level")
        return out

    def var_ir_operator(self) -> bfp_varstencil:
        """The finest operator with 26-bit faces used by ir_iterate_bfp (variable coefficients)."""
        out = bfp_varstencil()
        _check(_lib.bfp_hierarchy_var_ir_operator(self.h, C.byref(out)), "bfp_hierarchy_var_ir_operator")
        return out

    def close(self):
        if self.h:
            _lib.bfp_hierarchy_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self, stream=None) -> dict:
        host = (C.c_uint64 * 8)()
        _check(_lib.bfp_hierarchy_read_stats(self.h, host, _stream(stream)), "bfp_hierarchy_read_stats")
        keys = ("calls", "recomputed", "overflow", "underflow", "saturated", "ir_residuals", "ir_recomputed")
        return {k: int(host[i]) for i, k in enumerate(keys)}

    def finest_stats(self, stream=None) -> dict:
        """The finest level's counters (bfp_hierarchy_read_finest_stats)."""
        host = (C.c_uint64 * 8)()
        _check(_lib.bfp_hierarchy_read_finest_stats(self.h, host, _stream(stream)),
               "bfp_hierarchy_read_finest_stats")
        keys = ("calls", "recomputed", "overflow", "underflow", "saturated", "ir_residuals", "ir_recomputed")
        return {k: int(host[i]) for i, k in enumerate(keys)}

    def reset_stats(self, stream=None):
        _check(_lib.bfp_hierarchy_reset_stats(self.h, _stream(stream)), "bfp_hierarchy_reset_stats")

    def vcycle(self, r, y, stream=None):
        if isinstance(r, FltVector):
            _check(_lib.flt_vcycle(self.h, C.byref(r.struct()), C.byref(y.struct()), _stream(stream)),
                   "flt_vcycle")
            return
        _check(_lib.bfp_vcycle(self.h, C.byref(r.struct()), C.byref(y.struct()), _stream(stream)), "bfp_vcycle")

    def ir_iterate(self, f, x, k: int, stream=None):
        _check(_lib.bfp_ir_iterate(self.h, C.c_void_p(f.data_ptr()), C.c_void_p(x.data_ptr()), int(k),
                                   _stream(stream)), "bfp_ir_iterate")

    def ir_iterate_bfp(self, b, x, k: int, stream=None):
        """k IR steps with BFP x (updated in place) and BFP b' (bfp_ir_iterate_bfp)."""
        _check(_lib.bfp_ir_iterate_bfp(self.h, C.byref(b.struct()), C.byref(x.struct()), int(k), _stream(stream)),
               "bfp_ir_iterate_bfp")

    def rhs_scale(self) -> float:
        """s with b' = s f on the finest level."""
        out = C.c_double()
        _check(_lib.bfp_hierarchy_rhs_scale(self.h, C.byref(out)), "bfp_hierarchy_rhs_scale")
        return out.value

    def ir_residual(self, f, x, r, stream=None):
        _check(_lib.bfp_ir_residual(self.h, C.c_void_p(f.data_ptr()), C.c_void_p(x.data_ptr()),
                                    C.byref(r.struct()), _stream(stream)), "bfp_ir_residual")

    def fmg(self, f, x, stream=None):
        _check(_lib.bfp_fmg(self.h, C.c_void_p(f.data_ptr()), C.c_void_p(x.data_ptr()), _stream(stream)),
               "bfp_fmg")

    def ir_solve(self, f, x, max_iter=50, tol=1e-10, fmg_start=True, stall_fallback=False, stream=None):
        o = bfp_ir_opts()
        o.max_iter, o.tol, o.fmg_start = int(max_iter), float(tol), int(bool(fmg_start))
        o.stall_fallback = int(bool(stall_fallback))
        rep = bfp_ir_report()
        rc = _lib.ir_solve(self.h, C.c_void_p(f.data_ptr()), C.c_void_p(x.data_ptr()), C.byref(o), C.byref(rep),
                           _stream(stream))
        if rc not in (0, -7):
            raise BFPError(rc, "ir_solve")
        return rep


class Batch:
    """Owns a bfp_batch: independent hierarchies solved together in one graph launch."""

    def __init__(self, opts_list):
        n = len(opts_list)
        arr = (bfp_solver_opts * n)(*opts_list)
        b = C.c_void_p()
        _check(_lib.bfp_batch_create(arr, n, C.byref(b)), "bfp_batch_create")
        self.b, self.count = b, n

    def close(self):
        if self.b:
            _lib.bfp_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, fs, xs, ir_steps, fmg=True, stream=None):
        """[FMG] + ir_steps[i] IR-V steps for every instance, one graph launch on stream."""
        n = self.count
        fa = (C.c_void_p * n)(*[f.data_ptr() for f in fs])
        xa = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
        ka = (C.c_int32 * n)(*[int(k) for k in ir_steps])
        _check(_lib.bfp_batch_solve(self.b, fa, xa, ka, int(bool(fmg)), _stream(stream)), "bfp_batch_solve")

    def solve_one(self, i, f, x, ir_steps, fmg=True, stream=None):
        """Instance i alone, as its own graph launch."""
        _check(_lib.bfp_batch_solve_one(self.b, int(i), C.c_void_p(f.data_ptr()), C.c_void_p(x.data_ptr()),
                                        int(ir_steps), int(bool(fmg)), _stream(stream)), "bfp_batch_solve_one")

    def info(self):
        """(groups run as merged launches, instances on branches of their own) of the last captured solve."""
        g, sep = C.c_int32(), C.c_int32()
        _check(_lib.bfp_batch_info(self.b, C.byref(g), C.byref(sep)), "bfp_batch_info")
        return int(g.value), int(sep.value)

    def times(self):
        """ms from the launch start to the end of each instance's last op (waits for the launch)."""
        ms = (C.c_float * self.count)()
        _check(_lib.bfp_batch_times(self.b, ms), "bfp_batch_times")
        return [float(v) for v in ms]


def bfp_ir_update(x, y, stream=None):
    _check(_lib.bfp_ir_update(C.c_void_p(x.data_ptr()), C.byref(y.struct()), _stream(stream)), "bfp_ir_update")


def ir_solve(h: Hierarchy, f, x, **kw):
    return h.ir_solve(f, x, **kw)


def exported_symbols():
    """Names of the C ABI functions this binding declares."""
    return sorted(_sig)
