"""Out-of-bounds writes: every op and solver call on odd shapes, with each vector's mantissas, meta
block, the FP64 arrays and the qcomp windows carved out of larger buffers whose guard bands are
filled with a sentinel.  After the calls the guard bands must be unchanged (no kernel writes outside
its arrays) and the results must equal the same calls on ordinary allocations.  This stands in for a
memory checker, which is not available on this machine."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2307_00124_gb300 as bfp  # noqa: E402
from bfp_inputs import manufactured_rhs, random_mantissas  # noqa: E402

pytestmark = pytest.mark.gpu

GUARD = 4096           # bytes of guard band on each side (a multiple of 16: keeps the 16-byte alignment)
SENT = 0x5A


class Arena:
    """Carves tensors out of one byte buffer with a sentinel guard band around each."""

    def __init__(self):
        self.bufs = []

    def take(self, shape, dtype):
        n = int(np.prod(shape)) * torch.tensor([], dtype=dtype).element_size()
        raw = torch.full((GUARD + n + GUARD,), SENT, dtype=torch.uint8, device="cuda")
        self.bufs.append((raw, n))
        return raw[GUARD:GUARD + n].view(dtype).view(shape)

    def intact(self):
        torch.cuda.synchronize()
        for raw, n in self.bufs:
            if not (bool((raw[:GUARD] == SENT).all()) and bool((raw[GUARD + n:] == SENT).all())):
                return False
        return True


def vec(arena, shape, w, m=None, e=0):
    """A BFPVector in guarded memory (mantissas from m, or zeros)."""
    v0 = bfp.BFPVector(shape, w)
    mant = arena.take(tuple(v0.mant.shape), v0.mant.dtype)
    meta = arena.take((8,), torch.int64)
    mant.zero_()
    meta.zero_()
    v = bfp.BFPVector(shape, w, mant=mant, meta=meta)
    if m is not None:
        ref = bfp.BFPVector.from_mantissas(m, e, w)
        v.mant.copy_(ref.mant)
        v.meta.copy_(ref.meta)
    return v


@pytest.mark.parametrize("shape,w", [((37, 61), 16), ((13, 9, 23), 16), ((5, 3), 8), ((45, 29), 24)])
@pytest.mark.parametrize("mode", [bfp.QCOMP, bfp.NNQCOMP])
def test_ops_write_only_their_arrays(shape, w, mode):
    nd = len(shape)
    ar = Arena()
    A = bfp.bfp_laplace_stencil(nd, 0.8 if nd == 2 else 6 / 7)
    ym, rm = random_mantissas(shape, w, 1), random_mantissas(shape, w, 2, "smooth")
    y, r = vec(ar, shape, w, ym, -12), vec(ar, shape, w, rm, -10)
    outs = [vec(ar, shape, w) for _ in range(4)]
    tmp = ar.take((outs[0].rows, outs[0].ld), torch.int32)
    st = ar.take((8,), torch.int64)
    st.zero_()
    q = bfp.q(w, mode, tmp=tmp if mode == bfp.QCOMP else None)
    bfp.bfp_jacobi(A, y, r, outs[0], q, st)
    bfp.bfp_jacobi(A, None, r, outs[1], q, st)
    bfp.bfp_residual(A, y, r, outs[2], q, st)
    bfp.bfp_stencil_apply(A, y, outs[3], q, st)
    cs = tuple((s - 1) // 2 for s in shape)
    if min(cs) >= 1:
        rc = vec(ar, cs, w)
        bfp.bfp_restrict(r, rc, q, st)
        yo = vec(ar, shape, w)
        bfp.bfp_prolong(rc, y, yo, q, st)
        bfp.bfp_prolong(rc, None, yo, q, st)
    z = vec(ar, shape, w)
    bfp.bfp_axpy(bfp.scalar(3, -1), y, bfp.scalar(-5, 0), r, z, q, st)
    bfp.bfp_normalize(y, z, q, st)
    xd = ar.take(shape, torch.float64)
    bfp.bfp_to_f64(y, xd)
    bfp.bfp_from_f64(xd, z)
    assert ar.intact()
    # the same calls on ordinary allocations give the same results
    ref = bfp.BFPVector(shape, w)
    tmp2 = torch.zeros((ref.rows, ref.ld), dtype=torch.int32, device="cuda")
    y2, r2 = bfp.BFPVector.from_mantissas(ym, -12, w), bfp.BFPVector.from_mantissas(rm, -10, w)
    bfp.bfp_jacobi(A, y2, r2, ref, bfp.q(w, mode, tmp=tmp2 if mode == bfp.QCOMP else None))
    torch.cuda.synchronize()
    assert ref.exponent == outs[0].exponent and np.array_equal(ref.mantissas(), outs[0].mantissas())


@pytest.mark.parametrize("nd,n,mode", [(2, 63, bfp.QCOMP), (2, 127, bfp.NNQCOMP), (3, 15, bfp.QCOMP)])
def test_solver_writes_only_its_arrays(nd, n, mode):
    """FMG, IR-V steps, the IR residual and update on caller arrays in guarded memory."""
    ar = Arena()
    o = bfp.bfp_solver_opts_default(nd, n, 16)
    o.mode = mode
    h = bfp.Hierarchy(o)
    fh = manufactured_rhs(nd, n)
    f = ar.take(fh.shape, torch.float64)
    f.copy_(torch.from_numpy(fh))
    x = ar.take(fh.shape, torch.float64)
    x.zero_()
    r = vec(ar, (n,) * nd, 16)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        h.fmg(f, x)
        h.ir_iterate(f, x, 2)
        h.ir_residual(f, x, r)
        bfp.bfp_ir_update(x, r)
    stream.synchronize()
    assert ar.intact()
    h2 = bfp.Hierarchy(o)
    f2 = torch.from_numpy(fh).cuda()
    x2 = torch.zeros_like(f2)
    with torch.cuda.stream(stream):
        h2.fmg(f2, x2)
        h2.ir_iterate(f2, x2, 2)
    stream.synchronize()
    r2 = bfp.BFPVector((n,) * nd, 16)
    h2.ir_residual(f2, x2, r2)
    bfp.bfp_ir_update(x2, r2)
    torch.cuda.synchronize()
    assert torch.equal(x, x2)
    h.close()
    h2.close()
