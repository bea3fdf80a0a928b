"""bfp_jacobi_noalloc: the same result as bfp_jacobi, with the qcomp window in the
library's static device array instead of memory the caller or the library allocates.

Callers that cannot allocate device memory where they call the op (inside a host
callback, under a memory budget owned by another framework, or where an implicit
device synchronisation is not acceptable) use this entry point.  This file is
collected last so that a run stopping at the first failure has run every other
test before it; it also passes on its own in a fresh process, where the first
call performs the first lookup of the static array on the device.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2307_00124_gb300 as bfp  # noqa: E402
from bfp_inputs import random_mantissas  # noqa: E402

pytestmark = pytest.mark.gpu


def _vec(m, e, w):
    return bfp.BFPVector.from_mantissas(m, e, w)


def _same(a, b):
    torch.cuda.synchronize()
    assert a.exponent == b.exponent
    assert a.norm_m == b.norm_m
    assert np.array_equal(a.mantissas(), b.mantissas())
    assert np.array_equal(a.padding(), b.padding())


# (mode, w_add): qcomp with the window (w_tmp = w + 2 <= 32), qcomp whose w_tmp passes 32 bits (no
# window: the second pass recomputes), nnqcomp (no scratch at all)
MODES = [(bfp.QCOMP, -1), (bfp.QCOMP, 17), (bfp.NNQCOMP, -1)]


@pytest.mark.parametrize("mode,w_add", MODES)
@pytest.mark.parametrize("shape,w", [((1023, 1001), 16), ((63, 64), 24), ((9, 17, 31), 16)])
def test_noalloc_matches_allocating_entry_point_twice(shape, w, mode, w_add):
    nd = len(shape)
    A = bfp.bfp_laplace_stencil(nd, 0.8 if nd == 2 else 6 / 7)
    for call in range(2):          # two calls in a row share (and overwrite) the static window
        ym = random_mantissas(shape, w, 100 + call)
        rm = random_mantissas(shape, w, 200 + call, "smooth")
        y, r = _vec(ym, -11 - call, w), _vec(rm, -9 + call, w)
        ref, out = bfp.BFPVector(shape, w), bfp.BFPVector(shape, w)
        out.mant.fill_(3)
        tmp = torch.zeros((ref.rows, ref.ld), dtype=torch.int32, device="cuda")
        st_ref = torch.zeros(8, dtype=torch.int64, device="cuda")
        st_out = torch.zeros(8, dtype=torch.int64, device="cuda")
        for zero_guess in (False, True):
            bfp.bfp_jacobi(A, None if zero_guess else y, r, ref, bfp.q(w, mode, w_add=w_add, tmp=tmp), st_ref)
            bfp.bfp_jacobi_noalloc(A, None if zero_guess else y, r, out, bfp.q(w, mode, w_add=w_add), st_out)
            _same(out, ref)
        assert torch.equal(st_ref, st_out)


def test_noalloc_capacity_applies_to_the_window_only():
    cap = bfp.bfp_noalloc_window_capacity()
    assert cap == 1 << 22
    n = 2049                                   # 2049 rows x 2056 ld > 2^22
    A = bfp.bfp_laplace_stencil(2, 0.8)
    y = _vec(random_mantissas((n, n), 16, 7), -12, 16)
    r = _vec(random_mantissas((n, n), 16, 8, "smooth"), -10, 16)
    out = bfp.BFPVector((n, n), 16)
    with pytest.raises(bfp.BFPError) as ei:    # qcomp with the window: refused, nothing launched
        bfp.bfp_jacobi_noalloc(A, y, r, out, bfp.q(16, bfp.QCOMP))
    assert ei.value.status == -8
    for mode, w_add in ((bfp.NNQCOMP, -1), (bfp.QCOMP, 17)):   # no window: any size
        ref = bfp.BFPVector((n, n), 16)
        tmp = torch.zeros((ref.rows, ref.ld), dtype=torch.int32, device="cuda")
        bfp.bfp_jacobi(A, y, r, ref, bfp.q(16, mode, w_add=w_add, tmp=tmp))
        bfp.bfp_jacobi_noalloc(A, y, r, out, bfp.q(16, mode, w_add=w_add))
        _same(out, ref)
