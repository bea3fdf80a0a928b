// bfp_capi_star.cu -- C ABI: star-stencil ops (Alg. espmv / egemv on the
// 5- and 7-point Laplacian): bfp_stencil_apply, bfp_residual, bfp_jacobi,
// bfp_cheby.
#include "bfp_desc.h"
#include "bfp_star2d.cuh"

using namespace bfp;

namespace {

int32_t check_stencil(const bfp_stencil* A, const bfp_vec* v) {
  if (!A || (A->ndim != 2 && A->ndim != 3) || A->ndim != v->ndim) return BFP_ERR_ARG;
  if (A->center >= (1 << 15) || A->center < -(1 << 15) || A->nbr >= (1 << 15) || A->nbr < -(1 << 15))
    return BFP_ERR_ARG;
  if (A->omega.m >= (1ll << 31) || A->omega.m < -(1ll << 31)) return BFP_ERR_ARG;
  return BFP_OK;
}

template <int KIND, int ND>
int32_t star_launch(const bfp_vec* yv, const bfp_vec* rv, const QDesc& d, const bfp_vec* out, int64_t c,
                    int64_t n, int64_t mw, bool wide_in, cudaStream_t s) {
  if (ND == 2) {
    if (wide_in) return launch_star2d<int32_t, KIND>(vin(yv), vin(rv), c, n, mw, d, out, s, !yv || yv->w <= 30);
    return launch_star2d<int16_t, KIND>(vin(yv), vin(rv), c, n, mw, d, out, s);
  }
  if (!wide_in && !is32(out)) return launch_star3d16<KIND>(vin(yv), vin(rv), c, n, mw, d, out, s);
  if (wide_in) {
    OpStar<int32_t, KIND, ND> op{vin(yv), vin(rv), c, n, mw};
    return launch_quant(op, d, out, s);
  }
  OpStar<int16_t, KIND, ND> op{vin(yv), vin(rv), c, n, mw};
  return launch_quant(op, d, out, s);
}

template <int KIND>
int32_t star_dispatch(int nd, const bfp_vec* yv, const bfp_vec* rv, const QDesc& d, const bfp_vec* out,
                      int64_t c, int64_t n, int64_t mw, bool wide_in, cudaStream_t s) {
  if (nd == 2) return star_launch<KIND, 2>(yv, rv, d, out, c, n, mw, wide_in, s);
  return star_launch<KIND, 3>(yv, rv, d, out, c, n, mw, wide_in, s);
}

}  // namespace

extern "C" {

int32_t bfp_stencil_apply(const bfp_stencil* A, const bfp_vec* x, const bfp_vec* z, const bfp_q* q,
                          const bfp_stats* st, bfp_stream stream) {
  int32_t rc;
  if ((rc = check_vec(x)) || (rc = check_vec(z)) || (rc = check_stencil(A, x))) return rc;
  if (!same_shape(x, z)) return BFP_ERR_SHAPE;
  if (overlaps(x, z)) return BFP_ERR_ARG;
  QDesc d = blank_desc();
  int rule = 0;
  if ((rc = desc_apply(A, x->w, d, &rule)) || (rc = fill_q(d, q, z, rule))) return rc;
  d.meta_a = x->meta; d.meta_out = z->meta; d.stats = st ? st->counters : nullptr;
  return star_dispatch<kApply>(A->ndim, x, nullptr, d, z, A->center, A->nbr, 0, is32(x), as_stream(stream));
}

int32_t bfp_residual(const bfp_stencil* A, const bfp_vec* y, const bfp_vec* r, const bfp_vec* rv,
                     const bfp_q* q, const bfp_stats* st, bfp_stream stream) {
  int32_t rc;
  if ((rc = check_vec_wide(y)) || (rc = check_vec_wide(r)) || (rc = check_vec(rv)) || (rc = check_stencil(A, y)))
    return rc;
  if (!same_shape(y, r) || !same_shape(y, rv)) return BFP_ERR_SHAPE;
  const bool wide = is64(y) || is64(r) || is32(y) != is32(r);   // int64 or mixed storage
  if (overlaps(y, rv) || overlaps(r, rv)) return BFP_ERR_ARG;
  QDesc d = blank_desc();
  int rule = 0;
  if ((rc = desc_residual(A, y->w, r->w, d, &rule)) || (rc = fill_q(d, q, rv, rule))) return rc;
  d.meta_a = y->meta; d.meta_b = r->meta; d.meta_out = rv->meta; d.stats = st ? st->counters : nullptr;
  if (wide) {   // int64 operands or mixed storage: the generic row kernel
    if (A->ndim == 2)
      return launch_quant(OpResW<2>{vin(y), vin(r), esize(y), esize(r), A->center, A->nbr}, d, rv, as_stream(stream));
    return launch_quant(OpResW<3>{vin(y), vin(r), esize(y), esize(r), A->center, A->nbr}, d, rv, as_stream(stream));
  }
  return star_dispatch<kResidual>(A->ndim, y, r, d, rv, A->center, A->nbr, 0, is32(y), as_stream(stream));
}

int32_t bfp_cheby(const bfp_stencil* A, bfp_scalar c1, bfp_scalar c2, const bfp_vec* r, const bfp_vec* y_out,
                  const bfp_q* q, const bfp_stats* st, bfp_stream stream) {
  int32_t rc;
  if ((rc = check_vec(r)) || (rc = check_vec(y_out)) || (rc = check_stencil(A, r))) return rc;
  if (!same_shape(r, y_out)) return BFP_ERR_SHAPE;
  if (overlaps(r, y_out)) return BFP_ERR_ARG;
  QDesc d = blank_desc();
  int rule = 0;
  int64_t Tc = 0, Tn = 0;
  if ((rc = desc_cheby(A, c1, c2, r->w, d, &rule, &Tc, &Tn)) || (rc = fill_q(d, q, y_out, rule))) return rc;
  d.meta_a = r->meta; d.meta_out = y_out->meta; d.stats = st ? st->counters : nullptr;
  // T r is a stencil apply with T's coefficients
  return star_dispatch<kApply>(A->ndim, r, nullptr, d, y_out, Tc, Tn, 0, is32(r), as_stream(stream));
}

int32_t bfp_jacobi(const bfp_stencil* A, const bfp_vec* y, const bfp_vec* r, const bfp_vec* y_out,
                   const bfp_q* q, const bfp_stats* st, bfp_stream stream) {
  int32_t rc;
  if ((rc = check_vec(r)) || (rc = check_vec(y_out)) || (rc = check_stencil(A, r))) return rc;
  if (!same_shape(r, y_out)) return BFP_ERR_SHAPE;
  if (y) {
    if ((rc = check_vec(y))) return rc;
    if (!same_shape(y, r)) return BFP_ERR_SHAPE;
    if (overlaps(y, y_out)) return BFP_ERR_ARG;
  }
  if (overlaps(r, y_out)) return BFP_ERR_ARG;
  QDesc d = blank_desc();
  int rule = 0;
  if ((rc = desc_jacobi(A, y ? y->w : 0, r->w, d, &rule)) || (rc = fill_q(d, q, y_out, rule))) return rc;
  d.meta_out = y_out->meta; d.stats = st ? st->counters : nullptr;
  cudaStream_t s = as_stream(stream);
  const int64_t mw = A->omega.m;
  if (!y) {
    d.meta_b = r->meta;
    return star_dispatch<kJacobi0>(A->ndim, r, r, d, y_out, 0, 0, mw, is32(r), s);
  }
  int64_t Sc, Sn, eS;
  if ((rc = jacobi_operator(A, &Sc, &Sn, &eS))) return rc;
  d.meta_a = y->meta; d.meta_b = r->meta;
  if (is32(y) != is32(r)) {   // mixed storage (progressive widths): the generic row kernel
    if (A->ndim == 2) return launch_quant(OpJacD<2>{vin(y), vin(r), esize(y), esize(r), Sc, Sn, mw}, d, y_out, s);
    return launch_quant(OpJacD<3>{vin(y), vin(r), esize(y), esize(r), Sc, Sn, mw}, d, y_out, s);
  }
  return star_dispatch<kJacobi>(A->ndim, y, r, d, y_out, Sc, Sn, mw, is32(y), s);
}

}  // extern "C"
