// bfp_capi_star.cu -- C ABI: star-stencil ops (Alg. espmv / egemv on the
// 5- and 7-point Laplacian): bfp_stencil_apply, bfp_residual, bfp_jacobi.
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
    if (wide_in) return launch_star2d<int32_t, KIND>(vin(yv), vin(rv), c, n, mw, d, out, s);
    return launch_star2d<int16_t, KIND>(vin(yv), vin(rv), c, n, mw, d, out, s);
  }
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

int64_t iabs(int64_t v) { return v < 0 ? -v : v; }

}  // namespace

extern "C" {

int32_t bfp_stencil_apply(const bfp_stencil* A, const bfp_vec* x, const bfp_vec* z, const bfp_q* q,
                          const bfp_stats* st, bfp_stream stream) {
  int32_t rc;
  if ((rc = check_vec(x)) || (rc = check_vec(z)) || (rc = check_stencil(A, x))) return rc;
  if (!same_shape(x, z)) return BFP_ERR_SHAPE;
  if (overlaps(x, z)) return BFP_ERR_ARG;
  QDesc d = blank_desc();
  if ((rc = fill_q(d, q, z, 2))) return rc;
  const int mA = 2 * A->ndim + 1;
  const int wA = hmsb(A->center) > hmsb(A->nbr) ? hmsb(A->center) : hmsb(A->nbr);
  d.meta_a = x->meta; d.meta_out = z->meta; d.stats = st ? st->counters : nullptr;
  d.ch = A->e; d.ha = 1; d.two = 0;
  d.hbits = wA + x->w + clog2(mA);                 // Alg. espmv-setup width
  d.ng = 1; d.gv[0] = 0;                           // gamma = ||A||_inf ||x||
  d.gm[0] = (uint64_t)(iabs(A->center) + 2 * A->ndim * iabs(A->nbr)); d.ge[0] = A->e;
  return star_dispatch<kApply>(A->ndim, x, nullptr, d, z, A->center, A->nbr, 0, is32(x), as_stream(stream));
}

int32_t bfp_residual(const bfp_stencil* A, const bfp_vec* y, const bfp_vec* r, const bfp_vec* rv,
                     const bfp_q* q, const bfp_stats* st, bfp_stream stream) {
  int32_t rc;
  if ((rc = check_vec(y)) || (rc = check_vec(r)) || (rc = check_vec(rv)) || (rc = check_stencil(A, y))) return rc;
  if (!same_shape(y, r) || !same_shape(y, rv)) return BFP_ERR_SHAPE;
  if (is32(y) != is32(r)) return BFP_ERR_ARG;
  if (overlaps(y, rv) || overlaps(r, rv)) return BFP_ERR_ARG;
  QDesc d = blank_desc();
  if ((rc = fill_q(d, q, rv, 4))) return rc;     // Table tab:estimates, V residual: w_add = 4
  const int mA = 2 * A->ndim + 1;
  const int wA = hmsb(A->center) > hmsb(A->nbr) ? hmsb(A->center) : hmsb(A->nbr);
  d.meta_a = y->meta; d.meta_b = r->meta; d.meta_out = rv->meta; d.stats = st ? st->counters : nullptr;
  d.ch = A->e; d.ha = 1;                          // A y at e_A + e_y
  d.cl = 0; d.lb = 1;                             // -r at e_r
  d.two = 1;
  d.hbits = wA + y->w + clog2(mA);
  d.lbits = r->w + 1;
  // gamma = 1/4 (2 c1 + 1) ||r|| with c1 = 2 omega  ->  (|omega| + 1/4) ||r||
  const int64_t om = iabs(A->omega.m), oe = A->omega.e;
  uint64_t cm;
  int64_t ce;
  if (oe <= -2) { cm = (uint64_t)om + (1ull << (-2 - oe)); ce = oe; }
  else {
    if (oe + 2 > 30) return BFP_ERR_ARG;
    cm = ((uint64_t)om << (oe + 2)) + 1ull; ce = -2;
  }
  if (cm >= (1ull << 32)) return BFP_ERR_ARG;
  d.ng = 1; d.gv[0] = 1; d.gm[0] = cm; d.ge[0] = ce;
  return star_dispatch<kResidual>(A->ndim, y, r, d, rv, A->center, A->nbr, 0, is32(y), as_stream(stream));
}

int32_t bfp_jacobi(const bfp_stencil* A, const bfp_vec* y, const bfp_vec* r, const bfp_vec* y_out,
                   const bfp_q* q, const bfp_stats* st, bfp_stream stream) {
  int32_t rc;
  if ((rc = check_vec(r)) || (rc = check_vec(y_out)) || (rc = check_stencil(A, r))) return rc;
  if (!same_shape(r, y_out)) return BFP_ERR_SHAPE;
  if (y) {
    if ((rc = check_vec(y))) return rc;
    if (!same_shape(y, r)) return BFP_ERR_SHAPE;
    if (is32(y) != is32(r)) return BFP_ERR_ARG;
    if (overlaps(y, y_out)) return BFP_ERR_ARG;
  }
  if (overlaps(r, y_out)) return BFP_ERR_ARG;
  QDesc d = blank_desc();
  if ((rc = fill_q(d, q, y_out, 2))) return rc;   // Table tab:estimates, relaxation: w_add = 2
  const int64_t mw = A->omega.m, ew = A->omega.e;
  const int mA = 2 * A->ndim + 1;
  d.meta_out = y_out->meta; d.stats = st ? st->counters : nullptr;
  cudaStream_t s = as_stream(stream);
  if (!y) {
    // omega r at e_omega + e_r
    d.meta_b = r->meta;
    d.ch = ew; d.hb = 1; d.two = 0;
    d.hbits = hmsb(mw) + r->w;
    d.ng = 1; d.gv[0] = 1; d.gm[0] = (uint64_t)iabs(mw); d.ge[0] = ew;
    return star_dispatch<kJacobi0>(A->ndim, r, r, d, y_out, 0, 0, mw, is32(r), s);
  }
  // S = I - omega A as one BFP block: e_S = min(0, e_omega + e_A), k = e_omega + e_A - e_S
  const int64_t eS = (ew + A->e) < 0 ? (ew + A->e) : 0;
  const int64_t k = ew + A->e - eS;
  if (-eS > 40 || k > 40) return BFP_ERR_ARG;
  const int64_t Sc = ((int64_t)1 << (-eS)) - ((mw * A->center) << k);
  const int64_t Sn = -((mw * A->nbr) << k);
  if (Sc >= (1ll << 31) || Sc < -(1ll << 31) || Sn >= (1ll << 31) || Sn < -(1ll << 31)) return BFP_ERR_WIDTH;
  const int wS = hmsb(Sc) > hmsb(Sn) ? hmsb(Sc) : hmsb(Sn);
  d.meta_a = y->meta; d.meta_b = r->meta;
  d.ch = eS; d.ha = 1;                            // S y at e_S + e_y  (Alg. egemv: alpha = 1)
  d.cl = ew; d.lb = 1;                            // omega r at e_omega + e_r  (beta = omega)
  d.two = 1;
  d.hbits = wS + y->w + clog2(mA);
  d.lbits = hmsb(mw) + r->w;
  // gamma = ||S||_inf ||y|| + |omega| ||r||
  d.ng = 2;
  d.gv[0] = 0; d.gm[0] = (uint64_t)(iabs(Sc) + 2 * A->ndim * iabs(Sn)); d.ge[0] = eS;
  d.gv[1] = 1; d.gm[1] = (uint64_t)iabs(mw); d.ge[1] = ew;
  return star_dispatch<kJacobi>(A->ndim, y, r, d, y_out, Sc, Sn, mw, is32(y), s);
}

}  // extern "C"
