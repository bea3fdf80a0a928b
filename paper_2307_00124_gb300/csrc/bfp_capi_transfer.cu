// bfp_capi_transfer.cu -- C ABI: grid transfers of the V-cycle and FMG
// (full-weighting restriction R~, bilinear/trilinear prolongation P).
#include "bfp_host.h"

using namespace bfp;

namespace {

bool coarse_of(const bfp_vec* f, const bfp_vec* c) {
  if (f->ndim != c->ndim || f->ndim < 2) return false;
  for (int i = 0; i < f->ndim; ++i)
    if (f->n[i] != 2 * c->n[i] + 1) return false;
  return true;
}

template <int ND>
int32_t restrict_launch(const bfp_vec* rf, const bfp_vec* rc, const QDesc& d, cudaStream_t s) {
  if (is32(rf)) return launch_quant(OpRestrict<int32_t, ND>{vin(rf), rc->n[1]}, d, rc, s);
  return launch_quant(OpRestrict<int16_t, ND>{vin(rf), rc->n[1]}, d, rc, s);
}

template <int ND, bool CORR>
int32_t prolong_launch(const bfp_vec* dc, const bfp_vec* y, const bfp_vec* out, const QDesc& d, cudaStream_t s) {
  VIn yv = vin(y ? y : out);   // carries the fine shape; not read when CORR is false
  if (!CORR) yv.m = nullptr;
  if (is32(dc)) return launch_quant(OpProlong<int32_t, ND, CORR>{vin(dc), yv}, d, out, s);
  return launch_quant(OpProlong<int16_t, ND, CORR>{vin(dc), yv}, d, out, s);
}

}  // namespace

extern "C" {

int32_t bfp_restrict(const bfp_vec* r_f, const bfp_vec* r_c, const bfp_q* q, const bfp_stats* st,
                     bfp_stream stream) {
  int32_t rc;
  if ((rc = check_vec(r_f)) || (rc = check_vec(r_c))) return rc;
  if (!coarse_of(r_f, r_c)) return BFP_ERR_SHAPE;
  if (overlaps(r_f, r_c)) return BFP_ERR_ARG;
  QDesc d = blank_desc();
  if ((rc = fill_q(d, q, r_c, 6))) return rc;    // Table tab:estimates, restriction: w_add = 6
  const int nd = r_f->ndim;
  const int64_t eR = nd == 2 ? -2 : -4;           // R~ = P^T (2D), P^T / 2 (3D)
  int mR = 1;
  for (int i = 0; i < nd; ++i) mR *= 3;
  d.meta_a = r_f->meta; d.meta_out = r_c->meta; d.stats = st ? st->counters : nullptr;
  d.ch = eR; d.ha = 1; d.two = 0;
  d.hbits = hmsb(1ll << nd) + r_f->w + clog2(mR);  // Alg. espmv-setup with m_R = 3^d
  d.ng = 1; d.gv[0] = 0;                           // gamma = ||R~||_inf ||r_v||  (||R~|| = 4)
  d.gm[0] = nd == 2 ? 16 : 64; d.ge[0] = eR;
  cudaStream_t s = as_stream(stream);
  return nd == 2 ? restrict_launch<2>(r_f, r_c, d, s) : restrict_launch<3>(r_f, r_c, d, s);
}

int32_t bfp_prolong(const bfp_vec* dc, const bfp_vec* y, const bfp_vec* y_out, const bfp_q* q,
                    const bfp_stats* st, bfp_stream stream) {
  int32_t rc;
  if ((rc = check_vec(dc)) || (rc = check_vec(y_out))) return rc;
  if (!coarse_of(y_out, dc)) return BFP_ERR_SHAPE;
  if (overlaps(dc, y_out)) return BFP_ERR_ARG;
  if (y) {
    if ((rc = check_vec(y))) return rc;
    if (!same_shape(y, y_out)) return BFP_ERR_SHAPE;
    if (is32(y) != is32(dc)) return BFP_ERR_ARG;
    if (overlaps(y, y_out)) return BFP_ERR_ARG;
  }
  QDesc d = blank_desc();
  // Table tab:estimates: V correction w_add = 1, FMG interpolation w_add = 0
  if ((rc = fill_q(d, q, y_out, y ? 1 : 0))) return rc;
  const int nd = dc->ndim;
  const int64_t eP = -nd;                          // P mantissas prod(2 or 1) at e = -d
  const int wP = hmsb(1ll << nd);
  d.meta_out = y_out->meta; d.stats = st ? st->counters : nullptr;
  d.meta_a = dc->meta;
  d.ch = eP; d.ha = 1;
  d.hbits = wP + dc->w + nd + 1;                   // w_P + w_d + ceil(log2 m_P), sign of -P d
  // ||P||_inf = 1 = 2^d * 2^-d
  if (y) {
    d.meta_b = y->meta;
    d.cl = 0; d.lb = 1; d.two = 1;
    d.lbits = y->w + 1;
    d.ng = 2;                                      // gamma = ||y|| + ||P|| ||d||
    d.gv[0] = 1; d.gm[0] = 1; d.ge[0] = 0;
    d.gv[1] = 0; d.gm[1] = 1ull << nd; d.ge[1] = eP;
  } else {
    d.two = 0;
    d.ng = 1;                                      // gamma = ||P|| ||x||
    d.gv[0] = 0; d.gm[0] = 1ull << nd; d.ge[0] = eP;
  }
  cudaStream_t s = as_stream(stream);
  if (nd == 2) return y ? prolong_launch<2, true>(dc, y, y_out, d, s) : prolong_launch<2, false>(dc, y, y_out, d, s);
  return y ? prolong_launch<3, true>(dc, y, y_out, d, s) : prolong_launch<3, false>(dc, y, y_out, d, s);
}

}  // extern "C"
