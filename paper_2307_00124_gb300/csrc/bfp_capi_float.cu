// bfp_capi_float.cu -- C ABI of the float baselines (flt_jacobi, flt_residual,
// flt_restrict, flt_prolong): argument checks and launches of the kernels in
// bfp_float.cuh.  Not part of the paper's method.
#include <cmath>

#include "bfp_float.cuh"
#include "bfp_flt_host.h"

namespace bfp {
namespace {

int32_t stencil_coefs(const bfp_stencil* A, float* c, float* nb, float* om) {
  if (!A || (A->ndim != 2 && A->ndim != 3)) return BFP_ERR_ARG;
  const double cc = std::ldexp((double)A->center, (int)A->e), nn = std::ldexp((double)A->nbr, (int)A->e);
  const double oo = std::ldexp((double)A->omega.m, (int)A->omega.e);
  *c = (float)cc; *nb = (float)nn; *om = (float)oo;
  // the dyadic coefficients must be exact in FP32
  if ((double)*c != cc || (double)*nb != nn || (double)*om != oo) return BFP_ERR_WIDTH;
  return BFP_OK;
}

template <int KIND>
int32_t fstar(const bfp_stencil* A, const flt_vec* y, const flt_vec* r, const flt_vec* out, cudaStream_t s) {
  float c, nb, om;
  int32_t e = stencil_coefs(A, &c, &nb, &om);
  if (e) return e;
  if ((e = check_fvec(r)) || (e = check_fvec(out))) return e;
  if (KIND != kJacobi0) {
    if ((e = check_fvec(y))) return e;
    if (!same_fshape(y, out) || y->dtype != out->dtype) return BFP_ERR_SHAPE;
    if (foverlaps(y, out)) return BFP_ERR_ARG;
  }
  if (!same_fshape(r, out) || r->dtype != out->dtype || out->ndim != A->ndim) return BFP_ERR_SHAPE;
  if (foverlaps(r, out)) return BFP_ERR_ARG;
  const FVIn yv = KIND != kJacobi0 ? fvin(y) : fvin(r), rv = fvin(r);
  const FVOut o = fvout(out);
  const bool bf = out->dtype == FLT_BF16;
  if (out->ndim == 2) {
    const int64_t ny = out->n[1];
    if (ny == 0) return BFP_OK;
    const int rs = pick_rows(ny >= 2048 ? 16 : (ny >= 1024 ? 8 : (ny >= 256 ? 4 : 2)), 64);
    const dim3 g((unsigned)((out->ld + 255) / 256), (unsigned)((ny + 4 * rs - 1) / (4 * rs)));
    if (bf) k_fstar2d<uint16_t, KIND><<<g, 128, 0, s>>>(yv, rv, c, nb, om, o, rs);
    else k_fstar2d<float, KIND><<<g, 128, 0, s>>>(yv, rv, c, nb, om, o, rs);
  } else {
    const int64_t items = out->ld * out->n[1] * out->n[2];
    if (items == 0) return BFP_OK;
    const unsigned g = grid_for(items, 256);
    if (bf) k_fstar3d<uint16_t, KIND><<<g, 256, 0, s>>>(yv, rv, c, nb, om, o);
    else k_fstar3d<float, KIND><<<g, 256, 0, s>>>(yv, rv, c, nb, om, o);
  }
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

}  // namespace

int32_t flt_restrict_impl(const flt_vec* rf, const flt_vec* rc, cudaStream_t s) {
  int32_t e;
  if ((e = check_fvec(rf)) || (e = check_fvec(rc))) return e;
  if (rf->ndim != rc->ndim || rf->dtype != rc->dtype) return BFP_ERR_SHAPE;
  for (int i = 0; i < rf->ndim; ++i)
    if (rf->n[i] != 2 * rc->n[i] + 1) return BFP_ERR_SHAPE;
  if (foverlaps(rf, rc)) return BFP_ERR_ARG;
  const int64_t items = rc->ld * rc->n[1] * rc->n[2];
  if (items == 0) return BFP_OK;
  const unsigned g = grid_for(items, 256);
  const bool bf = rc->dtype == FLT_BF16;
  if (rc->ndim == 2) {
    if (bf) k_frestrict<uint16_t, 2><<<g, 256, 0, s>>>(fvin(rf), fvout(rc));
    else k_frestrict<float, 2><<<g, 256, 0, s>>>(fvin(rf), fvout(rc));
  } else {
    if (bf) k_frestrict<uint16_t, 3><<<g, 256, 0, s>>>(fvin(rf), fvout(rc));
    else k_frestrict<float, 3><<<g, 256, 0, s>>>(fvin(rf), fvout(rc));
  }
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

int32_t flt_prolong_impl(const flt_vec* d, const flt_vec* y, const flt_vec* out, cudaStream_t s) {
  int32_t e;
  if ((e = check_fvec(d)) || (e = check_fvec(out))) return e;
  if (d->ndim != out->ndim || d->dtype != out->dtype) return BFP_ERR_SHAPE;
  for (int i = 0; i < d->ndim; ++i)
    if (out->n[i] != 2 * d->n[i] + 1) return BFP_ERR_SHAPE;
  if (foverlaps(d, out)) return BFP_ERR_ARG;
  if (y) {
    if ((e = check_fvec(y))) return e;
    if (!same_fshape(y, out) || y->dtype != out->dtype) return BFP_ERR_SHAPE;
    if (foverlaps(y, out)) return BFP_ERR_ARG;
  }
  const int64_t items = out->ld * out->n[1] * out->n[2];
  if (items == 0) return BFP_OK;
  const unsigned g = grid_for(items, 256);
  const bool bf = out->dtype == FLT_BF16;
  const FVIn dv = fvin(d), yv = fvin(y ? y : out);
  const FVOut o = fvout(out);
#define BFP_FPRO(S, ND)                                                     \
  do {                                                                      \
    if (y) k_fprolong<S, ND, true><<<g, 256, 0, s>>>(dv, yv, o);            \
    else k_fprolong<S, ND, false><<<g, 256, 0, s>>>(dv, yv, o);             \
  } while (0)
  if (out->ndim == 2) {
    if (bf) BFP_FPRO(uint16_t, 2);
    else BFP_FPRO(float, 2);
  } else {
    if (bf) BFP_FPRO(uint16_t, 3);
    else BFP_FPRO(float, 3);
  }
#undef BFP_FPRO
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

int32_t flt_jacobi_impl(const bfp_stencil* A, const flt_vec* y, const flt_vec* r, const flt_vec* out,
                        cudaStream_t s) {
  return y ? fstar<kJacobi>(A, y, r, out, s) : fstar<kJacobi0>(A, nullptr, r, out, s);
}

int32_t flt_residual_impl(const bfp_stencil* A, const flt_vec* y, const flt_vec* r, const flt_vec* out,
                          cudaStream_t s) {
  if (!y) return BFP_ERR_ARG;
  return fstar<kResidual>(A, y, r, out, s);
}

}  // namespace bfp

extern "C" {

int32_t flt_jacobi(const bfp_stencil* A, const flt_vec* y, const flt_vec* r, const flt_vec* out,
                   bfp_stream stream) {
  return bfp::flt_jacobi_impl(A, y, r, out, (cudaStream_t)stream);
}

int32_t flt_residual(const bfp_stencil* A, const flt_vec* y, const flt_vec* r, const flt_vec* out,
                     bfp_stream stream) {
  return bfp::flt_residual_impl(A, y, r, out, (cudaStream_t)stream);
}

int32_t flt_restrict(const flt_vec* r_f, const flt_vec* r_c, bfp_stream stream) {
  return bfp::flt_restrict_impl(r_f, r_c, (cudaStream_t)stream);
}

int32_t flt_prolong(const flt_vec* d, const flt_vec* y, const flt_vec* out, bfp_stream stream) {
  return bfp::flt_prolong_impl(d, y, out, (cudaStream_t)stream);
}

}  // extern "C"
