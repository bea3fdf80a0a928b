// bfp_flt_host.h -- host helpers of the float baselines: flt_vec checks and
// views, and the launchers shared by the C ABI and the float hierarchy.
#pragma once

#include "bfp_float.cuh"
#include "bfp_host.h"

namespace bfp {

inline int64_t fbytes(const flt_vec* v) { return v->dtype == FLT_BF16 ? 2 : 4; }

inline int32_t check_fvec(const flt_vec* v) {
  if (!v || !v->data) return BFP_ERR_ARG;
  if (v->dtype != FLT_F32 && v->dtype != FLT_BF16) return BFP_ERR_ARG;
  if (v->ndim < 2 || v->ndim > 3) return BFP_ERR_SHAPE;
  for (int i = 0; i < 3; ++i)
    if (v->n[i] < 0) return BFP_ERR_SHAPE;
  if (v->ndim == 2 && v->n[2] != 1) return BFP_ERR_SHAPE;
  if (v->ld < v->n[0] || v->ld % 8 != 0 || v->ld <= 0) return BFP_ERR_SHAPE;
  if (reinterpret_cast<uintptr_t>(v->data) % 16 != 0) return BFP_ERR_SHAPE;
  return BFP_OK;
}

inline bool same_fshape(const flt_vec* a, const flt_vec* b) {
  return a->ndim == b->ndim && a->n[0] == b->n[0] && a->n[1] == b->n[1] && a->n[2] == b->n[2];
}

inline bool foverlaps(const flt_vec* a, const flt_vec* b) {
  if (!a || !b) return false;
  const char* a0 = (const char*)a->data;
  const char* a1 = a0 + a->n[1] * a->n[2] * a->ld * fbytes(a);
  const char* b0 = (const char*)b->data;
  const char* b1 = b0 + b->n[1] * b->n[2] * b->ld * fbytes(b);
  return a0 < b1 && b0 < a1;
}

inline FVIn fvin(const flt_vec* v) { return FVIn{v->data, v->ld, v->n[0], v->n[1], v->n[2]}; }
inline FVOut fvout(const flt_vec* v) { return FVOut{v->data, v->ld, v->n[0], v->n[1], v->n[2]}; }

int32_t flt_jacobi_impl(const bfp_stencil* A, const flt_vec* y, const flt_vec* r, const flt_vec* out, cudaStream_t s);
int32_t flt_residual_impl(const bfp_stencil* A, const flt_vec* y, const flt_vec* r, const flt_vec* out,
                          cudaStream_t s);
int32_t flt_restrict_impl(const flt_vec* rf, const flt_vec* rc, cudaStream_t s);
int32_t flt_prolong_impl(const flt_vec* d, const flt_vec* y, const flt_vec* out, cudaStream_t s);

}  // namespace bfp
