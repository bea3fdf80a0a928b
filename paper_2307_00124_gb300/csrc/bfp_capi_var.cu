// bfp_capi_var.cu -- C ABI: the variable-coefficient 5-point operator of
// -div(k grad u) (2D; a workload beside the paper's model problem, not in the
// paper): bfp_var_apply, bfp_var_residual, bfp_var_jacobi.
//
// Each op forms its exact result per element in int64 and quantises it
// through the generic two-group quantiser (qcomp / nnqcomp, Alg. qcomp and
// Alg. nnqcomp):
//   apply    : H = A'x = c x - (k_W x_W + k_E x_E + k_S x_S + k_N x_N)  at e_k + e_x
//   residual : H = A'y at e_k + e_y,  L = -r at e_r
//   jacobi   : H = y 2^s - q A'y at e_q + e_k + e_y (s = -(e_q + e_k)),  L = q r at e_q + e_r
//   jacobi0  : H = q r at e_q + e_r
// with c = k_W + k_E + k_S + k_N exact.  The face arrays share e_k (one BFP
// block, int16 or, for apply / residual, int32 mantissas); q is the per-point
// smoother weight block.
#include "bfp_desc.h"
#include "bfp_star2d.cuh"

using namespace bfp;

namespace {

struct VarView {
  VIn k[4];   // W, E, S, N
  VIn q;
};

VIn kview(const void* p, const bfp_varstencil* A) {
  VIn v;
  v.m = p;
  v.ld = A->ld;
  v.nx = A->n[0];
  v.ny = A->n[1];
  v.nz = 1;
  return v;
}

template <class T, int KIND, class TK = int16_t>
struct OpVar {
  static constexpr int kMinBlocks = 3;   // 85 registers: three 256-thread blocks per SM
  VIn y, r;
  VarView A;
  int32_t s;   // jacobi: left shift of y into the H group
  // A'y = k_W (y - y_W) + k_E (y - y_E) + k_S (y - y_S) + k_N (y - y_N), exactly c y - sum k_f y_f
  // (c = sum k_f); one face at a time keeps few registers live.  With int16 y and faces each
  // difference fits 17 bits and each product one 32 x 32 -> 64 multiply.
  __device__ __forceinline__ void operator()(int64_t row, int64_t c0, int64_t (&H)[8], int64_t (&L)[8]) const {
    constexpr bool kNarrow = sizeof(T) == 2 && sizeof(TK) == 2;
    if (KIND == kJacobi0) {
      int32_t rv[8], qv[8];
      ld8<T>(r, row, c0, rv);
      ldv<int16_t, 8>(A.q, row, c0, qv);
#pragma unroll
      for (int k = 0; k < 8; ++k) { H[k] = (int64_t)qv[k] * rv[k]; L[k] = 0; }
      return;
    }
    const int64_t ny = y.ny;
    int32_t ctr[8], nb[8], kf[8];
    ld8<T>(y, row, c0, ctr);
    auto add_face = [&](int f, bool first) {
      ldv<TK, 8>(A.k[f], row, c0, kf);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        int64_t term;
        if (kNarrow) term = (int64_t)kf[k] * (int32_t)(ctr[k] - nb[k]);
        else term = (int64_t)kf[k] * ((int64_t)ctr[k] - nb[k]);
        H[k] = first ? term : H[k] + term;
      }
    };
    {   // W and E: the row shifted by one, with the halo words
      const int32_t wv = (int32_t)ld1<T>(y, row, c0 - 1), ev = (int32_t)ld1<T>(y, row, c0 + 8);
#pragma unroll
      for (int k = 0; k < 8; ++k) nb[k] = k == 0 ? wv : ctr[k - 1];
      add_face(0, true);
#pragma unroll
      for (int k = 0; k < 8; ++k) nb[k] = k == 7 ? ev : ctr[k + 1];
      add_face(1, false);
    }
    ld8<T>(y, row - 1, c0, nb);                   // rows outside the grid read 0
    add_face(2, false);
    ld8<T>(y, row + 1 < ny ? row + 1 : -1, c0, nb);
    add_face(3, false);
    if (KIND == kApply) {
#pragma unroll
      for (int k = 0; k < 8; ++k) L[k] = 0;
      return;
    }
    int32_t rv[8];
    ld8<T>(r, row, c0, rv);
    if (KIND == kResidual) {
#pragma unroll
      for (int k = 0; k < 8; ++k) L[k] = -(int64_t)rv[k];
      return;
    }
    int32_t qv[8];
    ldv<int16_t, 8>(A.q, row, c0, qv);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      H[k] = (int64_t)((uint64_t)(int64_t)ctr[k] << s) - (int64_t)qv[k] * H[k];
      L[k] = (int64_t)qv[k] * rv[k];
    }
  }
};

bool wide_k(const bfp_varstencil* A) { return A->k_storage == 32; }

int32_t check_var(const bfp_varstencil* A, bool need_q) {
  if (!A || A->n[0] < 0 || A->n[1] < 0 || A->ld < A->n[0] || A->ld % 8 != 0 || A->ld <= 0) return BFP_ERR_ARG;
  if (A->k_storage != 0 && A->k_storage != 16 && A->k_storage != 32) return BFP_ERR_ARG;
  if (need_q && wide_k(A)) return BFP_ERR_ARG;
  for (int f = 0; f < 4; ++f)
    if (!A->k[f] || reinterpret_cast<uintptr_t>(A->k[f]) % 16 != 0) return BFP_ERR_ARG;
  if (need_q && (!A->q || reinterpret_cast<uintptr_t>(A->q) % 16 != 0)) return BFP_ERR_ARG;
  if (A->a_norm < 0 || A->a_norm >= (1ll << (wide_k(A) ? 34 : 20))) return BFP_ERR_ARG;
  if (A->q_norm < 0 || A->q_norm >= (1ll << 15)) return BFP_ERR_ARG;
  return BFP_OK;
}

bool var_shape(const bfp_varstencil* A, const bfp_vec* v) {
  return v->ndim == 2 && v->n[0] == A->n[0] && v->n[1] == A->n[1];
}

VarView view(const bfp_varstencil* A) {
  VarView v;
  for (int f = 0; f < 4; ++f) v.k[f] = kview(A->k[f], A);
  v.q = kview(A->q ? A->q : A->k[0], A);
  return v;
}

template <int KIND>
int32_t var_launch(const bfp_varstencil* A, const bfp_vec* y, const bfp_vec* r, const QDesc& d, const bfp_vec* out,
                   int32_t s, cudaStream_t st) {
  const bfp_vec* in = y ? y : r;
  const VIn yv = vin(y ? y : r), rv = vin(r ? r : in);
  // int16 throughout, on a grid large enough: the staged kernel
  if (!wide_k(A) && !is32(in) && !is32(out) && (!r || !is32(r)) && star16_var_fills(out)) {
    VarRow va;
    const VarView v = view(A);
    for (int f = 0; f < 4; ++f) va.k[f] = v.k[f];
    va.q = v.q;
    va.s = s;
    return launch_star16_var<KIND>(yv, rv, va, d, out, st);
  }
  if (KIND != kJacobi && KIND != kJacobi0 && wide_k(A)) {   // int32 faces: apply / residual only
    if (is32(in)) return launch_quant(OpVar<int32_t, KIND, int32_t>{yv, rv, view(A), s}, d, out, st);
    return launch_quant(OpVar<int16_t, KIND, int32_t>{yv, rv, view(A), s}, d, out, st);
  }
  if (is32(in)) return launch_quant(OpVar<int32_t, KIND>{yv, rv, view(A), s}, d, out, st);
  return launch_quant(OpVar<int16_t, KIND>{yv, rv, view(A), s}, d, out, st);
}

}  // namespace

extern "C" {

int32_t bfp_var_apply(const bfp_varstencil* A, const bfp_vec* x, const bfp_vec* z, const bfp_q* q,
                      const bfp_stats* st, bfp_stream stream) {
  int32_t rc;
  if ((rc = check_var(A, false)) || (rc = check_vec(x)) || (rc = check_vec(z))) return rc;
  if (!var_shape(A, x) || !same_shape(x, z)) return BFP_ERR_SHAPE;
  if (x->w > 32) return BFP_ERR_WIDTH;
  if (overlaps(x, z)) return BFP_ERR_ARG;
  QDesc d = blank_desc();
  int rule = 0;
  if ((rc = desc_var_apply(A, x->w, d, &rule)) || (rc = fill_q(d, q, z, rule))) return rc;
  d.meta_a = x->meta; d.meta_out = z->meta; d.stats = st ? st->counters : nullptr;
  return var_launch<kApply>(A, x, nullptr, d, z, 0, as_stream(stream));
}

int32_t bfp_var_residual(const bfp_varstencil* A, const bfp_vec* y, const bfp_vec* r, const bfp_vec* rv,
                         const bfp_q* q, const bfp_stats* st, bfp_stream stream) {
  int32_t rc;
  if ((rc = check_var(A, false)) || (rc = check_vec(y)) || (rc = check_vec(r)) || (rc = check_vec(rv))) return rc;
  if (!var_shape(A, y) || !same_shape(y, r) || !same_shape(y, rv)) return BFP_ERR_SHAPE;
  if (y->w > 32 || r->w > 32) return BFP_ERR_WIDTH;
  if (is32(y) != is32(r)) return BFP_ERR_ARG;
  if (overlaps(y, rv) || overlaps(r, rv)) return BFP_ERR_ARG;
  QDesc d = blank_desc();
  int rule = 0;
  if ((rc = desc_var_residual(A, y->w, r->w, d, &rule)) || (rc = fill_q(d, q, rv, rule))) return rc;
  d.meta_a = y->meta; d.meta_b = r->meta; d.meta_out = rv->meta; d.stats = st ? st->counters : nullptr;
  return var_launch<kResidual>(A, y, r, d, rv, 0, as_stream(stream));
}

int32_t bfp_var_jacobi(const bfp_varstencil* A, const bfp_vec* y, const bfp_vec* r, const bfp_vec* y_out,
                       const bfp_q* q, const bfp_stats* st, bfp_stream stream) {
  int32_t rc;
  if ((rc = check_var(A, true)) || (rc = check_vec(r)) || (rc = check_vec(y_out))) return rc;
  if (!var_shape(A, r) || !same_shape(r, y_out)) return BFP_ERR_SHAPE;
  if (r->w > 24) return BFP_ERR_WIDTH;
  if (overlaps(r, y_out)) return BFP_ERR_ARG;
  QDesc d = blank_desc();
  int rule = 0;
  int32_t s = 0;
  if (!y) {
    if ((rc = desc_var_jacobi(A, 0, r->w, d, &rule, &s)) || (rc = fill_q(d, q, y_out, rule))) return rc;
    d.meta_b = r->meta; d.meta_out = y_out->meta; d.stats = st ? st->counters : nullptr;
    return var_launch<kJacobi0>(A, nullptr, r, d, y_out, 0, as_stream(stream));
  }
  if ((rc = check_vec(y))) return rc;
  if (!same_shape(y, r)) return BFP_ERR_SHAPE;
  if (y->w > 24) return BFP_ERR_WIDTH;
  if (is32(y) != is32(r)) return BFP_ERR_ARG;
  if (overlaps(y, y_out)) return BFP_ERR_ARG;
  if ((rc = desc_var_jacobi(A, y->w, r->w, d, &rule, &s)) || (rc = fill_q(d, q, y_out, rule))) return rc;
  d.meta_a = y->meta; d.meta_b = r->meta; d.meta_out = y_out->meta; d.stats = st ? st->counters : nullptr;
  return var_launch<kJacobi>(A, y, r, d, y_out, s, as_stream(stream));
}

}  // extern "C"
