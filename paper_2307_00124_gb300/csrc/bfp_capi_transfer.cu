// bfp_capi_transfer.cu -- C ABI: grid transfers of the V-cycle and FMG
// (full-weighting restriction R~, bilinear/trilinear prolongation P).
#include "bfp_desc.h"
#include "bfp_transfer2d.cuh"

using namespace bfp;

namespace {

bool coarse_of(const bfp_vec* f, const bfp_vec* c) {
  if (f->ndim != c->ndim || f->ndim < 2) return false;
  for (int i = 0; i < f->ndim; ++i)
    if (f->n[i] != 2 * c->n[i] + 1) return false;
  return true;
}

// Rows per warp strip (<= 16: the kernels keep a per-strip mask of general-path rows): 8 on large
// levels; below 1024 rows one op's grid is a few CTAs and a strip's serial row steps set the op's
// latency, so strips stay at one or two rows there.  A launch recorded for a batched solve runs
// over many instances at once and fills the GPU anyway: taller strips there (fewer CTAs, each
// planning and committing once).
int rows_per_warp(int64_t rows) {
  if (launch_recorder()) return pick_rows(rows >= 1024 ? 8 : (rows >= 256 ? 4 : (rows >= 64 ? 2 : 1)), 16);
  return pick_rows(rows >= 1024 ? 8 : (rows >= 512 ? 2 : 1), 16);
}

int32_t launch_checks(const QDesc& d) {
  if (d.hbits > 62 || (d.two && d.lbits > 62)) return BFP_ERR_WIDTH;
  return BFP_OK;
}

// T: the fine mantissas (int16; or int32 of at most 27 bits with an int32 output)
template <class T = int16_t>
int32_t restrict2d16(const bfp_vec* rf, const bfp_vec* rc, const QDesc& d, cudaStream_t s) {
  int32_t e = launch_checks(d);
  if (e) return e;
  const int64_t ny = rc->n[1];
  const int rs = rows_per_warp(ny);
  const int64_t strips = (ny + 4 * rs - 1) / (4 * rs);
  const int64_t cols = sizeof(T) == 4 ? 128 : 256;   // coarse columns per warp chunk
  const dim3 grid((unsigned)((rc->ld + cols - 1) / cols), (unsigned)(strips > 0 ? strips : 1));
  const VOut o = vout(rc);
  static bool carved = false;   // the staging rings want the shared-memory carveout
  if (!carved) {
    cudaFuncSetAttribute(k_restrict2d16<true, false, T>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_restrict2d16<false, false, T>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_restrict2d16<true, true, T>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_restrict2d16<false, true, T>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    carved = true;
  }
  if (zero_accumulators(d.meta_out, s) != cudaSuccess) return BFP_ERR_CUDA;
  const TransferP P{vin(rf), vin(rf), d, o, rs};
  if (d.mode == kQcomp)
    launch_rec<TransferP, &k_restrict2d16<true, false, T>, &k_restrict2d16<true, true, T>>(grid, 128, 0, s, P);
  launch_rec<TransferP, &k_restrict2d16<false, false, T>, &k_restrict2d16<false, true, T>>(grid, 128, 0, s, P);
  note_launches(d.mode == kQcomp ? 2 : 1);
  return cudaGetLastError() == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

int32_t restrict3d16(const bfp_vec* rf, const bfp_vec* rc, const QDesc& d, cudaStream_t s) {
  int32_t e = launch_checks(d);
  if (e) return e;
  const int64_t ny = rc->n[1], nz = rc->n[2];
  if (nz > 65535) return BFP_ERR_SHAPE;
  const int rs = pick_rows(ny >= 128 ? 8 : (ny >= 32 ? 4 : 2), 16);
  const int64_t strips = (ny + kR3Warps * rs - 1) / (kR3Warps * rs);
  const dim3 grid((unsigned)((rc->ld + 255) / 256), (unsigned)(strips > 0 ? strips : 1), (unsigned)(nz > 0 ? nz : 1));
  VOut o = vout(rc);
  if (nz == 0) o.ny = 0;
  static bool carved = false;
  if (!carved) {
    cudaFuncSetAttribute(k_restrict3d16<true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_restrict3d16<false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    carved = true;
  }
  if (zero_accumulators(d.meta_out, s) != cudaSuccess) return BFP_ERR_CUDA;
  if (d.mode == kQcomp) k_restrict3d16<true><<<grid, 32 * kR3Warps, 0, s>>>(vin(rf), d, o, rs);
  k_restrict3d16<false><<<grid, 32 * kR3Warps, 0, s>>>(vin(rf), d, o, rs);
  note_launches(d.mode == kQcomp ? 2 : 1);
  return cudaGetLastError() == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

// staged interpolation, int16 (2D or 3D, grid z: fine planes) or int32 mantissas (2D)
template <bool CORR, int ND, class T = int16_t>
int32_t prolong16(const bfp_vec* dc, const bfp_vec* y, const bfp_vec* out, const QDesc& d, cudaStream_t s) {
  int32_t e = launch_checks(d);
  if (e) return e;
  const int64_t pairs = (out->n[1] + 1) / 2;
  const int rs = rows_per_warp(ND == 3 ? 4 * pairs : pairs);
  const int64_t nzf = ND == 3 ? out->n[2] : 1;
  if (nzf > 65535) return BFP_ERR_SHAPE;
  const int64_t strips = (pairs + 4 * rs - 1) / (4 * rs);
  const int64_t cols = sizeof(T) == 4 ? 128 : 256;   // fine columns per warp chunk
  const dim3 grid((unsigned)((out->ld + cols - 1) / cols), (unsigned)(strips > 0 ? strips : 1), (unsigned)nzf);
  const VOut o = vout(out);
  VIn yv = vin(y ? y : out);
  if (!CORR) yv.m = nullptr;
  static bool carved = false;
  if (!carved) {
    cudaFuncSetAttribute(k_prolong16<CORR, true, ND, false, T>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_prolong16<CORR, false, ND, false, T>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if constexpr (ND == 2) {
      cudaFuncSetAttribute(k_prolong16<CORR, true, 2, true, T>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      cudaFuncSetAttribute(k_prolong16<CORR, false, 2, true, T>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    carved = true;
  }
  if (zero_accumulators(d.meta_out, s) != cudaSuccess) return BFP_ERR_CUDA;
  const TransferP P{vin(dc), yv, d, o, rs};
  if constexpr (ND == 2) {   // recordable for batched solves
    if (d.mode == kQcomp)
      launch_rec<TransferP, &k_prolong16<CORR, true, 2, false, T>, &k_prolong16<CORR, true, 2, true, T>>(grid, 128, 0, s, P);
    launch_rec<TransferP, &k_prolong16<CORR, false, 2, false, T>, &k_prolong16<CORR, false, 2, true, T>>(grid, 128, 0, s, P);
  } else {
    if (d.mode == kQcomp) k_prolong16<CORR, true, ND><<<grid, 128, 0, s>>>(P, nullptr);
    k_prolong16<CORR, false, ND><<<grid, 128, 0, s>>>(P, nullptr);
  }
  note_launches(d.mode == kQcomp ? 2 : 1);
  return cudaGetLastError() == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

template <int ND>
int32_t restrict_launch(const bfp_vec* rf, const bfp_vec* rc, const QDesc& d, cudaStream_t s) {
  if (ND == 2 && !is32(rf)) return restrict2d16(rf, rc, d, s);
  // int32 fine mantissas of at most 27 bits (the nine-point sum exact in int32) into an int32 output
  if (ND == 2 && is32(rf) && !is64(rf) && is32(rc) && !is64(rc) && rf->w <= 27) return restrict2d16<int32_t>(rf, rc, d, s);
  if (ND == 3 && !is32(rf)) return restrict3d16(rf, rc, d, s);
  if (is32(rf)) return launch_quant(OpRestrict<int32_t, ND>{vin(rf), rc->n[1]}, d, rc, s);
  return launch_quant(OpRestrict<int16_t, ND>{vin(rf), rc->n[1]}, d, rc, s);
}

template <int ND, bool CORR>
int32_t prolong_launch(const bfp_vec* dc, const bfp_vec* y, const bfp_vec* out, const QDesc& d, cudaStream_t s) {
  if (CORR && is32(dc) != is32(y)) {   // mixed storage (progressive widths): y's storage at run time
    if (is32(dc)) return launch_quant(OpProlong<int32_t, ND, true, int64_t>{vin(dc), vin(y), esize(y)}, d, out, s);
    return launch_quant(OpProlong<int16_t, ND, true, int64_t>{vin(dc), vin(y), esize(y)}, d, out, s);
  }
  if (!is32(dc)) return prolong16<CORR, ND>(dc, y, out, d, s);
  // int32 mantissas (d of at most 29 bits: P_m d exact in int32; y int32 when corrected) into an int32 output
  if constexpr (ND == 2) {
    if (!is64(dc) && dc->w <= 29 && is32(out) && !is64(out) && (!CORR || !is64(y)))
      return prolong16<CORR, ND, int32_t>(dc, y, out, d, s);
  }
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
  const int nd = r_f->ndim;
  int rule = 0;
  if ((rc = desc_restrict(nd, r_f->w, d, &rule)) || (rc = fill_q(d, q, r_c, rule))) return rc;
  d.meta_a = r_f->meta; d.meta_out = r_c->meta; d.stats = st ? st->counters : nullptr;
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
    if (overlaps(y, y_out)) return BFP_ERR_ARG;
  }
  QDesc d = blank_desc();
  const int nd = dc->ndim;
  int rule = 0;
  if ((rc = desc_prolong(nd, dc->w, y ? y->w : 0, d, &rule)) || (rc = fill_q(d, q, y_out, rule))) return rc;
  d.meta_out = y_out->meta; d.stats = st ? st->counters : nullptr;
  d.meta_a = dc->meta;
  if (y) d.meta_b = y->meta;
  cudaStream_t s = as_stream(stream);
  if (nd == 2) return y ? prolong_launch<2, true>(dc, y, y_out, d, s) : prolong_launch<2, false>(dc, y, y_out, d, s);
  return y ? prolong_launch<3, true>(dc, y, y_out, d, s) : prolong_launch<3, false>(dc, y, y_out, d, s);
}

}  // extern "C"
