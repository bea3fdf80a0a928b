// bfp_host.h -- host-side validation, view construction and launch helpers
// shared by the C ABI translation units.
#pragma once

#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "bfp/bfp.h"
#include "bfp_ops.cuh"

namespace bfp {

// Counts every kernel this library enqueues (directly or into a captured graph).
void note_launches(int n);

// When set (by the multigrid driver, for the ops it enqueues), the output meta
// accumulators have already been zeroed for this op and the per-op memset is
// skipped.  Thread-local: other host threads calling the C ABI are unaffected.
bool& prezeroed();
struct PrezeroedScope {
  bool saved;
  PrezeroedScope() : saved(prezeroed()) { prezeroed() = true; }
  ~PrezeroedScope() { prezeroed() = saved; }
};

// Rows per warp strip of the row-walking kernels: the launchers' size
// heuristic unless a solver with a tuned schedule set an override for the ops
// it enqueues (thread-local, like PrezeroedScope).
int& tile_rows_override();
struct TileScope {
  int saved;
  explicit TileScope(int rows) : saved(tile_rows_override()) { if (rows > 0) tile_rows_override() = rows; }
  ~TileScope() { tile_rows_override() = saved; }
};
// Cap on the ops' default w_add (Table tab:estimates values): w_tmp = w_out + min(w_add*, cap)
// for ops enqueued inside the scope (negative: no cap; thread-local).
int& wadd_cap();
struct WaddScope {
  int saved;
  explicit WaddScope(int cap) : saved(wadd_cap()) { wadd_cap() = cap; }
  ~WaddScope() { wadd_cap() = saved; }
};
inline int capped_wadd(int rule, int cap) { return cap >= 0 && cap < rule ? cap : rule; }
inline int pick_rows(int heuristic, int cap) {
  const int v = tile_rows_override();
  return v > 0 ? (v < cap ? v : cap) : heuristic;
}

// ---- launch records (batched solves) ------------------------------------------
//
// While a recorder is installed (thread-local), the launch sites of the kernels
// that have a batched form, and the zeroing / device-to-device copies of the
// solver, append a record instead of enqueueing work.  A batched solve records
// the schedule of every instance, then replays records at the same position of
// instances with the same schedule as ONE launch of the batched kernel form
// (blockIdx.z = instance, parameters read from a device array).

using BatchedLaunch = void (*)(dim3 grid, dim3 block, size_t smem, cudaStream_t s, const void* params, int count);

struct LaunchRec {
  int32_t op = 0;                    // 0: kernel, 1: zero bytes, 2: device-to-device copy
  BatchedLaunch launch = nullptr;    // op 0: the batched form of the kernel
  dim3 grid, block;
  size_t smem = 0;
  std::vector<unsigned char> params; // op 0: the kernel's parameter struct
  void* dst = nullptr;               // ops 1, 2
  const void* src = nullptr;
  size_t bytes = 0;
};

std::vector<LaunchRec>*& launch_recorder();

// The batched form of kernel KB (parameters P[count] in device memory, grid z = count).
// Launch with programmatic stream serialization: the kernel may start while the previous kernel in
// the stream finishes; every kernel launched this way waits (pdl_wait) before its memory accesses.
template <class P, void (*K)(const P, const P*)>
inline void launch_pdl(dim3 g, dim3 b, size_t smem, cudaStream_t s, const P& p, const P* pb) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, K, p, pb);
}

template <class P, void (*KB)(const P, const P*)>
void batched_launch(dim3 g, dim3 b, size_t smem, cudaStream_t s, const void* params, int count) {
  launch_pdl<P, KB>(dim3(g.x, g.y, (unsigned)count), b, smem, s, P{}, reinterpret_cast<const P*>(params));
}

// Launches K1 with parameters p, or records it (with its batched form KB) while a recorder is installed.
template <class P, void (*K1)(const P, const P*), void (*KB)(const P, const P*)>
inline void launch_rec(dim3 g, dim3 b, size_t smem, cudaStream_t s, const P& p) {
  if (std::vector<LaunchRec>* r = launch_recorder()) {
    LaunchRec rec;
    rec.launch = &batched_launch<P, KB>;
    rec.grid = g;
    rec.block = b;
    rec.smem = smem;
    rec.params.resize(sizeof(P));
    std::memcpy(rec.params.data(), &p, sizeof(P));
    r->push_back(std::move(rec));
    return;
  }
  launch_pdl<P, K1>(g, b, smem, s, p, static_cast<const P*>(nullptr));
}

// cudaMemsetAsync(p, 0, bytes) / a device-to-device cudaMemcpyAsync, or their records.
inline cudaError_t mem_zero(void* p, size_t bytes, cudaStream_t s) {
  if (std::vector<LaunchRec>* r = launch_recorder()) {
    LaunchRec rec;
    rec.op = 1;
    rec.dst = p;
    rec.bytes = bytes;
    r->push_back(std::move(rec));
    return cudaSuccess;
  }
  return cudaMemsetAsync(p, 0, bytes, s);
}
inline cudaError_t mem_copy(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (std::vector<LaunchRec>* r = launch_recorder()) {
    LaunchRec rec;
    rec.op = 2;
    rec.dst = dst;
    rec.src = src;
    rec.bytes = bytes;
    r->push_back(std::move(rec));
    return cudaSuccess;
  }
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
}

inline cudaError_t zero_accumulators(int64_t* meta_out, cudaStream_t s) {
  if (prezeroed()) return cudaSuccess;
  return mem_zero(meta_out + 1, (BFP_META_WORDS - 1) * sizeof(int64_t), s);
}

inline cudaStream_t as_stream(bfp_stream s) { return reinterpret_cast<cudaStream_t>(s); }

inline int hmsb(int64_t z) {  // host msb (Sec. 2 signed width)
  uint64_t v = (uint64_t)(z ^ (z >> 63));
  int b = 0;
  while (v) { ++b; v >>= 1; }
  return b + 1;
}

inline int clog2(int64_t m) {
  int b = 0;
  uint64_t v = (uint64_t)(m - 1);
  while (v) { ++b; v >>= 1; }
  return b;
}

inline bool is32(const bfp_vec* v) { return v->w > 16; }
// int64 mantissas (33 <= w <= 62): accepted only by the ops that check with check_vec_wide
inline bool is64(const bfp_vec* v) { return v->w > 32; }
inline int esize(const bfp_vec* v) { return v->w > 32 ? 8 : (v->w > 16 ? 4 : 2); }

inline int32_t check_vec_w(const bfp_vec* v, int wmax) {
  if (!v || !v->mant || !v->meta) return BFP_ERR_ARG;
  if (v->w < 1 || v->w > wmax) return BFP_ERR_ARG;
  if (v->ndim < 1 || v->ndim > 3) return BFP_ERR_SHAPE;
  for (int i = 0; i < 3; ++i)
    if (v->n[i] < 0) return BFP_ERR_SHAPE;
  for (int i = v->ndim; i < 3; ++i)
    if (v->n[i] != 1) return BFP_ERR_SHAPE;
  if (v->ld < v->n[0] || v->ld % 8 != 0 || v->ld <= 0) return BFP_ERR_SHAPE;
  if (reinterpret_cast<uintptr_t>(v->mant) % 16 != 0) return BFP_ERR_SHAPE;
  if (reinterpret_cast<uintptr_t>(v->meta) % 8 != 0) return BFP_ERR_SHAPE;
  return BFP_OK;
}
inline int32_t check_vec(const bfp_vec* v) { return check_vec_w(v, 32); }
inline int32_t check_vec_wide(const bfp_vec* v) { return check_vec_w(v, 62); }

inline int64_t rows_of(const bfp_vec* v) { return v->n[1] * v->n[2]; }

inline bool same_shape(const bfp_vec* a, const bfp_vec* b) {
  return a->ndim == b->ndim && a->n[0] == b->n[0] && a->n[1] == b->n[1] && a->n[2] == b->n[2];
}

inline bool overlaps(const bfp_vec* a, const bfp_vec* b) {
  if (!a || !b) return false;
  const char* a0 = (const char*)a->mant;
  const char* a1 = a0 + (rows_of(a) * a->ld) * esize(a);
  const char* b0 = (const char*)b->mant;
  const char* b1 = b0 + (rows_of(b) * b->ld) * esize(b);
  bool mant = a0 < b1 && b0 < a1 && rows_of(a) > 0 && rows_of(b) > 0;
  bool meta = (a->meta < b->meta + BFP_META_WORDS) && (b->meta < a->meta + BFP_META_WORDS);
  return mant || meta;
}

inline VIn vin(const bfp_vec* v) {
  VIn r;
  r.m = v ? v->mant : nullptr;
  r.ld = v ? v->ld : 8;
  r.nx = v ? v->n[0] : 0;
  r.ny = v ? v->n[1] : 1;
  r.nz = v ? v->n[2] : 1;
  return r;
}

inline VOut vout(const bfp_vec* v) {
  VOut r;
  r.m = v->mant;
  r.ld = v->ld;
  r.nx = v->n[0];
  r.ny = v->n[1];
  r.nz = v->n[2];
  r.is32 = is32(v) ? 1 : 0;
  r.is64 = is64(v) ? 1 : 0;
  return r;
}

inline int sm_count() {
  static int cached = 0;
  if (!cached) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || cached <= 0)
      cached = 148;
  }
  return cached;
}

inline unsigned grid_for(int64_t work_items, int threads) {
  int64_t b = (work_items + threads - 1) / threads;
  int64_t cap = (int64_t)sm_count() * 8;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// Fills the quantisation fields of a QDesc from a bfp_q; w_add_rule is the
// op's Table tab:estimates value.
inline int32_t fill_q(QDesc& d, const bfp_q* q, const bfp_vec* out, int w_add_rule, bool wide_ok = false) {
  if (!q || q->w_out < 1 || q->w_out > (wide_ok ? 62 : 32) || q->w_out != out->w) return BFP_ERR_ARG;
  if (q->mode != BFP_QCOMP && q->mode != BFP_NNQCOMP) return BFP_ERR_ARG;
  int w_add = q->w_add < 0 ? capped_wadd(w_add_rule, wadd_cap()) : q->w_add;
  d.mode = q->mode;
  d.w_out = q->w_out;
  d.w_tmp = q->w_out + w_add;
  d.use_tmp = (q->mode == BFP_QCOMP && q->tmp != nullptr && d.w_tmp <= 32) ? 1 : 0;
  d.tmp = d.use_tmp ? q->tmp : nullptr;
  if (d.use_tmp && reinterpret_cast<uintptr_t>(q->tmp) % 16 != 0) return BFP_ERR_SHAPE;
  d.has_gamma = q->has_gamma ? 1 : 0;
  if (q->has_gamma && q->gamma.m < 0) return BFP_ERR_ARG;
  d.gamma_m = q->gamma.m;
  d.gamma_e = q->gamma.e;
  return BFP_OK;
}

inline QDesc blank_desc() {
  QDesc d;
  std::memset(&d, 0, sizeof(d));
  return d;
}

// memset of the output meta's accumulators, then the pass(es) of the op.
template <class Op>
inline int32_t launch_quant(const Op& op, const QDesc& q, const bfp_vec* out, cudaStream_t s) {
  if (q.hbits > 62 || (q.two && q.lbits > 62)) return BFP_ERR_WIDTH;
  VOut o = vout(out);
  const int threads = 256;
  const int64_t items = rows_of(out) * (out->ld / 8);
  unsigned g = grid_for(items, threads);
  if (zero_accumulators(q.meta_out, s) != cudaSuccess) return BFP_ERR_CUDA;
  if (q.mode == kQcomp) k_quant<Op, true><<<g, threads, 0, s>>>(op, q, o);
  k_quant<Op, false><<<g, threads, 0, s>>>(op, q, o);
  note_launches(q.mode == kQcomp ? 2 : 1);
  return cudaGetLastError() == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

// The same for an output with int64 mantissas (33 <= w_out <= 62).
template <class Op>
inline int32_t launch_quant_wide(const Op& op, const QDesc& q, const bfp_vec* out, cudaStream_t s) {
  if (q.hbits > 62 || (q.two && q.lbits > 62)) return BFP_ERR_WIDTH;
  VOut o = vout(out);
  const int threads = 256;
  const int64_t items = rows_of(out) * (out->ld / 8);
  unsigned g = grid_for(items, threads);
  if (zero_accumulators(q.meta_out, s) != cudaSuccess) return BFP_ERR_CUDA;
  if (q.mode == kQcomp) k_quant_wide<Op, true><<<g, threads, 0, s>>>(op, q, o);
  k_quant_wide<Op, false><<<g, threads, 0, s>>>(op, q, o);
  note_launches(q.mode == kQcomp ? 2 : 1);
  return cudaGetLastError() == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

}  // namespace bfp
