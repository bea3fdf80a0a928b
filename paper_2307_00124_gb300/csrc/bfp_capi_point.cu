// bfp_capi_point.cu -- C ABI: helpers and the pointwise BFP ops
// (normalise, axpby, dot, FP64 <-> BFP conversion).
#include <atomic>
#include <cmath>

#include "bfp_host.h"

using namespace bfp;

namespace bfp {
static std::atomic<long long> g_launches{0};
std::vector<LaunchRec>*& launch_recorder();
void note_launches(int n) {
  if (launch_recorder()) return;   // recorded, not launched (a batched replay counts its own launches)
  g_launches.fetch_add(n, std::memory_order_relaxed);
}
bool& prezeroed() {
  static thread_local bool flag = false;
  return flag;
}
int& tile_rows_override() {
  static thread_local int rows = 0;
  return rows;
}
int& wadd_cap() {
  static thread_local int cap = -1;
  return cap;
}
std::vector<LaunchRec>*& launch_recorder() {
  static thread_local std::vector<LaunchRec>* rec = nullptr;
  return rec;
}
}  // namespace bfp

namespace {

// ---- FP64 -> BFP (quant() of Alg. ir, read as floor) ---------------------

// Exact split of a double: v = M * 2^E (|M| < 2^53).  Returns false for NaN/Inf.
__device__ __forceinline__ bool f64_split(double v, int64_t& M, int64_t& E) {
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  const int ex = (int)((b >> 52) & 0x7ff);
  const uint64_t fr = b & ((1ull << 52) - 1);
  if (ex == 0x7ff) return false;
  if (ex == 0) { M = (int64_t)fr; E = -1074; }
  else { M = (int64_t)(fr | (1ull << 52)); E = ex - 1075; }
  if (b >> 63) M = -M;
  return true;
}

constexpr int64_t kF64KeyOffset = 4096;   // keeps the msb key positive for atomicMax
constexpr int64_t kF64EStar = -1074;      // every double is a multiple of 2^-1074

struct FromF64P {
  const double* x;
  VOut out;
  int64_t* meta_out;
  int32_t w, pass1;
};

// B: a batched launch, grid z the instance, parameters Pb[z]
template <bool B = false>
__global__ void __launch_bounds__(256) k_from_f64(const __grid_constant__ FromF64P P1,
                                                  const FromF64P* __restrict__ Pb) {
  pdl_wait();
  const FromF64P& P = B ? Pb[blockIdx.z] : P1;
  const double* __restrict__ x = P.x;
  const VOut& out = P.out;
  int64_t* meta_out = P.meta_out;
  const int w = P.w;
  const bool pass1 = P.pass1 != 0;
  const int64_t nvec = out.ld >> 3, rows = out.ny * out.nz, total = rows * nvec;
  int64_t e_out = 0;
  if (!pass1) {
    const int64_t key = meta_out[kMetaMu];
    const int64_t mu_abs = key > 0 ? key - kF64KeyOffset : kF64EStar + 1;
    e_out = mu_abs - w;
  }
  Red red = {0, 0, 0};
  bool bad = false;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / nvec, c0 = (idx - row * nvec) << 3;
    int64_t o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      o[k] = 0;
      const int64_t c = c0 + k;
      if (c >= out.nx) continue;
      int64_t M = 0, E = kF64EStar;
      if (!f64_split(x[row * out.nx + c], M, E)) { bad = true; continue; }
      if (pass1) {
        const int64_t mv = M == 0 ? kF64EStar + 1 : msb64(M) + E;
        red.key = max(red.key, (long long)(mv + kF64KeyOffset));
      } else {
        const int64_t sh = E - e_out;
        const int64_t v = sh >= 0 ? (int64_t)((uint64_t)M << (sh > 63 ? 63 : sh)) : (M >> (-sh > 63 ? 63 : -sh));
        o[k] = v;
        red.nrm = max(red.nrm, (long long)(v < 0 ? -v : v));
      }
    }
    if (!pass1) {
      if (out.is64) {
        stw8(out, row, c0, o);
      } else {
        int32_t o32[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) o32[k] = (int32_t)o[k];
        st8(out, row, c0, o32);
      }
    }
  }
  if (bad) atomicOr((unsigned long long*)&meta_out[BFP_META_FLAGS], 1ull);
  block_commit(red, meta_out, nullptr, pass1);
  if (!pass1 && blockIdx.x == 0 && threadIdx.x == 0) meta_out[0] = e_out;
}

struct ToF64P {
  VIn x;
  const int64_t* meta;
  double* out;
};

template <class T, bool B = false>
__global__ void __launch_bounds__(256) k_to_f64(const __grid_constant__ ToF64P P1, const ToF64P* __restrict__ Pb) {
  pdl_wait();
  const ToF64P& P = B ? Pb[blockIdx.z] : P1;
  const VIn& x = P.x;
  const int64_t* meta = P.meta;
  double* __restrict__ out = P.out;
  const int64_t rows = x.ny * x.nz, total = rows * x.nx;
  int64_t e = meta[0];
  const int ei = (int)(e > 4000 ? 4000 : (e < -4000 ? -4000 : e));
  const T* m = reinterpret_cast<const T*>(x.m);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / x.nx, c = idx - row * x.nx;
    out[idx] = ldexp((double)m[row * x.ld + c], ei);
  }
}

// ---- exact dot product (Sec. 2 remark: one wide accumulator, one final shift) ----

template <class T>
__global__ void __launch_bounds__(256) k_dot(const VIn x, const VIn y, int64_t* out) {
  const int64_t rows = x.ny * x.nz, total = rows * x.nx;
  const T* a = reinterpret_cast<const T*>(x.m);
  const T* b = reinterpret_cast<const T*>(y.m);
  i128 acc = 0;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / x.nx, c = idx - row * x.nx;
    acc += (i128)((int64_t)a[row * x.ld + c] * (int64_t)b[row * y.ld + c]);
  }
  // block reduction of the 128-bit partial sums
  __shared__ long long s_lo[8], s_hi[8];
  uint64_t lo = (uint64_t)acc;
  int64_t hi = (int64_t)(acc >> 64);
  for (int o = 16; o > 0; o >>= 1) {
    uint64_t lo2 = (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)lo, o);
    int64_t hi2 = (int64_t)__shfl_xor_sync(0xffffffffu, (long long)hi, o);
    i128 s = (((i128)hi << 64) | (i128)lo) + (((i128)hi2 << 64) | (i128)lo2);
    lo = (uint64_t)s;
    hi = (int64_t)(s >> 64);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { s_lo[wid] = (long long)lo; s_hi[wid] = (long long)hi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    i128 s = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += ((i128)s_hi[k] << 64) | (i128)(uint64_t)s_lo[k];
    // 32-bit limbs: three unsigned, the top one signed (two's complement sums)
    const u128 u = (u128)s;
    atomicAdd((unsigned long long*)&out[2], (unsigned long long)(uint32_t)(u));
    atomicAdd((unsigned long long*)&out[3], (unsigned long long)(uint32_t)(u >> 32));
    atomicAdd((unsigned long long*)&out[4], (unsigned long long)(uint32_t)(u >> 64));
    atomicAdd((unsigned long long*)&out[5], (unsigned long long)(int64_t)(s >> 96));
  }
}

__global__ void k_dot_finish(const int64_t* mx, const int64_t* my, int64_t* out, int w_out) {
  const i128 s = (i128)(uint64_t)out[2] + ((i128)(uint64_t)out[3] << 32) + ((i128)(uint64_t)out[4] << 64) +
                 ((i128)out[5] << 96);
  const int64_t e_star = mx[0] + my[0];
  const int mu = msb128(s);
  const int lam = mu - w_out;   // Alg. qcomp: lambda_out = mu* - w_out
  i128 m = lam >= 0 ? (s >> lam) : (i128)((u128)s << (-lam));
  out[0] = (int64_t)m;
  out[1] = e_star + lam;
}

// ---- max |m| of a block (the norm word of its meta) -------------------------------

template <class T>
__global__ void __launch_bounds__(256) k_block_norm(const VIn x, int64_t* meta) {
  const int64_t rows = x.ny * x.nz, total = rows * x.nx;
  const T* m = reinterpret_cast<const T*>(x.m);
  long long mx = 0;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / x.nx, c = idx - row * x.nx;
    const long long v = (long long)m[row * x.ld + c];
    mx = max(mx, v < 0 ? -v : v);
  }
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax((long long*)&meta[1], mx);
}

}  // namespace

// ---------------------------------------------------------------------------

extern "C" {

const char* bfp_status_str(int32_t st) {
  switch (st) {
    case BFP_OK: return "ok";
    case BFP_ERR_ARG: return "invalid argument";
    case BFP_ERR_SHAPE: return "invalid shape, leading dimension or alignment";
    case BFP_ERR_WIDTH: return "exact intermediate wider than 62 bits";
    case BFP_ERR_CUDA: return "CUDA runtime error";
    case BFP_ERR_NONFINITE: return "non-finite FP64 input";
    case BFP_ERR_TIMEOUT: return "bounded device wait timed out";
    case BFP_ERR_NOCONV: return "iteration limit reached";
    case BFP_ERR_CAPACITY: return "size exceeds the fixed static scratch capacity";
    default: return "unknown status";
  }
}

int32_t bfp_version(void) { return 100; }

int64_t bfp_kernel_launches(void) { return (int64_t)g_launches.load(); }

int64_t bfp_pitch(int64_t n0) { return n0 <= 0 ? 8 : ((n0 + 7) / 8) * 8; }

int32_t bfp_scalar_from_double(double x, int32_t w, bfp_scalar* out) {
  if (!out || w < 1 || w > 32 || !std::isfinite(x)) return BFP_ERR_ARG;
  if (x == 0.0) { out->m = 0; out->e = 0; return BFP_OK; }
  // exact split x = M 2^E (|M| < 2^53), then the smallest e with floor(x / 2^e) in X_w.
  // At e0 = msb(M) + E - w - 2 the floor needs >= w + 1 bits, so e0 is below the
  // minimum; fitting is monotone in e, so the first e that fits is the minimum.
  int ex = 0;
  double fm = std::frexp(x, &ex);
  int64_t M = (int64_t)std::ldexp(fm, 53);
  int64_t E = ex - 53;
  int64_t e = (int64_t)hmsb(M) + E - w - 2;
  int64_t m = 0;
  for (;;) {
    int64_t sh = E - e;
    m = sh >= 0 ? (int64_t)((uint64_t)M << sh) : (sh <= -63 ? (M >> 63) : (M >> (-sh)));
    if (hmsb(m) <= w) break;
    ++e;
  }
  out->m = m;
  out->e = e;
  return BFP_OK;
}

int32_t bfp_laplace_stencil(int32_t ndim, double omega, int32_t w_omega, bfp_stencil* out) {
  if (!out || (ndim != 2 && ndim != 3) || !(omega > 0.0)) return BFP_ERR_ARG;
  std::memset(out, 0, sizeof(*out));
  out->ndim = ndim;
  if (ndim == 2) { out->center = 4; out->nbr = -1; out->e = -2; }
  else { out->center = 6; out->nbr = -1; out->e = -3; }
  const double pscale = ndim == 2 ? 4.0 : 8.0;
  return bfp_scalar_from_double(omega * pscale / (2.0 * ndim), w_omega, &out->omega);
}

int32_t bfp_normalize(const bfp_vec* x, const bfp_vec* out, const bfp_q* q, const bfp_stats* st,
                      bfp_stream stream) {
  int32_t rc;
  if ((rc = check_vec_wide(x)) || (rc = check_vec_wide(out))) return rc;
  if (!same_shape(x, out)) return BFP_ERR_SHAPE;
  if (overlaps(x, out)) return BFP_ERR_ARG;
  QDesc d = blank_desc();
  if ((rc = fill_q(d, q, out, 2, true))) return rc;
  d.meta_a = x->meta;
  d.meta_out = out->meta;
  d.stats = st ? st->counters : nullptr;
  d.ch = 0; d.ha = 1; d.two = 0; d.hbits = x->w;
  d.ng = 1; d.gv[0] = 0; d.gm[0] = 1; d.ge[0] = 0;   // gamma = ||x||
  cudaStream_t s = as_stream(stream);
  if (is64(x) || is64(out)) {
    const OpCopyW op{vin(x), esize(x)};
    return is64(out) ? launch_quant_wide(op, d, out, s) : launch_quant(op, d, out, s);
  }
  if (is32(x)) return launch_quant(OpCopy<int32_t>{vin(x)}, d, out, s);
  return launch_quant(OpCopy<int16_t>{vin(x)}, d, out, s);
}

int32_t bfp_axpy(bfp_scalar a, const bfp_vec* x, bfp_scalar b, const bfp_vec* y, const bfp_vec* z,
                 const bfp_q* q, const bfp_stats* st, bfp_stream stream) {
  int32_t rc;
  if ((rc = check_vec_wide(x)) || (rc = check_vec_wide(y)) || (rc = check_vec_wide(z))) return rc;
  if (!same_shape(x, y) || !same_shape(x, z)) return BFP_ERR_SHAPE;
  if (overlaps(x, z) || overlaps(y, z)) return BFP_ERR_ARG;
  if (a.m >= (1ll << 31) || a.m < -(1ll << 31) || b.m >= (1ll << 31) || b.m < -(1ll << 31)) return BFP_ERR_ARG;
  QDesc d = blank_desc();
  if ((rc = fill_q(d, q, z, 2, true))) return rc;
  d.meta_a = x->meta; d.meta_b = y->meta; d.meta_out = z->meta;
  d.stats = st ? st->counters : nullptr;
  d.ch = a.e; d.ha = 1;                 // alpha x at e_alpha + e_x (Alg. eaxpby-setup)
  d.cl = b.e; d.lb = 1;                 // beta y at e_beta + e_y
  d.two = 1;
  d.hbits = hmsb(a.m) + x->w;
  d.lbits = hmsb(b.m) + y->w;
  d.ng = 2;                             // gamma = |alpha| ||x|| + |beta| ||y||
  d.gv[0] = 0; d.gm[0] = (uint64_t)(a.m < 0 ? -a.m : a.m); d.ge[0] = a.e;
  d.gv[1] = 1; d.gm[1] = (uint64_t)(b.m < 0 ? -b.m : b.m); d.ge[1] = b.e;
  cudaStream_t s = as_stream(stream);
  if (is64(x) || is64(y) || is64(z)) {
    const OpAxpyW op{vin(x), vin(y), esize(x), esize(y), a.m, b.m};
    return is64(z) ? launch_quant_wide(op, d, z, s) : launch_quant(op, d, z, s);
  }
  if (is32(x)) {
    if (is32(y)) return launch_quant(OpAxpy<int32_t, int32_t>{vin(x), vin(y), a.m, b.m}, d, z, s);
    return launch_quant(OpAxpy<int32_t, int16_t>{vin(x), vin(y), a.m, b.m}, d, z, s);
  }
  if (is32(y)) return launch_quant(OpAxpy<int16_t, int32_t>{vin(x), vin(y), a.m, b.m}, d, z, s);
  return launch_quant(OpAxpy<int16_t, int16_t>{vin(x), vin(y), a.m, b.m}, d, z, s);
}

int32_t bfp_from_f64(const double* x, const bfp_vec* out, bfp_stream stream) {
  int32_t rc;
  if (!x) return BFP_ERR_ARG;
  if ((rc = check_vec_wide(out))) return rc;
  cudaStream_t s = as_stream(stream);
  VOut o = vout(out);
  const int64_t items = rows_of(out) * (out->ld / 8);
  unsigned g = grid_for(items, 256);
  if (mem_zero(out->meta + 1, (BFP_META_WORDS - 1) * sizeof(int64_t), s) != cudaSuccess) return BFP_ERR_CUDA;
  launch_rec<FromF64P, &k_from_f64<>, &k_from_f64<true>>(g, 256, 0, s, FromF64P{x, o, out->meta, out->w, 1});
  launch_rec<FromF64P, &k_from_f64<>, &k_from_f64<true>>(g, 256, 0, s, FromF64P{x, o, out->meta, out->w, 0});
  note_launches(2);
  return cudaGetLastError() == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

int32_t bfp_to_f64(const bfp_vec* x, double* out, bfp_stream stream) {
  int32_t rc;
  if (!out) return BFP_ERR_ARG;
  if ((rc = check_vec_wide(x))) return rc;
  cudaStream_t s = as_stream(stream);
  const int64_t total = rows_of(x) * x->n[0];
  if (total == 0) return BFP_OK;
  unsigned g = grid_for(total, 256);
  const ToF64P P{vin(x), x->meta, out};
  if (is64(x)) launch_rec<ToF64P, &k_to_f64<long long>, &k_to_f64<long long, true>>(g, 256, 0, s, P);
  else if (is32(x)) launch_rec<ToF64P, &k_to_f64<int32_t>, &k_to_f64<int32_t, true>>(g, 256, 0, s, P);
  else launch_rec<ToF64P, &k_to_f64<int16_t>, &k_to_f64<int16_t, true>>(g, 256, 0, s, P);
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

int32_t bfp_dot(const bfp_vec* x, const bfp_vec* y, int32_t w_out, int64_t* out, bfp_stream stream) {
  int32_t rc;
  if ((rc = check_vec(x)) || (rc = check_vec(y))) return rc;
  if (!out || w_out < 1 || w_out > 62) return BFP_ERR_ARG;
  if (!same_shape(x, y) || is32(x) != is32(y)) return BFP_ERR_SHAPE;
  cudaStream_t s = as_stream(stream);
  if (cudaMemsetAsync(out, 0, BFP_META_WORDS * sizeof(int64_t), s) != cudaSuccess) return BFP_ERR_CUDA;
  const int64_t total = rows_of(x) * x->n[0];
  unsigned g = grid_for(total, 256);
  if (is32(x)) k_dot<int32_t><<<g, 256, 0, s>>>(vin(x), vin(y), out);
  else k_dot<int16_t><<<g, 256, 0, s>>>(vin(x), vin(y), out);
  k_dot_finish<<<1, 1, 0, s>>>(x->meta, y->meta, out, w_out);
  note_launches(2);
  return cudaGetLastError() == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

int32_t bfp_block_norm(const bfp_vec* x, bfp_stream stream) {
  int32_t rc;
  if ((rc = check_vec_wide(x))) return rc;
  cudaStream_t s = as_stream(stream);
  if (cudaMemsetAsync(x->meta + 1, 0, sizeof(int64_t), s) != cudaSuccess) return BFP_ERR_CUDA;
  const int64_t total = rows_of(x) * x->n[0];
  if (total == 0) return BFP_OK;
  unsigned g = grid_for(total, 256);
  if (is64(x)) k_block_norm<long long><<<g, 256, 0, s>>>(vin(x), x->meta);
  else if (is32(x)) k_block_norm<int32_t><<<g, 256, 0, s>>>(vin(x), x->meta);
  else k_block_norm<int16_t><<<g, 256, 0, s>>>(vin(x), x->meta);
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

}  // extern "C"
