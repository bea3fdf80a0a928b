// bfp_mg.cu -- BFP multigrid driver: V(nu1,nu2)-cycle (Alg. v-cycle with damped
// Jacobi), FP64 iterative refinement (Alg. ir with FP64 residual and update),
// and full multigrid (Alg. fmg).  Host code enqueues stream-ordered launches
// of the BFP ops; exponents and norms stay on the device.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "bfp_coarse.cuh"
#include "bfp_desc.h"
#include "bfp_flt_host.h"
#include "bfp_ir2d.cuh"

using namespace bfp;

namespace {

// A named NVTX range around the enqueueing of one solver phase (host side: the
// ranges show the driver's structure per level and op; a replayed graph shows
// only the ranges of its capture).
struct Nvtx {
  Nvtx(const char* what, int level) {
    char name[64];
    std::snprintf(name, sizeof(name), "bfp %s level %d", what, level);
    nvtxRangePushA(name);
  }
  ~Nvtx() { nvtxRangePop(); }
};

// ---- FP64 kernels with a fixed evaluation order --------------------------------
//
// The IR residual is r = b' - A' x with b' = s * f (s = h^2 / 2^p, exact) and
// A'x = c*x + nb*(((W + E) + S) + N [+ B + T]) evaluated with explicitly
// rounded operations (no contraction), so it is bitwise reproducible on any
// IEEE-754 machine that evaluates the same sequence.

struct Grid {
  int64_t nx, ny, nz;
};

__device__ __forceinline__ double at(const double* __restrict__ x, const Grid& g, int64_t i, int64_t j, int64_t k) {
  if (i < 0 || i >= g.nx || j < 0 || j >= g.ny || k < 0 || k >= g.nz) return 0.0;
  return x[i + g.nx * (j + g.ny * k)];
}

template <int ND>
__device__ __forceinline__ double ir_res(const double* __restrict__ b, double bscale, const double* __restrict__ x,
                                         const Grid& g, int64_t i, int64_t j, int64_t k, double cdiag, double cnb) {
  double s = __dadd_rn(at(x, g, i - 1, j, k), at(x, g, i + 1, j, k));
  s = __dadd_rn(s, at(x, g, i, j - 1, k));
  s = __dadd_rn(s, at(x, g, i, j + 1, k));
  if (ND == 3) {
    s = __dadd_rn(s, at(x, g, i, j, k - 1));
    s = __dadd_rn(s, at(x, g, i, j, k + 1));
  }
  const int64_t idx = i + g.nx * (j + g.ny * k);
  const double ax = __dadd_rn(__dmul_rn(cdiag, x[idx]), __dmul_rn(cnb, s));
  return __dsub_rn(__dmul_rn(b[idx], bscale), ax);
}

// 3D IR residual with the Alg. qcomp window (as k_ir2d): pass 1 max msb + w_tmp window
// from the previous residual's gamma, pass 2 narrows the window or recomputes.  The residual is
// ir_res<3>'s sequence with the power-of-two scalings done on the exponent field (bit-identical).
template <bool PASS1>
__global__ void __launch_bounds__(256) k_ir3d(const IrArgs a, const Grid g) {
  __shared__ IrPlan sp;
  if (threadIdx.x == 0) sp = ir_plan(a, PASS1);
  __syncthreads();
  const IrPlan& p = sp;
  if (PASS1 && blockIdx.x == 0 && threadIdx.x == 0) a.meta[4] = *a.gamma_mu;
  const int64_t nvec = a.out.ld >> 3, rows = g.ny * g.nz, total = rows * nvec;
  Red red = {0, 0, 0};
  bool bad = false;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / nvec, c0 = (idx - row * nvec) << 3;
    const int64_t j = row % g.ny, k = row / g.ny;
    int32_t o[8];
    if (!PASS1 && p.narrow) {
      const int sh = (int)(p.e_out - p.e_tmp);
      const int4* src = reinterpret_cast<const int4*>(a.tmp + row * a.out.ld + c0);
      const int4 u0 = src[0], u1 = src[1];
      const int32_t t[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        o[q] = c0 + q < g.nx ? (t[q] >> sh) : 0;
        red.nrm = max(red.nrm, (long long)(o[q] < 0 ? -o[q] : o[q]));
      }
      st8(a.out, row, c0, o);
      continue;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      o[q] = 0;
      const int64_t i = c0 + q;
      if (i >= g.nx) continue;
      double s = __dadd_rn(at(a.x, g, i - 1, j, k), at(a.x, g, i + 1, j, k));
      s = __dadd_rn(s, at(a.x, g, i, j - 1, k));
      s = __dadd_rn(s, at(a.x, g, i, j + 1, k));
      s = __dadd_rn(s, at(a.x, g, i, j, k - 1));
      s = __dadd_rn(s, at(a.x, g, i, j, k + 1));
      const int64_t xi = i + g.nx * (j + g.ny * k);
      const double cx = a.cdiag == 0.75 ? mul_three_quarters(a.x[xi]) : __dmul_rn(a.cdiag, a.x[xi]);
      const double ax = __dadd_rn(cx, -scale_pow2(s, a.nbshift, -a.cnb));
      const double r = __dsub_rn(scale_pow2(a.b[xi], a.bshift, a.bscale), ax);
      int64_t M = 0, E = -1074;
      if (!split_double(r, M, E)) { bad = true; continue; }
      if (PASS1) {
        const int64_t mv = M == 0 ? -1073 : msb64(M) + E;
        red.key = max(red.key, (long long)(mv + kIrKeyOff));
        if (p.window) a.tmp[row * a.out.ld + i] = wrap_bits((uint64_t)fshift(M, E - p.e_tmp), a.w_tmp);
      } else {
        const int64_t v = fshift(M, E - p.e_out);
        o[q] = (int32_t)v;
        red.nrm = max(red.nrm, (long long)(v < 0 ? -v : v));
      }
    }
    if (!PASS1) st8(a.out, row, c0, o);
  }
  if (bad) atomicOr((unsigned long long*)&a.meta[BFP_META_FLAGS], 1ull);
  block_commit(red, a.meta, nullptr, PASS1);
  if (!PASS1 && blockIdx.x == 0 && threadIdx.x == 0) ir_finish(a, p);
}

// ||b' - A' x||_inf (for ir_solve's host-side stopping test)
template <int ND>
__global__ void __launch_bounds__(256) k_ir_resnorm(const double* __restrict__ b, double bscale,
                                                    const double* __restrict__ x, Grid g, double cdiag,
                                                    double cnb, unsigned long long* out) {
  const int64_t total = g.nx * g.ny * g.nz;
  double mx = 0.0, mb = 0.0;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % g.nx, j = (idx / g.nx) % g.ny, k = idx / (g.nx * g.ny);
    mx = fmax(mx, fabs(ir_res<ND>(b, bscale, x, g, i, j, k, cdiag, cnb)));
    mb = fmax(mb, fabs(__dmul_rn(b[idx], bscale)));
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mb = fmax(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], (unsigned long long)__double_as_longlong(mx));   // non-negative doubles order as integers
    atomicMax(&out[1], (unsigned long long)__double_as_longlong(mb));
  }
}

// FP64 IR residual of the variable-coefficient operator (2D, dense n x n):
// r = b' - (c x - (((k_W x_W + k_E x_E) + k_S x_S) + k_N x_N)), every product and sum
// correctly rounded in this order, zero outside the grid.
__global__ void __launch_bounds__(256) k_var_res64(const double* __restrict__ b, double bscale,
                                                   const double* __restrict__ x, const double* __restrict__ kw,
                                                   const double* __restrict__ ke, const double* __restrict__ ks,
                                                   const double* __restrict__ kn, const double* __restrict__ c64,
                                                   int64_t n, double* __restrict__ r) {
  const int64_t total = n * n;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % n, j = idx / n;
    const double W = i > 0 ? x[idx - 1] : 0.0, E = i + 1 < n ? x[idx + 1] : 0.0;
    const double S = j > 0 ? x[idx - n] : 0.0, N = j + 1 < n ? x[idx + n] : 0.0;
    double s = __dadd_rn(__dmul_rn(kw[idx], W), __dmul_rn(ke[idx], E));
    s = __dadd_rn(s, __dmul_rn(ks[idx], S));
    s = __dadd_rn(s, __dmul_rn(kn[idx], N));
    const double ax = __dsub_rn(__dmul_rn(c64[idx], x[idx]), s);
    r[idx] = __dsub_rn(__dmul_rn(b[idx], bscale), ax);
  }
}

// max |r| and max |b' scale| (ir_solve's stopping test)
__global__ void __launch_bounds__(256) k_absmax2(const double* __restrict__ r, const double* __restrict__ b,
                                                 double bscale, int64_t total, unsigned long long* out) {
  double mx = 0.0, mb = 0.0;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    mx = fmax(mx, fabs(r[idx]));
    mb = fmax(mb, fabs(__dmul_rn(b[idx], bscale)));
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mb = fmax(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], (unsigned long long)__double_as_longlong(mx));
    atomicMax(&out[1], (unsigned long long)__double_as_longlong(mb));
  }
}

// ---- float baselines: FP64 IR residual rounded to FP32 (then BF16), update, conversions ----

template <class S>
__device__ __forceinline__ void fstore_f64(void* p, int64_t o, double v) {
  const float f = __double2float_rn(v);
  if (sizeof(S) == 4) reinterpret_cast<float*>(p)[o] = f;
  else reinterpret_cast<unsigned short*>(p)[o] = (unsigned short)f32_to_bf16(f);
}

template <class S>
__device__ __forceinline__ double fload_f64(const void* p, int64_t o) {
  if (sizeof(S) == 4) return (double)reinterpret_cast<const float*>(p)[o];
  return (double)bf16_to_f32(reinterpret_cast<const unsigned short*>(p)[o]);
}

// r = storage(RN32(b' - A'x)) with the FP64 residual of ir_res (fixed order)
template <int ND, class S>
__global__ void __launch_bounds__(256) k_fir_residual(const double* __restrict__ b, double bscale,
                                                      const double* __restrict__ x, Grid g, double cdiag, double cnb,
                                                      FVOut out) {
  const int64_t total = out.ld * g.ny * g.nz;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % out.ld, row = idx / out.ld, j = row % g.ny, k = row / g.ny;
    const double r = i < g.nx ? ir_res<ND>(b, bscale, x, g, i, j, k, cdiag, cnb) : 0.0;
    fstore_f64<S>(out.p, idx, r);
  }
}

// x <- x + y (y widened exactly, one FP64 rounding); kUpdRows rows of loads in flight
template <class S>
__global__ void __launch_bounds__(256) k_fir_update(double* __restrict__ x, const FVIn y) {
  const int64_t rows = y.ny * y.nz;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= y.nx) return;
  for (int64_t r0 = (int64_t)blockIdx.y * kUpdRows; r0 < rows; r0 += (int64_t)gridDim.y * kUpdRows) {
    double xv[kUpdRows], yv[kUpdRows];
#pragma unroll
    for (int k = 0; k < kUpdRows; ++k) {
      const int64_t row = r0 + k;
      if (row < rows) {
        xv[k] = x[row * y.nx + i];
        yv[k] = fload_f64<S>(y.p, row * y.ld + i);
      }
    }
#pragma unroll
    for (int k = 0; k < kUpdRows; ++k) {
      const int64_t row = r0 + k;
      if (row < rows) x[row * y.nx + i] = __dadd_rn(xv[k], yv[k]);
    }
  }
}

// dense doubles (n^d) <-> float vectors (padding written as 0)
template <class S>
__global__ void __launch_bounds__(256) k_f64_to_flt(const double* __restrict__ x, FVOut out) {
  const int64_t total = out.ld * out.ny * out.nz;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % out.ld, row = idx / out.ld;
    fstore_f64<S>(out.p, idx, i < out.nx ? x[row * out.nx + i] : 0.0);
  }
}

template <class S>
__global__ void __launch_bounds__(256) k_flt_to_f64(const FVIn v, double* __restrict__ x) {
  const int64_t total = v.nx * v.ny * v.nz;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % v.nx, row = idx / v.nx;
    x[idx] = fload_f64<S>(v.p, row * v.ld + i);
  }
}

// x <- x + m 2^e (the FP64 update of Alg. ir, sign flipped with the residual)
template <class T>
__global__ void __launch_bounds__(256) k_ir_update(double* __restrict__ x, const VIn y, const int64_t* meta) {
  const int64_t total = y.nx * y.ny * y.nz;
  const int64_t e = meta[0];
  const int ei = (int)(e > 4000 ? 4000 : (e < -4000 ? -4000 : e));
  const T* m = reinterpret_cast<const T*>(y.m);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / y.nx, c = idx - row * y.nx;
    x[idx] = __dadd_rn(x[idx], ldexp((double)m[row * y.ld + c], ei));
  }
}

// b_c = R~ (bscale * b_f), deltas in lexicographic order (outer axis first)
struct RestrictF64P {
  const double* bf;
  double bscale;
  Grid gf;
  double* bc;
  Grid gc;
  double rscale;
};

// B: a batched launch, grid z the instance, parameters Pb[z]
template <int ND, bool B = false>
__global__ void __launch_bounds__(256) k_restrict_f64(const __grid_constant__ RestrictF64P P1,
                                                      const RestrictF64P* __restrict__ Pb) {
  pdl_wait();
  const RestrictF64P& P = B ? Pb[blockIdx.z] : P1;
  const double* __restrict__ bf = P.bf;
  const double bscale = P.bscale, rscale = P.rscale;
  const Grid gf = P.gf, gc = P.gc;
  double* __restrict__ bc = P.bc;
  const int64_t total = gc.nx * gc.ny * gc.nz;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = idx % gc.nx, J = (idx / gc.nx) % gc.ny, K = idx / (gc.nx * gc.ny);
    double acc = 0.0;
    const int zr = ND == 3 ? 1 : 0;
    for (int dz = -zr; dz <= zr; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const double wgt = (double)((2 - abs(dx)) * (2 - abs(dy)) * (ND == 3 ? (2 - abs(dz)) : 1)) * rscale;
          const int64_t fi = 2 * I + 1 + dx, fj = 2 * J + 1 + dy, fk = ND == 3 ? 2 * K + 1 + dz : 0;
          const double v = __dmul_rn(bf[fi + gf.nx * (fj + gf.ny * fk)], bscale);
          acc = __dadd_rn(acc, __dmul_rn(wgt, v));
        }
    bc[idx] = acc;
  }
}

// ---- hierarchy ---------------------------------------------------------------------

// Face width of the finest operator in the IR residual with BFP x and b: the largest face gets
// 25 significant bits, so ||A'||_inf < 2^28 and A'x fits the quantiser's 62-bit group bound
// (msb(||A'||_inf) + w_x + 1 <= 62) for x up to 32 bits.
constexpr int kIrFaceBits = 26;

struct Level {
  int64_t n = 0;
  int w = 0;                      // width of this level's op results (progressive precision)
  int64_t* slots = nullptr;       // meta blocks of this level's op call sites (zeroed once per step)
  int nslots = 0;
  bfp_vec r{}, ya{}, yb{}, rv{};  // BFP buffers (mantissa + meta)
  bfp_vec rir{};                  // the level's IR residual when r's storage is the finer width's
  void* tmp = nullptr;            // qcomp window (int32)
  double* b = nullptr;            // FP64 right-hand side (levels >= 1)
  double* x = nullptr;            // FP64 iterate (levels >= 1)
  flt_vec fr{}, fya{}, fyb{}, frv{};   // float baselines: the same buffers as float vectors
  // variable coefficients: the level's operator, its unquantised FP64 faces and centre
  // (dense n x n) and the FP64 IR residual before quantisation
  bfp_varstencil vs{};
  bfp_varstencil vs_ir{};         // finest level only: the faces at kIrFaceBits (int32) for the BFP IR
  double* kf64[4] = {nullptr, nullptr, nullptr, nullptr};
  double* c64 = nullptr;
  double* r64 = nullptr;
};

}  // namespace

struct bfp_hierarchy {
  bfp_solver_opts o;
  bfp_stencil A;
  std::vector<Level> lv;
  std::vector<void*> allocs;
  uint64_t* stats = nullptr;             // counters of levels >= 1 and the on-chip coarse cycle
  uint64_t* stats0 = nullptr;            // counters of the finest level's separately launched ops
  int ir_first = 0;                      // the IR step being enqueued is an FMG level's first
  unsigned long long* norms = nullptr;   // 2 words for the residual norm
  int64_t* ir_gam = nullptr;             // per level: previous IR residual mu* (+2^40), 0 = unknown
  int64_t* arena = nullptr;              // all call-site meta blocks, contiguous
  size_t arena_words = 0;
  // on-chip coarse V-cycle: levels kc.. run in one CTA (kc = nlevels: disabled)
  int kc = 0;
  int coarse_wide = 0;                   // the on-chip cycle's storage: int32 (1) or int16 (0)
  CoarseBuf* d_bufs = nullptr;
  int nbufs = 0;
  int smem_bytes = 0;
  int meta_off = 0, ops_off = 0, bufs_off = 0, data_off = 0;
  std::vector<CoarseOp*> d_ops;          // per start level k >= kc
  std::vector<int> nops, rbuf, ybuf, runk;
  int var = 0;                           // variable-coefficient operator (bfp_hierarchy_create_var)
  int cheby = 0;                         // V(1,0) with the Chebyshev relaxation (opts.smoother)
  bfp_scalar c1{}, c2{};                 // its quantised coefficients (Alg. cheby-nodes, scaled for A')
  bfp_stencil Ares{};                    // A with omega = c1 / 2: the V residual's gamma (2 c1 + 1)/4 ||r||
  bfp_vec y0{};                          // spare finest-level buffer for ir steps
  flt_vec fy0{};                         // its float counterpart (float hierarchies)
  // captured IR step
  cudaGraphExec_t graph = nullptr;
  const double* graph_f = nullptr;
  double* graph_x = nullptr;
  cudaStream_t graph_stream = nullptr;
  // IR with a BFP iterate: scratch copy of x, and two captured steps x -> xt -> x
  bfp_vec xt{};
  size_t xt_bytes = 0;
  cudaGraphExec_t graph2 = nullptr;
  bfp_vec graph2_b{}, graph2_x{};
  cudaStream_t graph2_stream = nullptr;
};

namespace {

void* dalloc(bfp_hierarchy* h, size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, bytes < 16 ? 16 : bytes) != cudaSuccess) return nullptr;
  h->allocs.push_back(p);
  return p;
}

bool make_vec(bfp_hierarchy* h, bfp_vec& v, int nd, int64_t n, int w) {
  std::memset(&v, 0, sizeof(v));
  v.w = w;
  v.ndim = nd;
  v.n[0] = n; v.n[1] = n; v.n[2] = nd == 3 ? n : 1;
  v.ld = bfp_pitch(n);
  const size_t bytes = (size_t)(v.n[1] * v.n[2] * v.ld) * (w > 16 ? 4 : 2);
  v.mant = dalloc(h, bytes);
  v.meta = (int64_t*)dalloc(h, BFP_META_WORDS * sizeof(int64_t));
  if (!v.mant || !v.meta) return false;
  cudaMemset(v.mant, 0, bytes);
  cudaMemset(v.meta, 0, BFP_META_WORDS * sizeof(int64_t));
  return true;
}

bool make_fvec(bfp_hierarchy* h, flt_vec& v, int nd, int64_t n, int dtype) {
  std::memset(&v, 0, sizeof(v));
  v.dtype = dtype;
  v.ndim = nd;
  v.n[0] = n; v.n[1] = n; v.n[2] = nd == 3 ? n : 1;
  v.ld = bfp_pitch(n);
  const size_t bytes = (size_t)(v.n[1] * v.n[2] * v.ld) * (dtype == FLT_BF16 ? 2 : 4);
  v.data = dalloc(h, bytes);
  if (!v.data) return false;
  cudaMemset(v.data, 0, bytes);
  return true;
}

inline bool is_float(const bfp_hierarchy* h) { return h->o.arith != BFP_ARITH_BFP; }
inline int fdtype(const bfp_hierarchy* h) { return h->o.arith == BFP_ARITH_BF16 ? FLT_BF16 : FLT_F32; }

inline double pscale(int nd) { return nd == 2 ? 4.0 : 8.0; }

// Chebyshev relaxation (Alg. cheby-nodes, Alg. solver-setup).  rho: the largest eigenvalue of
// A x = lambda D x on level 5 (h = 1/32), 1 + cos(pi/32), as a literal (the correctly rounded
// double) so that no libm call enters the coefficients.
constexpr double kChebRho = 1.995184726672197;
constexpr double kChebEta = 0.15;

// c1, c2 of two Chebyshev steps on [eta rho, rho] for D^-1 A, scaled for A' (diagonal d: c1 / d,
// c2 / d^2) and floor-quantised to w_omega bits.
int32_t cheby_setup(const bfp_solver_opts* o, const bfp_stencil& A, bfp_scalar* c1q, bfp_scalar* c2q) {
  const double eta = o->cheby_eta, rho = kChebRho;
  const double alpha = 0.5 * (1.0 + eta) * rho;
  const double c = 0.5 * (1.0 - eta) * rho;
  const double beta = alpha - (c * c) / (2.0 * alpha);
  const double c1 = 2.0 / beta, c2 = -1.0 / (alpha * beta);
  const double d = (2.0 * o->ndim) / pscale(o->ndim);
  int32_t rc = bfp_scalar_from_double(c1 / d, o->w_omega, c1q);
  if (!rc) rc = bfp_scalar_from_double((c2 / d) / d, o->w_omega, c2q);
  if (rc) return rc;
  int64_t Tc, Tn, eT;
  return cheby_operator(&A, *c1q, *c2q, &Tc, &Tn, &eT);
}

struct Q {
  bfp_q q;
  bfp_stats st;
};

Q make_q(const bfp_hierarchy* h, const Level& L) {
  Q r;
  std::memset(&r, 0, sizeof(r));
  r.q.w_out = L.w;
  r.q.w_add = -1;
  r.q.mode = h->o.mode;
  r.q.tmp = (h->o.mode == BFP_QCOMP && h->o.use_tmp) ? L.tmp : nullptr;
  r.st.counters = &L == &h->lv[0] ? h->stats0 : h->stats;   // the finest level counts apart
  return r;
}

#define TRY(x)                         \
  do {                                 \
    int32_t _rc = (x);                 \
    if (_rc != BFP_OK) return _rc;     \
  } while (0)

// ---- on-chip coarse V-cycle -------------------------------------------------

struct CoarseLevelBufs {
  int r, y0, y1;
};

// One op of the on-chip schedule on level l: the QDesc the C ABI op would build (meta pointers
// unused; qcomp without the window buffer) and the op's coefficients.
// The operator whose omega feeds the V residual's gamma rule: with the Chebyshev relaxation the
// rule (2 c1 + 1)/4 ||r|| is (omega + 1/4) ||r|| at omega = c1 / 2.
const bfp_stencil* res_op(const bfp_hierarchy* h) { return h->cheby ? &h->Ares : &h->A; }

int32_t make_coarse_op(const bfp_hierarchy* h, int l, int kind, int a, int b, int out, CoarseOp* res) {
  const int nd = h->o.ndim;
  // result width: level l's; input widths for the exact-width bounds: y, r_v on level l at w_l, the
  // right-hand side at most w_(l-1) (the finer level's restriction), d from level l+1 at w_(l+1)
  const int w = h->lv[l].w;
  const int wr = l > 0 ? h->lv[l - 1].w : w;
  const int wc = l + 1 < (int)h->lv.size() ? h->lv[l + 1].w : w;
  CoarseOp op;
  std::memset(&op, 0, sizeof(op));
  op.kind = kind; op.a = a; op.b = b; op.out = out;
  QDesc& d = op.q;
  int rule = 0;
  int32_t rc = BFP_OK;
  switch (kind) {
    case cJac0: rc = desc_jacobi(&h->A, 0, wr, d, &rule); op.mw = h->A.omega.m; break;
    case cJac: {
      int64_t Sc, Sn, eS;
      rc = desc_jacobi(&h->A, w, wr, d, &rule);
      if (!rc) rc = jacobi_operator(&h->A, &Sc, &Sn, &eS);
      op.c = Sc; op.nb = Sn; op.mw = h->A.omega.m;
      break;
    }
    case cRes: rc = desc_residual(res_op(h), w, wr, d, &rule); op.c = h->A.center; op.nb = h->A.nbr; break;
    case cCheb: {   // T r as a damped-Jacobi op reading r for y, with no omega r term
      int64_t Tc = 0, Tn = 0;
      rc = desc_cheby(&h->A, h->c1, h->c2, wr, d, &rule, &Tc, &Tn);
      op.kind = cJac; op.a = b; op.c = Tc; op.nb = Tn; op.mw = 0;
      break;
    }
    case cRestrict: rc = desc_restrict(nd, w, d, &rule); break;
    default: rc = desc_prolong(nd, wc, w, d, &rule); break;
  }
  if (rc) return rc;
  if (d.hbits > 62 || (d.two && d.lbits > 62)) return BFP_ERR_WIDTH;
  if (op.c != (int32_t)op.c || op.nb != (int32_t)op.nb || op.mw != (int32_t)op.mw) return BFP_ERR_WIDTH;
  d.mode = h->o.mode;
  d.w_out = w;
  d.w_tmp = w + capped_wadd(rule, h->o.w_add_max);
  d.use_tmp = 0;
  op.solo = h->lv[l + (kind == cRestrict ? 1 : 0)].n <= 15 ? 1 : 0;   // output level size
  set_fold_consts(op);
  *res = op;
  return BFP_OK;
}

// Flattens the V-cycle schedule of levels l.. (the same op order as vcycle_rec)
int32_t coarse_flatten(const bfp_hierarchy* h, int l, int rbuf, const std::vector<CoarseLevelBufs>& lb,
                       std::vector<CoarseOp>& ops, int* res) {
  const bool coarsest = (l + 1 == (int)h->lv.size());
  const int nu1 = coarsest ? h->o.coarse_sweeps : h->o.nu1;
  const CoarseLevelBufs& B = lb[l - h->kc];
  int cur = B.y0, oth = B.y1;
  auto push = [&](int kind, int a, int b, int out) -> int32_t {
    CoarseOp op;
    TRY(make_coarse_op(h, l, kind, a, b, out, &op));
    ops.push_back(op);
    return BFP_OK;
  };
  if (h->cheby) {   // V(1,0): relaxation; residual, restriction, coarse correction
    TRY(push(cCheb, -1, rbuf, cur));
    if (!coarsest) {
      const int rnext = lb[l + 1 - h->kc].r;
      TRY(push(cRes, cur, rbuf, oth));
      TRY(push(cRestrict, oth, -1, rnext));
      int d = -1;
      TRY(coarse_flatten(h, l + 1, rnext, lb, ops, &d));
      TRY(push(cProlong, d, cur, oth)); std::swap(cur, oth);
    }
    *res = cur;
    return BFP_OK;
  }
  TRY(push(cJac0, -1, rbuf, cur));
  for (int i = 1; i < nu1; ++i) { TRY(push(cJac, cur, rbuf, oth)); std::swap(cur, oth); }
  if (!coarsest) {
    const int rnext = lb[l + 1 - h->kc].r;
    TRY(push(cRes, cur, rbuf, oth));                   // r_v (kept in the free ping-pong buffer)
    TRY(push(cRestrict, oth, -1, rnext));
    int d = -1;
    TRY(coarse_flatten(h, l + 1, rnext, lb, ops, &d));
    TRY(push(cProlong, d, cur, oth)); std::swap(cur, oth);
    for (int i = 0; i < h->o.nu2; ++i) { TRY(push(cJac, cur, rbuf, oth)); std::swap(cur, oth); }
  }
  *res = cur;
  return BFP_OK;
}

// Marks the first run of identical solo damped-Jacobi sweeps on a level of <= 32 points that
// alternate between two buffers (the coarsest level's sweeps), which the kernel runs with the grid
// in registers; returns its first op (ops.size(): none).
int mark_sweep_run(std::vector<CoarseOp>& ops, const std::vector<CoarseBuf>& bufs) {
  auto same = [&](const CoarseOp& x, const CoarseOp& p) {
    return x.kind == cJac && x.solo && !x.sync_before && x.a == p.out && x.out == p.a && x.b == p.b &&
           x.c == p.c && x.nb == p.nb && x.mw == p.mw && std::memcmp(&x.q, &p.q, sizeof(QDesc)) == 0;
  };
  for (size_t i = 0; i < ops.size(); ++i) {
    const CoarseOp& o = ops[i];
    if (!(o.kind == cJac && o.solo && o.a >= 0 && o.a != o.out && (int64_t)bufs[o.out].n * bufs[o.out].n <= 32))
      continue;
    size_t e = i + 1;
    while (e < ops.size() && same(ops[e], ops[e - 1])) ++e;
    if (e - i > 1) {
      ops[i].run = (int32_t)(e - i);
      return (int)i;
    }
  }
  return (int)ops.size();
}

// The coarsest level's sweeps in one launch (k_sweep_run) when the level has at most 32 points
// and int16 mantissas.
bool sweep_run_fits(const bfp_hierarchy* h, int k) {
  const int64_t n = h->lv[k].n;
  const int64_t np = h->o.ndim == 3 ? n * n * n : n * n;
  const bool narrow = h->lv[k].w <= 16 && (k == 0 || h->lv[k - 1].w <= 16);   // int16 r and y
  return !h->cheby && narrow && np >= 1 && np <= 32 && k + 1 == (int)h->lv.size();
}

int32_t sweep_run(bfp_hierarchy* h, int k, const bfp_vec* r, const bfp_vec* y, cudaStream_t s) {
  SweepRunArgs a;
  std::memset(&a, 0, sizeof(a));
  if (h->var) {   // the level's bfp_var_jacobi descriptors
    const bfp_varstencil& V = h->lv[k].vs;
    const int w = h->lv[k].w, wr = k > 0 ? h->lv[k - 1].w : w;
    for (int t = 0; t < 2; ++t) {
      CoarseOp& op = t == 0 ? a.op0 : a.op1;
      op.kind = t == 0 ? cVarJac0 : cVarJac;
      op.a = t == 0 ? -1 : 0;
      op.solo = 1;
      int rule = 0;
      int32_t sh = 0;
      TRY(desc_var_jacobi(&V, t == 0 ? 0 : w, wr, op.q, &rule, &sh));
      if (op.q.hbits > 62 || (op.q.two && op.q.lbits > 62)) return BFP_ERR_WIDTH;
      op.q.mode = h->o.mode;
      op.q.w_out = w;
      op.q.w_tmp = w + capped_wadd(rule, h->o.w_add_max);
      op.q.use_tmp = 0;
      set_fold_consts(op);
      if (t == 1) a.s = sh;
    }
    a.var = 1;
    auto view = [&](const void* p) {
      VIn v;
      v.m = p; v.ld = V.ld; v.nx = V.n[0]; v.ny = V.n[1]; v.nz = 1;
      return v;
    };
    for (int f = 0; f < 4; ++f) a.kf[f] = view(V.k[f]);
    a.kq = view(V.q);
  } else {
    TRY(make_coarse_op(h, k, cJac0, -1, 0, 0, &a.op0));
    TRY(make_coarse_op(h, k, cJac, 0, 0, 0, &a.op1));
  }
  a.sweeps = h->o.coarse_sweeps;
  a.n = (int32_t)h->lv[k].n;
  a.nd = h->o.ndim;
  a.r = vin(r);
  a.r_meta = r->meta;
  a.y = vout(y);
  a.y_meta = y->meta;
  a.stats = h->stats;
  launch_rec<SweepRunArgs, &k_sweep_run<false>, &k_sweep_run<true>>(dim3(1), dim3(32), 0, s, a);
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

bool allow_coarse_smem(bool is32, int optin) {
  cudaFuncAttributes fa;
  const cudaError_t e0 = is32 ? cudaFuncGetAttributes(&fa, k_coarse_vcycle<int32_t, false>)
                              : cudaFuncGetAttributes(&fa, k_coarse_vcycle<int16_t, false>);
  if (e0 != cudaSuccess) return false;
  const int dyn = optin - (int)fa.sharedSizeBytes;
  cudaError_t e1 = is32
      ? cudaFuncSetAttribute(k_coarse_vcycle<int32_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn)
      : cudaFuncSetAttribute(k_coarse_vcycle<int16_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
  if (e1 == cudaSuccess)   // the batched form (one CTA per instance) needs the same shared memory
    e1 = is32 ? cudaFuncSetAttribute(k_coarse_vcycle<int32_t, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn)
              : cudaFuncSetAttribute(k_coarse_vcycle<int16_t, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
  return e1 == cudaSuccess;
}

// Chooses kc and uploads the op lists; kc = nlevels disables the on-chip path.
int32_t coarse_setup(bfp_hierarchy* h) {
  const int nl = (int)h->lv.size();
  h->kc = nl;
  if (h->o.ndim != 2) return BFP_OK;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return BFP_OK;
  const int budget = optin - 2048;   // the kernel's static shared memory is a few hundred bytes
  int eb = h->o.w > 16 ? 4 : 2;
  const int nmax = h->o.coarse_onchip == 1 || h->o.coarse_onchip > 127 ? 127 : h->o.coarse_onchip;   // 4 columns per lane
  auto buf_bytes = [&](int64_t n) { return ((n + 2) * (n + 2) * eb + 15) / 16 * 16; };
  // the largest start level (n <= 127) whose levels, schedule and tables fit in shared memory; the
  // kernel keeps one storage type, so with progressive widths the start level, the level above it
  // (its right-hand side) and every coarser level share the storage class
  for (int k = 0; k < nl; ++k) {
    if (h->lv[k].n > nmax) continue;
    // (widths fall towards the coarsest level: comparing the level above with the coarsest covers all)
    if ((h->lv[k > 0 ? k - 1 : 0].w > 16) != (h->lv[nl - 1].w > 16)) continue;
    eb = h->lv[k].w > 16 ? 4 : 2;
    const int64_t nops = (int64_t)(nl - 1 - k) * (h->o.nu1 + 3 + h->o.nu2) + h->o.coarse_sweeps;
    int64_t bytes = (int64_t)(nl - k) * 3 * (BFP_META_WORDS * 8 + (int64_t)sizeof(CoarseBuf)) + nops * (int64_t)sizeof(CoarseOp) + 64;
    for (int l = k; l < nl; ++l) bytes += 3 * buf_bytes(h->lv[l].n);
    if (bytes <= budget) { h->kc = k; break; }
  }
  if (h->kc == nl) return BFP_OK;
  eb = h->lv[h->kc].w > 16 ? 4 : 2;
  h->coarse_wide = eb == 4;
  const int nb = (nl - h->kc) * 3;
  const int max_ops = (nl - 1 - h->kc) * (h->o.nu1 + 3 + h->o.nu2) + h->o.coarse_sweeps;
  // layout: meta blocks | buffer table | op list | mantissa buffers (16-byte aligned)
  h->meta_off = 0;
  h->bufs_off = nb * BFP_META_WORDS * 8;
  h->ops_off = (int)(((int64_t)h->bufs_off + nb * (int64_t)sizeof(CoarseBuf) + 15) / 16 * 16);
  int off = (int)(((int64_t)h->ops_off + max_ops * (int64_t)sizeof(CoarseOp) + 15) / 16 * 16);
  h->data_off = off;
  std::vector<CoarseLevelBufs> lb;
  std::vector<CoarseBuf> bufs;
  for (int l = h->kc; l < nl; ++l) {
    CoarseLevelBufs B;
    int* ids[3] = {&B.r, &B.y0, &B.y1};
    for (int t = 0; t < 3; ++t) {
      *ids[t] = (int)bufs.size();
      bufs.push_back(CoarseBuf{off, (int32_t)h->lv[l].n});
      off += (int)buf_bytes(h->lv[l].n);
    }
    lb.push_back(B);
  }
  h->smem_bytes = off;
  h->nbufs = nb;
  h->d_bufs = (CoarseBuf*)dalloc(h, bufs.size() * sizeof(CoarseBuf));
  if (!h->d_bufs) return BFP_ERR_CUDA;
  cudaMemcpy(h->d_bufs, bufs.data(), bufs.size() * sizeof(CoarseBuf), cudaMemcpyHostToDevice);
  for (int k = h->kc; k < nl; ++k) {
    std::vector<CoarseOp> ops;
    int res = -1;
    TRY(coarse_flatten(h, k, lb[k - h->kc].r, lb, ops, &res));
    for (size_t i = 1; i < ops.size(); ++i) ops[i].sync_before = (ops[i - 1].solo && !ops[i].solo) ? 1 : 0;
    const int rk = mark_sweep_run(ops, bufs);
    if ((int)ops.size() > max_ops) return BFP_ERR_ARG;
    CoarseOp* d = (CoarseOp*)dalloc(h, ops.size() * sizeof(CoarseOp));
    if (!d) return BFP_ERR_CUDA;
    cudaMemcpy(d, ops.data(), ops.size() * sizeof(CoarseOp), cudaMemcpyHostToDevice);
    h->d_ops.push_back(d);
    h->nops.push_back((int)ops.size());
    h->rbuf.push_back(lb[k - h->kc].r);
    h->ybuf.push_back(res);
    h->runk.push_back(rk);
  }
  // the attribute is per kernel, shared by every hierarchy: allow the device maximum once rather than
  // this hierarchy's size (a later hierarchy with a smaller on-chip part must not shrink it)
  return allow_coarse_smem(h->coarse_wide != 0, optin) ? BFP_OK : BFP_ERR_CUDA;
}

int32_t coarse_vcycle(bfp_hierarchy* h, int k, const bfp_vec* r, const bfp_vec* out, cudaStream_t s) {
  const int i = k - h->kc;
  CoarseArgs a;
  std::memset(&a, 0, sizeof(a));
  a.ops = h->d_ops[i];
  a.nops = h->nops[i];
  a.run_k = h->runk[i];
  a.bufs = h->d_bufs;
  a.nbufs = h->nbufs;
  a.meta_off = h->meta_off;
  a.ops_off = h->ops_off;
  a.bufs_off = h->bufs_off;
  a.data_off = h->data_off;
  a.smem_bytes = h->smem_bytes;
  a.rin = vin(r);
  a.rin_meta = r->meta;
  a.rin_buf = h->rbuf[i];
  a.yout = vout(out);
  a.yout_meta = out->meta;
  a.yout_buf = h->ybuf[i];
  a.stats = h->stats;
  if (h->coarse_wide)
    launch_rec<CoarseArgs, &k_coarse_vcycle<int32_t, false>, &k_coarse_vcycle<int32_t, true>>(
        dim3(1), dim3(kCoarseThreads), h->smem_bytes, s, a);
  else
    launch_rec<CoarseArgs, &k_coarse_vcycle<int16_t, false>, &k_coarse_vcycle<int16_t, true>>(
        dim3(1), dim3(kCoarseThreads), h->smem_bytes, s, a);
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

// V(nu1, nu2) on level k: the approximate solution of A' y = r ends in bufA's
// mantissas; *res describes it (its meta block is a call-site slot of level k).
// Every op writes a meta block of its own (zeroed once per step), so the ops
// skip their per-op memset.
int32_t vcycle_rec(bfp_hierarchy* h, int k, const bfp_vec* r, const bfp_vec* bufA, const bfp_vec* bufB,
                   bfp_vec* res, cudaStream_t s) {
  Nvtx range("vcycle", k);
  Level& L = h->lv[k];
  Q q = make_q(h, L);
  int slot = 0;
  auto at_slot = [&](const bfp_vec* buf) {
    bfp_vec v = *buf;
    v.meta = L.slots + BFP_META_WORDS * (slot++);
    return v;
  };
  if (k >= h->kc) {                       // the rest of the cycle on one SM
    bfp_vec y = at_slot(bufA);
    TRY(coarse_vcycle(h, k, r, &y, s));
    *res = y;
    return BFP_OK;
  }
  const bool coarsest = (k + 1 == (int)h->lv.size());
  if (h->cheby) {   // V(1,0) of Alg. v-cycle: relax from 0, then the coarse correction
    bfp_vec cur = at_slot(coarsest ? bufA : bufB);
    TRY(bfp_cheby(&h->A, h->c1, h->c2, r, &cur, &q.q, &q.st, s));
    if (!coarsest) {
      Level& C = h->lv[k + 1];
      bfp_vec rv = at_slot(&L.rv);
      TRY(bfp_residual(&h->Ares, &cur, r, &rv, &q.q, &q.st, s));        // r_v = A y - r
      bfp_vec rc = at_slot(&C.r);
      rc.w = L.w;
      TRY(bfp_restrict(&rv, &rc, &q.q, &q.st, s));
      bfp_vec d;
      TRY(vcycle_rec(h, k + 1, &rc, &C.ya, &C.yb, &d, s));
      bfp_vec nx = at_slot(bufA);
      TRY(bfp_prolong(&d, &cur, &nx, &q.q, &q.st, s));                 // y = y - P d
      cur = nx;
    }
    *res = cur;
    return BFP_OK;
  }
  auto jacobi = [&](const bfp_vec* y, const bfp_vec* out) -> int32_t {
    return h->var ? bfp_var_jacobi(&L.vs, y, r, out, &q.q, &q.st, s) : bfp_jacobi(&h->A, y, r, out, &q.q, &q.st, s);
  };
  if (coarsest && sweep_run_fits(h, k)) {   // the coarsest level's sweeps in one launch
    bfp_vec y = at_slot(bufA);
    TRY(sweep_run(h, k, r, &y, s));
    *res = y;
    return BFP_OK;
  }
  const int nu1 = coarsest ? h->o.coarse_sweeps : h->o.nu1;
  // writes per level: 1 (omega r) + (nu1 - 1) sweeps [+ correction + nu2 sweeps]
  const int writes = coarsest ? nu1 : (nu1 + 1 + h->o.nu2);
  // choose the first target so that the last write lands in bufA
  const bfp_vec* curb = (writes % 2 == 1) ? bufA : bufB;
  const bfp_vec* othb = (curb == bufA) ? bufB : bufA;
  bfp_vec cur = at_slot(curb);
  TRY(jacobi(nullptr, &cur));                                          // relaxation from y = 0
  for (int i = 1; i < nu1; ++i) {
    bfp_vec nx = at_slot(othb);
    TRY(jacobi(&cur, &nx));
    cur = nx;
    std::swap(curb, othb);
  }
  if (!coarsest) {
    Level& C = h->lv[k + 1];
    bfp_vec rv = at_slot(&L.rv);
    if (h->var) TRY(bfp_var_residual(&L.vs, &cur, r, &rv, &q.q, &q.st, s));   // r_v = A y - r
    else TRY(bfp_residual(&h->A, &cur, r, &rv, &q.q, &q.st, s));
    bfp_vec rc = at_slot(&C.r);
    rc.w = L.w;                                                        // restricted at this level's width
    TRY(bfp_restrict(&rv, &rc, &q.q, &q.st, s));                       // r_c = R~ r_v
    bfp_vec d;
    TRY(vcycle_rec(h, k + 1, &rc, &C.ya, &C.yb, &d, s));               // d = V(r_c)
    bfp_vec nx = at_slot(othb);
    TRY(bfp_prolong(&d, &cur, &nx, &q.q, &q.st, s));                   // y = y - P d
    cur = nx;
    std::swap(curb, othb);
    for (int i = 0; i < h->o.nu2; ++i) {
      bfp_vec nx2 = at_slot(othb);
      TRY(jacobi(&cur, &nx2));
      cur = nx2;
      std::swap(curb, othb);
    }
  }
  *res = cur;
  return BFP_OK;
}

int slots_needed(const bfp_solver_opts& o, bool coarsest) {
  // IR residual + relaxations [+ residual, restriction, correction, post-relaxations]
  return 1 + (coarsest ? o.coarse_sweeps : (o.nu1 + 3 + o.nu2));
}

cudaError_t zero_arena(bfp_hierarchy* h, cudaStream_t s) {
  return mem_zero(h->arena, h->arena_words * sizeof(int64_t), s);
}

Grid grid_of(int nd, int64_t n) { return Grid{n, n, nd == 3 ? n : 1}; }

// r (BFP, width w, normalised) = quant(b' - A' x) on level k (Alg. ir residual line)
int32_t ir_residual_q(bfp_hierarchy* h, int k, const double* b, double bscale, const double* x, const bfp_vec* r,
                      cudaStream_t s) {
  if (h->var) {   // variable coefficients: the FP64 residual, then quant() (bfp_from_f64)
    const Level& L = h->lv[k];
    k_var_res64<<<grid_for(L.n * L.n, 256), 256, 0, s>>>(b, bscale, x, L.kf64[0], L.kf64[1], L.kf64[2], L.kf64[3],
                                                         L.c64, L.n, L.r64);
    note_launches(1);
    if (cudaGetLastError() != cudaSuccess) return BFP_ERR_CUDA;
    return bfp_from_f64(L.r64, r, s);
  }
  const int nd = h->o.ndim;
  const Grid g = grid_of(nd, h->lv[k].n);
  const double cdiag = (2.0 * nd) / pscale(nd), cnb = -1.0 / pscale(nd);
  VOut o = vout(r);
  const int64_t items = rows_of(r) * (r->ld / 8);
  const unsigned gr = grid_for(items, 256);
  if (zero_accumulators(r->meta, s) != cudaSuccess) return BFP_ERR_CUDA;
  IrArgs a;
  a.b = b; a.bscale = bscale; a.x = x; a.nx = g.nx; a.ny = g.ny; a.cdiag = cdiag; a.cnb = cnb;
  int bsh = 0;
  while (std::ldexp(1.0, -bsh) > bscale && bsh < 1100) ++bsh;   // bscale = 2^-bsh (n + 1 = 2^J)
  if (std::ldexp(1.0, -bsh) != bscale || cnb != -1.0 / pscale(nd)) return BFP_ERR_ARG;
  a.bshift = bsh;
  a.nbshift = nd == 2 ? 2 : 3;                   // nb = -2^-nbshift
  a.out = o; a.meta = r->meta;
  a.w = r->w;
  // Table tab:estimates, IR residual: w_add = 4 (i > 1), 5 for the first step on an FMG level
  // (gamma from the coarser level's last residual)
  a.w_tmp = r->w + capped_wadd(h->ir_first ? 5 : 4, h->o.w_add_max);
  a.tmp = (h->lv[k].tmp && a.w_tmp <= 32) ? (int32_t*)h->lv[k].tmp : nullptr;
  a.gamma_mu = h->ir_gam + k;
  a.stats = k == 0 ? h->stats0 : h->stats;
  if (nd == 2) {
    if (cdiag != 1.0) return BFP_ERR_ARG;
    const int rs = pick_rows(g.ny >= 2048 ? 16 : (g.ny >= 1024 ? 8 : (g.ny >= 256 ? 4 : 2)), 64);
    const dim3 grid2((unsigned)((g.nx + kIrCols - 1) / kIrCols),
                     (unsigned)((g.ny + (int64_t)kIrWarps * rs - 1) / ((int64_t)kIrWarps * rs)));
    launch_rec<IrP, &k_ir2d<true>, &k_ir2d<true, true>>(grid2, 128, 0, s, IrP{a, rs});
    launch_rec<IrP, &k_ir2d<false>, &k_ir2d<false, true>>(grid2, 128, 0, s, IrP{a, rs});
  } else {
    k_ir3d<true><<<gr, 256, 0, s>>>(a, g);
    k_ir3d<false><<<gr, 256, 0, s>>>(a, g);
  }
  note_launches(2);
  return cudaGetLastError() == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

int32_t ir_update(double* x, const bfp_vec* y, cudaStream_t s) {
  const int64_t total = y->n[0] * y->n[1] * y->n[2];
  if (total == 0) return BFP_OK;
  const int64_t rows = y->n[1] * y->n[2];
  const int64_t rblocks = (rows + kUpdRows - 1) / kUpdRows;
  const dim3 gu((unsigned)((y->n[0] + 255) / 256), (unsigned)(rblocks < 65535 ? rblocks : 65535));
  const UpdP P{x, vin(y), y->meta};
  if (y->w > 16) launch_rec<UpdP, &k_ir_update2<int32_t>, &k_ir_update2<int32_t, true>>(gu, 256, 0, s, P);
  else launch_rec<UpdP, &k_ir_update2<int16_t>, &k_ir_update2<int16_t, true>>(gu, 256, 0, s, P);
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

// ---- float baselines: the same V(nu1, nu2) schedule on float vectors ----

int32_t flt_vcycle_rec(bfp_hierarchy* h, int k, const flt_vec* r, const flt_vec* bufA, const flt_vec* bufB,
                       flt_vec* res, cudaStream_t s) {
  Level& L = h->lv[k];
  const bool coarsest = (k + 1 == (int)h->lv.size());
  const int nu1 = coarsest ? h->o.coarse_sweeps : h->o.nu1;
  const int writes = coarsest ? nu1 : (nu1 + 1 + h->o.nu2);
  const flt_vec* curb = (writes % 2 == 1) ? bufA : bufB;   // the last write lands in bufA
  const flt_vec* othb = (curb == bufA) ? bufB : bufA;
  TRY(flt_jacobi_impl(&h->A, nullptr, r, curb, s));
  for (int i = 1; i < nu1; ++i) {
    TRY(flt_jacobi_impl(&h->A, curb, r, othb, s));
    std::swap(curb, othb);
  }
  if (!coarsest) {
    Level& C = h->lv[k + 1];
    TRY(flt_residual_impl(&h->A, curb, r, &L.frv, s));        // r_v = A'y - r
    TRY(flt_restrict_impl(&L.frv, &C.fr, s));
    flt_vec d;
    TRY(flt_vcycle_rec(h, k + 1, &C.fr, &C.fya, &C.fyb, &d, s));
    TRY(flt_prolong_impl(&d, curb, othb, s));                 // y - P d
    std::swap(curb, othb);
    for (int i = 0; i < h->o.nu2; ++i) {
      TRY(flt_jacobi_impl(&h->A, curb, r, othb, s));
      std::swap(curb, othb);
    }
  }
  *res = *curb;
  return BFP_OK;
}

int32_t flt_ir_step(bfp_hierarchy* h, int k, const double* b, double bscale, double* x, cudaStream_t s) {
  Level& L = h->lv[k];
  const int nd = h->o.ndim;
  const Grid g = grid_of(nd, L.n);
  const double cdiag = (2.0 * nd) / pscale(nd), cnb = -1.0 / pscale(nd);
  const FVOut ro = fvout(&L.fr);
  const unsigned gr = grid_for(L.fr.ld * g.ny * g.nz, 256);
  const bool bf = L.fr.dtype == FLT_BF16;
#define BFP_FIR(ND)                                                                             \
  do {                                                                                          \
    if (bf) k_fir_residual<ND, uint16_t><<<gr, 256, 0, s>>>(b, bscale, x, g, cdiag, cnb, ro);   \
    else k_fir_residual<ND, float><<<gr, 256, 0, s>>>(b, bscale, x, g, cdiag, cnb, ro);         \
  } while (0)
  if (nd == 2) BFP_FIR(2);
  else BFP_FIR(3);
#undef BFP_FIR
  note_launches(1);
  const flt_vec* A = (k == 0) ? &h->fy0 : &L.fya;
  flt_vec y;
  TRY(flt_vcycle_rec(h, k, &L.fr, A, &L.fyb, &y, s));
  const int64_t rows = y.n[1] * y.n[2];
  const int64_t rblocks = (rows + kUpdRows - 1) / kUpdRows;
  const dim3 gu((unsigned)((y.n[0] + 255) / 256), (unsigned)(rblocks < 65535 ? rblocks : 65535));
  if (bf) k_fir_update<uint16_t><<<gu, 256, 0, s>>>(x, fvin(&y));
  else k_fir_update<float><<<gu, 256, 0, s>>>(x, fvin(&y));
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

int32_t ir_step(bfp_hierarchy* h, int k, const double* b, double bscale, double* x, cudaStream_t s) {
  if (is_float(h)) return flt_ir_step(h, k, b, bscale, x, s);
  Nvtx range("ir_step", k);
  Level& L = h->lv[k];
  if (zero_arena(h, s) != cudaSuccess) return BFP_ERR_CUDA;   // every call-site meta of this step
  PrezeroedScope pz;
  bfp_vec r = L.rir.mant ? L.rir : L.r;
  r.w = L.w;                                                  // quantised to this level's width
  r.meta = L.slots + BFP_META_WORDS * (L.nslots - 1);         // the IR residual's own slot
  TRY(ir_residual_q(h, k, b, bscale, x, &r, s));
  const bfp_vec* A = (k == 0) ? &h->y0 : &L.ya;
  const bfp_vec* B = &L.yb;
  bfp_vec y;
  TRY(vcycle_rec(h, k, &r, A, B, &y, s));
  return ir_update(x, &y, s);
}

// One step of Alg. ir with BFP x and b on the finest level:
//   r = A'x - b (qcomp, level width), y = V(r), x_out = x - y (qcomp, x_out->w bits).
// x_out must not overlap x (the two qcomp passes read x twice).
int32_t ir_step_bfp(bfp_hierarchy* h, const bfp_vec* b, const bfp_vec* x, const bfp_vec* x_out, cudaStream_t s) {
  Level& L = h->lv[0];
  if (zero_arena(h, s) != cudaSuccess) return BFP_ERR_CUDA;
  bfp_vec y;
  {
    PrezeroedScope pz;
    Q q = make_q(h, L);
    q.q.mode = BFP_QCOMP;
    q.q.tmp = h->o.use_tmp ? L.tmp : nullptr;
    bfp_vec r = L.r;
    r.w = L.w;
    r.meta = L.slots + BFP_META_WORDS * (L.nslots - 1);   // the IR residual's own slot
    if (h->var) TRY(bfp_var_residual(&L.vs_ir, x, b, &r, &q.q, &q.st, s));
    else TRY(bfp_residual(&h->A, x, b, &r, &q.q, &q.st, s));
    TRY(vcycle_rec(h, 0, &r, &h->y0, &L.yb, &y, s));
  }
  // x_out's meta is not an arena slot: the op zeroes it itself
  Q q = make_q(h, L);
  q.q.w_out = x_out->w;
  q.q.w_add = 0;                 // Table tab:estimates, IR correction row (gamma ||x|| + ||y||)
  q.q.mode = BFP_QCOMP;
  q.q.tmp = nullptr;
  const bfp_scalar one{1, 0}, minus_one{-1, 0};
  return bfp_axpy(one, x, minus_one, &y, x_out, &q.q, &q.st, s);
}

int32_t ir_bfp_direct(bfp_hierarchy* h, const bfp_vec* b, const bfp_vec* x, int32_t k, cudaStream_t s) {
  for (int32_t i = 0; i < k; ++i) {
    const bool even = (i % 2) == 0;
    TRY(ir_step_bfp(h, b, even ? x : &h->xt, even ? &h->xt : x, s));
  }
  return BFP_OK;
}

// ---- variable coefficients: host setup of every level's operator ----

double harmonic(double a, double b) { return ((2.0 * a) * b) / (a + b); }

// Level l's operator from the node values K ((n+2)^2, [y][x], boundary included): faces,
// one-exponent int16 face block, integer smoother weights, FP64 faces for the IR residual.
int32_t var_level_setup(bfp_hierarchy* h, Level& L, const std::vector<double>& K) {
  const int64_t n = L.n, m = n + 2, ld = bfp_pitch(n), pts = n * n;
  std::vector<double> F[4];
  for (auto& f : F) f.assign((size_t)pts, 0.0);
  double M = 0.0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      const double c = K[(j + 1) * m + i + 1];
      const int64_t p = j * n + i;
      F[0][p] = harmonic(K[(j + 1) * m + i], c);
      F[1][p] = harmonic(c, K[(j + 1) * m + i + 2]);
      F[2][p] = harmonic(K[j * m + i + 1], c);
      F[3][p] = harmonic(c, K[(j + 2) * m + i + 1]);
      for (auto& f : F) {
        if (!(f[p] > 0.0) || !std::isfinite(f[p])) return BFP_ERR_ARG;
        M = f[p] > M ? f[p] : M;
      }
    }
  int fe = 0;
  std::frexp(M, &fe);
  const int64_t e_k = fe - 15;                      // the largest face: 15 significant bits
  std::vector<int16_t> km[4];
  for (auto& v : km) v.assign((size_t)(n * ld), 0);
  std::vector<int64_t> c((size_t)pts, 0);
  int64_t cmin = INT64_MAX, cmax = 0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      const int64_t p = j * n + i;
      int64_t sum = 0;
      for (int f = 0; f < 4; ++f) {
        const double v = std::floor(std::ldexp(F[f][p], (int)-e_k));
        if (v < 0.0 || v >= 32768.0) return BFP_ERR_ARG;
        km[f][j * ld + i] = (int16_t)v;
        sum += (int64_t)v;
      }
      c[p] = sum;
      cmin = sum < cmin ? sum : cmin;
      cmax = sum > cmax ? sum : cmax;
    }
  if (cmin <= 0) return BFP_ERR_ARG;
  // q_i = floor(omega_m 2^s / c_i), the largest s with max q < 2^15
  const int64_t wm = h->A.omega.m;
  if (wm <= 0 || wm >= (1ll << 16)) return BFP_ERR_ARG;
  const int64_t lim = cmin << 15;                   // omega_m 2^s < lim
  auto bitlen = [](int64_t v) { int b = 0; while (v) { ++b; v >>= 1; } return b; };
  auto fits = [&](int sv) { return sv >= 0 ? (wm << sv) < lim : wm < (lim << -sv); };
  int sh = bitlen(lim) - bitlen(wm);
  while (!fits(sh)) --sh;
  while (sh < 40 && fits(sh + 1)) ++sh;
  std::vector<int16_t> qm((size_t)(n * ld), 0);
  int64_t qmax = 0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      const int64_t ci = c[j * n + i];
      const int64_t qv = sh >= 0 ? (wm << sh) / ci : wm / (ci << -sh);
      qm[j * ld + i] = (int16_t)qv;
      qmax = qv > qmax ? qv : qmax;
    }
  std::vector<double> c64((size_t)pts);
  for (int64_t p = 0; p < pts; ++p) c64[p] = ((F[0][p] + F[1][p]) + F[2][p]) + F[3][p];
  // device copies
  const size_t kb = (size_t)(n * ld) * sizeof(int16_t), fb = (size_t)pts * sizeof(double);
  int16_t* dk[4];
  for (int f = 0; f < 4; ++f) {
    dk[f] = (int16_t*)dalloc(h, kb ? kb : 16);
    L.kf64[f] = (double*)dalloc(h, fb ? fb : 16);
    if (!dk[f] || !L.kf64[f]) return BFP_ERR_CUDA;
    if (kb && cudaMemcpy(dk[f], km[f].data(), kb, cudaMemcpyHostToDevice) != cudaSuccess) return BFP_ERR_CUDA;
    if (fb && cudaMemcpy(L.kf64[f], F[f].data(), fb, cudaMemcpyHostToDevice) != cudaSuccess) return BFP_ERR_CUDA;
  }
  int16_t* dq = (int16_t*)dalloc(h, kb ? kb : 16);
  L.c64 = (double*)dalloc(h, fb ? fb : 16);
  L.r64 = (double*)dalloc(h, fb ? fb : 16);
  if (!dq || !L.c64 || !L.r64) return BFP_ERR_CUDA;
  if (kb && cudaMemcpy(dq, qm.data(), kb, cudaMemcpyHostToDevice) != cudaSuccess) return BFP_ERR_CUDA;
  if (fb && cudaMemcpy(L.c64, c64.data(), fb, cudaMemcpyHostToDevice) != cudaSuccess) return BFP_ERR_CUDA;
  bfp_varstencil& V = L.vs;
  V.n[0] = n; V.n[1] = n; V.ld = ld;
  for (int f = 0; f < 4; ++f) V.k[f] = dk[f];
  V.e_k = e_k;
  V.q = dq;
  V.e_q = h->A.omega.e - e_k - sh;
  V.a_norm = 2 * cmax;
  V.q_norm = qmax;
  V.omega = h->A.omega;
  V.k_storage = 16;
  if (&L != &h->lv[0]) return BFP_OK;
  // the finest level's faces again at kIrFaceBits (int32): the IR residual's operator when x and
  // b are BFP blocks (bfp_ir_iterate_bfp)
  const int64_t e_w = fe - (kIrFaceBits - 1);
  const size_t wb = (size_t)(n * ld) * sizeof(int32_t);
  std::vector<int32_t> kw((size_t)(n * ld), 0);
  int64_t wmax = 0;
  std::vector<int64_t> cw((size_t)pts, 0);
  for (int f = 0; f < 4; ++f) {
    for (int64_t j = 0; j < n; ++j)
      for (int64_t i = 0; i < n; ++i) {
        const double v = std::floor(std::ldexp(F[f][j * n + i], (int)-e_w));
        if (v < 0.0 || v >= 2147483648.0) return BFP_ERR_ARG;
        kw[j * ld + i] = (int32_t)v;
        cw[j * n + i] += (int64_t)v;
      }
    int32_t* d = (int32_t*)dalloc(h, wb ? wb : 16);
    if (!d) return BFP_ERR_CUDA;
    if (wb && cudaMemcpy(d, kw.data(), wb, cudaMemcpyHostToDevice) != cudaSuccess) return BFP_ERR_CUDA;
    L.vs_ir.k[f] = d;
  }
  for (int64_t v : cw) wmax = v > wmax ? v : wmax;
  bfp_varstencil& W = L.vs_ir;
  W.n[0] = n; W.n[1] = n; W.ld = ld;
  W.e_k = e_w;
  W.q = nullptr;
  W.e_q = 0;
  W.a_norm = 2 * wmax;
  W.q_norm = 0;
  W.omega = h->A.omega;
  W.k_storage = 32;
  return BFP_OK;
}

int32_t var_setup(bfp_hierarchy* h, const double* k_nodes) {
  int64_t mprev = h->o.n + 2;
  std::vector<double> K(k_nodes, k_nodes + mprev * mprev);
  for (size_t l = 0; l < h->lv.size(); ++l) {
    Level& L = h->lv[l];
    if (l > 0) {   // injection: coarse node c sits on fine node 2c
      const int64_t m = L.n + 2;
      std::vector<double> Kc((size_t)(m * m));
      for (int64_t j = 0; j < m; ++j)
        for (int64_t i = 0; i < m; ++i) Kc[j * m + i] = K[(2 * j) * mprev + 2 * i];
      K.swap(Kc);
      mprev = m;
    }
    TRY(var_level_setup(h, L, K));
  }
  return BFP_OK;
}

double bscale_of(const bfp_hierarchy* h) {
  const double hh = 1.0 / (double)(h->o.n + 1);
  return h->var ? hh * hh : hh * hh / pscale(h->o.ndim);   // an exact power of two for n + 1 = 2^J
}

}  // namespace

extern "C" {

int32_t bfp_solver_opts_default(int32_t ndim, int64_t n, int32_t w, bfp_solver_opts* o) {
  if (!o || (ndim != 2 && ndim != 3)) return BFP_ERR_ARG;
  std::memset(o, 0, sizeof(*o));
  o->ndim = ndim;
  o->n = n;
  o->w = w;
  o->mode = BFP_QCOMP;
  o->nu1 = 2;
  o->nu2 = 2;
  o->coarse_sweeps = 32;
  o->n_fmg = 2;
  o->omega = ndim == 2 ? 0.8 : 6.0 / 7.0;
  o->w_omega = 16;
  o->use_tmp = 1;
  o->use_graph = 1;
  o->coarse_onchip = 63;
  o->arith = BFP_ARITH_BFP;
  o->tile_rows = 0;
  o->smoother = BFP_SMOOTH_JACOBI;
  o->cheby_eta = kChebEta;
  o->w_add_max = -1;
  return BFP_OK;
}

void bfp_hierarchy_destroy(bfp_hierarchy* h) {
  if (!h) return;
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->graph2) cudaGraphExecDestroy(h->graph2);
  for (void* p : h->allocs) cudaFree(p);
  delete h;
}

int32_t bfp_hierarchy_create(const bfp_solver_opts* o, bfp_hierarchy** out) {
  if (!o || !out) return BFP_ERR_ARG;
  *out = nullptr;
  if ((o->ndim != 2 && o->ndim != 3) || o->w < 1 || o->w > 32) return BFP_ERR_ARG;
  if (o->nu1 < 1 || o->nu2 < 0 || o->coarse_sweeps < 1 || o->n_fmg < 1) return BFP_ERR_ARG;
  if (o->mode != BFP_QCOMP && o->mode != BFP_NNQCOMP) return BFP_ERR_ARG;
  if (o->arith != BFP_ARITH_BFP && o->arith != BFP_ARITH_FP32 && o->arith != BFP_ARITH_BF16) return BFP_ERR_ARG;
  if (o->tile_rows < 0 || o->tile_rows > 64) return BFP_ERR_ARG;
  if (o->w_step < 0 || (o->w_step > 0 && o->arith != BFP_ARITH_BFP)) return BFP_ERR_ARG;
  if (o->smoother != BFP_SMOOTH_JACOBI && o->smoother != BFP_SMOOTH_CHEBY) return BFP_ERR_ARG;
  if (o->w_add_max > 32) return BFP_ERR_ARG;
  if (o->smoother == BFP_SMOOTH_CHEBY && (o->arith != BFP_ARITH_BFP || !(o->cheby_eta > 0.0 && o->cheby_eta < 1.0)))
    return BFP_ERR_ARG;
  // n = 2^J - 1 with J >= 2
  if (o->n < 3 || ((o->n + 1) & o->n) != 0) return BFP_ERR_SHAPE;
  bfp_hierarchy* h = new (std::nothrow) bfp_hierarchy();
  if (!h) return BFP_ERR_ARG;
  h->o = *o;
  int32_t rc = bfp_laplace_stencil(o->ndim, o->omega, o->w_omega, &h->A);
  if (rc) { delete h; return rc; }
  h->Ares = h->A;
  if (o->smoother == BFP_SMOOTH_CHEBY) {
    h->cheby = 1;
    rc = cheby_setup(o, h->A, &h->c1, &h->c2);
    if (rc) { delete h; return rc; }
    h->Ares.omega.m = h->c1.m;
    h->Ares.omega.e = h->c1.e - 1;
  }
  for (int64_t n = o->n; n >= 3; n = (n - 1) / 2) {
    Level L;
    L.n = n;
    const int64_t wk = (int64_t)o->w - (int64_t)h->lv.size() * o->w_step, wmin = o->w < 2 ? o->w : 2;
    L.w = (int)(wk > wmin ? wk : wmin);         // w_k = max(w - k w_step, min(w, 2))
    h->lv.push_back(L);
    if (n == 3) break;
  }
  const int nd = o->ndim;
  bool ok = true;
  const bool flt = is_float(h);
  for (size_t k = 0; k < h->lv.size() && ok; ++k) {
    Level& L = h->lv[k];
    if (flt) {
      const int dt = fdtype(h);
      ok = make_fvec(h, L.fr, nd, L.n, dt) && make_fvec(h, L.fya, nd, L.n, dt) && make_fvec(h, L.fyb, nd, L.n, dt) &&
           make_fvec(h, L.frv, nd, L.n, dt);
    } else {
      // storage follows w; a level's right-hand side r holds the finer level's restriction, so
      // it takes the finer width's storage (progressive widths), and where that storage differs
      // from the level's own, the level's FMG IR residual gets a buffer of its own (rir)
      const int wr = k == 0 ? L.w : h->lv[k - 1].w;
      ok = make_vec(h, L.r, nd, L.n, wr) && make_vec(h, L.ya, nd, L.n, L.w) &&
           make_vec(h, L.yb, nd, L.n, L.w) && make_vec(h, L.rv, nd, L.n, L.w);
      if (ok && (wr > 16) != (L.w > 16)) ok = make_vec(h, L.rir, nd, L.n, L.w);
    }
    const int64_t pts = L.n * L.n * (nd == 3 ? L.n : 1);
    if (ok && o->use_tmp && !flt) {
      L.tmp = dalloc(h, (size_t)(L.r.n[1] * L.r.n[2] * L.r.ld) * 4);
      ok = L.tmp != nullptr;
    }
    if (ok && k > 0) {
      L.b = (double*)dalloc(h, pts * sizeof(double));
      L.x = (double*)dalloc(h, pts * sizeof(double));
      ok = L.b && L.x;
    }
  }
  ok = ok && (flt ? make_fvec(h, h->fy0, nd, o->n, fdtype(h)) : make_vec(h, h->y0, nd, o->n, o->w));
  if (ok) {
    size_t words = 0;
    for (size_t k = 0; k < h->lv.size(); ++k) {
      h->lv[k].nslots = slots_needed(*o, k + 1 == h->lv.size());
      words += (size_t)h->lv[k].nslots * BFP_META_WORDS;
    }
    h->arena = (int64_t*)dalloc(h, words * sizeof(int64_t));
    h->arena_words = words;
    ok = h->arena != nullptr;
    size_t off = 0;
    for (size_t k = 0; ok && k < h->lv.size(); ++k) {
      h->lv[k].slots = h->arena + off;
      off += (size_t)h->lv[k].nslots * BFP_META_WORDS;
    }
    if (ok) cudaMemset(h->arena, 0, words * sizeof(int64_t));
  }
  h->kc = (int)h->lv.size();
  if (ok && o->coarse_onchip && !flt) {
    int32_t crc = coarse_setup(h);
    if (crc) { bfp_hierarchy_destroy(h); return crc; }
  }
  if (ok) {
    h->stats = (uint64_t*)dalloc(h, 16 * sizeof(uint64_t));
    h->stats0 = h->stats ? h->stats + 8 : nullptr;
    h->norms = (unsigned long long*)dalloc(h, 2 * sizeof(unsigned long long));
    h->ir_gam = (int64_t*)dalloc(h, h->lv.size() * sizeof(int64_t));
    ok = h->stats && h->norms && h->ir_gam;
    if (ok) cudaMemset(h->stats, 0, 16 * sizeof(uint64_t));
    if (ok) cudaMemset(h->ir_gam, 0, h->lv.size() * sizeof(int64_t));
  }
  if (!ok || cudaDeviceSynchronize() != cudaSuccess) {
    bfp_hierarchy_destroy(h);
    return BFP_ERR_CUDA;
  }
  *out = h;
  return BFP_OK;
}

int32_t bfp_hierarchy_create_var(const bfp_solver_opts* o, const double* k_nodes, bfp_hierarchy** out) {
  if (!o || !k_nodes || !out) return BFP_ERR_ARG;
  *out = nullptr;
  if (o->ndim != 2 || o->arith != BFP_ARITH_BFP || o->w > 24 || o->smoother != BFP_SMOOTH_JACOBI) return BFP_ERR_ARG;
  if (o->w_step > 0 && o->w > 16) return BFP_ERR_ARG;   // the variable ops take one storage for y and r
  bfp_solver_opts oo = *o;
  oo.coarse_onchip = 0;                              // the on-chip cycle has the constant operator only
  bfp_hierarchy* h = nullptr;
  int32_t rc = bfp_hierarchy_create(&oo, &h);
  if (rc) return rc;
  h->var = 1;
  rc = var_setup(h, k_nodes);
  if (rc == BFP_OK && cudaDeviceSynchronize() != cudaSuccess) rc = BFP_ERR_CUDA;
  if (rc) {
    bfp_hierarchy_destroy(h);
    return rc;
  }
  *out = h;
  return BFP_OK;
}

int32_t bfp_hierarchy_var_level(const bfp_hierarchy* h, int32_t level, bfp_varstencil* out) {
  if (!h || !out || !h->var || level < 0 || level >= (int32_t)h->lv.size()) return BFP_ERR_ARG;
  *out = h->lv[level].vs;
  return BFP_OK;
}

int32_t bfp_hierarchy_var_ir_operator(const bfp_hierarchy* h, bfp_varstencil* out) {
  if (!h || !out || !h->var) return BFP_ERR_ARG;
  *out = h->lv[0].vs_ir;
  return BFP_OK;
}

static int32_t read_counters(bfp_hierarchy* h, uint64_t* host8, bool finest_only, bfp_stream stream) {
  if (!h || !host8) return BFP_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  uint64_t both[16];
  if (cudaMemcpyAsync(both, h->stats, 16 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return BFP_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return BFP_ERR_CUDA;
  for (int i = 0; i < 8; ++i) host8[i] = both[8 + i] + (finest_only ? 0 : both[i]);
  return BFP_OK;
}

int32_t bfp_hierarchy_read_stats(bfp_hierarchy* h, uint64_t* host8, bfp_stream stream) {
  return read_counters(h, host8, false, stream);
}

int32_t bfp_hierarchy_read_finest_stats(bfp_hierarchy* h, uint64_t* host8, bfp_stream stream) {
  return read_counters(h, host8, true, stream);
}

int32_t bfp_hierarchy_reset_stats(bfp_hierarchy* h, bfp_stream stream) {
  if (!h) return BFP_ERR_ARG;
  return cudaMemsetAsync(h->stats, 0, 16 * sizeof(uint64_t), as_stream(stream)) == cudaSuccess ? BFP_OK
                                                                                                : BFP_ERR_CUDA;
}

int32_t bfp_vcycle(bfp_hierarchy* h, const bfp_vec* r, const bfp_vec* y, bfp_stream stream) {
  if (!h || !r || !y || is_float(h)) return BFP_ERR_ARG;
  int32_t rc;
  if ((rc = check_vec(r)) || (rc = check_vec(y))) return rc;
  const Level& L = h->lv[0];
  if (r->w != h->o.w || y->w != h->o.w || r->n[0] != L.n || !same_shape(r, &L.r) || !same_shape(y, &L.r))
    return BFP_ERR_SHAPE;
  if (overlaps(r, y)) return BFP_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  if (zero_arena(h, s) != cudaSuccess) return BFP_ERR_CUDA;
  PrezeroedScope pz;
  TileScope ts(h->o.tile_rows);
  WaddScope wz(h->o.w_add_max);
  bfp_vec res;
  TRY(vcycle_rec(h, 0, r, y, &h->y0, &res, s));
  // the result's mantissas are in y; its exponent and norm are in a call-site slot
  if (cudaMemcpyAsync(y->meta, res.meta, BFP_META_WORDS * sizeof(int64_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return BFP_ERR_CUDA;
  return BFP_OK;
}

static int32_t ir_iterate_direct(bfp_hierarchy* h, const double* f, double* x, int32_t k, cudaStream_t s) {
  TileScope ts(h->o.tile_rows);
  WaddScope wz(h->o.w_add_max);
  const double bs = bscale_of(h);
  for (int i = 0; i < k; ++i) TRY(ir_step(h, 0, f, bs, x, s));
  return BFP_OK;
}

int32_t bfp_ir_iterate(bfp_hierarchy* h, const double* f, double* x, int32_t k, bfp_stream stream) {
  if (!h || !f || !x || k < 0) return BFP_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  if (k == 0) return BFP_OK;
  if (!h->o.use_graph || s == nullptr) return ir_iterate_direct(h, f, x, k, s);
  // one IR step captured once per (f, x, stream) and replayed
  if (!h->graph || h->graph_f != f || h->graph_x != x || h->graph_stream != s) {
    if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return BFP_ERR_CUDA;
    int32_t rc = ir_iterate_direct(h, f, x, 1, s);
    cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (rc != BFP_OK) { if (g) cudaGraphDestroy(g); return rc; }
    if (ce != cudaSuccess) return BFP_ERR_CUDA;
    ce = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) { h->graph = nullptr; return BFP_ERR_CUDA; }
    h->graph_f = f; h->graph_x = x; h->graph_stream = s;
  }
  for (int i = 0; i < k; ++i)
    if (cudaGraphLaunch(h->graph, s) != cudaSuccess) return BFP_ERR_CUDA;
  return BFP_OK;
}

static bool same_vec(const bfp_vec& a, const bfp_vec& b) { return std::memcmp(&a, &b, sizeof(bfp_vec)) == 0; }

int32_t bfp_ir_iterate_bfp(bfp_hierarchy* h, const bfp_vec* b, const bfp_vec* x, int32_t k, bfp_stream stream) {
  if (!h || !b || !x || k < 0 || is_float(h)) return BFP_ERR_ARG;
  int32_t rc;
  if ((rc = check_vec_wide(b)) || (rc = check_vec_wide(x))) return rc;
  const Level& L = h->lv[0];
  if (!same_shape(b, &L.r) || !same_shape(x, &L.r)) return BFP_ERR_SHAPE;
  if (h->var && (is64(b) || is64(x))) return BFP_ERR_WIDTH;   // A'x with 26-bit faces: x <= 32 bits
  if (overlaps(b, x)) return BFP_ERR_ARG;
  if (x->ld != L.r.ld) return BFP_ERR_SHAPE;
  if (k == 0) return BFP_OK;
  cudaStream_t s = as_stream(stream);
  // scratch iterate with x's storage (pitch and rows of the finest level)
  const size_t bytes = (size_t)(L.r.n[1] * L.r.n[2] * L.r.ld) * esize(x);
  if (!h->xt.mant || h->xt_bytes != bytes) {
    void* m = dalloc(h, bytes);
    int64_t* meta = (int64_t*)dalloc(h, BFP_META_WORDS * sizeof(int64_t));
    if (!m || !meta) return BFP_ERR_CUDA;
    h->xt_bytes = bytes;
    h->xt.mant = m;
    h->xt.meta = meta;
  }
  h->xt.w = x->w; h->xt.ndim = x->ndim; h->xt.ld = x->ld;
  for (int d = 0; d < 3; ++d) h->xt.n[d] = x->n[d];
  if (overlaps(b, &h->xt) || overlaps(x, &h->xt)) return BFP_ERR_ARG;
  TileScope ts(h->o.tile_rows);
  WaddScope wz(h->o.w_add_max);
  const int32_t pairs = k / 2;
  if (pairs > 0 && h->o.use_graph && s != nullptr) {
    // two steps (x -> xt -> x) captured once per (b, x, stream) and replayed
    if (!h->graph2 || !same_vec(h->graph2_b, *b) || !same_vec(h->graph2_x, *x) || h->graph2_stream != s) {
      if (h->graph2) { cudaGraphExecDestroy(h->graph2); h->graph2 = nullptr; }
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return BFP_ERR_CUDA;
      rc = ir_bfp_direct(h, b, x, 2, s);
      cudaError_t ce = cudaStreamEndCapture(s, &g);
      if (rc != BFP_OK) { if (g) cudaGraphDestroy(g); return rc; }
      if (ce != cudaSuccess) return BFP_ERR_CUDA;
      ce = cudaGraphInstantiate(&h->graph2, g, 0);
      cudaGraphDestroy(g);
      if (ce != cudaSuccess) { h->graph2 = nullptr; return BFP_ERR_CUDA; }
      h->graph2_b = *b; h->graph2_x = *x; h->graph2_stream = s;
    }
    for (int32_t i = 0; i < pairs; ++i)
      if (cudaGraphLaunch(h->graph2, s) != cudaSuccess) return BFP_ERR_CUDA;
  } else if (pairs > 0) {
    TRY(ir_bfp_direct(h, b, x, 2 * pairs, s));
  }
  if (k % 2 == 1) {   // the last step lands in the scratch copy: move it back
    TRY(ir_bfp_direct(h, b, x, 1, s));
    if (cudaMemcpyAsync(x->mant, h->xt.mant, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(x->meta, h->xt.meta, BFP_META_WORDS * sizeof(int64_t), cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
      return BFP_ERR_CUDA;
  }
  return BFP_OK;
}

int32_t bfp_hierarchy_rhs_scale(const bfp_hierarchy* h, double* out) {
  if (!h || !out) return BFP_ERR_ARG;
  *out = bscale_of(h);
  return BFP_OK;
}

int32_t bfp_fmg(bfp_hierarchy* h, const double* f, double* x, bfp_stream stream) {
  if (!h || !f || !x) return BFP_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  TileScope ts(h->o.tile_rows);
  WaddScope wz(h->o.w_add_max);
  const int nd = h->o.ndim;
  const int nl = (int)h->lv.size();
  const double rscale = nd == 2 ? 0.25 : 0.0625;   // R~ = P^T (2D), P^T/2 (3D): weights prod(2-|d|) * 2^e_R
  const double bs0 = bscale_of(h);
  // right-hand sides b_k = R~ b_{k-1}, b_0 = s f
  for (int k = 1; k < nl; ++k) {
    const Level& F = h->lv[k - 1];
    Level& Cc = h->lv[k];
    const double* bf = (k == 1) ? f : F.b;
    const double sc = (k == 1) ? bs0 : 1.0;
    const int64_t tot = Cc.n * Cc.n * (nd == 3 ? Cc.n : 1);
    const RestrictF64P P{bf, sc, grid_of(nd, F.n), Cc.b, grid_of(nd, Cc.n), rscale};
    if (nd == 2)
      launch_rec<RestrictF64P, &k_restrict_f64<2>, &k_restrict_f64<2, true>>(grid_for(tot, 256), 256, 0, s, P);
    else k_restrict_f64<3><<<grid_for(tot, 256), 256, 0, s>>>(P, nullptr);
    note_launches(1);
  }
  if (mem_zero(h->ir_gam, nl * sizeof(int64_t), s) != cudaSuccess) return BFP_ERR_CUDA;
  for (int k = nl - 1; k >= 0; --k) {
    Level& L = h->lv[k];
    double* xk = (k == 0) ? x : L.x;
    const int64_t tot = L.n * L.n * (nd == 3 ? L.n : 1);
    if (k == nl - 1) {
      if (mem_zero(xk, tot * sizeof(double), s) != cudaSuccess) return BFP_ERR_CUDA;
    } else {
      Level& Cc = h->lv[k + 1];
      if (is_float(h)) {
        // float baselines: x_k = P x_{k+1} in the vectors' format
        const flt_vec* xf = (k == 0) ? &h->fy0 : &L.fya;
        const bool bf = xf->dtype == FLT_BF16;
        const unsigned g1 = grid_for(Cc.fya.ld * Cc.fya.n[1] * Cc.fya.n[2], 256);
        if (bf) k_f64_to_flt<uint16_t><<<g1, 256, 0, s>>>(Cc.x, fvout(&Cc.fya));
        else k_f64_to_flt<float><<<g1, 256, 0, s>>>(Cc.x, fvout(&Cc.fya));
        TRY(flt_prolong_impl(&Cc.fya, nullptr, xf, s));
        const unsigned g2 = grid_for(tot, 256);
        if (bf) k_flt_to_f64<uint16_t><<<g2, 256, 0, s>>>(fvin(xf), xk);
        else k_flt_to_f64<float><<<g2, 256, 0, s>>>(fvin(xf), xk);
        note_launches(2);
      } else {
        // x_k = P x_{k+1} at width w (Alg. fmg interpolation line, qspmv)
        TRY(bfp_from_f64(Cc.x, &Cc.ya, s));
        Q q = make_q(h, L);
        bfp_vec* xf = (k == 0) ? &h->y0 : &L.ya;
        TRY(bfp_prolong(&Cc.ya, nullptr, xf, &q.q, &q.st, s));
        TRY(bfp_to_f64(xf, xk, s));
      }
    }
    const double* bk = (k == 0) ? f : L.b;
    const double sc = (k == 0) ? bs0 : 1.0;
    if (k < nl - 1) {   // first step: gamma from the coarser level's last IR residual (i = 1 row)
      if (mem_copy(h->ir_gam + k, h->ir_gam + k + 1, sizeof(int64_t), s) !=
          cudaSuccess)
        return BFP_ERR_CUDA;
    }
    for (int i = 0; i < h->o.n_fmg; ++i) {
      h->ir_first = (i == 0 && k < nl - 1) ? 1 : 0;
      const int32_t rc = ir_step(h, k, bk, sc, xk, s);
      h->ir_first = 0;
      TRY(rc);
    }
  }
  return cudaGetLastError() == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

int32_t bfp_ir_residual(bfp_hierarchy* h, const double* f, const double* x, const bfp_vec* r, bfp_stream stream) {
  if (!h || !f || !x || !r || is_float(h)) return BFP_ERR_ARG;
  int32_t rc;
  if ((rc = check_vec(r))) return rc;
  if (!same_shape(r, &h->lv[0].r)) return BFP_ERR_SHAPE;
  return ir_residual_q(h, 0, f, bscale_of(h), x, r, as_stream(stream));
}

int32_t flt_vcycle(bfp_hierarchy* h, const flt_vec* r, const flt_vec* y, bfp_stream stream) {
  if (!h || !r || !y || !is_float(h)) return BFP_ERR_ARG;
  int32_t rc;
  if ((rc = check_fvec(r)) || (rc = check_fvec(y))) return rc;
  const Level& L = h->lv[0];
  if (!same_fshape(r, &L.fr) || !same_fshape(y, &L.fr) || r->dtype != fdtype(h) || y->dtype != fdtype(h))
    return BFP_ERR_SHAPE;
  if (foverlaps(r, y)) return BFP_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  TileScope ts(h->o.tile_rows);
  WaddScope wz(h->o.w_add_max);
  flt_vec res;
  return flt_vcycle_rec(h, 0, r, y, &h->fy0, &res, s);   // the result lands in y (bufA)
}

int32_t bfp_ir_update(double* x, const bfp_vec* y, bfp_stream stream) {
  if (!x) return BFP_ERR_ARG;
  int32_t rc;
  if ((rc = check_vec(y))) return rc;
  return ir_update(x, y, as_stream(stream));
}

int32_t ir_solve(bfp_hierarchy* h, const double* f, double* x, const bfp_ir_opts* o, bfp_ir_report* rep,
                 bfp_stream stream) {
  if (!h || !f || !x || !o || !rep) return BFP_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  TileScope ts(h->o.tile_rows);
  WaddScope wz(h->o.w_add_max);
  std::memset(rep, 0, sizeof(*rep));
  rep->fallback_at = -1;
  if (o->fmg_start) TRY(bfp_fmg(h, f, x, s));
  double hist[2] = {-1.0, -1.0};   // residual norms one and two steps back
  const int nd = h->o.ndim;
  const Grid g = grid_of(nd, h->o.n);
  const double cdiag = (2.0 * nd) / pscale(nd), cnb = -1.0 / pscale(nd);
  const double bs = bscale_of(h);
  const int64_t tot = g.nx * g.ny * g.nz;
  for (int it = 0;; ++it) {
    if (cudaMemsetAsync(h->norms, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess) return BFP_ERR_CUDA;
    if (h->var) {
      const Level& L = h->lv[0];
      k_var_res64<<<grid_for(tot, 256), 256, 0, s>>>(f, bs, x, L.kf64[0], L.kf64[1], L.kf64[2], L.kf64[3], L.c64,
                                                     L.n, L.r64);
      k_absmax2<<<grid_for(tot, 256), 256, 0, s>>>(L.r64, f, bs, tot, h->norms);
      note_launches(2);
    } else {
      if (nd == 2) k_ir_resnorm<2><<<grid_for(tot, 256), 256, 0, s>>>(f, bs, x, g, cdiag, cnb, h->norms);
      else k_ir_resnorm<3><<<grid_for(tot, 256), 256, 0, s>>>(f, bs, x, g, cdiag, cnb, h->norms);
      note_launches(1);
    }
    unsigned long long hn[2] = {0, 0};
    if (cudaMemcpyAsync(hn, h->norms, sizeof(hn), cudaMemcpyDeviceToHost, s) != cudaSuccess) return BFP_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return BFP_ERR_CUDA;
    double rn, bn;
    std::memcpy(&rn, &hn[0], 8);
    std::memcpy(&bn, &hn[1], 8);
    rep->iterations = it;
    rep->res_inf = rn;
    rep->res0_inf = bn;
    if (rn <= o->tol * bn) { rep->converged = 1; return BFP_OK; }
    if (it >= o->max_iter) return BFP_ERR_NOCONV;
    if (o->stall_fallback && h->o.mode == BFP_NNQCOMP && rep->fallback_at < 0 && hist[1] >= 0.0 &&
        rn > 0.5 * hist[1])
      rep->fallback_at = it;
    hist[1] = hist[0];
    hist[0] = rn;
    if (rep->fallback_at >= 0) {   // the V-cycle ops of this step with qcomp
      const int32_t mode = h->o.mode;
      h->o.mode = BFP_QCOMP;
      const int32_t rc = ir_step(h, 0, f, bs, x, s);
      h->o.mode = mode;
      TRY(rc);
    } else {
      TRY(ir_step(h, 0, f, bs, x, s));
    }
  }
}

}  // extern "C"

// ---- batched solve: many independent instances in one graph launch ----------------

struct bfp_batch {
  std::vector<bfp_hierarchy*> h;
  std::vector<bfp_solver_opts> opts;   // per instance (instances with equal options form a group)
  void* pbuf = nullptr;                 // device copy of the merged launches' parameters
  size_t pbuf_bytes = 0;
  int merged_groups = 0, fallback_instances = 0;   // of the last captured solve
  std::vector<cudaStream_t> st;        // one capture branch per instance
  std::vector<cudaEvent_t> join, tend;
  cudaEvent_t fork = nullptr, tstart = nullptr;
  cudaGraphExec_t graph = nullptr;
  std::vector<const double*> gf;       // the arguments the graph was captured with
  std::vector<double*> gx;
  std::vector<int32_t> gk;
  int32_t gfmg = -1;
  cudaStream_t gs = nullptr;
  // per-instance graphs (one launch per instance)
  struct One {
    cudaGraphExec_t g = nullptr;
    const double* f = nullptr;
    double* x = nullptr;
    int32_t k = -1, fmg = -1;
    cudaStream_t s = nullptr;
  };
  std::vector<One> one;
};

namespace {

// FMG (optional) then k IR-V steps of one instance on stream s (direct launches)
int32_t instance_solve(bfp_hierarchy* h, const double* f, double* x, int32_t k, int32_t fmg, cudaStream_t s) {
  TileScope ts(h->o.tile_rows);
  WaddScope wz(h->o.w_add_max);
  if (fmg) TRY(bfp_fmg(h, f, x, s));
  const double bs = bscale_of(h);
  for (int i = 0; i < k; ++i) TRY(ir_step(h, 0, f, bs, x, s));
  return BFP_OK;
}

// Zeroing and small device-to-device copies of many instances in one launch (grid z: instance).
__global__ void __launch_bounds__(256) k_zero_many(void* const* __restrict__ dst, size_t bytes) {
  unsigned char* d = reinterpret_cast<unsigned char*>(dst[blockIdx.z]);
  const size_t words = bytes / 8;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (size_t)gridDim.x * blockDim.x)
    reinterpret_cast<unsigned long long*>(d)[i] = 0ull;
  for (size_t i = words * 8 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < bytes;
       i += (size_t)gridDim.x * blockDim.x)
    d[i] = 0;
}
__global__ void __launch_bounds__(256) k_copy_many(void* const* __restrict__ dst, const void* const* __restrict__ src,
                                                   size_t bytes) {
  unsigned char* d = reinterpret_cast<unsigned char*>(dst[blockIdx.z]);
  const unsigned char* a = reinterpret_cast<const unsigned char*>(src[blockIdx.z]);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < bytes; i += (size_t)gridDim.x * blockDim.x)
    d[i] = a[i];
}

// The schedule of one instance (FMG and k IR-V steps) as launch records.  Returns false when any
// part of it has no batched form: the work the recorder did not take is captured on a private
// stream instead, and a non-empty capture means the schedule cannot be merged.
bool record_instance(bfp_hierarchy* h, const double* f, double* x, int32_t k, int32_t fmg, cudaStream_t cap,
                     std::vector<LaunchRec>* out) {
  out->clear();
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
  launch_recorder() = out;
  const int32_t rc = instance_solve(h, f, x, k, fmg, cap);
  launch_recorder() = nullptr;
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(cap, &g);
  size_t nodes = 1;
  if (ce == cudaSuccess && g) cudaGraphGetNodes(g, nullptr, &nodes);
  if (g) cudaGraphDestroy(g);
  (void)cudaGetLastError();
  return rc == BFP_OK && ce == cudaSuccess && nodes == 0;
}

bool same_rec(const LaunchRec& a, const LaunchRec& b) {
  if (a.op != b.op) return false;
  if (a.op == 0)
    return a.launch == b.launch && a.grid.x == b.grid.x && a.grid.y == b.grid.y && a.grid.z == b.grid.z &&
           a.block.x == b.block.x && a.smem == b.smem && a.params.size() == b.params.size();
  return a.bytes == b.bytes;
}

// One position of a group's merged schedule: the members still running there and where their
// parameters (kernels) or pointers (zeroing, copies) sit in the parameter buffer.
struct MergedPos {
  const LaunchRec* rec;          // the first member's record (kind, grid, sizes)
  int count;                     // members with a record at this position
  size_t off;                    // byte offset in the parameter buffer
};

}  // namespace

extern "C" {

void bfp_batch_destroy(bfp_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->pbuf) cudaFree(b->pbuf);
  for (auto& o : b->one)
    if (o.g) cudaGraphExecDestroy(o.g);
  for (bfp_hierarchy* h : b->h) bfp_hierarchy_destroy(h);
  for (cudaStream_t s : b->st) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  for (cudaEvent_t e : b->tend) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->tstart) cudaEventDestroy(b->tstart);
  delete b;
}

int32_t bfp_batch_create(const bfp_solver_opts* opts, int32_t count, bfp_batch** out) {
  if (!opts || !out || count < 1) return BFP_ERR_ARG;
  *out = nullptr;
  bfp_batch* b = new (std::nothrow) bfp_batch();
  if (!b) return BFP_ERR_ARG;
  for (int32_t i = 0; i < count; ++i) {
    bfp_hierarchy* h = nullptr;
    const int32_t rc = bfp_hierarchy_create(&opts[i], &h);
    if (rc) { bfp_batch_destroy(b); return rc; }
    b->h.push_back(h);
    b->opts.push_back(opts[i]);
    cudaStream_t s = nullptr;
    cudaEvent_t j = nullptr, t = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&j, cudaEventDisableTiming) != cudaSuccess || cudaEventCreate(&t) != cudaSuccess) {
      if (s) cudaStreamDestroy(s);
      if (j) cudaEventDestroy(j);
      bfp_batch_destroy(b);
      return BFP_ERR_CUDA;
    }
    b->st.push_back(s);
    b->join.push_back(j);
    b->tend.push_back(t);
  }
  b->one.resize(count);
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&b->tstart) != cudaSuccess) {
    bfp_batch_destroy(b);
    return BFP_ERR_CUDA;
  }
  *out = b;
  return BFP_OK;
}

int32_t bfp_batch_solve(bfp_batch* b, const double* const* f, double* const* x, const int32_t* ir_steps, int32_t fmg,
                        bfp_stream stream) {
  if (!b || !f || !x || !ir_steps) return BFP_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  if (s == nullptr) return BFP_ERR_ARG;   // capture needs a created stream
  const size_t n = b->h.size();
  for (size_t i = 0; i < n; ++i)
    if (!f[i] || !x[i] || ir_steps[i] < 0) return BFP_ERR_ARG;
  bool same = b->graph && b->gs == s && b->gfmg == fmg;
  for (size_t i = 0; same && i < n; ++i) same = b->gf[i] == f[i] && b->gx[i] == x[i] && b->gk[i] == ir_steps[i];
  if (!same) {
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    // groups: instances with equal options run the same schedule (up to their step counts)
    std::vector<std::vector<int>> groups;
    for (size_t i = 0; i < n; ++i) {
      bool placed = false;
      for (auto& g : groups)
        if (std::memcmp(&b->opts[g[0]], &b->opts[i], sizeof(bfp_solver_opts)) == 0) {
          g.push_back((int)i);
          placed = true;
          break;
        }
      if (!placed) groups.push_back({(int)i});
    }
    // record every member's schedule; a group merges when every record has a batched form and the
    // members' schedules agree position by position (a shorter one is a prefix of the longest)
    std::vector<std::vector<LaunchRec>> recs(n);
    std::vector<char> merged(groups.size(), 0);
    cudaStream_t cap = nullptr;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return BFP_ERR_CUDA;
    for (size_t gi = 0; gi < groups.size(); ++gi) {
      bool ok = true;
      int longest = groups[gi][0];
      for (int m : groups[gi]) {
        ok = ok && record_instance(b->h[m], f[m], x[m], ir_steps[m], fmg, cap, &recs[m]);
        if (ok && recs[m].size() > recs[longest].size()) longest = m;
      }
      const std::vector<LaunchRec>& L = recs[longest];
      for (int m : groups[gi])
        for (size_t p2 = 0; ok && p2 < recs[m].size(); ++p2) ok = same_rec(recs[m][p2], L[p2]);
      merged[gi] = ok ? 1 : 0;
      if (!ok)
        for (int m : groups[gi]) recs[m].clear();
    }
    cudaStreamDestroy(cap);
    // the merged launches' parameters (kernels) and pointer arrays (zeroing, copies), position by position
    std::vector<std::vector<MergedPos>> pos(groups.size());
    std::vector<unsigned char> host;
    auto put = [&](const void* p3, size_t bytes) {
      const size_t off = host.size();
      host.resize(off + bytes);
      std::memcpy(host.data() + off, p3, bytes);
    };
    for (size_t gi = 0; gi < groups.size(); ++gi) {
      if (!merged[gi]) continue;
      size_t len = 0;
      for (int m : groups[gi]) len = recs[m].size() > len ? recs[m].size() : len;
      for (size_t p2 = 0; p2 < len; ++p2) {
        host.resize((host.size() + 15) / 16 * 16);
        MergedPos mp{nullptr, 0, host.size()};
        for (int m : groups[gi]) {
          if (recs[m].size() <= p2) continue;
          const LaunchRec& r = recs[m][p2];
          if (!mp.rec) mp.rec = &r;
          ++mp.count;
          if (r.op == 0) put(r.params.data(), r.params.size());
          else put(&r.dst, sizeof(void*));
        }
        if (mp.rec->op == 2)
          for (int m : groups[gi])
            if (recs[m].size() > p2) put(&recs[m][p2].src, sizeof(void*));
        pos[gi].push_back(mp);
      }
    }
    if (host.size() > b->pbuf_bytes) {
      if (b->pbuf) cudaFree(b->pbuf);
      b->pbuf = nullptr;
      b->pbuf_bytes = 0;
      if (cudaMalloc(&b->pbuf, host.size()) != cudaSuccess) return BFP_ERR_CUDA;
      b->pbuf_bytes = host.size();
    }
    if (!host.empty() && cudaMemcpy(b->pbuf, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return BFP_ERR_CUDA;
    unsigned char* dev = reinterpret_cast<unsigned char*>(b->pbuf);

    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) return BFP_ERR_CUDA;
    int32_t rc = BFP_OK;
    if (cudaEventRecordWithFlags(b->tstart, s, cudaEventRecordExternal) != cudaSuccess ||
        cudaEventRecord(b->fork, s) != cudaSuccess)
      rc = BFP_ERR_CUDA;
    int nmerged = 0, nfallback = 0;
    for (size_t gi = 0; rc == BFP_OK && gi < groups.size(); ++gi) {
      if (!merged[gi]) {   // one capture branch per member, the single-instance launches
        for (int m : groups[gi]) {
          ++nfallback;
          if (cudaStreamWaitEvent(b->st[m], b->fork, 0) != cudaSuccess) { rc = BFP_ERR_CUDA; break; }
          rc = instance_solve(b->h[m], f[m], x[m], ir_steps[m], fmg, b->st[m]);
          if (rc) break;
          if (cudaEventRecordWithFlags(b->tend[m], b->st[m], cudaEventRecordExternal) != cudaSuccess ||
              cudaEventRecord(b->join[m], b->st[m]) != cudaSuccess || cudaStreamWaitEvent(s, b->join[m], 0) != cudaSuccess)
            rc = BFP_ERR_CUDA;
        }
        continue;
      }
      ++nmerged;
      const int first = groups[gi][0];
      cudaStream_t gs = b->st[first];
      if (cudaStreamWaitEvent(gs, b->fork, 0) != cudaSuccess) { rc = BFP_ERR_CUDA; break; }
      for (int m : groups[gi])
        if (recs[m].empty() && cudaEventRecordWithFlags(b->tend[m], gs, cudaEventRecordExternal) != cudaSuccess)
          rc = BFP_ERR_CUDA;
      for (size_t p2 = 0; rc == BFP_OK && p2 < pos[gi].size(); ++p2) {
        const MergedPos& mp = pos[gi][p2];
        const LaunchRec& r = *mp.rec;
        if (r.op == 0) {
          r.launch(r.grid, r.block, r.smem, gs, dev + mp.off, mp.count);
        } else {
          const size_t words = (r.bytes + 7) / 8;
          const unsigned gx = (unsigned)(words / 256 + 1 > 1024 ? 1024 : words / 256 + 1);
          void* const* dsts = reinterpret_cast<void* const*>(dev + mp.off);
          if (r.op == 1) k_zero_many<<<dim3(gx, 1, (unsigned)mp.count), 256, 0, gs>>>(dsts, r.bytes);
          else k_copy_many<<<dim3(gx, 1, (unsigned)mp.count), 256, 0, gs>>>(
              dsts, reinterpret_cast<const void* const*>(dev + mp.off + mp.count * sizeof(void*)), r.bytes);
        }
        note_launches(1);
        for (int m : groups[gi])   // members whose schedule ends here
          if (recs[m].size() == p2 + 1 &&
              cudaEventRecordWithFlags(b->tend[m], gs, cudaEventRecordExternal) != cudaSuccess)
            rc = BFP_ERR_CUDA;
      }
      if (rc == BFP_OK && (cudaEventRecord(b->join[first], gs) != cudaSuccess ||
                           cudaStreamWaitEvent(s, b->join[first], 0) != cudaSuccess))
        rc = BFP_ERR_CUDA;
    }
    if (rc == BFP_OK && cudaGetLastError() != cudaSuccess) rc = BFP_ERR_CUDA;
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (rc != BFP_OK || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return rc != BFP_OK ? rc : BFP_ERR_CUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) { b->graph = nullptr; return BFP_ERR_CUDA; }
    b->gf.assign(f, f + n);
    b->gx.assign(x, x + n);
    b->gk.assign(ir_steps, ir_steps + n);
    b->gfmg = fmg;
    b->gs = s;
    b->merged_groups = nmerged;
    b->fallback_instances = nfallback;
  }
  return cudaGraphLaunch(b->graph, s) == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

int32_t bfp_batch_solve_one(bfp_batch* b, int32_t i, const double* f, double* x, int32_t ir_steps, int32_t fmg,
                            bfp_stream stream) {
  if (!b || i < 0 || i >= (int32_t)b->h.size() || !f || !x || ir_steps < 0) return BFP_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  if (s == nullptr) return BFP_ERR_ARG;
  bfp_batch::One& o = b->one[i];
  if (!o.g || o.f != f || o.x != x || o.k != ir_steps || o.fmg != fmg || o.s != s) {
    if (o.g) { cudaGraphExecDestroy(o.g); o.g = nullptr; }
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) return BFP_ERR_CUDA;
    const int32_t rc = instance_solve(b->h[i], f, x, ir_steps, fmg, s);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (rc != BFP_OK || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return rc != BFP_OK ? rc : BFP_ERR_CUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&o.g, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) { o.g = nullptr; return BFP_ERR_CUDA; }
    o.f = f; o.x = x; o.k = ir_steps; o.fmg = fmg; o.s = s;
  }
  return cudaGraphLaunch(o.g, s) == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

int32_t bfp_batch_info(const bfp_batch* b, int32_t* merged_groups, int32_t* separate_instances) {
  if (!b || !merged_groups || !separate_instances) return BFP_ERR_ARG;
  *merged_groups = b->merged_groups;
  *separate_instances = b->fallback_instances;
  return BFP_OK;
}

int32_t bfp_batch_times(bfp_batch* b, float* ms) {
  if (!b || !ms || !b->graph) return BFP_ERR_ARG;
  for (size_t i = 0; i < b->h.size(); ++i) {
    if (cudaEventSynchronize(b->tend[i]) != cudaSuccess) return BFP_ERR_CUDA;
    if (cudaEventElapsedTime(&ms[i], b->tstart, b->tend[i]) != cudaSuccess) return BFP_ERR_CUDA;
  }
  return BFP_OK;
}

}  // extern "C"
