// bfp_ir2d.cuh -- FP64 iterative-refinement kernels for the 2D finest levels.
//
// Residual r = b' - A' x quantised to a normalised BFP block (Alg. ir residual
// line with FP64 arithmetic): r is evaluated with explicitly rounded
// operations in a fixed order, so it is bitwise reproducible.  The
// quantisation follows Alg. qcomp: pass 1 finds mu* = max_i (msb(M_i) + E_i)
// and stores a w_tmp-bit window guessed from gamma = the previous residual's
// norm (Table tab:estimates, IR residual row, w_add = 4); pass 2 narrows the
// window when it captured every significant bit and otherwise recomputes r.
//
// Layout: FP64 vectors are dense (row stride n), so a lane owns the
// interleaved columns cb + 32 k + lane (k < kIrV): every warp access is a
// contiguous 256-byte line whatever the row alignment.  A warp walks a strip
// of rows keeping x rows j-1, j, j+1 (and j+2, prefetched) in registers; the
// f row and the edge values are also loaded one row ahead.
#pragma once

#include "bfp_host.h"

namespace bfp {

constexpr int kIrV = 2;            // doubles per lane
constexpr int kIrCols = 32 * kIrV;
constexpr int kIrWarps = 4;
constexpr int64_t kIrKeyOff = 4096;

struct IrArgs {
  const double* b;   // right-hand side (scaled by bscale on the fly)
  double bscale;     // 2^-bshift
  int32_t bshift;
  int32_t nbshift;   // nb = -2^-nbshift
  const double* x;
  int64_t nx, ny;
  double cdiag, cnb;
  VOut out;          // BFP residual
  int64_t* meta;     // its meta block
  int32_t* tmp;      // qcomp window (int32, out layout) or null
  int64_t* gamma_mu; // previous residual's mu* (+ offset; 0 = unknown) in / out
  uint64_t* stats;   // [5] IR residual quantisations, [6] of which recomputed
  int w, w_tmp;
};

__device__ __forceinline__ bool split_double(double v, int64_t& M, int64_t& E) {
  const uint64_t bits = (uint64_t)__double_as_longlong(v);
  const int ex = (int)((bits >> 52) & 0x7ff);
  const uint64_t fr = bits & ((1ull << 52) - 1);
  if (ex == 0x7ff) return false;
  if (ex == 0) { M = (int64_t)fr; E = -1074; }
  else { M = (int64_t)(fr | (1ull << 52)); E = ex - 1075; }
  if (bits >> 63) M = -M;
  return true;
}

// Rare-case fallbacks kept out of line: inlined, the compiler would evaluate
// them speculatively and occupy GB300's low-rate FP64 pipe on every element.
__device__ __noinline__ double dmul_slow(double v, double factor) { return __dmul_rn(v, factor); }

// v * 2^-k for k >= 0 (exact): exponent-field arithmetic when v and the result
// are normal, the rounded multiply otherwise (zeros, subnormals, Inf/NaN).
// Either way the result equals __dmul_rn(v, 2^-k) bit for bit.
__device__ __forceinline__ double scale_pow2(double v, int k, double factor) {
  const uint64_t bits = (uint64_t)__double_as_longlong(v);
  const int ex = (int)((bits >> 52) & 0x7ff);
  if (ex > k && ex != 0x7ff) return __longlong_as_double((long long)(bits - ((uint64_t)k << 52)));
  return dmul_slow(v, factor);
}


// 0.75 v correctly rounded (the centre term of the 3D A'x), computed on the integer pipe: the product of
// the 53-bit significand m by 3 is exact in 55 bits and is rounded once to 53 bits, to nearest with ties
// to even, exactly as the IEEE multiply rounds it.  Zero, subnormal, tiny, huge and non-finite v (whose
// result may leave the normal range) take the rounded multiply, out of line.  Bit for bit
// __dmul_rn(0.75, v).
__device__ __forceinline__ double mul_three_quarters(double v) {
  const uint64_t bits = (uint64_t)__double_as_longlong(v);
  const int ex = (int)((bits >> 52) & 0x7ff);
  if (ex < 3 || ex > 2045) return dmul_slow(v, 0.75);
  const uint64_t M = 3ull * ((bits & ((1ull << 52) - 1)) | (1ull << 52));   // in [3 2^52, 3 2^53)
  const int sh = (M >> 54) ? 2 : 1;                                          // bits above the 53 kept
  uint64_t q = M >> sh;
  const uint64_t rem = M & ((1ull << sh) - 1), half = 1ull << (sh - 1);
  if (rem > half || (rem == half && (q & 1ull))) ++q;
  int e = ex - 2 + sh;
  if (q >> 53) { q >>= 1; ++e; }                                             // rounded up to 2^53
  return __longlong_as_double((long long)((bits & (1ull << 63)) | ((uint64_t)e << 52) | (q & ((1ull << 52) - 1))));
}

// floor(M 2^sh) for any sh (caller guarantees the fit when sh > 0)
__device__ __forceinline__ int64_t fshift(int64_t M, int64_t sh) {
  if (sh >= 0) return (int64_t)((uint64_t)M << (sh > 63 ? 63 : sh));
  return M >> (-sh > 63 ? 63 : -sh);
}

struct IrPlan {
  int64_t e_out, e_tmp, gam;
  int32_t window, narrow, recompute;
};

// Pass 1: the window exponent from gamma = the previous residual's mu (0: none);
// pass 2: e_out from mu* and the narrow / recompute decision of Alg. qcomp.
__device__ __forceinline__ IrPlan ir_plan(const IrArgs& a, bool pass1) {
  IrPlan p;
  const int64_t g = pass1 ? *a.gamma_mu : a.meta[4];
  p.window = (a.tmp != nullptr && g != 0) ? 1 : 0;
  p.gam = g - (int64_t(1) << 40);              // msb value of gamma (encoded with an offset)
  p.e_tmp = p.gam - a.w_tmp;
  p.e_out = 0;
  p.narrow = 0;
  p.recompute = 1;
  if (!pass1) {
    const int64_t key = a.meta[kMetaMu];
    const int64_t mu_abs = key > 0 ? key - kIrKeyOff : -1073;
    p.e_out = mu_abs - a.w;
    const bool ovf = p.gam < mu_abs, unf = (mu_abs - a.w) < (p.gam - a.w_tmp);
    p.narrow = (p.window && !ovf && !unf) ? 1 : 0;
    p.recompute = !p.narrow;
  }
  return p;
}

// after pass 2 (one thread): the result exponent, the next residual's gamma, the counters
__device__ __forceinline__ void ir_finish(const IrArgs& a, const IrPlan& p) {
  a.meta[0] = p.e_out;
  *a.gamma_mu = p.e_out + a.w + (int64_t(1) << 40);   // gamma of the next IR residual
  if (a.stats) {
    atomicAdd((unsigned long long*)&a.stats[5], 1ull);
    if (p.recompute) atomicAdd((unsigned long long*)&a.stats[6], 1ull);
  }
}

struct IrP {
  IrArgs a;
  int32_t rs;
};

// B: a batched launch, grid z the instance, parameters Pb[z]
template <bool PASS1, bool B = false>
__global__ void __launch_bounds__(128) k_ir2d(const __grid_constant__ IrP P1, const IrP* __restrict__ Pb) {
  pdl_wait();
  const IrP& P = B ? Pb[blockIdx.z] : P1;
  const IrArgs& a = P.a;
  const int rs = P.rs;
  __shared__ IrPlan sp;
  if (threadIdx.x == 0) sp = ir_plan(a, PASS1);
  __syncthreads();
  const IrPlan& p = sp;
  if (PASS1 && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) a.meta[4] = *a.gamma_mu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t cb = (int64_t)blockIdx.x * kIrCols;
  const int64_t j0 = ((int64_t)blockIdx.y * kIrWarps + warp) * rs;
  const int64_t j1 = j0 + rs < a.ny ? j0 + rs : a.ny;
  Red red = {0, 0, 0};
  bool bad = false;
  const int64_t nx = a.nx;

  if (!PASS1 && p.narrow) {
    // window hit: 8 consecutive columns per lane, 4 rows of the warp's tile at a time
    const int sh = (int)(p.e_out - p.e_tmp);
    const int64_t col = cb + (lane & 7) * 8;
    uint32_t nrm = 0;
    if (col < a.out.ld) {
      // four rows per lane in flight: all loads of a group before any store
      for (int64_t jb = j0 + (lane >> 3); jb < j1; jb += 16) {
        int4 u[4][2];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const int64_t j = jb + 4 * g;
          if (j < j1) {
            const int4* src = reinterpret_cast<const int4*>(a.tmp + j * a.out.ld + col);
            u[g][0] = src[0];
            u[g][1] = src[1];
          }
        }
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const int64_t j = jb + 4 * g;
          if (j >= j1) break;
          int32_t o[8] = {u[g][0].x, u[g][0].y, u[g][0].z, u[g][0].w, u[g][1].x, u[g][1].y, u[g][1].z, u[g][1].w};
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            o[k] = col + k < nx ? (o[k] >> sh) : 0;   // padding columns [nx, ld) are written as 0
            const uint32_t av = (uint32_t)(o[k] < 0 ? -o[k] : o[k]);
            nrm = av > nrm ? av : nrm;
          }
          stv<8>(a.out, j, col, o);
        }
      }
    }
    red.nrm = max(red.nrm, (long long)nrm);
  } else if (j0 < j1) {
    auto ldrow = [&](int64_t j, double (&v)[kIrV]) {
#pragma unroll
      for (int k = 0; k < kIrV; ++k) {
        const int64_t i = cb + 32 * k + lane;
        v[k] = (j >= 0 && j < a.ny && i < nx) ? __ldg(a.x + j * nx + i) : 0.0;
      }
    };
    double xm[kIrV], xc[kIrV], xp[kIrV], xpp[kIrV];
    ldrow(j0 - 1, xm);
    ldrow(j0, xc);
    ldrow(j0 + 1, xp);
    // f row j and the x edge values of row j (lanes 0, 31), loaded one row ahead
    auto ldb = [&](int64_t j, double (&v)[kIrV], double& we, double& ee) {
#pragma unroll
      for (int k = 0; k < kIrV; ++k) {
        const int64_t i = cb + 32 * k + lane;
        v[k] = (j < j1 && i < nx) ? __ldg(a.b + j * nx + i) : 0.0;
      }
      we = (j < j1 && lane == 0 && cb > 0) ? __ldg(a.x + j * nx + cb - 1) : 0.0;
      ee = (j < j1 && lane == 31 && cb + kIrCols < nx) ? __ldg(a.x + j * nx + cb + kIrCols) : 0.0;
    };
    double bn[kIrV], wn, en;
    ldb(j0, bn, wn, en);
    for (int64_t j = j0; j < j1; ++j) {
      ldrow(j + 2, xpp);
      double bv[kIrV];
#pragma unroll
      for (int k = 0; k < kIrV; ++k) bv[k] = bn[k];
      const double wedge = wn, eedge = en;
      ldb(j + 1, bn, wn, en);
#pragma unroll
      for (int k = 0; k < kIrV; ++k) {
        const int64_t i = cb + 32 * k + lane;
        double wv = __shfl_up_sync(0xffffffffu, xc[k], 1);
        double ev = __shfl_down_sync(0xffffffffu, xc[k], 1);
        const double wprev = __shfl_sync(0xffffffffu, xc[k > 0 ? k - 1 : 0], 31);
        const double enext = __shfl_sync(0xffffffffu, xc[k < kIrV - 1 ? k + 1 : kIrV - 1], 0);
        if (lane == 0) wv = k > 0 ? wprev : wedge;
        if (lane == 31) ev = k < kIrV - 1 ? enext : eedge;
        if (i >= nx) {
          if (!PASS1 && i < a.out.ld) {   // padding columns [nx, ld) are written as 0
            if (a.out.is32) reinterpret_cast<int32_t*>(a.out.m)[j * a.out.ld + i] = 0;
            else reinterpret_cast<int16_t*>(a.out.m)[j * a.out.ld + i] = 0;
          }
          continue;
        }
        // r = b' - A'x, A'x = c x + nb (((W + E) + S) + N): fixed order, explicit rounding.
        // In 2D c = 1 (1 * x = x exactly) and nb, bscale are powers of two (exact scalings).
        double s = __dadd_rn(wv, ev);
        s = __dadd_rn(s, xm[k]);
        s = __dadd_rn(s, xp[k]);
        const double ax = __dadd_rn(xc[k], -scale_pow2(s, a.nbshift, -a.cnb));
        const double r = __dsub_rn(scale_pow2(bv[k], a.bshift, a.bscale), ax);
        int64_t M = 0, E = -1074;
        if (!split_double(r, M, E)) { bad = true; continue; }
        if (PASS1) {
          const int64_t mv = M == 0 ? -1073 : msb64(M) + E;
          red.key = max(red.key, (long long)(mv + kIrKeyOff));
          if (p.window) a.tmp[j * a.out.ld + i] = wrap_bits((uint64_t)fshift(M, E - p.e_tmp), a.w_tmp);
        } else {
          const int64_t v = fshift(M, E - p.e_out);
          red.nrm = max(red.nrm, (long long)(v < 0 ? -v : v));
          if (a.out.is32) reinterpret_cast<int32_t*>(a.out.m)[j * a.out.ld + i] = (int32_t)v;
          else reinterpret_cast<int16_t*>(a.out.m)[j * a.out.ld + i] = (int16_t)v;
        }
      }
#pragma unroll
      for (int k = 0; k < kIrV; ++k) { xm[k] = xc[k]; xc[k] = xp[k]; xp[k] = xpp[k]; }
    }
  }
  if (bad) atomicOr((unsigned long long*)&a.meta[BFP_META_FLAGS], 1ull);
  pdl_trigger();
  block_commit(red, a.meta, nullptr, PASS1);
  if (!PASS1 && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) ir_finish(a, p);
}

// x <- x + m 2^e (FP64 update of Alg. ir): a thread owns one column of
// kUpdRows consecutive rows and issues all of their loads before any add.
constexpr int kUpdRows = 8;
struct UpdP {
  double* x;
  VIn y;
  const int64_t* meta;
};

template <class T, bool B = false>
__global__ void __launch_bounds__(256) k_ir_update2(const __grid_constant__ UpdP P1, const UpdP* __restrict__ Pb) {
  pdl_wait();
  const UpdP& P = B ? Pb[blockIdx.z] : P1;
  double* __restrict__ x = P.x;
  const VIn& y = P.y;
  const int64_t* meta = P.meta;
  const int64_t e = meta[0];
  const int64_t rows = y.ny * y.nz;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= y.nx) return;
  const T* m = reinterpret_cast<const T*>(y.m);
  for (int64_t r0 = (int64_t)blockIdx.y * kUpdRows; r0 < rows; r0 += (int64_t)gridDim.y * kUpdRows) {
    double xv[kUpdRows];
    int32_t mv[kUpdRows];
#pragma unroll
    for (int k = 0; k < kUpdRows; ++k) {
      const int64_t row = r0 + k;
      if (row < rows) {
        xv[k] = x[row * y.nx + i];
        mv[k] = (int32_t)__ldg(m + row * y.ld + i);
      }
    }
#pragma unroll
    for (int k = 0; k < kUpdRows; ++k) {
      const int64_t row = r0 + k;
      if (row < rows) x[row * y.nx + i] = __dadd_rn(xv[k], mant_pow2(mv[k], e));
    }
  }
}

}  // namespace bfp
