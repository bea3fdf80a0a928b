// bfp_star2d.cuh -- 2D five-point stencil ops (apply, residual, damped Jacobi)
// as row-walking kernels.
//
// Layout: a warp owns a 256-column chunk (8 consecutive mantissas per lane,
// one 16-byte load for int16) and walks a strip of rows; the rows above and
// below live in registers (rolling window, prefetched two rows ahead), the
// west/east neighbours come from the adjacent lanes by shuffle, and only
// lanes 0 and 31 load one extra mantissa each.  Every input byte is read
// from DRAM about once.  The exact results go through the shared quantiser
// (quant8): qcomp pass 1 (mu* and the w_tmp window), qcomp pass 2 / nnqcomp
// (the w_out result).
#pragma once

#include "bfp_host.h"
#include "bfp_star2d16.cuh"

namespace bfp {

constexpr int kStarWarps = 4;     // warps per CTA, stacked over consecutive row strips
constexpr int kStarV = 4;         // mantissas per lane
constexpr int kStarCols = 32 * kStarV;

// Loads kStarV mantissas of row j at this lane's columns (0 outside the grid).
template <class T>
struct RowLoader {
  const T* col;      // base + c0
  int64_t ld;
  int ny;
  bool ok;           // lane inside the row (c0 < min(nx, ld))
  int nvalid;        // valid columns of this lane's chunk (kStarV unless it holds column nx-1)
  __device__ __forceinline__ void operator()(int j, int32_t (&o)[kStarV]) const {
    if (ok && j >= 0 && j < ny) {
      const T* p = col + (int64_t)j * ld;
      if (sizeof(T) == 2) {
        const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
        o[0] = (int32_t)(int16_t)(u.x & 0xffffu); o[1] = (int32_t)(int16_t)(u.x >> 16);
        o[2] = (int32_t)(int16_t)(u.y & 0xffffu); o[3] = (int32_t)(int16_t)(u.y >> 16);
      } else {
        const int4 u = __ldg(reinterpret_cast<const int4*>(p));
        o[0] = u.x; o[1] = u.y; o[2] = u.z; o[3] = u.w;
      }
      if (nvalid < kStarV) {
#pragma unroll
        for (int k = 0; k < kStarV; ++k)
          if (k >= nvalid) o[k] = 0;
      }
    } else {
#pragma unroll
      for (int k = 0; k < kStarV; ++k) o[k] = 0;
    }
  }
};

template <class T>
__device__ __forceinline__ RowLoader<T> row_loader(const VIn& v, int64_t c0) {
  RowLoader<T> L;
  L.col = reinterpret_cast<const T*>(v.m) + c0;
  L.ld = v.ld;
  L.ny = (int)(v.ny * v.nz);
  L.ok = v.m != nullptr && c0 < v.nx && c0 < v.ld;
  const int64_t nv = v.nx - c0;
  L.nvalid = nv >= kStarV ? kStarV : (nv > 0 ? (int)nv : 0);
  return L;
}

// One output row chunk of the fast path: Z_k = cy*y_k + cn*ns_k + cr*r_k exactly in int64
// (the exponent alignment of App. B folded into the coefficients), then a uniform
// right shift by t < 32 (one funnel shift), saturation by comparing Z with the
// precomputed bounds (nnqcomp), or the bit width of Z (qcomp pass 1).
struct FastRow {
  int64_t zmax, zmin;   // v > hi  <=>  Z > zmax ;  v < lo  <=>  Z < zmin
  int32_t hi, lo;
  uint32_t t;           // < 32
  uint32_t tl;          // pass 1: left shift of the window
  int32_t w, clamp;
};

__device__ __forceinline__ FastRow make_fast_row(const Fast& fq) {
  FastRow f;
  f.t = (uint32_t)fq.t;
  f.tl = (uint32_t)fq.tl;
  f.w = fq.w;
  f.clamp = fq.clamp;
  f.hi = (int32_t)((1ll << (fq.w - 1)) - 1);
  f.lo = (int32_t)(-(1ll << (fq.w - 1)));
  f.zmax = (int64_t)(((uint64_t)((int64_t)f.hi + 1) << f.t) - 1);
  f.zmin = (int64_t)((uint64_t)(int64_t)f.lo << f.t);
  return f;
}

template <bool PASS1, bool NARROW32>
__device__ __forceinline__ void fast_row(const int64_t (&zc)[3], const int32_t (&yv)[kStarV],
                                         const int32_t (&nsv)[kStarV], const int32_t (&rv)[kStarV],
                                         const FastRow& fr, int nvalid, long long& key, uint32_t& nrm, int& sat,
                                         int32_t (&o)[kStarV]) {
#pragma unroll
  for (int k = 0; k < kStarV; ++k) {
    int64_t Z;
    if (NARROW32) Z = (int64_t)(int32_t)zc[0] * yv[k] + (int64_t)(int32_t)zc[1] * nsv[k] + (int64_t)(int32_t)zc[2] * rv[k];
    else Z = zc[0] * (int64_t)yv[k] + zc[1] * (int64_t)nsv[k] + zc[2] * (int64_t)rv[k];
    const bool valid = k < nvalid;
    const uint32_t zlo = (uint32_t)(uint64_t)Z, zhi = (uint32_t)((uint64_t)Z >> 32);
    const int32_t v = (int32_t)__funnelshift_r(zlo, zhi, fr.t);   // low 32 bits of Z >> t
    if (PASS1) {
      if (valid) key = max(key, (long long)(256 + msb64(Z)));
      const int s = 32 - fr.w;
      o[k] = valid ? ((int32_t)((uint32_t)v << fr.tl << s) >> s) : 0;   // decr to w_tmp bits
    } else {
      int32_t vi = v;
      if (fr.clamp) {
        const bool above = Z > fr.zmax, below = Z < fr.zmin;
        vi = above ? fr.hi : (below ? fr.lo : v);
        sat += ((above || below) && valid) ? 1 : 0;
      }
      vi = valid ? vi : 0;
      o[k] = vi;
      const uint32_t av = (uint32_t)(vi < 0 ? -vi : vi);
      nrm = av > nrm ? av : nrm;
    }
  }
}

template <class T, int KIND, bool PASS1>
__global__ void __launch_bounds__(128, 8) k_star2d(const VIn y, const VIn r, const int32_t c, const int32_t nb,
                                                   const int32_t mw, const QDesc q, const VOut out, const int rs,
                                                   const int nsfit) {
  __shared__ Plan sp;
  if (threadIdx.x == 0) {
    build_plan(q, sp);
    if (!PASS1 && q.mode == kQcomp) plan_from_mu(sp, q.meta_out[kMetaMu]);
  }
  __syncthreads();
  const Plan& p = sp;
  Fast fq = make_fast(p, PASS1);
  if (fq.t >= 32) fq.ok = 0;          // the register fast path shifts by less than 32
  const FastRow fr = make_fast_row(fq);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * kStarCols + lane * kStarV;
  const int ny = (int)out.ny;
  const int j0 = (int)(((int64_t)blockIdx.y * kStarWarps + warp) * rs);
  const int j1 = j0 + rs < ny ? j0 + rs : ny;
  const bool act = c0 < out.ld;
  Red red = {0, 0, 0};
  uint32_t nrm32 = 0;
  int sat = 0;
  int32_t* tmp = (PASS1 && p.use_tmp && !p.guarded) ? reinterpret_cast<int32_t*>(q.tmp) : nullptr;
  // Z = cy*y + cn*ns + cr*r with the group shifts folded into the coefficients
  int64_t zc[3];
  if (KIND == kJacobi0) {
    zc[0] = 0; zc[1] = 0; zc[2] = (int64_t)((uint64_t)(int64_t)mw << fq.dh);
  } else {
    zc[0] = (int64_t)((uint64_t)(int64_t)c << fq.dh);
    zc[1] = (int64_t)((uint64_t)(int64_t)nb << fq.dh);
    zc[2] = KIND == kApply ? 0 : (KIND == kResidual ? -(int64_t)(1ull << fq.dl) : (int64_t)((uint64_t)(int64_t)mw << fq.dl));
  }
  // folded coefficients in 32 bits: Z from 32 x 32 -> 64-bit products (the mantissas and the neighbour
  // sum are 32-bit: int16 storage, or int32 inputs of at most 30 bits, nsfit)
  const bool small = zc[0] == (int32_t)zc[0] && zc[1] == (int32_t)zc[1] && zc[2] == (int32_t)zc[2];
  const bool reg = sizeof(T) == 2 || nsfit != 0;   // register path: the neighbour sum exact in int32
  const RowLoader<T> ly = row_loader<T>(y, c0), lr = row_loader<T>(r, c0);
  const int nvalid = (int)(out.nx - c0 >= kStarV ? kStarV : (out.nx - c0 > 0 ? out.nx - c0 : 0));

  auto emit = [&](int j, const int32_t (&o)[kStarV]) {
    if (PASS1) {
      if (tmp) *reinterpret_cast<int4*>(tmp + (int64_t)j * out.ld + c0) = make_int4(o[0], o[1], o[2], o[3]);
    } else {
      stv<kStarV>(out, j, c0, o);
    }
  };

  if (!PASS1 && p.narrow) {
    for (int j = j0; j < j1; ++j)
      if (act) narrowv<kStarV>(reinterpret_cast<const int32_t*>(q.tmp), p, out, j, c0, red);
  } else if (KIND == kJacobi0) {
    const int32_t zero[kStarV] = {0, 0, 0, 0};
    for (int j = j0; j < j1; ++j) {
      int32_t b[kStarV];
      lr(j, b);
      if (!act) continue;
      if (fq.ok) {
        int32_t o[kStarV];
        if (small) fast_row<PASS1, true>(zc, zero, zero, b, fr, nvalid, red.key, nrm32, sat, o);
        else fast_row<PASS1, false>(zc, zero, zero, b, fr, nvalid, red.key, nrm32, sat, o);
        emit(j, o);
      } else {
        auto hl = [&](int k, int64_t& H, int64_t& L) { H = (int64_t)mw * (int64_t)b[k]; L = 0; };
        quantvf<PASS1, kStarV>(hl, p, fq, out, tmp, j, c0, red);
      }
    }
  } else if (j0 < j1) {
    int32_t ym[kStarV], yc[kStarV], yp[kStarV], ypp[kStarV], rc[kStarV], rn[kStarV];
    ly(j0 - 1, ym);
    ly(j0, yc);
    ly(j0 + 1, yp);
    if (KIND != kApply) lr(j0, rc);
    else {
#pragma unroll
      for (int k = 0; k < kStarV; ++k) rc[k] = 0;
    }
    const T* yrow = reinterpret_cast<const T*>(y.m);
    for (int j = j0; j < j1; ++j) {
      // prefetch: two rows of y and one row of r ahead
      ly(j + 2, ypp);
      if (KIND != kApply) lr(j + 1, rn);
      int32_t wv = __shfl_up_sync(0xffffffffu, yc[kStarV - 1], 1);
      int32_t ev = __shfl_down_sync(0xffffffffu, yc[0], 1);
      if (lane == 0) wv = (c0 > 0 && c0 - 1 < y.nx) ? (int32_t)__ldg(yrow + (int64_t)j * y.ld + c0 - 1) : 0;
      if (lane == 31) ev = (c0 + kStarV < y.nx) ? (int32_t)__ldg(yrow + (int64_t)j * y.ld + c0 + kStarV) : 0;
      int32_t ns[kStarV];   // int16 inputs only (fast path): |ns| <= 2^17
#pragma unroll
      for (int k = 0; k < kStarV; ++k) {
        const uint32_t wk = (uint32_t)(k == 0 ? wv : yc[k - 1]);
        const uint32_t ek = (uint32_t)(k == kStarV - 1 ? ev : yc[k + 1]);
        ns[k] = reg ? (int32_t)(((wk + ek) + (uint32_t)ym[k]) + (uint32_t)yp[k]) : 0;
      }
      if (act) {
        if (fq.ok && reg) {
          int32_t o[kStarV];
          if (small) fast_row<PASS1, true>(zc, yc, ns, rc, fr, nvalid, red.key, nrm32, sat, o);
          else fast_row<PASS1, false>(zc, yc, ns, rc, fr, nvalid, red.key, nrm32, sat, o);
          emit(j, o);
        } else {
          typedef typename std::conditional<sizeof(T) == 2, int32_t, int64_t>::type S;
          auto hl = [&](int k, int64_t& H, int64_t& L) {
            const S wk = k == 0 ? (S)wv : (S)yc[k - 1];
            const S ek = k == kStarV - 1 ? (S)ev : (S)yc[k + 1];
            const S nss = ((wk + ek) + (S)ym[k]) + (S)yp[k];
            H = (int64_t)c * (int64_t)yc[k] + (int64_t)nb * (int64_t)nss;
            L = KIND == kApply ? 0 : (KIND == kResidual ? -(int64_t)rc[k] : (int64_t)mw * (int64_t)rc[k]);
          };
          quantvf<PASS1, kStarV>(hl, p, fq, out, tmp, j, c0, red);
        }
      }
#pragma unroll
      for (int k = 0; k < kStarV; ++k) {
        ym[k] = yc[k];
        yc[k] = yp[k];
        yp[k] = ypp[k];
        if (KIND != kApply) rc[k] = rn[k];
      }
    }
  }
  red.nrm = max(red.nrm, (long long)nrm32);
  red.sat += sat;
  block_commit(red, q.meta_out, q.stats, PASS1);
  if (!PASS1) op_epilogue(q, p);
}

// staged kernel (int16 mantissas, 2D or 3D; int32 mantissas, 2D), zero_accumulators already issued;
// rs rows per warp
template <int KIND, int ND, class T = int16_t>
inline int32_t launch_star16(const VIn& y, const VIn& r, int32_t c, int32_t nb, int32_t mw, const QDesc& q,
                             const VOut& o, int rs, cudaStream_t s) {
  static bool carved = false;   // the staging ring wants the shared-memory carveout (7 CTAs / SM in 2D, 5 in 3D)
  if (!carved) {
    cudaFuncSetAttribute(k_star16<KIND, true, ND, false, false, T>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_star16<KIND, false, ND, false, false, T>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if constexpr (ND == 2) {
      cudaFuncSetAttribute(k_star16<KIND, true, 2, false, true, T>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      cudaFuncSetAttribute(k_star16<KIND, false, 2, false, true, T>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    carved = true;
  }
  // columns per warp chunk: 4 int32, 16 int16 (2D) or 8 int16 (3D) mantissas per lane
  constexpr int64_t kCols = sizeof(T) == 4 ? kS16Cols / 2 : (ND == 2 ? 2 * kS16Cols : kS16Cols);
  const int64_t strips = (o.ny + 4 * (int64_t)rs - 1) / (4 * (int64_t)rs);
  const int64_t chunks = (o.ld + kCols - 1) / kCols;
  const dim3 g((unsigned)(chunks > 0 ? chunks : 1), (unsigned)(strips > 0 ? strips : 1),
               (unsigned)(ND == 3 ? o.nz : 1));
  const Star16P P{y, r, c, nb, mw, q, o, rs, VarRow{}};
  if constexpr (ND == 2) {   // recordable for batched solves
    if (q.mode == kQcomp)
      launch_rec<Star16P, &k_star16<KIND, true, 2, false, false, T>, &k_star16<KIND, true, 2, false, true, T>>(g, 128, 0, s, P);
    launch_rec<Star16P, &k_star16<KIND, false, 2, false, false, T>, &k_star16<KIND, false, 2, false, true, T>>(g, 128, 0, s, P);
  } else {
    if (q.mode == kQcomp) k_star16<KIND, true, ND><<<g, 128, 0, s>>>(P, nullptr);
    k_star16<KIND, false, ND><<<g, 128, 0, s>>>(P, nullptr);
  }
  note_launches(q.mode == kQcomp ? 2 : 1);
  return cudaGetLastError() == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

// Rows per warp strip of the variable-coefficient staged kernel.
inline int star16_var_rows(int64_t ny) { return pick_rows(ny >= 2048 ? 16 : (ny >= 1024 ? 8 : (ny >= 256 ? 4 : 2)), 32); }

// The staged kernel pays off once its grid (256-column chunks x strips) fills the GPU about
// twice over (three CTAs per SM): on smaller grids the row walk's per-row latency is exposed and
// the generic row kernel, with more independent work per SM, is faster (measured per level of the
// 2047^2 hierarchy: 1.3x faster at 2047^2, slower from 1023^2 down).
inline bool star16_var_fills(const bfp_vec* out) {
  const int64_t ny = out->n[1], rs = star16_var_rows(ny);
  const int64_t ctas = ((out->ld + kS16Cols - 1) / kS16Cols) * ((ny + 4 * rs - 1) / (4 * rs));
  return ctas >= 3 * (int64_t)sm_count();
}

// 2D variable-coefficient op (int16 y, r, faces, weights and result) through the staged kernel
template <int KIND>
inline int32_t launch_star16_var(const VIn& y, const VIn& r, const VarRow& va, const QDesc& q, const bfp_vec* out,
                                 cudaStream_t s) {
  if (q.hbits > 62 || (q.two && q.lbits > 62)) return BFP_ERR_WIDTH;
  static bool carved = false;
  if (!carved) {
    cudaFuncSetAttribute(k_star16<KIND, true, 2, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_star16<KIND, false, 2, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    carved = true;
  }
  const VOut o = vout(out);
  const int rs = star16_var_rows(out->n[1]);   // <= 32: row masks
  if (zero_accumulators(q.meta_out, s) != cudaSuccess) return BFP_ERR_CUDA;
  const int64_t strips = (o.ny + 4 * (int64_t)rs - 1) / (4 * (int64_t)rs);
  const int64_t chunks = (o.ld + kS16Cols - 1) / kS16Cols;
  const dim3 g((unsigned)(chunks > 0 ? chunks : 1), (unsigned)(strips > 0 ? strips : 1), 1u);
  const Star16P P{y, r, 0, 0, 0, q, o, rs, va};
  if (q.mode == kQcomp) k_star16<KIND, true, 2, true><<<g, 128, 0, s>>>(P, nullptr);
  k_star16<KIND, false, 2, true><<<g, 128, 0, s>>>(P, nullptr);
  note_launches(q.mode == kQcomp ? 2 : 1);
  return cudaGetLastError() == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

// 3D seven-point op on int16 mantissas through the staged kernel
template <int KIND>
inline int32_t launch_star3d16(const VIn& y, const VIn& r, int64_t c64, int64_t nb64, int64_t mw64, const QDesc& q,
                               const bfp_vec* out, cudaStream_t s) {
  if (q.hbits > 62 || (q.two && q.lbits > 62)) return BFP_ERR_WIDTH;
  const VOut o = vout(out);
  if (o.nz > 65535) return BFP_ERR_SHAPE;
  const int64_t ny = out->n[1];
  const int rs = pick_rows(ny >= 256 ? 16 : (ny >= 64 ? 8 : 2), 32);   // <= 32: row masks
  if (zero_accumulators(q.meta_out, s) != cudaSuccess) return BFP_ERR_CUDA;
  VOut oo = o;
  if (KIND == kJacobi0) {   // no neighbours: all ny * nz rows as one plane
    oo.ny = o.ny * o.nz;
    oo.nz = 1;
    const int rs2 = pick_rows(oo.ny >= 2048 ? 16 : (oo.ny >= 1024 ? 8 : (oo.ny >= 256 ? 4 : 2)), 32);
    return launch_star16<KIND, 2>(y, r, 0, 0, (int32_t)mw64, q, oo, rs2, s);
  }
  if (oo.nz == 0) { oo.ny = 0; oo.nz = 1; }   // no planes: one (empty) plane still publishes the meta
  return launch_star16<KIND, 3>(y, r, (int32_t)c64, (int32_t)nb64, (int32_t)mw64, q, oo, rs, s);
}

template <class T, int KIND>
// nsfit: y's mantissas have at most 30 bits, so a sum of four neighbours is exact in int32
inline int32_t launch_star2d(const VIn& y, const VIn& r, int64_t c64, int64_t nb64, int64_t mw64, const QDesc& q,
                             const bfp_vec* out, cudaStream_t s, bool nsfit = true) {
  if (q.hbits > 62 || (q.two && q.lbits > 62)) return BFP_ERR_WIDTH;
  const int32_t c = (int32_t)c64, nb = (int32_t)nb64, mw = (int32_t)mw64;   // checked < 2^31 by the caller
  const VOut o = vout(out);
  const int64_t ny = out->n[1];
  const int rs = pick_rows(ny >= 2048 ? 16 : (ny >= 1024 ? 8 : (ny >= 256 ? 4 : 2)), 32);   // <= 32: row masks
  // the int16 staged kernel's lanes take 16 columns: half the rows per strip keep a level's CTA count
  const int rs16 = pick_rows(ny >= 2048 ? 8 : (ny >= 1024 ? 4 : (ny >= 256 ? 2 : 1)), 32);
  const int64_t chunks = (out->ld + kStarCols - 1) / kStarCols;
  const int64_t strips = (ny + (int64_t)kStarWarps * rs - 1) / ((int64_t)kStarWarps * rs);
  const dim3 grid((unsigned)chunks, (unsigned)(strips > 0 ? strips : 1));
  if (zero_accumulators(q.meta_out, s) != cudaSuccess) return BFP_ERR_CUDA;
  if (sizeof(T) == 2 && !o.is32) return launch_star16<KIND, 2>(y, r, c, nb, mw, q, o, rs16, s);
  // int32 mantissas of at most 30 bits in y and r (one storage class: the callers send mixed storage to
  // the generic row kernel) and an int32 output: the staged kernel with 128-column chunks (the range
  // test of its register path needs w_out <= 30)
  if (sizeof(T) == 4 && o.is32 && nsfit && q.w_out <= 30) return launch_star16<KIND, 2, int32_t>(y, r, c, nb, mw, q, o, rs, s);
  if (q.mode == kQcomp) k_star2d<T, KIND, true><<<grid, 128, 0, s>>>(y, r, c, nb, mw, q, o, rs, nsfit ? 1 : 0);
  k_star2d<T, KIND, false><<<grid, 128, 0, s>>>(y, r, c, nb, mw, q, o, rs, nsfit ? 1 : 0);
  note_launches(q.mode == kQcomp ? 2 : 1);
  return cudaGetLastError() == cudaSuccess ? BFP_OK : BFP_ERR_CUDA;
}

}  // namespace bfp
