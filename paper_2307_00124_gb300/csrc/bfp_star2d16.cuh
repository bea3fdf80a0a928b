// bfp_star2d16.cuh -- five-point stencil ops on int16 mantissas (w <= 16), the
// finest-level hot path of the V-cycle.
//
// A warp owns a 256-column chunk: each lane 8 consecutive mantissas (one
// 16-byte load per row and input), kept packed as int16 pairs.  The warp walks
// a strip of rows with the rows above and below in registers, prefetching
// the next two rows of y (and the edge mantissas lanes 0 and 31 need) and the
// next row of r, so three rows of loads are in flight per warp.
//
// Fast path (the exact integer Z fits in int64 and the output exponent is at
// or above Z's): Z = cy*y + cn*(W+E+S+N) + cr*r with the App. B exponent
// alignment folded into three 32-bit coefficients, the result is one funnel
// shift, and nnqcomp saturation is detected with one unsigned range test per
// element; a warp that sees a value outside X_w (or a plan outside the fast
// regime) recomputes that row through the general quantiser, kept out of line
// so that it costs no registers on the fast path.  qcomp pass 1 takes the bit
// width of the OR of |Z| (the max msb) and stores the w_tmp window.
#pragma once

#include "bfp_host.h"

namespace bfp {

constexpr int kS16Cols = 256;   // columns per warp chunk (32 lanes x 8)

struct Pk8 {
  uint32_t w[4];
};

__device__ __forceinline__ int32_t pk_get(const Pk8& p, int k) {
  const uint32_t word = p.w[k >> 1];
  return (k & 1) ? ((int32_t)word >> 16) : ((int32_t)(word << 16) >> 16);
}

struct Loader16 {
  const int16_t* col;   // row 0 of this lane's 8 columns
  int64_t ld;
  int ny;
  bool ok;              // any valid column in this lane
  uint32_t mask[4];     // zeroes the columns >= nx
  __device__ __forceinline__ Pk8 operator()(int j) const {
    Pk8 p;
    if (ok && j >= 0 && j < ny) {
      const uint4 u = __ldg(reinterpret_cast<const uint4*>(col + (int64_t)j * ld));
      p.w[0] = u.x & mask[0]; p.w[1] = u.y & mask[1]; p.w[2] = u.z & mask[2]; p.w[3] = u.w & mask[3];
    } else {
      p.w[0] = p.w[1] = p.w[2] = p.w[3] = 0u;
    }
    return p;
  }
};

__device__ __forceinline__ Loader16 loader16(const VIn& v, int64_t c0) {
  Loader16 L;
  L.col = reinterpret_cast<const int16_t*>(v.m) + c0;
  L.ld = v.ld;
  L.ny = (int)(v.ny * v.nz);
  L.ok = v.m != nullptr && c0 < v.nx && c0 < v.ld;
  const int64_t nv = v.nx - c0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t lo = (2 * i < nv) ? 0xffffu : 0u, hi = (2 * i + 1 < nv) ? 0xffff0000u : 0u;
    L.mask[i] = lo | hi;
  }
  return L;
}

// Inputs of one lane's 8 outputs, for the out-of-line general path.
struct Row8 {
  int32_t y[8], ym[8], yp[8], r[8];
  int32_t wv, ev;
};

template <bool PASS1, int KIND>
__device__ __noinline__ void slow_row8(const Row8& in, const Plan& p, const Fast& fq, const VOut& out, int32_t* tmp,
                                       int64_t row, int64_t c0, Red& red, int32_t c, int32_t nb, int32_t mw) {
  auto hl = [&](int k, int64_t& H, int64_t& L) {
    if (KIND == kJacobi0) {
      H = (int64_t)mw * (int64_t)in.r[k];
      L = 0;
      return;
    }
    const int64_t wk = k == 0 ? in.wv : in.y[k - 1];
    const int64_t ek = k == 7 ? in.ev : in.y[k + 1];
    const int64_t ns = wk + ek + in.ym[k] + in.yp[k];
    H = (int64_t)c * (int64_t)in.y[k] + (int64_t)nb * ns;
    L = KIND == kApply ? 0 : (KIND == kResidual ? -(int64_t)in.r[k] : (int64_t)mw * (int64_t)in.r[k]);
  };
  quantvf<PASS1, 8>(hl, p, fq, out, tmp, row, c0, red);
}

template <int KIND, bool PASS1>
__global__ void __launch_bounds__(128, 7) k_star2d16(const VIn y, const VIn r, const int32_t c, const int32_t nb,
                                                     const int32_t mw, const QDesc q, const VOut out, const int rs) {
  __shared__ Plan sp;
  if (threadIdx.x == 0) {
    build_plan(q, sp);
    if (!PASS1 && q.mode == kQcomp) plan_from_mu(sp, q.meta_out[kMetaMu]);
  }
  __syncthreads();
  const Plan& p = sp;
  const Fast fq = make_fast(p, PASS1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * kS16Cols + lane * 8;
  const int ny = (int)out.ny;
  const int j0 = (int)(((int64_t)blockIdx.y * 4 + warp) * rs);
  const int j1 = j0 + rs < ny ? j0 + rs : ny;
  const bool act = c0 < out.ld;
  Red red = {0, 0, 0};
  int32_t* tmp = (PASS1 && p.use_tmp && !p.guarded) ? reinterpret_cast<int32_t*>(q.tmp) : nullptr;

  // Z = cy*y + cn*ns + cr*r, the group shifts folded into the coefficients
  int64_t cy, cn, cr;
  if (KIND == kJacobi0) {
    cy = 0; cn = 0; cr = (int64_t)((uint64_t)(int64_t)mw << fq.dh);
  } else {
    cy = (int64_t)((uint64_t)(int64_t)c << fq.dh);
    cn = (int64_t)((uint64_t)(int64_t)nb << fq.dh);
    cr = KIND == kApply ? 0 : (KIND == kResidual ? -(int64_t)(1ull << fq.dl) : (int64_t)((uint64_t)(int64_t)mw << fq.dl));
  }
  const bool fast = fq.ok && fq.t < 32 && cy == (int32_t)cy && cn == (int32_t)cn && cr == (int32_t)cr;
  const int32_t cy32 = (int32_t)cy, cn32 = (int32_t)cn, cr32 = (int32_t)cr;
  const uint32_t t = (uint32_t)fq.t;
  const int sh = 32 - fq.w;                     // decr to fq.w bits (pass 1 window)
  // nnqcomp range: the result fits in X_w iff zmin <= Z <= zmax
  const int64_t zmin = (int64_t)((uint64_t)(-(1ll << (fq.w - 1))) << t);
  const uint64_t zrange = (uint64_t)(((uint64_t)1 << (fq.w - 1 + t)) * 2 - 1);
  const int64_t nvalid = out.nx - c0;

  const Loader16 ly = loader16(y, c0), lr = loader16(r, c0);
  // lane 0 needs the west neighbour of its first column, lane 31 the east one of its last
  const int16_t* yb = reinterpret_cast<const int16_t*>(y.m);
  const int64_t ecol = lane == 0 ? c0 - 1 : c0 + 8;
  const bool eok = (lane == 0 || lane == 31) && KIND != kJacobi0 && y.m != nullptr && ecol >= 0 && ecol < y.nx;
  auto ledge = [&](int j) -> int32_t {
    return (eok && j >= 0 && j < ny) ? (int32_t)__ldg(yb + (int64_t)j * y.ld + ecol) : 0;
  };

  uint32_t nrm = 0;
  uint64_t ormag = 0;

  auto emit_row = [&](int j, int32_t (&o)[8]) {
    if (nvalid < 8) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k >= nvalid) o[k] = 0;
    }
    if (PASS1) {
      if (tmp) {
        int4* d = reinterpret_cast<int4*>(tmp + (int64_t)j * out.ld + c0);
        d[0] = make_int4(o[0], o[1], o[2], o[3]);
        d[1] = make_int4(o[4], o[5], o[6], o[7]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint32_t a = (uint32_t)(o[k] < 0 ? -o[k] : o[k]);
        nrm = a > nrm ? a : nrm;
      }
      uint4 u;
      u.x = (uint32_t)(uint16_t)o[0] | ((uint32_t)(uint16_t)o[1] << 16);
      u.y = (uint32_t)(uint16_t)o[2] | ((uint32_t)(uint16_t)o[3] << 16);
      u.z = (uint32_t)(uint16_t)o[4] | ((uint32_t)(uint16_t)o[5] << 16);
      u.w = (uint32_t)(uint16_t)o[6] | ((uint32_t)(uint16_t)o[7] << 16);
      if (out.is32) {
        stv<8>(out, j, c0, o);
      } else {
        *reinterpret_cast<uint4*>(reinterpret_cast<int16_t*>(out.m) + (int64_t)j * out.ld + c0) = u;
      }
    }
  };

  if (!PASS1 && p.narrow) {
    for (int j = j0; j < j1; ++j)
      if (act) narrowv<8>(reinterpret_cast<const int32_t*>(q.tmp), p, out, j, c0, red);
  } else if (j0 < j1) {
    Pk8 ym, yc, yp, rc;
    int32_t ec = 0, ep = 0;
    if (KIND != kJacobi0) {
      ym = ly(j0 - 1); yc = ly(j0); yp = ly(j0 + 1);
      ec = ledge(j0); ep = ledge(j0 + 1);
    }
    if (KIND != kApply) rc = lr(j0);
    for (int j = j0; j < j1; ++j) {
      Pk8 ypp, rn;
      int32_t epp = 0;
      if (KIND != kJacobi0) { ypp = ly(j + 2); epp = ledge(j + 2); }
      if (KIND != kApply) rn = lr(j + 1);
      int32_t yv[8], wv = 0, ev = 0;
      if (KIND != kJacobi0) {
#pragma unroll
        for (int k = 0; k < 8; ++k) yv[k] = pk_get(yc, k);
        wv = __shfl_up_sync(0xffffffffu, yv[7], 1);
        ev = __shfl_down_sync(0xffffffffu, yv[0], 1);
        if (lane == 0) wv = ec;
        if (lane == 31) ev = ec;
      }
      if (act) {
        bool redo = !fast;
        int32_t o[8];
        if (fast) {
          bool ovf = false;
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            int64_t Z;
            if (KIND == kJacobi0) {
              Z = (int64_t)cr32 * pk_get(rc, k);
            } else {
              const int32_t wk = k == 0 ? wv : yv[k - 1];
              const int32_t ek = k == 7 ? ev : yv[k + 1];
              const int32_t ns = wk + ek + pk_get(ym, k) + pk_get(yp, k);
              Z = (int64_t)cy32 * yv[k] + (int64_t)cn32 * ns;
              if (KIND != kApply) Z += (int64_t)cr32 * pk_get(rc, k);
            }
            const int32_t v = (int32_t)__funnelshift_r((uint32_t)(uint64_t)Z, (uint32_t)((uint64_t)Z >> 32), t);
            if (PASS1) {
              if (k < nvalid) ormag |= (uint64_t)(Z ^ (Z >> 63));
              o[k] = (int32_t)((uint32_t)v << sh) >> sh;
            } else {
              if (fq.clamp) ovf |= ((uint64_t)Z - (uint64_t)zmin > zrange) && (k < nvalid);
              o[k] = v;
            }
          }
          if (!PASS1 && fq.clamp) redo = ovf;
        }
        if (!PASS1 && fq.clamp && fast) redo = __any_sync(__activemask(), redo);
        if (redo) {
          Row8 in;
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            in.y[k] = KIND == kJacobi0 ? 0 : pk_get(yc, k);
            in.ym[k] = KIND == kJacobi0 ? 0 : pk_get(ym, k);
            in.yp[k] = KIND == kJacobi0 ? 0 : pk_get(yp, k);
            in.r[k] = KIND == kApply ? 0 : pk_get(rc, k);
          }
          in.wv = wv;
          in.ev = ev;
          slow_row8<PASS1, KIND>(in, p, fq, out, tmp, j, c0, red, c, nb, mw);
        } else {
          emit_row(j, o);
        }
      }
      if (KIND != kJacobi0) { ym = yc; yc = yp; yp = ypp; ec = ep; ep = epp; }
      if (KIND != kApply) rc = rn;
    }
  }
  if (PASS1 && ormag) red.key = max(red.key, (long long)(256 + (64 - __clzll((long long)ormag)) + 1));
  if (PASS1 && fast && j0 < j1 && act && ormag == 0) red.key = max(red.key, 257ll);   // all-zero chunk: msb 1
  red.nrm = max(red.nrm, (long long)nrm);
  block_commit(red, q.meta_out, q.stats, PASS1);
  if (!PASS1) op_epilogue(q, p);
}

}  // namespace bfp
