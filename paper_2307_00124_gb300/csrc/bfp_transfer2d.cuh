// bfp_transfer2d.cuh -- 2D grid transfers on int16 mantissas as row-walking
// kernels: full-weighting restriction (Alg. v-cycle restriction line) and
// bilinear interpolation with or without the correction y - P d (Alg. v-cycle
// correction line, Alg. fmg interpolation line).  Same structure and the same
// register fast path / out-of-line general path as bfp_star2d16.cuh.
#pragma once

#include "bfp_star2d16.cuh"

namespace bfp {

__device__ __forceinline__ void unpack8(const uint4 u, int32_t (&o)[8]) {
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    o[2 * k] = (int32_t)(w[k] << 16) >> 16;
    o[2 * k + 1] = (int32_t)w[k] >> 16;
  }
}

// int16 row chunk of 8 at (row, c0) with zeros outside the grid
__device__ __forceinline__ void ldrow16(const VIn& v, int64_t row, int64_t c0, int32_t (&o)[8]) {
  if (row < 0 || row >= v.ny * v.nz || c0 >= v.nx || c0 >= v.ld) {
#pragma unroll
    for (int k = 0; k < 8; ++k) o[k] = 0;
    return;
  }
  unpack8(__ldg(reinterpret_cast<const uint4*>(reinterpret_cast<const int16_t*>(v.m) + row * v.ld + c0)), o);
  if (c0 + 8 > v.nx) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (c0 + k >= v.nx) o[k] = 0;
  }
}

__device__ __forceinline__ int32_t ld1_16(const VIn& v, int64_t row, int64_t col) {
  if (row < 0 || row >= v.ny * v.nz || col < 0 || col >= v.nx) return 0;
  return (int32_t)__ldg(reinterpret_cast<const int16_t*>(v.m) + row * v.ld + col);
}

// Emits one 8-wide output chunk from exact groups (H, L) through the fast path when the
// plan allows (no value outside X_w in the warp), else through the general quantiser.
// General-path fallback for one chunk (kept out of line).
template <bool PASS1>
__device__ __noinline__ void slow_hl8(const int32_t (&H)[8], const int32_t (&L)[8], const Plan& p, const VOut& out,
                                      int32_t* tmp, int64_t row, int64_t c0, Red& red) {
  int64_t H64[8], L64[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) { H64[k] = H[k]; L64[k] = L[k]; }
  quant8<PASS1>(H64, L64, p, out, tmp, row, c0, red);
}

template <bool PASS1>
__device__ __forceinline__ void emit_hl8(const int32_t (&H)[8], const int32_t (&L)[8], const Plan& p, const Fast& fq,
                                         bool fast, const VOut& out, int32_t* tmp, int64_t row, int64_t c0, Red& red,
                                         uint32_t& nrm, uint64_t& ormag) {
  const int64_t nvalid = out.nx - c0;
  int32_t o[8];
  bool redo = !fast;
  if (fast) {
    const int64_t hi = (1ll << (fq.w - 1)) - 1, lo = -(1ll << (fq.w - 1));
    bool ovf = false;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t Z = (int64_t)((uint64_t)(int64_t)H[k] << fq.dh) + (int64_t)((uint64_t)(int64_t)L[k] << fq.dl);
      const int64_t v = Z >> fq.t;
      const bool valid = k < nvalid;
      if (PASS1) {
        if (valid) ormag |= (uint64_t)(Z ^ (Z >> 63));
        o[k] = valid ? wrap_bits((uint64_t)v, fq.w) : 0;
      } else {
        if (fq.clamp) ovf |= (v > hi || v < lo) && valid;
        o[k] = valid ? (int32_t)v : 0;
      }
    }
    if (!PASS1 && fq.clamp) redo = __any_sync(__activemask(), ovf);
  }
  if (redo) {
    slow_hl8<PASS1>(H, L, p, out, tmp, row, c0, red);
    return;
  }
  if (PASS1) {
    if (tmp) {
      int4* d = reinterpret_cast<int4*>(tmp + row * out.ld + c0);
      d[0] = make_int4(o[0], o[1], o[2], o[3]);
      d[1] = make_int4(o[4], o[5], o[6], o[7]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t a = (uint32_t)(o[k] < 0 ? -o[k] : o[k]);
      nrm = a > nrm ? a : nrm;
    }
    stv<8>(out, row, c0, o);
  }
}

__device__ __forceinline__ void fold_key(Red& red, uint64_t ormag, bool any) {
  if (ormag) red.key = max(red.key, (long long)(256 + (64 - __clzll((long long)ormag)) + 1));
  else if (any) red.key = max(red.key, 257ll);
}

// r_c = R~ r_f: a warp owns 256 coarse columns (8 per lane: fine columns 2c0 .. 2c0+16)
// and walks coarse rows, keeping the horizontally weighted fine row 2J+2 for the next row.
template <bool PASS1>
__global__ void __launch_bounds__(128, 8) k_restrict2d16(const VIn f, const QDesc q, const VOut out, const int rs) {
  __shared__ Plan sp;
  if (threadIdx.x == 0) {
    build_plan(q, sp);
    if (!PASS1 && q.mode == kQcomp) plan_from_mu(sp, q.meta_out[kMetaMu]);
  }
  __syncthreads();
  const Plan& p = sp;
  const Fast fq = make_fast(p, PASS1);
  const bool fast = fq.ok;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * 256 + lane * 8;
  const int64_t ny = out.ny;
  const int64_t J0 = ((int64_t)blockIdx.y * 4 + warp) * rs;
  const int64_t J1 = J0 + rs < ny ? J0 + rs : ny;
  const bool act = c0 < out.ld;
  int32_t* tmp = (PASS1 && p.use_tmp && !p.guarded) ? reinterpret_cast<int32_t*>(q.tmp) : nullptr;
  Red red = {0, 0, 0};
  uint32_t nrm = 0;
  uint64_t ormag = 0;
  bool any = false;
  // h_k = f[2c] + 2 f[2c+1] + f[2c+2] for c = c0 + k of fine row fr
  auto hrow = [&](int64_t fr, int32_t (&h)[8]) {
    int32_t a[8], b[8];
    ldrow16(f, fr, 2 * c0, a);
    ldrow16(f, fr, 2 * c0 + 8, b);
    int32_t nxt = __shfl_down_sync(0xffffffffu, a[0], 1);
    if (lane == 31) nxt = ld1_16(f, fr, 2 * c0 + 16);
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = a[2 * k] + 2 * a[2 * k + 1] + (k < 3 ? a[2 * k + 2] : b[0]);
#pragma unroll
    for (int k = 0; k < 4; ++k) h[4 + k] = b[2 * k] + 2 * b[2 * k + 1] + (k < 3 ? b[2 * k + 2] : nxt);
  };
  if (!PASS1 && p.narrow) {
    for (int64_t J = J0; J < J1; ++J)
      if (act) narrowv<8>(reinterpret_cast<const int32_t*>(q.tmp), p, out, J, c0, red);
  } else if (J0 < J1) {
    int32_t hp[8];
    hrow(2 * J0, hp);
    for (int64_t J = J0; J < J1; ++J) {
      int32_t hm[8], hn[8];
      hrow(2 * J + 1, hm);
      hrow(2 * J + 2, hn);
      int32_t H[8], L[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) { H[k] = hp[k] + 2 * hm[k] + hn[k]; L[k] = 0; hp[k] = hn[k]; }
      if (act) {
        emit_hl8<PASS1>(H, L, p, fq, fast, out, tmp, J, c0, red, nrm, ormag);
        any = any || (out.nx - c0 > 0);
      }
    }
  }
  if (PASS1) fold_key(red, ormag, any);
  red.nrm = max(red.nrm, (long long)nrm);
  block_commit(red, q.meta_out, q.stats, PASS1);
  if (!PASS1) op_epilogue(q, p);
}

// y' = y - P d (CORR) or P d: a warp owns 256 fine columns (8 per lane: coarse
// columns c0/2 - 1 .. c0/2 + 3) and walks pairs of fine rows (2J, 2J+1), keeping
// the interpolated coarse row J - 1.
template <bool CORR, bool PASS1>
__global__ void __launch_bounds__(128, 8) k_prolong2d16(const VIn d, const VIn y, const QDesc q, const VOut out,
                                                        const int rs) {
  __shared__ Plan sp;
  if (threadIdx.x == 0) {
    build_plan(q, sp);
    if (!PASS1 && q.mode == kQcomp) plan_from_mu(sp, q.meta_out[kMetaMu]);
  }
  __syncthreads();
  const Plan& p = sp;
  const Fast fq = make_fast(p, PASS1);
  const bool fast = fq.ok;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * 256 + lane * 8;
  const int64_t ny = out.ny;                     // fine rows
  const int64_t P0 = ((int64_t)blockIdx.y * 4 + warp) * rs;   // first row pair (fine rows 2P0, 2P0+1)
  const int64_t P1 = P0 + rs;
  const bool act = c0 < out.ld;
  int32_t* tmp = (PASS1 && p.use_tmp && !p.guarded) ? reinterpret_cast<int32_t*>(q.tmp) : nullptr;
  Red red = {0, 0, 0};
  uint32_t nrm = 0;
  uint64_t ormag = 0;
  bool any = false;
  const int64_t C = c0 >> 1;                     // first coarse column of this lane (multiple of 4)
  // g_k: horizontal interpolation of coarse row J at fine columns c0 + k (mantissas at exponent -1)
  auto grow = [&](int64_t J, int32_t (&g)[8]) {
    int32_t dv[5];
    if (J >= 0 && J < d.ny && C < d.nx) {
      const uint2 u = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const int16_t*>(d.m) + J * d.ld + C));
      dv[1] = (int32_t)(u.x << 16) >> 16; dv[2] = (int32_t)u.x >> 16;
      dv[3] = (int32_t)(u.y << 16) >> 16; dv[4] = (int32_t)u.y >> 16;
#pragma unroll
      for (int k = 1; k < 5; ++k)
        if (C + k - 1 >= d.nx) dv[k] = 0;
    } else {
      dv[1] = dv[2] = dv[3] = dv[4] = 0;
    }
    dv[0] = __shfl_up_sync(0xffffffffu, dv[4], 1);
    if (lane == 0) dv[0] = (J >= 0 && J < d.ny) ? ld1_16(d, J, C - 1) : 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) g[k] = (k & 1) ? 2 * dv[(k + 1) / 2] : dv[k / 2] + dv[k / 2 + 1];
  };
  if (!PASS1 && p.narrow) {
    for (int64_t j = 2 * P0; j < 2 * P1 && j < ny; ++j)
      if (act) narrowv<8>(reinterpret_cast<const int32_t*>(q.tmp), p, out, j, c0, red);
  } else if (2 * P0 < ny) {
    int32_t gm[8];
    grow(P0 - 1, gm);
    for (int64_t P = P0; P < P1 && 2 * P < ny; ++P) {
      int32_t gc[8];
      grow(P, gc);
      // fine row 2P: coarse rows P-1, P (weights 1, 1); fine row 2P+1: coarse row P (weight 2)
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int64_t j = 2 * P + half;
        if (j >= ny) break;
        int32_t yv[8];
        if (CORR) ldrow16(y, j, c0, yv);
        int32_t H[8], L[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int32_t pd = half == 0 ? gm[k] + gc[k] : 2 * gc[k];
          H[k] = CORR ? -pd : pd;
          L[k] = CORR ? yv[k] : 0;
        }
        if (act) {
          emit_hl8<PASS1>(H, L, p, fq, fast, out, tmp, j, c0, red, nrm, ormag);
          any = any || (out.nx - c0 > 0);
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) gm[k] = gc[k];
    }
  }
  if (PASS1) fold_key(red, ormag, any);
  red.nrm = max(red.nrm, (long long)nrm);
  block_commit(red, q.meta_out, q.stats, PASS1);
  if (!PASS1) op_epilogue(q, p);
}

}  // namespace bfp
