// bfp_float.cuh -- the float baselines: FP32 and BF16-storage / FP32-arithmetic
// versions of the multigrid ops (damped Jacobi, residual, full weighting,
// interpolation + correction), for comparison with the BFP solver.  They are
// not part of the paper's method.
//
// Arithmetic: FP32, round to nearest, no contraction (explicit __f*_rn), in
// the order stated per op, so the results are reproducible bit for bit by any
// IEEE-754 FP32 evaluation of the same expressions.  BF16 vectors hold the
// upper 16 bits of an FP32 value; loads widen exactly, stores round to
// nearest-even.
//
// The 2D Jacobi / residual kernel follows the BFP five-point kernel: a warp
// owns a 256-column chunk (8 values per lane), rows staged per lane through a
// cp.async ring in shared memory with halo words at the chunk edges.  The
// transfers and all 3D ops are plain one-thread-per-output kernels.
#pragma once

#include <cuda_bf16.h>

#include "bfp_star2d16.cuh"

namespace bfp {

struct FVIn {
  const void* p;
  int64_t ld, nx, ny, nz;   // rows = ny * nz
};
struct FVOut {
  void* p;
  int64_t ld, nx, ny, nz;
};

__device__ __forceinline__ float bf16_to_f32(uint32_t h) { return __uint_as_float(h << 16); }
__device__ __forceinline__ uint32_t f32_to_bf16(float v) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v));
}

template <class S>
__device__ __forceinline__ float fld(const FVIn& v, int64_t row, int64_t col) {
  if (row < 0 || row >= v.ny * v.nz || col < 0 || col >= v.nx) return 0.0f;
  const int64_t o = row * v.ld + col;
  if (sizeof(S) == 4) return __ldg(reinterpret_cast<const float*>(v.p) + o);
  return bf16_to_f32(__ldg(reinterpret_cast<const unsigned short*>(v.p) + o));
}

template <class S>
__device__ __forceinline__ void fst(const FVOut& v, int64_t row, int64_t col, float x) {
  const int64_t o = row * v.ld + col;
  if (sizeof(S) == 4) reinterpret_cast<float*>(v.p)[o] = x;
  else reinterpret_cast<unsigned short*>(v.p)[o] = (unsigned short)f32_to_bf16(x);
}

// One point of a stencil op in the stated order:
//   s = (W + E) + (S + N) [+ (B + T)],  a = c y + nb s,
//   Jacobi: y + om (r - a);  residual: a - r;  Jacobi from 0: om r.
template <int KIND>
__device__ __forceinline__ float fpoint(float y, float w, float e, float s_, float n_, float b_, float t_, bool three,
                                        float r, float c, float nb, float om) {
  if (KIND == kJacobi0) return __fmul_rn(om, r);
  float s = __fadd_rn(__fadd_rn(w, e), __fadd_rn(s_, n_));
  if (three) s = __fadd_rn(s, __fadd_rn(b_, t_));
  const float a = __fadd_rn(__fmul_rn(c, y), __fmul_rn(nb, s));
  if (KIND == kResidual) return __fsub_rn(a, r);
  if (KIND == kApply) return a;
  return __fadd_rn(y, __fmul_rn(om, __fsub_rn(r, a)));
}

// ---------------------------------------------------------------------------
// 2D Jacobi / residual / Jacobi-from-zero, staged rows
// ---------------------------------------------------------------------------

template <class S>
struct FStage {
  static constexpr int kLaneWords = 2 * (int)sizeof(S);          // 8 values per lane
  static constexpr int kRowWords = 8 + 32 * kLaneWords;          // pad, halo, 32 slots, halo, pad
  static constexpr int kStages = sizeof(S) == 4 ? 5 : 6;
  static constexpr int kPerWord = 4 / (int)sizeof(S);
  uint32_t y[kStages][kRowWords];
  uint32_t r[kStages][32 * kLaneWords];
};

template <class S, int KIND>
__global__ void __launch_bounds__(128, 5) k_fstar2d(const FVIn y, const FVIn r, const float c, const float nb,
                                                    const float om, const FVOut out, const int rs) {
  using St = FStage<S>;
  constexpr int LW = St::kLaneWords, NS = St::kStages;
  __shared__ __align__(16) St stg[4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * 256 + lane * 8;
  const int ny = (int)out.ny;
  const int j0 = (int)(((int64_t)blockIdx.y * 4 + warp) * rs);
  const int j1 = j0 + rs < ny ? j0 + rs : ny;
  const bool act = c0 < out.ld;
  constexpr bool kUseY = KIND != kJacobi0;
  St& Sg = stg[warp];
  const int nyin = kUseY ? (int)(y.ny * y.nz) : 1, nrin = (int)(r.ny * r.nz);
  const bool ycol = kUseY && c0 < y.nx && c0 < y.ld, rcol = c0 < r.nx && c0 < r.ld;
  const char* yb = kUseY ? reinterpret_cast<const char*>(y.p) : nullptr;
  const char* rb = reinterpret_cast<const char*>(r.p);
  const int64_t yrow = kUseY ? y.ld * (int64_t)sizeof(S) : 0, rrow = r.ld * (int64_t)sizeof(S);
  // halo words: lane 0 the 4 bytes ending at column c0 - 1, lane 31 those starting at c0 + 8
  const int64_t hcol = lane == 0 ? c0 - St::kPerWord : c0 + 8;
  const bool hok = kUseY && (lane == 0 ? (c0 >= St::kPerWord && c0 - 1 < y.nx) : (lane == 31 && c0 + 8 < y.nx));
  const int hword = lane == 0 ? 3 : St::kRowWords - 4;
  int jy = j0 - 1;
  int64_t oy = kUseY ? (int64_t)jy * yrow + c0 * (int64_t)sizeof(S) : 0;
  int64_t orr = (int64_t)(jy - 1) * rrow + c0 * (int64_t)sizeof(S);
  auto issue = [&](int slot) {
    if (kUseY) {
      const bool in = (unsigned)jy < (unsigned)nyin;
      const bool ok = ycol && in;
#pragma unroll
      for (int h = 0; h < LW / 4; ++h)
        cp16(&Sg.y[slot][4 + LW * lane + 4 * h], yb + (ok ? oy + 16 * h : 0), ok ? 16u : 0u);
      const bool ek = hok && in;
      cp4_if(lane == 0 || lane == 31, &Sg.y[slot][hword],
             yb + (ek ? oy + (hcol - c0) * (int64_t)sizeof(S) : 0), ek ? 4u : 0u);
      oy += yrow;
    }
    {
      const bool ok = rcol && (unsigned)(jy - 1) < (unsigned)nrin;
#pragma unroll
      for (int h = 0; h < LW / 4; ++h)
        cp16(&Sg.r[slot][LW * lane + 4 * h], rb + (ok ? orr + 16 * h : 0), ok ? 16u : 0u);
      orr += rrow;
    }
    ++jy;
    cp_commit();
  };
  // the lane's columns at or beyond nx read as 0
  const int nvalid = (int)(out.nx - c0 < 8 ? (out.nx - c0 < 0 ? 0 : out.nx - c0) : 8);
  auto val = [&](const uint32_t* words, int k) -> float {
    float v;
    if (sizeof(S) == 4) v = __uint_as_float(words[k]);
    else v = bf16_to_f32((k & 1) ? (words[k >> 1] >> 16) : (words[k >> 1] & 0xffffu));
    return k < nvalid ? v : 0.0f;
  };
  auto one = [&](const uint32_t* row, int idx) -> float {   // one value of a staged y row (element index)
    if (sizeof(S) == 4) return __uint_as_float(row[idx]);
    return bf16_to_f32((idx & 1) ? (row[idx >> 1] >> 16) : (row[idx >> 1] & 0xffffu));
  };

  if (j0 < j1) {
#pragma unroll
    for (int s = 0; s < NS - 1; ++s) issue(s);
    int s0 = 0, s1 = 1, s2 = 2, sn = NS - 1;
    for (int j = j0; j < j1; ++j) {
      issue(sn);
      cp_wait<NS - 3>();
      __syncwarp();
      float o[8];
      uint32_t rw[LW];
#pragma unroll
      for (int h = 0; h < LW; ++h) rw[h] = Sg.r[s2][LW * lane + h];
      if (kUseY) {
        uint32_t ym[LW], yc[LW], yp[LW];
#pragma unroll
        for (int h = 0; h < LW; ++h) {
          ym[h] = Sg.y[s0][4 + LW * lane + h];
          yc[h] = Sg.y[s1][4 + LW * lane + h];
          yp[h] = Sg.y[s2][4 + LW * lane + h];
        }
        const int base = 4 * St::kPerWord + 8 * lane;   // element index of column c0 in the row
        const float wv = one(Sg.y[s1], base - 1), ev = one(Sg.y[s1], base + 8);
        float yv[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) yv[k] = val(yc, k);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float wk = k == 0 ? wv : yv[k - 1];
          const float ek = k == 7 ? ev : yv[k + 1];
          o[k] = fpoint<KIND>(yv[k], wk, ek, val(ym, k), val(yp, k), 0.0f, 0.0f, false, val(rw, k), c, nb, om);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = fpoint<KIND>(0.0f, 0, 0, 0, 0, 0, 0, false, val(rw, k), c, nb, om);
      }
      if (act) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (k >= nvalid) o[k] = 0.0f;   // padding columns are written as 0
        char* dst = reinterpret_cast<char*>(out.p) + ((int64_t)j * out.ld + c0) * (int64_t)sizeof(S);
        if (sizeof(S) == 4) {
          reinterpret_cast<float4*>(dst)[0] = make_float4(o[0], o[1], o[2], o[3]);
          reinterpret_cast<float4*>(dst)[1] = make_float4(o[4], o[5], o[6], o[7]);
        } else {
          uint4 u;
          u.x = f32_to_bf16(o[0]) | (f32_to_bf16(o[1]) << 16);
          u.y = f32_to_bf16(o[2]) | (f32_to_bf16(o[3]) << 16);
          u.z = f32_to_bf16(o[4]) | (f32_to_bf16(o[5]) << 16);
          u.w = f32_to_bf16(o[6]) | (f32_to_bf16(o[7]) << 16);
          *reinterpret_cast<uint4*>(dst) = u;
        }
      }
      sn = s0;
      s0 = s1;
      s1 = s2;
      s2 = s2 + 1 == NS ? 0 : s2 + 1;
    }
    cp_wait<0>();
  }
}

// ---------------------------------------------------------------------------
// 3D stencil ops: one thread per point
// ---------------------------------------------------------------------------

template <class S, int KIND>
__global__ void __launch_bounds__(256) k_fstar3d(const FVIn y, const FVIn r, const float c, const float nb,
                                                 const float om, const FVOut out) {
  const int64_t nx = out.nx, ny = out.ny, nz = out.nz, ld = out.ld;
  const int64_t total = ld * ny * nz;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % ld, row = idx / ld, j = row % ny, k = row / ny;
    if (i >= nx) { fst<S>(out, row, i, 0.0f); continue; }
    float v;
    const float rv = fld<S>(r, row, i);
    if (KIND == kJacobi0) {
      v = fpoint<KIND>(0, 0, 0, 0, 0, 0, 0, true, rv, c, nb, om);
    } else {
      auto at = [&](int64_t ii, int64_t jj, int64_t kk) -> float {
        if (jj < 0 || jj >= ny || kk < 0 || kk >= nz) return 0.0f;
        return fld<S>(y, kk * ny + jj, ii);
      };
      v = fpoint<KIND>(at(i, j, k), at(i - 1, j, k), at(i + 1, j, k), at(i, j - 1, k), at(i, j + 1, k),
                       at(i, j, k - 1), at(i, j, k + 1), true, rv, c, nb, om);
    }
    fst<S>(out, row, i, v);
  }
}

// ---------------------------------------------------------------------------
// Transfers (2D and 3D): one thread per output point
// ---------------------------------------------------------------------------

// r_c = 2^-2d * separable full weighting: along x (f0 + 2 f1) + f2, then the
// same along y [and z]; fine index of coarse I is 2I + 1.
template <class S, int ND>
__global__ void __launch_bounds__(256) k_frestrict(const FVIn f, const FVOut out) {
  const int64_t nx = out.nx, ny = out.ny, nz = out.nz, ld = out.ld;
  const int64_t total = ld * ny * nz;
  const float scale = ND == 2 ? 0.25f : 0.0625f;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = idx % ld, row = idx / ld, J = row % ny, K = row / ny;
    if (I >= nx) { fst<S>(out, row, I, 0.0f); continue; }
    auto hx = [&](int64_t fj, int64_t fk) -> float {
      if (fj < 0 || fj >= f.ny || fk < 0 || fk >= f.nz) return 0.0f;
      const int64_t fr = fk * f.ny + fj;
      return __fadd_rn(__fadd_rn(fld<S>(f, fr, 2 * I), __fmul_rn(2.0f, fld<S>(f, fr, 2 * I + 1))),
                       fld<S>(f, fr, 2 * I + 2));
    };
    auto hy = [&](int64_t fk) -> float {
      return __fadd_rn(__fadd_rn(hx(2 * J, fk), __fmul_rn(2.0f, hx(2 * J + 1, fk))), hx(2 * J + 2, fk));
    };
    float acc;
    if (ND == 2) acc = hy(0);
    else acc = __fadd_rn(__fadd_rn(hy(2 * K), __fmul_rn(2.0f, hy(2 * K + 1))), hy(2 * K + 2));
    fst<S>(out, row, I, __fmul_rn(scale, acc));
  }
}

// out = y - P d (CORR) or P d: separable interpolation, x first; on a coarse
// point the value, between two 0.5 a + 0.5 b.  Fine index i is on coarse
// (i - 1) / 2 when odd, between i/2 - 1 and i/2 when even.
template <class S, int ND, bool CORR>
__global__ void __launch_bounds__(256) k_fprolong(const FVIn d, const FVIn y, const FVOut out) {
  const int64_t nx = out.nx, ny = out.ny, nz = out.nz, ld = out.ld;
  const int64_t total = ld * ny * nz;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % ld, row = idx / ld, j = row % ny, k = row / ny;
    if (i >= nx) { fst<S>(out, row, i, 0.0f); continue; }
    auto dv = [&](int64_t I, int64_t J, int64_t K) -> float {
      if (J < 0 || J >= d.ny || K < 0 || K >= d.nz) return 0.0f;
      return fld<S>(d, K * d.ny + J, I);
    };
    auto gx = [&](int64_t J, int64_t K) -> float {
      if (i & 1) return dv((i - 1) >> 1, J, K);
      return __fadd_rn(__fmul_rn(0.5f, dv((i >> 1) - 1, J, K)), __fmul_rn(0.5f, dv(i >> 1, J, K)));
    };
    auto gy = [&](int64_t K) -> float {
      if (j & 1) return gx((j - 1) >> 1, K);
      return __fadd_rn(__fmul_rn(0.5f, gx((j >> 1) - 1, K)), __fmul_rn(0.5f, gx(j >> 1, K)));
    };
    float pd;
    if (ND == 2) pd = gy(0);
    else if (k & 1) pd = gy((k - 1) >> 1);
    else pd = __fadd_rn(__fmul_rn(0.5f, gy((k >> 1) - 1)), __fmul_rn(0.5f, gy(k >> 1)));
    fst<S>(out, row, i, CORR ? __fsub_rn(fld<S>(y, row, i), pd) : pd);
  }
}

}  // namespace bfp
