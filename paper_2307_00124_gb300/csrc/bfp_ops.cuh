// bfp_ops.cuh -- views, exact per-element computations ("comp-func" of
// Alg. qcomp) and the generic quantised row kernel shared by all BFP ops.
#pragma once

#include <type_traits>

#include "bfp_device.cuh"

namespace bfp {

// Read-only view of one BFP vector's mantissas.
struct VIn {
  const void* m;
  int64_t ld, nx, ny, nz;   // rows = ny * nz
};

// Write view of an output vector.
struct VOut {
  void* m;
  int64_t ld, nx, ny, nz;
  int32_t is32;
};

template <class T>
__device__ __forceinline__ int64_t ld1(const VIn& v, int64_t row, int64_t col) {
  if (col < 0 || col >= v.nx || row < 0 || row >= v.ny * v.nz) return 0;
  return (int64_t)__ldg(reinterpret_cast<const T*>(v.m) + row * v.ld + col);
}

// 8 consecutive mantissas of one row starting at c0 (c0 % 8 == 0).  Entries
// at columns >= nx, rows outside the vector, or vectors past ld read as 0
// (zero Dirichlet halo and padding).
template <class T>
__device__ __forceinline__ void ld8(const VIn& v, int64_t row, int64_t c0, int32_t (&o)[8]) {
  if (row < 0 || row >= v.ny * v.nz || c0 >= v.ld || c0 >= v.nx) {
#pragma unroll
    for (int k = 0; k < 8; ++k) o[k] = 0;
    return;
  }
  const T* p = reinterpret_cast<const T*>(v.m) + row * v.ld + c0;
  if (sizeof(T) == 2) {
    uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      o[2 * k] = (int32_t)(int16_t)(w[k] & 0xffffu);
      o[2 * k + 1] = (int32_t)(int16_t)(w[k] >> 16);
    }
  } else {
    int4 a = __ldg(reinterpret_cast<const int4*>(p));
    int4 b = __ldg(reinterpret_cast<const int4*>(p) + 1);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
  }
  if (c0 + 8 > v.nx) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (c0 + k >= v.nx) o[k] = 0;
  }
}

__device__ __forceinline__ void st8(const VOut& v, int64_t row, int64_t c0, const int32_t (&o)[8]) {
  if (v.is32) {
    int4* p = reinterpret_cast<int4*>(reinterpret_cast<int32_t*>(v.m) + row * v.ld + c0);
    p[0] = make_int4(o[0], o[1], o[2], o[3]);
    p[1] = make_int4(o[4], o[5], o[6], o[7]);
  } else {
    uint4 u;
    u.x = (uint32_t)(uint16_t)o[0] | ((uint32_t)(uint16_t)o[1] << 16);
    u.y = (uint32_t)(uint16_t)o[2] | ((uint32_t)(uint16_t)o[3] << 16);
    u.z = (uint32_t)(uint16_t)o[4] | ((uint32_t)(uint16_t)o[5] << 16);
    u.w = (uint32_t)(uint16_t)o[6] | ((uint32_t)(uint16_t)o[7] << 16);
    *reinterpret_cast<uint4*>(reinterpret_cast<int16_t*>(v.m) + row * v.ld + c0) = u;
  }
}

// ---------------------------------------------------------------------------
// Exact per-element computations.  Each fills H[k], L[k] (the two exponent
// groups of z*) for the 8 outputs at (row, c0 .. c0+7).
// ---------------------------------------------------------------------------

// x (normalise):  H = x
template <class T>
struct OpCopy {
  VIn x;
  __device__ __forceinline__ void operator()(int64_t row, int64_t c0, int64_t (&H)[8], int64_t (&L)[8]) const {
    int32_t a[8];
    ld8<T>(x, row, c0, a);
#pragma unroll
    for (int k = 0; k < 8; ++k) { H[k] = a[k]; L[k] = 0; }
  }
};

// axpby (Alg. eaxpby-row):  H = m_alpha x, L = m_beta y
template <class T>
struct OpAxpy {
  VIn x, y;
  int64_t am, bm;
  __device__ __forceinline__ void operator()(int64_t row, int64_t c0, int64_t (&H)[8], int64_t (&L)[8]) const {
    int32_t a[8], b[8];
    ld8<T>(x, row, c0, a);
    ld8<T>(y, row, c0, b);
#pragma unroll
    for (int k = 0; k < 8; ++k) { H[k] = am * a[k]; L[k] = bm * b[k]; }
  }
};

enum StarKind : int32_t { kApply = 0, kResidual = 1, kJacobi = 2, kJacobi0 = 3 };

// Star stencil ops (Alg. espmv-row / egemv-row on the 2*ndim+1 point stencil).
//   apply    : H = c x + n sum_nbrs(x)                 (z = A x)
//   residual : H = c y + n sum_nbrs(y), L = -r          (rv = A y - r)
//   jacobi   : H = sc y + sn sum_nbrs(y), L = m_w r     (S y + omega r, S = I - omega A)
//   jacobi0  : H = m_w r                                (omega r, zero initial guess)
template <class T, int KIND, int NDIM>
struct OpStar {
  VIn y, r;
  int64_t c, n, mw;
  __device__ __forceinline__ void operator()(int64_t row, int64_t c0, int64_t (&H)[8], int64_t (&L)[8]) const {
    typedef typename std::conditional<sizeof(T) == 2, int32_t, int64_t>::type S;
    if (KIND == kJacobi0) {
      int32_t b[8];
      ld8<T>(r, row, c0, b);
#pragma unroll
      for (int k = 0; k < 8; ++k) { H[k] = mw * b[k]; L[k] = 0; }
      return;
    }
    const int64_t nyy = y.ny;
    const int64_t yy = row % nyy;
    int32_t ctr[8], up[8], dn[8];
    ld8<T>(y, row, c0, ctr);
    if (yy > 0) ld8<T>(y, row - 1, c0, dn); else {
#pragma unroll
      for (int k = 0; k < 8; ++k) dn[k] = 0;
    }
    if (yy + 1 < nyy) ld8<T>(y, row + 1, c0, up); else {
#pragma unroll
      for (int k = 0; k < 8; ++k) up[k] = 0;
    }
    S ns[8];
    const int64_t wv = ld1<T>(y, row, c0 - 1), ev = ld1<T>(y, row, c0 + 8);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      S wk = k == 0 ? (S)wv : (S)ctr[k - 1];
      S ek = k == 7 ? (S)ev : (S)ctr[k + 1];
      ns[k] = ((wk + ek) + (S)dn[k]) + (S)up[k];
    }
    if (NDIM == 3) {
      const int64_t zz = row / nyy;
      int32_t bk[8], fr[8];
      if (zz > 0) ld8<T>(y, row - nyy, c0, bk); else {
#pragma unroll
        for (int k = 0; k < 8; ++k) bk[k] = 0;
      }
      if (zz + 1 < y.nz) ld8<T>(y, row + nyy, c0, fr); else {
#pragma unroll
        for (int k = 0; k < 8; ++k) fr[k] = 0;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) ns[k] += (S)bk[k] + (S)fr[k];
    }
    if (KIND == kApply) {
#pragma unroll
      for (int k = 0; k < 8; ++k) { H[k] = c * ctr[k] + n * (int64_t)ns[k]; L[k] = 0; }
    } else {
      int32_t b[8];
      ld8<T>(r, row, c0, b);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        H[k] = c * ctr[k] + n * (int64_t)ns[k];
        L[k] = KIND == kResidual ? -(int64_t)b[k] : mw * b[k];
      }
    }
  }
};

// Full-weighting restriction R~ (Alg. v-cycle restriction line):
// coarse node I gathers fine nodes 2I+1+delta with weights prod(2 - |delta|).
template <class T, int NDIM>
struct OpRestrict {
  VIn f;   // fine vector; coarse shape comes from the output view
  int64_t cny;
  __device__ __forceinline__ void hsum(int64_t frow, int64_t c0, int64_t (&h)[8]) const {
    // h[k] = f[2c+0] + 2 f[2c+1] + f[2c+2] for c = c0 + k
    int32_t a[8], b[8];
    const int64_t f0 = 2 * c0;
    ld8<T>(f, frow, f0, a);
    ld8<T>(f, frow, f0 + 8, b);
    const int64_t last = ld1<T>(f, frow, f0 + 16);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int64_t e2 = (2 * k + 2 < 8) ? a[2 * k + 2] : b[0];
      h[k] = (int64_t)a[2 * k] + 2 * (int64_t)a[2 * k + 1] + e2;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int64_t e2 = (2 * k + 2 < 8) ? b[2 * k + 2] : last;
      h[4 + k] = (int64_t)b[2 * k] + 2 * (int64_t)b[2 * k + 1] + e2;
    }
  }
  __device__ __forceinline__ void operator()(int64_t row, int64_t c0, int64_t (&H)[8], int64_t (&L)[8]) const {
    const int64_t J = row % cny, K = row / cny;
#pragma unroll
    for (int k = 0; k < 8; ++k) { H[k] = 0; L[k] = 0; }
    const int zr = NDIM == 3 ? 1 : 0;
    for (int dz = -zr; dz <= zr; ++dz) {
      for (int dy = -1; dy <= 1; ++dy) {
        const int64_t fy = 2 * J + 1 + dy;
        const int64_t fz = NDIM == 3 ? 2 * K + 1 + dz : 0;
        const int64_t wgt = (2 - (dy < 0 ? -dy : dy)) * (NDIM == 3 ? (2 - (dz < 0 ? -dz : dz)) : 1);
        int64_t h[8];
        hsum(fy + f.ny * fz, c0, h);
#pragma unroll
        for (int k = 0; k < 8; ++k) H[k] += wgt * h[k];
      }
    }
  }
};

// Interpolation P d (bilinear / trilinear), optionally with the correction
// y - P d (Alg. v-cycle correction line):  H = -P_m d (or +P_m d), L = y.
template <class T, int NDIM, bool CORRECT>
struct OpProlong {
  VIn d, y;
  __device__ __forceinline__ void hinterp(int64_t crow, int64_t c0, int64_t (&g)[8]) const {
    // fine column i: odd -> 2 d[(i-1)/2]; even -> d[i/2 - 1] + d[i/2]
    const int64_t C = c0 >> 1;   // first coarse column (multiple of 4)
    int64_t dv[5];
    dv[0] = ld1<T>(d, crow, C - 1);
#pragma unroll
    for (int k = 0; k < 4; ++k) dv[k + 1] = ld1<T>(d, crow, C + k);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      // fine col c0+k; even k -> d[C + k/2 - 1] + d[C + k/2]; odd k -> 2 d[C + (k-1)/2]
      if ((k & 1) == 0) g[k] = dv[k / 2] + dv[k / 2 + 1];
      else g[k] = 2 * dv[(k - 1) / 2 + 1];
    }
  }
  __device__ __forceinline__ void operator()(int64_t row, int64_t c0, int64_t (&H)[8], int64_t (&L)[8]) const {
    const int64_t fny = y.ny;   // fine rows per plane (y view carries the fine shape)
    const int64_t j = row % fny, kz = row / fny;
    int64_t acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0;
    // contributing coarse rows in y (and z): odd j -> J=(j-1)/2 weight 2; even -> j/2-1, j/2 weight 1
    int64_t Jy[2], wy[2];
    int ny_ = 0;
    if (j & 1) { Jy[0] = (j - 1) / 2; wy[0] = 2; ny_ = 1; }
    else { Jy[0] = j / 2 - 1; wy[0] = 1; Jy[1] = j / 2; wy[1] = 1; ny_ = 2; }
    int64_t Jz[2] = {0, 0}, wz[2] = {1, 1};
    int nz_ = 1;
    if (NDIM == 3) {
      if (kz & 1) { Jz[0] = (kz - 1) / 2; wz[0] = 2; nz_ = 1; }
      else { Jz[0] = kz / 2 - 1; wz[0] = 1; Jz[1] = kz / 2; wz[1] = 1; nz_ = 2; }
    }
    for (int a = 0; a < nz_; ++a) {
      for (int b = 0; b < ny_; ++b) {
        if (Jy[b] < 0 || Jy[b] >= d.ny) continue;
        if (NDIM == 3 && (Jz[a] < 0 || Jz[a] >= d.nz)) continue;
        int64_t g[8];
        hinterp(Jy[b] + d.ny * Jz[a], c0, g);
        const int64_t wgt = wy[b] * wz[a];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += wgt * g[k];
      }
    }
    if (CORRECT) {
      int32_t yv[8];
      ld8<T>(y, row, c0, yv);
#pragma unroll
      for (int k = 0; k < 8; ++k) { H[k] = -acc[k]; L[k] = yv[k]; }
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) { H[k] = acc[k]; L[k] = 0; }
    }
  }
};

// ---------------------------------------------------------------------------
// Generic quantised row kernel: each thread owns 8 consecutive outputs of a row.
//   PASS1 : qcomp first loop (mu* atomic max, optional w_tmp window store)
//   !PASS1: nnqcomp single pass, or qcomp second pass (narrow the window or
//           recompute, decided once from mu*)
// ---------------------------------------------------------------------------

template <class Acc, class Op, bool PASS1>
__device__ __forceinline__ void row_elems(const Op& op, const Plan& p, const VOut& out, int32_t* tmp,
                                          int64_t row, int64_t c0, Red& red) {
  int64_t H[8], L[8];
  op(row, c0, H, L);
  int32_t o[8];
  const int64_t nvalid = out.nx - c0;
  if (PASS1) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      Acc Z = combine<Acc>(H[k], L[k], p);
      if (k < nvalid) red.key = max(red.key, (long long)mu_key<Acc>(Z, H[k], L[k], p));
      o[k] = (k < nvalid) ? window<Acc>(Z, p) : 0;
    }
    if (tmp) {
      int4* q = reinterpret_cast<int4*>(tmp + row * out.ld + c0);
      q[0] = make_int4(o[0], o[1], o[2], o[3]);
      q[1] = make_int4(o[4], o[5], o[6], o[7]);
    }
  } else {
    int sat = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      // padding columns (k >= nvalid) may see a real neighbour through the stencil: skip them
      if (k < nvalid) {
        Acc Z = combine<Acc>(H[k], L[k], p);
        o[k] = finish<Acc>(Z, H[k], L[k], p, sat);
      } else {
        o[k] = 0;
      }
      long long a = o[k] < 0 ? -(long long)o[k] : (long long)o[k];
      red.nrm = max(red.nrm, a);
    }
    red.sat += sat;
    st8(out, row, c0, o);
  }
}

template <class Op, bool PASS1>
__global__ void __launch_bounds__(256) k_quant(const Op op, const QDesc q, const VOut out) {
  __shared__ Plan sp;
  if (threadIdx.x == 0) {
    build_plan(q, sp);
    if (!PASS1 && q.mode == kQcomp) plan_from_mu(sp, q.meta_out[kMetaMu]);
  }
  __syncthreads();
  const Plan p = sp;
  const int64_t nvec = out.ld >> 3;
  const int64_t rows = out.ny * out.nz;
  const int64_t total = rows * nvec;
  Red red = {0, 0, 0};
  int32_t* tmp = (PASS1 && p.use_tmp && !p.guarded) ? reinterpret_cast<int32_t*>(q.tmp) : nullptr;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / nvec;
    const int64_t c0 = (idx - row * nvec) << 3;
    if (!PASS1 && p.narrow) {
      // Alg. qcomp success branch: decr(w_tmp - w_out, tmp >> (lambda_out - lambda_tmp))
      const int4* src = reinterpret_cast<const int4*>(reinterpret_cast<const int32_t*>(q.tmp) + row * out.ld + c0);
      int4 a = src[0], b = src[1];
      const int32_t t[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
      const int s = (int)(p.e_out - p.e_tmp);
      int32_t o[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        o[k] = (c0 + k < out.nx) ? (t[k] >> s) : 0;
        long long av = o[k] < 0 ? -(long long)o[k] : (long long)o[k];
        red.nrm = max(red.nrm, av);
      }
      st8(out, row, c0, o);
      continue;
    }
    if (p.wide) row_elems<i128, Op, PASS1>(op, p, out, tmp, row, c0, red);
    else row_elems<int64_t, Op, PASS1>(op, p, out, tmp, row, c0, red);
  }
  block_commit(red, q.meta_out, q.stats, PASS1);
  if (!PASS1 && blockIdx.x == 0 && threadIdx.x == 0) {
    q.meta_out[0] = p.e_out;
    if (q.stats) {
      atomicAdd((unsigned long long*)&q.stats[0], 1ull);
      if (q.mode == kQcomp) {
        if (p.overflow || p.underflow) atomicAdd((unsigned long long*)&q.stats[1], 1ull);
        if (p.overflow) atomicAdd((unsigned long long*)&q.stats[2], 1ull);
        if (p.underflow) atomicAdd((unsigned long long*)&q.stats[3], 1ull);
      }
    }
  }
}

}  // namespace bfp
