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
  int32_t is64;   // int64 mantissas (33 <= w <= 62; outputs of k_quant_wide only)
};

template <class T>
__device__ __forceinline__ int64_t ld1(const VIn& v, int64_t row, int64_t col) {
  if (col < 0 || col >= v.nx || row < 0 || row >= v.ny * v.nz) return 0;
  return (int64_t)__ldg(reinterpret_cast<const T*>(v.m) + row * v.ld + col);
}

// V consecutive mantissas (V = 4, 8, or 16 for int16) of one row starting at c0 (c0 % V == 0).
// Entries at columns >= nx, rows outside the vector, or chunks past ld read as
// 0 (zero Dirichlet halo and padding).
template <class T, int V>
__device__ __forceinline__ void ldv(const VIn& v, int64_t row, int64_t c0, int32_t (&o)[V]) {
  if (row < 0 || row >= v.ny * v.nz || c0 >= v.ld || c0 >= v.nx) {
#pragma unroll
    for (int k = 0; k < V; ++k) o[k] = 0;
    return;
  }
  const T* p = reinterpret_cast<const T*>(v.m) + row * v.ld + c0;
  if (sizeof(T) == 2 && V == 16) {   // the second half only inside the row (ld is a multiple of 8)
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(p));
    const uint4 b = c0 + 8 < v.ld ? __ldg(reinterpret_cast<const uint4*>(p) + 1) : make_uint4(0u, 0u, 0u, 0u);
    const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      o[(2 * k) % V] = (int32_t)(int16_t)(w[k] & 0xffffu);
      o[(2 * k + 1) % V] = (int32_t)(int16_t)(w[k] >> 16);
    }
  } else if (sizeof(T) == 2) {
    uint32_t w[V / 2];
    if (V == 8) {
      const uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
      w[0] = u.x; w[1] = u.y;
      if (V == 8) { w[V == 8 ? 2 : 0] = u.z; w[V == 8 ? 3 : 1] = u.w; }
    } else {
      const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
      w[0] = u.x; w[1] = u.y;
    }
#pragma unroll
    for (int k = 0; k < V / 2; ++k) {
      o[2 * k] = (int32_t)(int16_t)(w[k] & 0xffffu);
      o[2 * k + 1] = (int32_t)(int16_t)(w[k] >> 16);
    }
  } else {
    const int4 a = __ldg(reinterpret_cast<const int4*>(p));
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    if (V == 8) {
      const int4 b = __ldg(reinterpret_cast<const int4*>(p) + 1);
      o[V == 8 ? 4 : 0] = b.x; o[V == 8 ? 5 : 1] = b.y; o[V == 8 ? 6 : 2] = b.z; o[V == 8 ? 7 : 3] = b.w;
    }
  }
  if (c0 + V > v.nx) {
#pragma unroll
    for (int k = 0; k < V; ++k)
      if (c0 + k >= v.nx) o[k] = 0;
  }
}

template <class T>
__device__ __forceinline__ void ld8(const VIn& v, int64_t row, int64_t c0, int32_t (&o)[8]) {
  ldv<T, 8>(v, row, c0, o);
}

template <int V>
__device__ __forceinline__ void stv(const VOut& v, int64_t row, int64_t c0, const int32_t (&o)[V]) {
  if constexpr (V == 16) {   // two halves of 8; the second only inside the row (ld is a multiple of 8)
    int32_t lo[8], hi[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) { lo[k] = o[k]; hi[k] = o[(k + 8) % V]; }
    stv<8>(v, row, c0, lo);
    if (c0 + 8 < v.ld) stv<8>(v, row, c0 + 8, hi);
    return;
  }
  if (v.is32) {
    int4* p = reinterpret_cast<int4*>(reinterpret_cast<int32_t*>(v.m) + row * v.ld + c0);
    p[0] = make_int4(o[0], o[1], o[2], o[3]);
    if (V == 8) p[1] = make_int4(o[V == 8 ? 4 : 0], o[V == 8 ? 5 : 1], o[V == 8 ? 6 : 2], o[V == 8 ? 7 : 3]);
  } else {
    uint32_t w[V / 2];
#pragma unroll
    for (int k = 0; k < V / 2; ++k) w[k] = (uint32_t)(uint16_t)o[2 * k] | ((uint32_t)(uint16_t)o[2 * k + 1] << 16);
    int16_t* p = reinterpret_cast<int16_t*>(v.m) + row * v.ld + c0;
    if (V == 8) *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[V == 8 ? 2 : 0], w[V == 8 ? 3 : 1]);
    else *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
  }
}

__device__ __forceinline__ void st8(const VOut& v, int64_t row, int64_t c0, const int32_t (&o)[8]) {
  stv<8>(v, row, c0, o);
}

// 8 mantissas of any storage (int16 / int32 / int64) widened to int64; the zero rules of ldv.
template <class T>
__device__ __forceinline__ void ldw8(const VIn& v, int64_t row, int64_t c0, int64_t (&o)[8]) {
  if constexpr (sizeof(T) != 8) {
    int32_t t[8];
    ldv<T, 8>(v, row, c0, t);
#pragma unroll
    for (int k = 0; k < 8; ++k) o[k] = t[k];
    return;
  } else {
  if (row < 0 || row >= v.ny * v.nz || c0 >= v.ld || c0 >= v.nx) {
#pragma unroll
    for (int k = 0; k < 8; ++k) o[k] = 0;
    return;
  }
  const longlong2* p = reinterpret_cast<const longlong2*>(reinterpret_cast<const long long*>(v.m) + row * v.ld + c0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const longlong2 a = __ldg(p + q);
    o[2 * q] = a.x;
    o[2 * q + 1] = a.y;
  }
  if (c0 + 8 > v.nx) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (c0 + k >= v.nx) o[k] = 0;
  }
  }
}

// 8 int64 mantissas (outputs of 33..62 bits).
__device__ __forceinline__ void stw8(const VOut& v, int64_t row, int64_t c0, const int64_t (&o)[8]) {
  longlong2* p = reinterpret_cast<longlong2*>(reinterpret_cast<long long*>(v.m) + row * v.ld + c0);
#pragma unroll
  for (int q = 0; q < 4; ++q) p[q] = make_longlong2(o[2 * q], o[2 * q + 1]);
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

// axpby (Alg. eaxpby-row):  H = m_alpha x, L = m_beta y (x, y stored as TX, TY)
template <class TX, class TY>
struct OpAxpy {
  VIn x, y;
  int64_t am, bm;
  __device__ __forceinline__ void operator()(int64_t row, int64_t c0, int64_t (&H)[8], int64_t (&L)[8]) const {
    int32_t a[8], b[8];
    ld8<TX>(x, row, c0, a);
    ld8<TY>(y, row, c0, b);
#pragma unroll
    for (int k = 0; k < 8; ++k) { H[k] = am * a[k]; L[k] = bm * b[k]; }
  }
};

// Storage chosen at run time (es = bytes per mantissa: 2, 4 or 8), widened to int64.
__device__ __forceinline__ void ldw8d(const VIn& v, int es, int64_t row, int64_t c0, int64_t (&o)[8]) {
  if (es == 8) ldw8<int64_t>(v, row, c0, o);
  else if (es == 4) ldw8<int32_t>(v, row, c0, o);
  else ldw8<int16_t>(v, row, c0, o);
}
__device__ __forceinline__ int64_t ld1d(const VIn& v, int es, int64_t row, int64_t col) {
  return es == 8 ? ld1<long long>(v, row, col) : (es == 4 ? ld1<int32_t>(v, row, col) : ld1<int16_t>(v, row, col));
}

// Ops on operands of any storage (the paths that take int64 mantissas, 33 <= w <= 62):
//   copy     : H = x                                   (normalise)
//   axpby    : H = m_alpha x, L = m_beta y             (Alg. eaxpby-row)
//   residual : H = c y + n sum_nbrs(y), L = -r         (r_v = A y - r on the star stencil)
struct OpCopyW {
  VIn x;
  int ex;
  __device__ __forceinline__ void operator()(int64_t row, int64_t c0, int64_t (&H)[8], int64_t (&L)[8]) const {
    ldw8d(x, ex, row, c0, H);
#pragma unroll
    for (int k = 0; k < 8; ++k) L[k] = 0;
  }
};

struct OpAxpyW {
  VIn x, y;
  int ex, ey;
  int64_t am, bm;
  __device__ __forceinline__ void operator()(int64_t row, int64_t c0, int64_t (&H)[8], int64_t (&L)[8]) const {
    int64_t a[8], b[8];
    ldw8d(x, ex, row, c0, a);
    ldw8d(y, ey, row, c0, b);
#pragma unroll
    for (int k = 0; k < 8; ++k) { H[k] = am * a[k]; L[k] = bm * b[k]; }
  }
};

template <int NDIM>
struct OpResW {
  VIn y, r;
  int ey, er;
  int64_t c, n;
  __device__ __forceinline__ void operator()(int64_t row, int64_t c0, int64_t (&H)[8], int64_t (&L)[8]) const {
    const int64_t nyy = y.ny, yy = row % nyy;
    int64_t ctr[8], nb[8], b[8];
    ldw8d(y, ey, row, c0, ctr);
    ldw8d(y, ey, yy > 0 ? row - 1 : -1, c0, nb);                 // rows outside the grid read 0
    ldw8d(y, ey, yy + 1 < nyy ? row + 1 : -1, c0, b);
    int64_t ns[8];
    const int64_t wv = ld1d(y, ey, row, c0 - 1), ev = ld1d(y, ey, row, c0 + 8);
#pragma unroll
    for (int k = 0; k < 8; ++k) ns[k] = (((k == 0 ? wv : ctr[k - 1]) + (k == 7 ? ev : ctr[k + 1])) + nb[k]) + b[k];
    if (NDIM == 3) {
      const int64_t zz = row / nyy;
      ldw8d(y, ey, zz > 0 ? row - nyy : -1, c0, nb);
      ldw8d(y, ey, zz + 1 < y.nz ? row + nyy : -1, c0, b);
#pragma unroll
      for (int k = 0; k < 8; ++k) ns[k] += nb[k] + b[k];
    }
    ldw8d(r, er, row, c0, b);
#pragma unroll
    for (int k = 0; k < 8; ++k) { H[k] = c * ctr[k] + n * ns[k]; L[k] = -b[k]; }
  }
};

// Damped Jacobi S y + m_w r with y and r of different storage (progressive widths: the right-hand
// side comes from the finer level's width):  H = sc y + sn sum_nbrs(y), L = m_w r.
template <int NDIM>
struct OpJacD {
  VIn y, r;
  int ey, er;
  int64_t c, n, mw;
  __device__ __forceinline__ void operator()(int64_t row, int64_t c0, int64_t (&H)[8], int64_t (&L)[8]) const {
    const int64_t nyy = y.ny, yy = row % nyy;
    int64_t ctr[8], nb[8], b[8];
    ldw8d(y, ey, row, c0, ctr);
    ldw8d(y, ey, yy > 0 ? row - 1 : -1, c0, nb);
    ldw8d(y, ey, yy + 1 < nyy ? row + 1 : -1, c0, b);
    int64_t ns[8];
    const int64_t wv = ld1d(y, ey, row, c0 - 1), ev = ld1d(y, ey, row, c0 + 8);
#pragma unroll
    for (int k = 0; k < 8; ++k) ns[k] = (((k == 0 ? wv : ctr[k - 1]) + (k == 7 ? ev : ctr[k + 1])) + nb[k]) + b[k];
    if (NDIM == 3) {
      const int64_t zz = row / nyy;
      ldw8d(y, ey, zz > 0 ? row - nyy : -1, c0, nb);
      ldw8d(y, ey, zz + 1 < y.nz ? row + nyy : -1, c0, b);
#pragma unroll
      for (int k = 0; k < 8; ++k) ns[k] += nb[k] + b[k];
    }
    ldw8d(r, er, row, c0, b);
#pragma unroll
    for (int k = 0; k < 8; ++k) { H[k] = c * ctr[k] + n * ns[k]; L[k] = mw * b[k]; }
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
// T: d's storage; TY: y's (int64_t: the storage given at run time by ey).
template <class T, int NDIM, bool CORRECT, class TY = T>
struct OpProlong {
  VIn d, y;
  int ey = 0;
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
      int64_t yv[8];
      if constexpr (sizeof(TY) == 8) ldw8d(y, ey, row, c0, yv);
      else ldw8<TY>(y, row, c0, yv);
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

// Quantises the 8 exact results of one row chunk; hl(k, H, L) yields the two
// exponent groups of element k.  The common case (an int64 combine suffices)
// is unrolled and computes each element on the fly; the rare wide / far-apart
// exponent case stages the groups in local memory and runs one element at a
// time in 128-bit, so that its registers do not add to the unrolled path's.
template <bool PASS1, int V, class HL>
__device__ __forceinline__ void quantvf(const HL& hl, const Plan& p, const Fast& fq, const VOut& out, int32_t* tmp,
                                        int64_t row, int64_t c0, Red& red, bool store = true) {
  int32_t o[V];
  const int64_t nvalid = out.nx - c0;
  int sat = 0;
  if (fq.ok) {
    const int64_t hi = (1ll << (fq.w - 1)) - 1, lo = -(1ll << (fq.w - 1));
#pragma unroll
    for (int k = 0; k < V; ++k) {
      int64_t H, L;
      hl(k, H, L);
      const int64_t Z = (int64_t)((uint64_t)H << fq.dh) + (int64_t)((uint64_t)L << fq.dl);
      const bool valid = k < nvalid;   // padding columns may see a real neighbour: masked
      if (PASS1) {
        if (valid) red.key = max(red.key, (long long)(256 + msb64(Z)));
        o[k] = valid ? wrap_bits((uint64_t)(Z >> fq.t) << fq.tl, fq.w) : 0;
      } else {
        int64_t v = Z >> fq.t;
        if (fq.clamp) {
          const bool c = v > hi || v < lo;
          v = v > hi ? hi : (v < lo ? lo : v);
          sat += (c && valid) ? 1 : 0;
        }
        o[k] = valid ? (int32_t)v : 0;
      }
    }
  } else {
    // general path (far-apart exponent groups, 128-bit combine, left-shifted
    // outputs): staged in local memory, one element at a time
    int64_t Hs[V], Ls[V];
    int32_t os[V];
#pragma unroll
    for (int k = 0; k < V; ++k) hl(k, Hs[k], Ls[k]);
#pragma unroll 1
    for (int k = 0; k < V; ++k) {
      os[k] = 0;
      if (k < nvalid) {
        if (p.wide) {
          const i128 Z = combine<i128>(Hs[k], Ls[k], p);
          if (PASS1) {
            red.key = max(red.key, (long long)mu_key<i128>(Z, Hs[k], Ls[k], p));
            os[k] = window<i128>(Z, p);
          } else {
            os[k] = finish<i128>(Z, Hs[k], Ls[k], p, sat);
          }
        } else {
          const int64_t Z = combine<int64_t>(Hs[k], Ls[k], p);
          if (PASS1) {
            red.key = max(red.key, (long long)mu_key<int64_t>(Z, Hs[k], Ls[k], p));
            os[k] = window<int64_t>(Z, p);
          } else {
            os[k] = finish<int64_t>(Z, Hs[k], Ls[k], p, sat);
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < V; ++k) o[k] = os[k];
  }
  if (PASS1) {
    if (tmp && store) {
      int4* q = reinterpret_cast<int4*>(tmp + row * out.ld + c0);
#pragma unroll
      for (int g = 0; g < V / 4; ++g)   // (past column c0 + 8 only inside the row: ld is a multiple of 8)
        if (g < 2 || c0 + 8 < out.ld) q[g] = make_int4(o[4 * g], o[4 * g + 1], o[4 * g + 2], o[4 * g + 3]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < V; ++k) red.nrm = max(red.nrm, (long long)(o[k] < 0 ? -(long long)o[k] : (long long)o[k]));
    red.sat += sat;
    if (store) stv<V>(out, row, c0, o);
  }
}

template <bool PASS1>
__device__ __forceinline__ void quant8(const int64_t (&H)[8], const int64_t (&L)[8], const Plan& p,
                                       const VOut& out, int32_t* tmp, int64_t row, int64_t c0, Red& red,
                                       bool store = true) {
  const Fast fq = make_fast(p, PASS1);
  quantvf<PASS1, 8>([&](int k, int64_t& h, int64_t& l) { h = H[k]; l = L[k]; }, p, fq, out, tmp, row, c0, red, store);
}

// Alg. qcomp success branch for one row chunk: decr(w_tmp - w_out, tmp >> (lambda_out - lambda_tmp)).
template <int V>
__device__ __forceinline__ void narrowv(const int32_t* tmp, const Plan& p, const VOut& out, int64_t row, int64_t c0,
                                        Red& red) {
  const int4* src = reinterpret_cast<const int4*>(tmp + row * out.ld + c0);
  int32_t t[V];
#pragma unroll
  for (int g = 0; g < V / 4; ++g) {   // (past column c0 + 8 only inside the row: ld is a multiple of 8)
    const int4 a = (g < 2 || c0 + 8 < out.ld) ? src[g] : make_int4(0, 0, 0, 0);
    t[4 * g] = a.x; t[4 * g + 1] = a.y; t[4 * g + 2] = a.z; t[4 * g + 3] = a.w;
  }
  const int s = (int)(p.e_out - p.e_tmp);
  int32_t o[V];
#pragma unroll
  for (int k = 0; k < V; ++k) {
    o[k] = (c0 + k < out.nx) ? (t[k] >> s) : 0;
    red.nrm = max(red.nrm, (long long)(o[k] < 0 ? -(long long)o[k] : (long long)o[k]));
  }
  stv<V>(out, row, c0, o);
}

__device__ __forceinline__ void narrow8(const int32_t* tmp, const Plan& p, const VOut& out, int64_t row, int64_t c0,
                                        Red& red) {
  narrowv<8>(tmp, p, out, row, c0, red);
}

// Final bookkeeping of a quantised op: e_out and the counters (block (0, 0, 0) only).
// first: this CTA is the op's first block (block (0, 0, 0); in a batched launch (0, 0) of its instance).
__device__ __forceinline__ void op_epilogue(const QDesc& q, const Plan& p,
                                            bool first = (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0)) {
  if (first && threadIdx.x == 0) {
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

// Resident blocks per SM an op asks the compiler for (Op::kMinBlocks; default 1).
template <class Op, class = void>
struct OpMinBlocks { static constexpr int value = 1; };
template <class Op>
struct OpMinBlocks<Op, std::void_t<decltype(Op::kMinBlocks)>> { static constexpr int value = Op::kMinBlocks; };

template <class Op, bool PASS1>
__global__ void __launch_bounds__(256, OpMinBlocks<Op>::value) k_quant(const Op op, const QDesc q, const VOut out) {
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
      narrow8(reinterpret_cast<const int32_t*>(q.tmp), p, out, row, c0, red);
      continue;
    }
    int64_t H[8], L[8];
    op(row, c0, H, L);
    quant8<PASS1>(H, L, p, out, tmp, row, c0, red);
  }
  block_commit(red, q.meta_out, q.stats, PASS1);
  if (!PASS1) op_epilogue(q, p);
}

// Quantisation of 8 exact results into int64 mantissas (33 <= w_out <= 62): the per-element
// general path of quantvf (no w_tmp window: qcomp recomputes in its second pass).
template <bool PASS1>
__device__ __forceinline__ void quant8_wide(const int64_t (&H)[8], const int64_t (&L)[8], const Plan& p,
                                            const VOut& out, int64_t row, int64_t c0, Red& red) {
  int64_t o[8];
  int sat = 0;
  const int64_t nvalid = out.nx - c0;
#pragma unroll 1
  for (int k = 0; k < 8; ++k) {
    o[k] = 0;
    if (k >= nvalid) continue;
    if (p.wide) {
      const i128 Z = combine<i128>(H[k], L[k], p);
      if (PASS1) red.key = max(red.key, (long long)mu_key<i128>(Z, H[k], L[k], p));
      else o[k] = finish<i128, int64_t>(Z, H[k], L[k], p, sat);
    } else {
      const int64_t Z = combine<int64_t>(H[k], L[k], p);
      if (PASS1) red.key = max(red.key, (long long)mu_key<int64_t>(Z, H[k], L[k], p));
      else o[k] = finish<int64_t, int64_t>(Z, H[k], L[k], p, sat);
    }
  }
  if (!PASS1) {
#pragma unroll
    for (int k = 0; k < 8; ++k) red.nrm = max(red.nrm, (long long)(o[k] < 0 ? -o[k] : o[k]));
    red.sat += sat;
    stw8(out, row, c0, o);
  }
}

template <class Op, bool PASS1>
__global__ void __launch_bounds__(256) k_quant_wide(const Op op, const QDesc q, const VOut out) {
  __shared__ Plan sp;
  if (threadIdx.x == 0) {
    build_plan(q, sp);
    if (!PASS1 && q.mode == kQcomp) plan_from_mu(sp, q.meta_out[kMetaMu]);
  }
  __syncthreads();
  const Plan p = sp;
  const int64_t nvec = out.ld >> 3;
  const int64_t total = out.ny * out.nz * nvec;
  Red red = {0, 0, 0};
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / nvec;
    const int64_t c0 = (idx - row * nvec) << 3;
    int64_t H[8], L[8];
    op(row, c0, H, L);
    quant8_wide<PASS1>(H, L, p, out, row, c0, red);
  }
  block_commit(red, q.meta_out, q.stats, PASS1);
  if (!PASS1) op_epilogue(q, p);
}

}  // namespace bfp
