// bfp_star2d16.cuh -- five- and seven-point stencil ops on int16 mantissas
// (w <= 16), the finest-level hot path of the V-cycle, and the 2D five-point ops
// on int32 mantissas of at most 30 bits (the same kernel with half the values
// per lane).
//
// A warp owns a 256-column chunk of a strip of rows of one plane: each lane 8
// consecutive mantissas (16 bytes per row and input; int32: 128 columns, 4 per
// lane).  Rows are staged through
// a per-lane ring of NS slots in shared memory with cp.async (16-byte copies,
// zero-filled outside the grid), issued NS - 3 rows ahead of the three-row
// window the lane reads back (rows j-1, j, j+1 of y and row j of r; in 3D also
// row j of the planes below and above, which the CTAs of those planes, resident
// at the same time, bring into L2).
// Every lane reads only what it copied itself, so a per-thread wait on the
// copy groups is the only synchronisation; the west / east neighbours at the
// chunk edges come from shuffles, lanes 0 and 31 copying the one extra
// mantissa pair they need.
//
// Fast path (the exact integer Z fits in int64 and the output exponent is at
// or above Z's): Z = cy*y + cn*(W+E+S+N) + cr*r with the App. B exponent
// alignment folded into three 32-bit coefficients; the result is one funnel
// shift.  When |Z| < 2^(31 + t) (from the op's msb bounds) the nnqcomp
// saturation test runs on the 32-bit results: the OR of v + 2^(w-1) over a
// row has no bit at or above w iff every v is in X_w; otherwise it is one
// unsigned range test on Z per element.
// A warp that sees a value outside X_w (or a plan outside the fast regime)
// recomputes that row through the general quantiser, kept out of line.  qcomp
// pass 1 takes the bit width of the OR of |Z| (the max msb) and stores the
// w_tmp window.  max |m| is kept on the packed results with 16x2 max / min.
#pragma once

#include <type_traits>

#include "bfp_host.h"

namespace bfp {

constexpr int kS16Cols = 256;   // columns per warp chunk (32 lanes x 8)
constexpr int kStages = 6;      // ring slots per lane (2D): the 3-row window + 3 rows in flight
constexpr int kStages3 = 5;     // 3D (four rows per stage): the window + 2 rows in flight

// A lane's mantissas of one row: 4 words (8 int16 or 4 int32) or 8 words (16 int16)
struct Pk8 {
  uint32_t w[8];
};

__device__ __forceinline__ int32_t pk_get(const Pk8& p, int k) {
  const uint32_t word = p.w[k >> 1];
  return (k & 1) ? ((int32_t)word >> 16) : (int32_t)(int16_t)(word & 0xffffu);
}

// c + the int16 mantissa k of p (sign-extended), one dp2a (FMA pipe): unpack and add in one instruction
__device__ __forceinline__ int32_t add_half(const Pk8& p, int k, int32_t c) {
  int32_t d;
  asm("dp2a.lo.s32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(p.w[k >> 1]), "r"((k & 1) ? 0x0100 : 0x0001), "r"(c));
  return d;
}

// mantissa k of a lane's 16 bytes: int16 (k < 8) or int32 (k < 4) storage
template <bool W32>
__device__ __forceinline__ int32_t vget(const Pk8& p, int k) {
  return W32 ? (int32_t)p.w[k & 3] : pk_get(p, k);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Asynchronous copies global -> shared; src_bytes 0 fills zeros (the source
// address is then not read; callers still pass an address inside the buffer).
__device__ __forceinline__ void cp16(void* dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
// predicated 4-byte copy (no branch: only lanes with p set issue it)
__device__ __forceinline__ void cp4_if(bool p, void* dst, const void* src, uint32_t src_bytes) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.b32 q, %3, 0;\n @q cp.async.ca.shared.global [%0], [%1], 4, %2;\n}\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(src_bytes), "r"((int)p)
      : "memory");
}

// Z = a*b + c with a 64-bit accumulator (one mad.wide)
__device__ __forceinline__ int64_t madw(int32_t a, int32_t b, int64_t c) {
  int64_t d;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}
__device__ __forceinline__ int64_t mulw(int32_t a, int32_t b) {
  int64_t d;
  asm("mul.wide.s32 %0, %1, %2;" : "=l"(d) : "r"(a), "r"(b));
  return d;
}
// the same with 32-bit shared-state-space destination addresses
__device__ __forceinline__ void cp16u(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp4u_if(bool p, uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.b32 q, %3, 0;\n @q cp.async.ca.shared.global [%0], [%1], 4, %2;\n}\n" ::"r"(dst),
      "l"(src), "r"(src_bytes), "r"((int)p)
      : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ uint32_t max_s16x2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("max.s16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ uint32_t min_s16x2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("min.s16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

// Per-point coefficients of the variable-coefficient operator (2D, int16 faces W, E, S, N and
// smoother weights q, in the output's layout; s: the left shift of y into the Jacobi H group).
// A'y = k_W (y - y_W) + k_E (y - y_E) + k_S (y - y_S) + k_N (y - y_N), exactly c y - sum k_f y_f.
struct VarRow {
  VIn k[4];
  VIn q;
  int32_t s;
};

// Inputs of one lane's NV outputs, for the out-of-line general path.
template <int NV>
struct RowIn {
  int32_t y[NV], ym[NV], yp[NV], r[NV], zm[NV], zp[NV];
  int32_t wv, ev;
};

// The general path for one lane's NV outputs of row j of plane kz (mantissas of type T): reloads its
// inputs from global memory (zero outside the grid) and quantises through quantvf.
template <bool PASS1, int KIND, int ND, bool VAR, class T = int16_t, int NV = 8>
__device__ __noinline__ void slow_row8(const VIn& y, const VIn& r, const Plan& p, const Fast& fq, const VOut& out,
                                       int32_t* tmp, int64_t j, int64_t kz, int64_t c0, Red& red, int32_t c,
                                       int32_t nb, int32_t mw, const VarRow& va) {
  RowIn<NV> in;
  int32_t kf[4][8], qv[8];
  if constexpr (VAR) {
    const int64_t row = kz * out.ny + j;
#pragma unroll
    for (int f = 0; f < 4; ++f) ldv<int16_t, 8>(va.k[f], row, c0, kf[f]);
    ldv<int16_t, 8>(va.q, row, c0, qv);
  }
  const int64_t ny = out.ny, row = kz * ny + j;
  if (KIND != kJacobi0) {
    ldv<T, NV>(y, row, c0, in.y);
    ldv<T, NV>(y, j > 0 ? row - 1 : -1, c0, in.ym);
    ldv<T, NV>(y, j + 1 < ny ? row + 1 : -1, c0, in.yp);
    ldv<T, NV>(y, ND == 3 && kz > 0 ? row - ny : -1, c0, in.zm);
    ldv<T, NV>(y, ND == 3 && kz + 1 < out.nz ? row + ny : -1, c0, in.zp);
    in.wv = (int32_t)ld1<T>(y, row, c0 - 1);
    in.ev = (int32_t)ld1<T>(y, row, c0 + NV);
  }
  if (KIND != kApply) ldv<T, NV>(r, row, c0, in.r);
  auto hl = [&](int k, int64_t& H, int64_t& L) {
    if constexpr (VAR) {
      if (KIND == kJacobi0) {
        H = (int64_t)qv[k] * in.r[k];
        L = 0;
        return;
      }
      const int64_t yk = in.y[k];
      const int64_t ay = (int64_t)kf[0][k] * (yk - (k == 0 ? in.wv : in.y[k - 1])) +
                         (int64_t)kf[1][k] * (yk - (k == NV - 1 ? in.ev : in.y[k + 1])) +
                         (int64_t)kf[2][k] * (yk - in.ym[k]) + (int64_t)kf[3][k] * (yk - in.yp[k]);
      if (KIND == kApply) { H = ay; L = 0; }
      else if (KIND == kResidual) { H = ay; L = -(int64_t)in.r[k]; }
      else { H = (int64_t)((uint64_t)yk << va.s) - (int64_t)qv[k] * ay; L = (int64_t)qv[k] * in.r[k]; }
      return;
    }
    if (KIND == kJacobi0) {
      H = (int64_t)mw * (int64_t)in.r[k];
      L = 0;
      return;
    }
    const int64_t wk = k == 0 ? in.wv : in.y[k - 1];
    const int64_t ek = k == NV - 1 ? in.ev : in.y[k + 1];
    const int64_t ns = wk + ek + in.ym[k] + in.yp[k] + in.zm[k] + in.zp[k];
    H = (int64_t)c * (int64_t)in.y[k] + (int64_t)nb * ns;
    L = KIND == kApply ? 0 : (KIND == kResidual ? -(int64_t)in.r[k] : (int64_t)mw * (int64_t)in.r[k]);
  };
  quantvf<PASS1, NV>(hl, p, fq, out, tmp, row, c0, red);
}

// Per-warp staging ring.  A y row is 136 words: 3 pad words, the west halo
// pair (columns c-2, c-1 of the chunk start c), 32 lane slots of 4 words, the
// east halo pair (columns c+256, c+257), 3 pad words; lane slots stay 16-byte
// aligned, and every west / east neighbour is one int16 load from the row.
// In 3D a stage also holds row j of the planes below (zm) and above (zp).
// LW: words per lane and row (4, or 8 for 16 int16 mantissas per lane); a y row is 8 + 32 LW words.
constexpr int kRowWords = 136;
template <int ND, int LW = 4>
struct __align__(16) Stage16 {
  // wide lanes: the window + 2 rows in flight (four warps' stages stay within 48 KB of static shared memory)
  static constexpr int N = LW == 8 ? kStages3 : kStages;
  uint32_t y[N][8 + 32 * LW];
  uint4 r[N][8 * LW];
};
template <>
struct __align__(16) Stage16<3, 4> {
  static constexpr int N = kStages3;
  uint32_t y[N][kRowWords];
  uint4 r[N][32];
  uint4 zm[N][32], zp[N][32];
};

// Parameters of one star-stencil op (one instance of a batched launch).
struct Star16P {
  VIn y, r;
  int32_t c, nb, mw;
  QDesc q;
  VOut out;
  int32_t rs;
  VarRow va;
};


// grid: (column chunks of 32 lanes x 16 bytes, strips of 4 * rs rows, planes); B: a batched launch of 2D
// ops, grid z the instance, parameters Pb[z].  T: the mantissa storage of y, r and the output, int16
// (8 per lane, 256-column chunks) or int32 (4 per lane, 128-column chunks; 2D constant-coefficient ops
// with mantissas of at most 30 bits, so the neighbour sum is exact in int32)
template <int KIND, bool PASS1, int ND, bool VAR = false, bool B = false, class T = int16_t>
__global__ void __launch_bounds__(128, (ND == 3 || VAR) ? 5 : (sizeof(T) == 2 ? 4 : 7))
    k_star16(const __grid_constant__ Star16P P1, const Star16P* __restrict__ Pb) {
  static_assert(!B || ND == 2, "batched launches are 2D");
  constexpr bool W32 = sizeof(T) == 4;
  static_assert(!W32 || (ND == 2 && !VAR), "int32 mantissas: 2D constant-coefficient ops");
  // 2D constant-coefficient int16 ops: 16 mantissas per lane (32 bytes per row and input), so that a
  // row's fixed per-lane work (copies, waits, loads, the range vote, stores) covers twice the points
  constexpr bool WIDE = !W32 && ND == 2 && !VAR;
  constexpr int NV = W32 ? 4 : (WIDE ? 16 : 8);   // mantissas per lane and row
  constexpr int LW = WIDE ? 8 : 4;                // words per lane and row
  constexpr int kRowW = 8 + 32 * LW;              // words of a staged y row
  constexpr int kCols = 32 * NV;                  // columns per warp chunk
  constexpr int64_t kEs = sizeof(T);              // bytes per mantissa
  pdl_wait();
  const Star16P& P = B ? Pb[blockIdx.z] : P1;
  const VIn& y = P.y;
  const VIn& r = P.r;
  const int32_t c = P.c, nb = P.nb, mw = P.mw;
  const QDesc& q = P.q;
  const VOut& out = P.out;
  const int rs = P.rs;
  const VarRow& va = P.va;
  constexpr int NS = Stage16<ND, LW>::N;
  __shared__ Plan sp;
  __shared__ Stage16<ND, LW> stg[4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * kCols + lane * NV;
  const int ny = (int)out.ny;
  const int kz = ND == 3 ? (int)blockIdx.z : 0;
  const int64_t rowoff = (int64_t)kz * ny;        // global row of the plane's row 0
  const int j0 = (int)(((int64_t)blockIdx.y * 4 + warp) * rs);
  const int j1 = j0 + rs < ny ? j0 + rs : ny;
  const bool act = c0 < out.ld;
  constexpr bool kUseY = KIND != kJacobi0, kUseR = KIND != kApply;
  // staging: stage s holds y row j0 - 1 + s and r (zm, zp) row j0 - 2 + s
  Stage16<ND, LW>& S = stg[warp];
  const int nyin = kUseY ? ny : 1, nrin = kUseR ? ny : 1;
  const bool ycol = kUseY && c0 < y.nx && c0 < y.ld, rcol = kUseR && c0 < r.nx && c0 < r.ld;
  // the second 16 bytes of a wide lane (columns c0 + 8 ..)
  const bool ycol1 = WIDE && kUseY && c0 + 8 < y.nx && c0 + 8 < y.ld;
  const bool rcol1 = WIDE && kUseR && c0 + 8 < r.nx && c0 + 8 < r.ld;
  const T* ybase = kUseY ? reinterpret_cast<const T*>(y.m) : nullptr;
  const T* rbase = kUseR ? reinterpret_cast<const T*>(r.m) : nullptr;
  // halo words: lane 0 copies (c0-2, c0-1) (int16; int32: c0-1) into word 3, lane 31 (c0+NV, c0+NV+1)
  // (int32: c0+4) into word kRowW - 4
  const int64_t ecol = lane == 0 ? c0 - (W32 ? 1 : 2) : c0 + NV;
  const bool eok = kUseY && (lane == 0 ? (c0 >= (W32 ? 1 : 2) && c0 - 1 < y.nx) : (lane == 31 && c0 + NV < y.nx));
  const int eword = lane == 0 ? 3 : kRowW - 4;
  // the next stage to issue: y row jy at byte offset oy, r row jy - 1 at byte offset orr (rows
  // outside the grid and lanes past the row are zero-filled)
  int jy = j0 - 1;
  int64_t oy = kUseY ? ((rowoff + jy) * y.ld + c0) * kEs : 0, orr = kUseR ? ((rowoff + jy - 1) * r.ld + c0) * kEs : 0;
  const int64_t ystride = kUseY ? y.ld * kEs : 0, rstride = kUseR ? r.ld * kEs : 0;
  // 3D: row jy - 1 of planes kz - 1 and kz + 1 (offsets used only when that plane exists)
  const bool zmok = ND == 3 && kUseY && kz > 0, zpok = ND == 3 && kUseY && kz + 1 < (int)out.nz;
  int64_t ozm = ND == 3 && kUseY ? ((rowoff - ny + jy - 1) * y.ld + c0) * 2 : 0;
  const int64_t zdelta = 2 * (int64_t)ny * y.ld * 2;
  const int64_t edelta = (ecol - c0) * kEs;
  const bool edge_lane = lane == 0 || lane == 31;
  const uint32_t ybytes = 16u, rbytes = 16u;
  const char* yb = reinterpret_cast<const char*>(ybase);
  const char* rb = reinterpret_cast<const char*>(rbase);
  constexpr uint32_t kYRowBytes = kRowW * 4, kRRowBytes = 32 * LW * 4;
  const uint32_t ydst = smem_u32(&S.y[0][4 + LW * lane]), edst = smem_u32(&S.y[0][eword]);
  const uint32_t rdst = smem_u32(&S.r[0][(LW / 4) * lane]);
  uint32_t zmdst = 0, zpdst = 0;
  if constexpr (ND == 3) {
    zmdst = smem_u32(&S.zm[0][lane]);
    zpdst = smem_u32(&S.zp[0][lane]);
  }
  // INT: an interior strip (every row it stages inside the grid, every lane's 8 columns inside
  // the row), so the copies need no bounds; with_r: stage s >= 2 (the r rows of stages 0, 1 are
  // never read)
  auto issue = [&](int slot, auto inttag, bool with_r) {
    constexpr bool INT = decltype(inttag)::value;
    if (kUseY) {
      const bool in = INT || (unsigned)jy < (unsigned)nyin;
      const bool ok = INT || (in && ycol);
      cp16u(ydst + (uint32_t)slot * kYRowBytes, yb + (ok ? oy : 0), ok ? ybytes : 0u);
      if constexpr (WIDE) {
        const bool ok1 = INT || (in && ycol1);
        cp16u(ydst + (uint32_t)slot * kYRowBytes + 16u, yb + (ok1 ? oy + 16 : 0), ok1 ? 16u : 0u);
      }
      const bool ek = eok && in;
      cp4u_if(edge_lane, edst + (uint32_t)slot * kYRowBytes, yb + (ek ? oy + edelta : 0), ek ? 4u : 0u);
      oy += ystride;
    }
    if (kUseR) {
      if (with_r) {
        const bool rin = (unsigned)(jy - 1) < (unsigned)nrin;
        const bool ok = INT || (rcol && rin);
        cp16u(rdst + (uint32_t)slot * kRRowBytes, rb + (ok ? orr : 0), ok ? rbytes : 0u);
        if constexpr (WIDE) {
          const bool ok1 = INT || (rcol1 && rin);
          cp16u(rdst + (uint32_t)slot * kRRowBytes + 16u, rb + (ok1 ? orr + 16 : 0), ok1 ? 16u : 0u);
        }
      }
      orr += rstride;
    }
    if (ND == 3 && kUseY) {
      const bool in = ycol && (unsigned)(jy - 1) < (unsigned)nyin;
      const bool okm = in && zmok, okp = in && zpok;
      cp16u(zmdst + (uint32_t)slot * kRRowBytes, yb + (okm ? ozm : 0), okm ? 16u : 0u);
      cp16u(zpdst + (uint32_t)slot * kRRowBytes, yb + (okp ? ozm + zdelta : 0), okp ? 16u : 0u);
      ozm += ystride;
    }
    ++jy;
    cp_commit();
  };
  // a lane's mantissas of the staged y / r row in `slot` (one or two 16-byte halves)
  auto rdy = [&](int slot) {
    Pk8 v;
    const uint4 a = *reinterpret_cast<const uint4*>(&S.y[slot][4 + LW * lane]);
    v.w[0] = a.x; v.w[1] = a.y; v.w[2] = a.z; v.w[3] = a.w;
    if constexpr (LW == 8) {
      const uint4 b = *reinterpret_cast<const uint4*>(&S.y[slot][8 + LW * lane]);
      v.w[LW - 4] = b.x; v.w[LW - 3] = b.y; v.w[LW - 2] = b.z; v.w[LW - 1] = b.w;
    }
    return v;
  };
  auto rdr = [&](int slot) {
    Pk8 v;
    const uint4 a = S.r[slot][(LW / 4) * lane];
    v.w[0] = a.x; v.w[1] = a.y; v.w[2] = a.z; v.w[3] = a.w;
    if constexpr (LW == 8) {
      const uint4 b = S.r[slot][(LW / 4) * lane + 1];
      v.w[LW - 4] = b.x; v.w[LW - 3] = b.y; v.w[LW - 2] = b.z; v.w[LW - 1] = b.w;
    }
    return v;
  };
  auto rd = [&](const uint4& u) {
    Pk8 v;
    v.w[0] = u.x; v.w[1] = u.y; v.w[2] = u.z; v.w[3] = u.w;
    return v;
  };

  // the first stages of the ring do not depend on the plan: issued before it is built (nnqcomp and
  // qcomp's first pass; qcomp's second pass may only narrow the window and loads nothing then)
  const int nst = j1 - j0 + 2;   // stages with a row that is read: y rows j0 - 1 .. j1
  const bool early = (PASS1 || q.mode == kNnqcomp) && j0 < j1;
  auto prologue = [&](auto inttag) {
#pragma unroll
    for (int s = 0; s < NS - 1; ++s) {
      if (s < nst) issue(s, inttag, s >= 2);
      else cp_commit();   // the ring's later stages are committed empty: the group count stays the same
    }
  };
  const bool with_mu = !PASS1 && q.mode == kQcomp;
  const MetaIn mi = threadIdx.x == 0 ? load_meta(q, with_mu) : MetaIn{0, 0, 0, 0, 0};
  if (early) prologue(std::false_type{});
  if (threadIdx.x == 0) build_plan_m(q, mi, with_mu, sp);
  __syncthreads();
  const Plan& p = sp;
  const Fast fq = make_fast(p, PASS1);
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
  const int32_t cy32 = (int32_t)cy, cn32 = (int32_t)cn, cr32 = (int32_t)cr;
  const uint32_t t = (uint32_t)fq.t;
  // |Z| <= 2^zb from the msb bounds of the two groups
  const int zb = q.two ? max(q.hbits + fq.dh, q.lbits + fq.dl) : q.hbits + fq.dh;
  // fast: Z exact in int64 (the plan's fast regime); fold: the group shifts folded into 32-bit
  // coefficients and t < 32, so Z is three mad.wide and the result one funnel shift (else
  // Z = (H << dh) + (L << dl) from the plain coefficients and the result Z >> t)
  const bool fast = fq.ok;
  const bool fold = !VAR && cy == (int32_t)cy && cn == (int32_t)cn && cr == (int32_t)cr && fq.t < 32;
  const uint32_t dh = (uint32_t)fq.dh, dl = (uint32_t)fq.dl;
  // saturation test on the 32-bit results when Z >> t is exact in int32, else on Z
  const bool v32 = zb - (int)fq.t <= 30;
  const int64_t zmin = (int64_t)((uint64_t)(-(1ll << (fq.w - 1))) << (t & 63));   // used only when t < 32
  const uint64_t zrange = (uint64_t)(((uint64_t)1 << ((fq.w - 1 + t) & 63)) * 2 - 1);
  const int sh = fq.w < 32 ? 32 - fq.w : 0;    // decr to fq.w bits (pass 1 window; wider windows are not kept)
  const uint32_t tl = (uint32_t)fq.tl;          // pass 1: the window's left shift (window below Ez)
  const uint32_t half = 1u << ((fq.w - 1) & 31);   // v in X_w iff v + 2^(w-1) in [0, 2^w)
  const int nvalid = (int)(out.nx - c0 < NV ? (out.nx - c0 < 0 ? 0 : out.nx - c0) : NV);
  const bool partial = nvalid < NV;

  uint32_t vmax = 0, vmin = 0;                  // packed 16x2 extremes of the results (int16)
  int32_t imax = 0, imin = 0;                   // extremes of the results (int32)
  uint32_t redo_rows = 0;
  uint64_t ormag = 0;
  if (!PASS1 && p.narrow) {
    for (int j = j0; j < j1; ++j)
      if (act) narrowv<NV>(reinterpret_cast<const int32_t*>(q.tmp), p, out, rowoff + j, c0, red);
  } else if (j0 < j1) {
    // the row walk, instantiated for both saturation tests (a uniform choice per CTA)
    auto walk = [&](auto v32tag, auto foldtag, auto inttag) {
      constexpr bool V32 = decltype(v32tag)::value, FOLD = decltype(foldtag)::value;
      constexpr bool INT = decltype(inttag)::value;
      if (!early) prologue(inttag);   // stage s = y row j0 - 1 + s
      // ring slots of stages i, i + 1, i + 2 and i + NS - 1 (= i - 1 mod NS)
      int s0 = 0, s1 = 1, s2 = 2, sn = NS - 1;
      for (int j = j0; j < j1; ++j) {
        const int i = j - j0;
        if (i + NS - 1 < nst) issue(sn, inttag, true);   // stage i + NS - 1, into the slot of row j - 2
        else cp_commit();
        [[maybe_unused]] int32_t kf[4][8], qv[8];   // this row's coefficients, loaded while the ring fills
        if constexpr (VAR) {
          if (KIND != kJacobi0) {
#pragma unroll
            for (int f = 0; f < 4; ++f) ldv<int16_t, 8>(va.k[f], rowoff + j, c0, kf[f]);
          }
          if (KIND == kJacobi || KIND == kJacobi0) ldv<int16_t, 8>(va.q, rowoff + j, c0, qv);
        }
        cp_wait<NS - 3>();                        // stages <= i + 2 have landed (own copies)
        __syncwarp();                             // ... and the other lanes' (neighbours, halo)
        Pk8 ym, yc, yp, rc, zm, zp;
        int32_t yv[NV], wv = 0, ev = 0;
        if (kUseY) {
          ym = rdy(s0);
          yc = rdy(s1);
          yp = rdy(s2);
  #pragma unroll
          for (int k = 0; k < NV; ++k) yv[k] = vget<W32>(yc, k);
          if (!INT && partial) {   // padding columns may hold anything: the east neighbour of the last column is 0
#pragma unroll
            for (int k = 0; k < NV; ++k)
              if (k >= nvalid) yv[k] = 0;
          }
          if constexpr (W32) {
            const int32_t* roww = reinterpret_cast<const int32_t*>(&S.y[s1][0]);
            wv = roww[3 + 4 * lane];              // column c0 - 1
            ev = roww[8 + 4 * lane];              // column c0 + 4
          } else {
            const int16_t* row = reinterpret_cast<const int16_t*>(&S.y[s1][0]);
            wv = row[7 + NV * lane];              // column c0 - 1
            ev = row[8 + NV * (lane + 1)];        // column c0 + NV
          }
          if constexpr (ND == 3) {
            zm = rd(S.zm[s2][lane]);
            zp = rd(S.zp[s2][lane]);
          }
        }
        if (kUseR) rc = rdr(s2);
        sn = s0;
        s0 = s1;
        s1 = s2;
        s2 = s2 + 1 == NS ? 0 : s2 + 1;
        if (INT || act) {
          bool redo = !fast;
          int32_t o[NV];
          bool ovf = false;
          if (fast) {
  #pragma unroll
            for (int k = 0; k < NV; ++k) {
              int64_t Z;
              if constexpr (VAR) {
                if (KIND == kJacobi0) {
                  Z = (int64_t)((uint64_t)mulw(qv[k], vget<W32>(rc, k)) << dh);
                } else {
                  const int32_t yk = yv[k];
                  int64_t ay = mulw(kf[0][k], yk - (k == 0 ? wv : yv[k - 1]));
                  ay = madw(kf[1][k], yk - (k == NV - 1 ? ev : yv[k + 1]), ay);
                  ay = madw(kf[2][k], yk - vget<W32>(ym, k), ay);
                  ay = madw(kf[3][k], yk - vget<W32>(yp, k), ay);
                  int64_t H = ay, L = 0;
                  if (KIND == kResidual) L = -(int64_t)vget<W32>(rc, k);
                  if (KIND == kJacobi) {
                    H = (int64_t)((uint64_t)(int64_t)yk << va.s) - (int64_t)qv[k] * ay;
                    L = mulw(qv[k], vget<W32>(rc, k));
                  }
                  Z = (int64_t)((uint64_t)H << dh) + (int64_t)((uint64_t)L << dl);
                }
              } else if (KIND == kJacobi0) {
                Z = FOLD ? mulw(cr32, vget<W32>(rc, k)) : (int64_t)((uint64_t)mulw(mw, vget<W32>(rc, k)) << dh);
              } else {
                const int32_t wk = k == 0 ? wv : yv[k - 1];
                const int32_t ek = k == NV - 1 ? ev : yv[k + 1];
                int32_t ns;
                if constexpr (W32) {
                  ns = wk + ek + vget<W32>(ym, k) + vget<W32>(yp, k);
                } else {
                  ns = add_half(yp, k, add_half(ym, k, wk + ek));
                  if (ND == 3) ns = add_half(zp, k, add_half(zm, k, ns));
                }
                if (FOLD) {
                  Z = madw(cn32, ns, mulw(cy32, yv[k]));
                  if (KIND != kApply) Z = madw(cr32, vget<W32>(rc, k), Z);
                } else {
                  const int64_t H = madw(nb, ns, mulw(c, yv[k]));
                  const int64_t L = KIND == kApply ? 0 : (KIND == kResidual ? -(int64_t)vget<W32>(rc, k)
                                                                              : mulw(mw, vget<W32>(rc, k)));
                  Z = (int64_t)((uint64_t)H << dh) + (int64_t)((uint64_t)L << dl);
                }
              }
              const int32_t v = FOLD ? (int32_t)__funnelshift_r((uint32_t)(uint64_t)Z, (uint32_t)((uint64_t)Z >> 32), t)
                                   : (int32_t)(Z >> t);
              if (PASS1) {
                if (INT || k < nvalid) ormag |= (uint64_t)(Z ^ (Z >> 63));
                o[k] = (int32_t)(((uint32_t)v << tl) << sh) >> sh;
              } else {
                o[k] = v;
                if (!V32 && fq.clamp) ovf |= ((uint64_t)Z - (uint64_t)zmin > zrange) && (INT || k < nvalid);
              }
            }
            if (!INT && partial) {
  #pragma unroll
              for (int k = 0; k < NV; ++k)
                if (k >= nvalid) o[k] = 0;
            }
            if (!PASS1 && fq.clamp) {
              if (V32) {
                uint32_t acc = 0;
  #pragma unroll
                for (int k = 0; k < NV; ++k) acc |= (uint32_t)o[k] + half;
                redo = (acc >> fq.w) != 0u;
              } else {
                redo = ovf;
              }
            }
          }
          if (!PASS1 && fq.clamp && fast) redo = __any_sync(__activemask(), redo);
          if (redo) {
            redo_rows |= 1u << i;                 // recomputed after the loop
          } else if (PASS1) {
            if (tmp) {
              int4* d = reinterpret_cast<int4*>(tmp + (rowoff + j) * out.ld + c0);
#pragma unroll
              for (int g = 0; g < NV / 4; ++g)   // (a wide lane's second half only inside the row)
                if (g < 2 || c0 + 8 < out.ld) d[g] = make_int4(o[4 * g], o[4 * g + 1], o[4 * g + 2], o[4 * g + 3]);
            }
          } else if constexpr (W32) {
            imax = max(imax, max(max(o[0], o[1]), max(o[2], o[3])));
            imin = min(imin, min(min(o[0], o[1]), min(o[2], o[3])));
            *reinterpret_cast<int4*>(reinterpret_cast<int32_t*>(out.m) + (rowoff + j) * out.ld + c0) =
                make_int4(o[0], o[1], o[2], o[3]);
          } else {
            uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<int16_t*>(out.m) + (rowoff + j) * out.ld + c0);
#pragma unroll
            for (int g = 0; g < NV / 8; ++g) {
              uint4 u;
              u.x = __byte_perm((uint32_t)o[8 * g], (uint32_t)o[8 * g + 1], 0x5410);
              u.y = __byte_perm((uint32_t)o[8 * g + 2], (uint32_t)o[8 * g + 3], 0x5410);
              u.z = __byte_perm((uint32_t)o[8 * g + 4], (uint32_t)o[8 * g + 5], 0x5410);
              u.w = __byte_perm((uint32_t)o[8 * g + 6], (uint32_t)o[8 * g + 7], 0x5410);
              vmax = max_s16x2(vmax, max_s16x2(max_s16x2(u.x, u.y), max_s16x2(u.z, u.w)));
              vmin = min_s16x2(vmin, min_s16x2(min_s16x2(u.x, u.y), min_s16x2(u.z, u.w)));
              if (g == 0 || c0 + 8 < out.ld) dst[g] = u;   // a wide lane's second half only inside the row
            }
          }
        }
      }
      cp_wait<0>();
    };
    // interior strip: y rows j0 - 1 .. j1 inside the plane, the chunk's columns inside the row
    const bool xfull = (int64_t)blockIdx.x * kCols + kCols <= out.nx;
    const bool interior = xfull && (!kUseY || (j0 >= 1 && j1 < ny));
    const std::false_type no;
    if constexpr (VAR) {   // per-point coefficients: no folded constants
      if (v32 && interior) walk(std::true_type{}, no, std::true_type{});
      else if (v32) walk(std::true_type{}, no, no);
      else walk(no, no, no);
    } else if (fold && v32 && interior) walk(std::true_type{}, std::true_type{}, std::true_type{});
    else if (fold) {
      if (v32) walk(std::true_type{}, std::true_type{}, no);
      else walk(std::false_type{}, std::true_type{}, no);
    } else {
      if (v32) walk(std::true_type{}, std::false_type{}, no);
      else walk(std::false_type{}, std::false_type{}, no);
    }
    // rows a warp sent to the general path (warp-uniform mask; rs <= 32)
    for (uint32_t m = redo_rows; m != 0u; m &= m - 1u) {
      const int j = j0 + __ffs(m) - 1;
      if (act) slow_row8<PASS1, KIND, ND, VAR, T, NV>(y, r, p, fq, out, tmp, j, kz, c0, red, c, nb, mw, va);
    }
  }
  if (!PASS1) {
    if constexpr (W32) {
      red.nrm = max(red.nrm, max((long long)imax, -(long long)imin));
    } else {
      const int32_t mx = max((int32_t)vmax >> 16, (int32_t)(int16_t)(vmax & 0xffffu));
      const int32_t mn = min((int32_t)vmin >> 16, (int32_t)(int16_t)(vmin & 0xffffu));
      red.nrm = max(red.nrm, (long long)max(mx, -mn));
    }
  }
  if (PASS1 && ormag) red.key = max(red.key, (long long)(256 + (64 - __clzll((long long)ormag)) + 1));
  if (PASS1 && fast && j0 < j1 && act && ormag == 0 && nvalid > 0) red.key = max(red.key, 257ll);   // all-zero chunk: msb 1
  pdl_trigger();
  block_commit(red, q.meta_out, q.stats, PASS1);
  if (!PASS1) op_epilogue(q, p, blockIdx.x == 0 && blockIdx.y == 0 && (B || blockIdx.z == 0));
}

}  // namespace bfp
