// bfp_transfer2d.cuh -- grid transfers on int16 mantissas (2D and 3D) and on
// int32 mantissas (2D): full-weighting restriction (Alg. v-cycle restriction
// line) and bilinear interpolation with or without the correction y - P d
// (Alg. v-cycle correction line, Alg. fmg interpolation line).
//
// Same structure as bfp_star2d16.cuh: a warp owns a 256-column chunk (int32:
// 128) of a strip of output rows, input rows are staged per warp through a cp.async
// ring in shared memory (with halo words for the one neighbour mantissa a
// chunk needs from the next / previous chunk), the exact groups H (the
// transfer stencil) and L (the correction's y) are combined as
// Z = kh*H + kl*L with the App. B exponent alignment folded into kh, kl, and
// rows a warp cannot finish on the register path are recomputed after the
// walk through the general quantiser.
#pragma once

#include <type_traits>

#include "bfp_star2d16.cuh"

namespace bfp {

__device__ __forceinline__ void unpack8(const uint4 u, int32_t (&o)[8]) {
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    o[2 * k] = (int32_t)(int16_t)(w[k] & 0xffffu);
    o[2 * k + 1] = (int32_t)w[k] >> 16;
  }
}

__device__ __forceinline__ int32_t ld1_16(const VIn& v, int64_t row, int64_t col) {
  if (row < 0 || row >= v.ny * v.nz || col < 0 || col >= v.nx) return 0;
  return (int32_t)__ldg(reinterpret_cast<const int16_t*>(v.m) + row * v.ld + col);
}
template <class T>
__device__ __forceinline__ int32_t ld1_t(const VIn& v, int64_t row, int64_t col) {
  if (row < 0 || row >= v.ny * v.nz || col < 0 || col >= v.nx) return 0;
  return (int32_t)__ldg(reinterpret_cast<const T*>(v.m) + row * v.ld + col);
}

__device__ __forceinline__ void cp8(void* dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}

// General-path fallback for one chunk (kept out of line).
template <bool PASS1>
__device__ __noinline__ void slow_hl8(const int32_t (&H)[8], const int32_t (&L)[8], const Plan& p, const VOut& out,
                                      int32_t* tmp, int64_t row, int64_t c0, Red& red) {
  int64_t H64[8], L64[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) { H64[k] = H[k]; L64[k] = L[k]; }
  quant8<PASS1>(H64, L64, p, out, tmp, row, c0, red);
}

// The same for NV outputs (NV = 4: a lane of the int32 kernels).
template <bool PASS1, int NV>
__device__ __noinline__ void slow_hlv(const int32_t (&H)[NV], const int32_t (&L)[NV], const Plan& p, const VOut& out,
                                      int32_t* tmp, int64_t row, int64_t c0, Red& red) {
  const Fast fq = make_fast(p, PASS1);
  quantvf<PASS1, NV>([&](int k, int64_t& h, int64_t& l) { h = H[k]; l = L[k]; }, p, fq, out, tmp, row, c0, red);
}

// Uniform per-CTA constants of the register path: Z = kh H + kl L, v = Z >> t.
struct EmitC {
  bool fast;          // register path usable
  bool fold;          // Z = kh H + kl L with 32-bit kh, kl (else (H << dh) + (L << dl))
  uint32_t dh, dl;
  bool v32;           // |Z| < 2^(31 + t): saturation tested on the 32-bit results
  int32_t kh, kl;
  uint32_t t;
  uint32_t tl;        // pass 1: left shift of the window (window below the exact exponent)
  int w, sh;          // result width, 32 - w (pass 1 window decr)
  uint32_t half;      // 2^(w-1)
  int64_t zmin;
  uint64_t zrange;
};

__device__ __forceinline__ EmitC make_emit(const Fast& fq, const QDesc& q, int32_t hsign, bool pass1) {
  EmitC e;
  const bool dh_ok = fq.dh <= 30, dl_ok = fq.dl <= 30;
  e.kh = dh_ok ? hsign * (int32_t)(1u << (fq.dh & 31)) : 0;
  e.kl = dl_ok ? (int32_t)(1u << (fq.dl & 31)) : 0;
  e.fast = fq.ok && fq.w <= 32;
  e.fold = dh_ok && dl_ok && fq.t < 32;
  e.dh = (uint32_t)fq.dh;
  e.dl = (uint32_t)fq.dl;
  e.kh = e.fold ? e.kh : hsign;   // unfolded: H carries its sign, Z = (hsign H << dh) + (L << dl)
  e.t = (uint32_t)fq.t;
  e.tl = (uint32_t)fq.tl;
  const int zb = q.two ? max(q.hbits + fq.dh, q.lbits + fq.dl) : q.hbits + fq.dh;
  e.v32 = zb - fq.t <= 30;
  e.w = fq.w;
  e.sh = 32 - fq.w;
  e.half = 1u << ((fq.w - 1) & 31);
  e.zmin = (int64_t)((uint64_t)(-(1ll << (fq.w - 1))) << (fq.t & 63));
  e.zrange = (uint64_t)(((uint64_t)1 << ((fq.w - 1 + fq.t) & 63)) * 2 - 1);
  (void)pass1;
  return e;
}

// One lane's NV (8, or 4 for int32 inputs) outputs on the register path; returns true when the warp must
// recompute the row on the general path (nnqcomp saturation, or no fast path).
template <bool PASS1, bool V32, bool FOLD, int NV = 8>
__device__ __forceinline__ bool emit8(const EmitC& e, const Fast& fq, const int32_t (&H)[NV], const int32_t (&L)[NV],
                                      bool two, int nvalid, bool partial, const VOut& out, int32_t* tmp, int64_t row,
                                      int64_t c0, uint64_t& ormag, uint32_t& vmax, uint32_t& vmin) {
  int32_t o[NV];
  bool ovf = false;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    int64_t Z;
    if (FOLD) {
      Z = two ? madw(e.kl, L[k], mulw(e.kh, H[k])) : mulw(e.kh, H[k]);
    } else {
      Z = (int64_t)((uint64_t)(int64_t)(e.kh * H[k]) << e.dh);
      if (two) Z += (int64_t)((uint64_t)(int64_t)L[k] << e.dl);
    }
    const int32_t v = FOLD ? (int32_t)__funnelshift_r((uint32_t)(uint64_t)Z, (uint32_t)((uint64_t)Z >> 32), e.t)
                           : (int32_t)(Z >> e.t);
    if (PASS1) {
      if (k < nvalid) ormag |= (uint64_t)(Z ^ (Z >> 63));
      o[k] = (int32_t)(((uint32_t)v << e.tl) << e.sh) >> e.sh;
    } else {
      o[k] = v;
      if (!V32 && fq.clamp) ovf |= ((uint64_t)Z - (uint64_t)e.zmin > e.zrange) && (k < nvalid);
    }
  }
  if (partial) {
#pragma unroll
    for (int k = 0; k < NV; ++k)
      if (k >= nvalid) o[k] = 0;
  }
  bool redo = false;
  if (!PASS1 && fq.clamp) {
    if (V32) {
      uint32_t acc = 0;
#pragma unroll
      for (int k = 0; k < NV; ++k) acc |= (uint32_t)o[k] + e.half;
      redo = (acc >> e.w) != 0u;
    } else {
      redo = ovf;
    }
    redo = __any_sync(__activemask(), redo);
  }
  if (redo) return true;
  constexpr int H8 = NV > 4 ? 4 : 0;   // index base of the second group of four (NV = 8)
  if (PASS1) {
    if (tmp) {
      int4* d = reinterpret_cast<int4*>(tmp + row * out.ld + c0);
      d[0] = make_int4(o[0], o[1], o[2], o[3]);
      if (NV == 8) d[1] = make_int4(o[H8], o[H8 + 1], o[H8 + 2], o[H8 + 3]);
    }
  } else if (out.is32) {
    int4* d = reinterpret_cast<int4*>(reinterpret_cast<int32_t*>(out.m) + row * out.ld + c0);
    d[0] = make_int4(o[0], o[1], o[2], o[3]);
    if (NV == 8) d[1] = make_int4(o[H8], o[H8 + 1], o[H8 + 2], o[H8 + 3]);
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const uint32_t a = (uint32_t)(o[k] < 0 ? -o[k] : o[k]);
      m = a > m ? a : m;
    }
    vmax = max(vmax, m);   // (int32 outputs: vmax holds max |v| directly, vmin unused)
  } else {
    uint4 u;
    u.x = __byte_perm((uint32_t)o[0], (uint32_t)o[1], 0x5410);
    u.y = __byte_perm((uint32_t)o[2], (uint32_t)o[3], 0x5410);
    u.z = NV == 8 ? __byte_perm((uint32_t)o[H8], (uint32_t)o[H8 + 1], 0x5410) : u.x;
    u.w = NV == 8 ? __byte_perm((uint32_t)o[H8 + 2], (uint32_t)o[H8 + 3], 0x5410) : u.y;
    vmax = max_s16x2(vmax, max_s16x2(max_s16x2(u.x, u.y), max_s16x2(u.z, u.w)));
    vmin = min_s16x2(vmin, min_s16x2(min_s16x2(u.x, u.y), min_s16x2(u.z, u.w)));
    int16_t* dst = reinterpret_cast<int16_t*>(out.m) + row * out.ld + c0;
    if (NV == 8) *reinterpret_cast<uint4*>(dst) = u;
    else *reinterpret_cast<uint2*>(dst) = make_uint2(u.x, u.y);
  }
  return false;
}

__device__ __forceinline__ long long packed_norm(uint32_t vmax, uint32_t vmin, bool is32) {
  if (is32) return (long long)vmax;
  const int32_t mx = max((int32_t)vmax >> 16, (int32_t)(int16_t)(vmax & 0xffffu));
  const int32_t mn = min((int32_t)vmin >> 16, (int32_t)(int16_t)(vmin & 0xffffu));
  return (long long)max(mx, -mn);
}

__device__ __forceinline__ void fold_key(Red& red, uint64_t ormag, bool any) {
  if (ormag) red.key = max(red.key, (long long)(256 + (64 - __clzll((long long)ormag)) + 1));
  else if (any) red.key = max(red.key, 257ll);
}

// ---------------------------------------------------------------------------
// Restriction r_c = R~ r_f.  A lane owns 8 coarse columns c0.. (fine columns
// 2c0 .. 2c0+16); a stage is one fine row: 32 lane slots of 32 bytes, then the
// east halo pair (the next chunk's first fine pair).
// ---------------------------------------------------------------------------
constexpr int kRStages = 8;
constexpr int kRRowWords = 4 + 256 + 4;
struct __align__(16) StageR {
  uint32_t f[kRStages][kRRowWords];
};

// H of coarse row J from global memory (general path; fine mantissas of type T)
template <class T = int16_t, int NV = 8>
__device__ __forceinline__ void restrict_hl_global(const VIn& f, int64_t J, int64_t c0, int32_t (&H)[NV]) {
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const int64_t fi = 2 * (c0 + k) + 1, fj = 2 * J + 1;
    int32_t acc = 0;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx)
        acc += (2 - (dx < 0 ? -dx : dx)) * (2 - (dy < 0 ? -dy : dy)) * ld1_t<T>(f, fj + dy, fi + dx);
    H[k] = acc;
  }
}

template <bool PASS1, class T = int16_t, int NV = 8>
__device__ __noinline__ void restrict_slow(const VIn& f, const Plan& p, const VOut& out, int32_t* tmp, int64_t J,
                                           int64_t c0, Red& red) {
  int32_t H[NV], L[NV];
  restrict_hl_global<T, NV>(f, J, c0, H);
#pragma unroll
  for (int k = 0; k < NV; ++k) L[k] = 0;
  slow_hlv<PASS1, NV>(H, L, p, out, tmp, J, c0, red);
}

// Parameters of one restriction / interpolation op (one instance of a batched launch).
struct TransferP {
  VIn f;       // restriction: fine input; interpolation: the coarse d
  VIn y;       // interpolation: y of the correction
  QDesc q;
  VOut out;
  int32_t rs;
};

// B: a batched launch of 2D ops, grid z the instance, parameters Pb[z].  T: the fine mantissas, int16
// (a lane owns 8 coarse columns, 16 fine ones) or int32 (4 coarse, 8 fine; at most 27 bits, so the
// nine-point sum is exact in int32); either way a lane stages 32 bytes of a fine row.
template <bool PASS1, bool B = false, class T = int16_t>
__global__ void __launch_bounds__(128, 6) k_restrict2d16(const __grid_constant__ TransferP P1,
                                                        const TransferP* __restrict__ Pb) {
  constexpr bool W32 = sizeof(T) == 4;
  constexpr int NV = W32 ? 4 : 8;           // coarse columns per lane
  constexpr int kSeg = 16 / (int)sizeof(T);  // fine mantissas per 16-byte copy
  pdl_wait();
  const TransferP& P = B ? Pb[blockIdx.z] : P1;
  const VIn& f = P.f;
  const QDesc& q = P.q;
  const VOut& out = P.out;
  const int rs = P.rs;
  __shared__ Plan sp;
  __shared__ StageR stg[4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * (32 * NV) + lane * NV;
  const int64_t fc = 2 * c0;
  const int ny = (int)out.ny;
  const int J0 = (int)(((int64_t)blockIdx.y * 4 + warp) * rs);
  const int J1 = J0 + rs < ny ? J0 + rs : ny;
  const bool act = c0 < out.ld;
  const int nvalid = (int)(out.nx - c0 < NV ? (out.nx - c0 < 0 ? 0 : out.nx - c0) : NV);
  const bool partial = nvalid < NV;
  // fine columns fc + m, m < 2 NV, beyond nx read as 0 (partial chunks only)
  const int fvalid = (int)(f.nx - fc < 2 * NV ? (f.nx - fc < 0 ? 0 : f.nx - fc) : 2 * NV);
  uint32_t fmask[8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
    fmask[i] = W32 ? ((i < fvalid) ? 0xffffffffu : 0u)
                   : (((2 * i < fvalid) ? 0xffffu : 0u) | ((2 * i + 1 < fvalid) ? 0xffff0000u : 0u));
  const bool fpartial = fvalid < 2 * NV;

  StageR& S = stg[warp];
  const int nfin = (int)(f.ny * f.nz);
  const T* fb = reinterpret_cast<const T*>(f.m);
  const bool seg0 = fc < f.nx && fc < f.ld, seg1 = fc + kSeg < f.nx && fc + kSeg < f.ld;
  const bool hok = lane == 31 && fc + 2 * NV < f.nx;
  // the next stage to issue: fine row jf (stage s holds fine row 2 J0 + s)
  int jf = 2 * J0;
  int64_t of = (int64_t)jf * f.ld + fc;
  auto issue = [&](int slot) {
    const bool in = (unsigned)jf < (unsigned)nfin;
    cp16(&S.f[slot][4 + 8 * lane], fb + ((in && seg0) ? of : 0), (in && seg0) ? 16u : 0u);
    cp16(&S.f[slot][8 + 8 * lane], fb + ((in && seg1) ? of + kSeg : 0), (in && seg1) ? 16u : 0u);
    const bool hk = hok && in;
    cp4_if(lane == 31, &S.f[slot][kRRowWords - 4], fb + (hk ? of + 2 * NV : 0), hk ? 4u : 0u);
    of += f.ld;
    ++jf;
  };
  // prologue: fine rows 2 J0 .. 2 J0 + 5 in three groups of two; it does not depend on the plan and is
  // issued before the plan is built (nnqcomp and qcomp's first pass)
  auto prologue = [&]() {
#pragma unroll
    for (int g = 0; g < 3; ++g) {
      issue(2 * g);
      issue(2 * g + 1);
      cp_commit();
    }
  };
  const bool early = (PASS1 || q.mode == kNnqcomp) && J0 < J1;
  const bool with_mu = !PASS1 && q.mode == kQcomp;
  const MetaIn mi = threadIdx.x == 0 ? load_meta(q, with_mu) : MetaIn{0, 0, 0, 0, 0};
  if (early) prologue();
  if (threadIdx.x == 0) build_plan_m(q, mi, with_mu, sp);
  __syncthreads();
  const Plan& p = sp;
  const Fast fq = make_fast(p, PASS1);
  const EmitC ec = make_emit(fq, q, 1, PASS1);
  Red red = {0, 0, 0};
  int32_t* tmp = (PASS1 && p.use_tmp && !p.guarded) ? reinterpret_cast<int32_t*>(q.tmp) : nullptr;
  // h_k = f[2c] + 2 f[2c+1] + f[2c+2] for c = c0 + k of the fine row in `slot`
  auto hrow = [&](int slot, int32_t (&h)[NV]) {
    const uint4 a = *reinterpret_cast<const uint4*>(&S.f[slot][4 + 8 * lane]);
    const uint4 b = *reinterpret_cast<const uint4*>(&S.f[slot][8 + 8 * lane]);
    uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    if (fpartial) {
#pragma unroll
      for (int i = 0; i < 8; ++i) w[i] &= fmask[i];
    }
    if constexpr (W32) {   // fine values 2k, 2k + 1 in words 2k, 2k + 1; the next lane's first (or the halo)
      const int32_t nxt = reinterpret_cast<const int32_t*>(&S.f[slot][0])[4 + 8 * (lane + 1)];
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const int32_t v2 = k < NV - 1 ? (int32_t)w[2 * k + 2 < 8 ? 2 * k + 2 : 0] : nxt;
        h[k] = (int32_t)w[2 * k] + 2 * (int32_t)w[2 * k + 1] + v2;
      }
    } else {
      const int32_t nxt = reinterpret_cast<const int16_t*>(&S.f[slot][0])[8 + 16 * (lane + 1)];
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const int32_t v0 = (int32_t)(int16_t)(w[k] & 0xffffu), v1 = (int32_t)w[k] >> 16;
        const int32_t v2 = k < NV - 1 ? (int32_t)(int16_t)(w[k + 1 < 8 ? k + 1 : 0] & 0xffffu) : nxt;
        h[k] = v0 + 2 * v1 + v2;
      }
    }
  };

  uint32_t vmax = 0, vmin = 0, redo_rows = 0;
  uint64_t ormag = 0;
  bool any = false;
  if (!PASS1 && p.narrow) {
    for (int J = J0; J < J1; ++J)
      if (act) narrowv<NV>(reinterpret_cast<const int32_t*>(q.tmp), p, out, J, c0, red);
  } else if (J0 < J1) {
    auto walk = [&](auto v32tag, auto foldtag) {
      constexpr bool V32 = decltype(v32tag)::value, FOLD = decltype(foldtag)::value;
      if (!early) prologue();
      cp_wait<2>();
      __syncwarp();
      int32_t hp[NV];
      hrow(0, hp);
      for (int J = J0; J < J1; ++J) {
        const int i = J - J0;
        __syncwarp();                           // every lane is done with the slots reused below
        issue((2 * i + 6) & (kRStages - 1));    // fine rows 2J + 6, 2J + 7 into the slots of 2J - 2, 2J - 1
        issue((2 * i + 7) & (kRStages - 1));
        cp_commit();
        cp_wait<2>();                           // fine rows <= 2J + 3 have landed
        __syncwarp();
        int32_t hm[NV], hn[NV];
        hrow((2 * i + 1) & (kRStages - 1), hm);
        hrow((2 * i + 2) & (kRStages - 1), hn);
        int32_t H[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) { H[k] = hp[k] + 2 * hm[k] + hn[k]; hp[k] = hn[k]; }
        if (act) {
          bool redo = !ec.fast;
          if (ec.fast)   // one exact group: the L argument is not read
            redo = emit8<PASS1, V32, FOLD, NV>(ec, fq, H, H, false, nvalid, partial, out, tmp, J, c0, ormag, vmax, vmin);
          if (redo) redo_rows |= 1u << i;
          any = any || nvalid > 0;
        }
      }
      cp_wait<0>();
    };
    if (ec.fold) {
      if (ec.v32) walk(std::true_type{}, std::true_type{});
      else walk(std::false_type{}, std::true_type{});
    } else {
      if (ec.v32) walk(std::true_type{}, std::false_type{});
      else walk(std::false_type{}, std::false_type{});
    }
    for (uint32_t m = redo_rows; m != 0u; m &= m - 1u) {
      const int J = J0 + __ffs(m) - 1;
      if (act) restrict_slow<PASS1, T, NV>(f, p, out, tmp, J, c0, red);
    }
  }
  if (PASS1) fold_key(red, ormag, any && ec.fast);
  else red.nrm = max(red.nrm, packed_norm(vmax, vmin, out.is32 != 0));
  pdl_trigger();
  block_commit(red, q.meta_out, q.stats, PASS1);
  if (!PASS1) op_epilogue(q, p, blockIdx.x == 0 && blockIdx.y == 0 && (B || blockIdx.z == 0));
}

// ---------------------------------------------------------------------------
// 3D restriction.  A warp owns a 256-column chunk of coarse rows J0.. of coarse
// plane K; a stage is fine row jf of the fine planes 2K, 2K+1, 2K+2, combined
// as v = f0 + 2 f1 + f2 before the horizontal sums.  Stages are three times the
// 2D size, so a CTA has two warps and a ring of six fine rows: rows 2J+1 ..
// 2J+3 in use or landed, rows 2J+4, 2J+5 in flight.
// ---------------------------------------------------------------------------
constexpr int kR3Slots = 6;
constexpr int kR3Warps = 2;
struct __align__(16) StageR3 {
  uint32_t f[kR3Slots][3][kRRowWords];
};

template <bool PASS1>
__device__ __noinline__ void restrict3_slow(const VIn& f, const Plan& p, const VOut& out, int32_t* tmp, int64_t J,
                                            int64_t K, int64_t c0, Red& red) {
  int32_t H[8], L[8];
  const int64_t fny = f.ny;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int64_t fi = 2 * (c0 + k) + 1, fj = 2 * J + 1, fk = 2 * K + 1;
    int32_t acc = 0;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx)
          acc += (2 - (dx < 0 ? -dx : dx)) * (2 - (dy < 0 ? -dy : dy)) * (2 - (dz < 0 ? -dz : dz)) *
                 ld1_16(f, (fk + dz) * fny + fj + dy, fi + dx);
    H[k] = acc;
    L[k] = 0;
  }
  slow_hl8<PASS1>(H, L, p, out, tmp, K * out.ny + J, c0, red);
}

// grid: (256-column chunks, strips of kR3Warps * rs coarse rows, coarse planes)
template <bool PASS1>
__global__ void __launch_bounds__(64) k_restrict3d16(const VIn f, const QDesc q, const VOut out, const int rs) {
  __shared__ Plan sp;
  __shared__ StageR3 stg[kR3Warps];
  if (threadIdx.x == 0) {
    build_plan(q, sp);
    if (!PASS1 && q.mode == kQcomp) plan_from_mu(sp, q.meta_out[kMetaMu]);
  }
  __syncthreads();
  const Plan& p = sp;
  const Fast fq = make_fast(p, PASS1);
  const EmitC ec = make_emit(fq, q, 1, PASS1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * 256 + lane * 8;
  const int64_t fc = 2 * c0;
  const int ny = (int)out.ny;                    // coarse rows per plane
  const int K = (int)blockIdx.z;
  const int64_t crow0 = (int64_t)K * ny;
  const int J0 = (int)(((int64_t)blockIdx.y * kR3Warps + warp) * rs);
  const int J1 = J0 + rs < ny ? J0 + rs : ny;
  const bool act = c0 < out.ld;
  Red red = {0, 0, 0};
  int32_t* tmp = (PASS1 && p.use_tmp && !p.guarded) ? reinterpret_cast<int32_t*>(q.tmp) : nullptr;
  const int nvalid = (int)(out.nx - c0 < 8 ? (out.nx - c0 < 0 ? 0 : out.nx - c0) : 8);
  const bool partial = nvalid < 8;
  const int fvalid = (int)(f.nx - fc < 16 ? (f.nx - fc < 0 ? 0 : f.nx - fc) : 16);
  uint32_t fmask[8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
    fmask[i] = ((2 * i < fvalid) ? 0xffffu : 0u) | ((2 * i + 1 < fvalid) ? 0xffff0000u : 0u);
  const bool fpartial = fvalid < 16;

  StageR3& S = stg[warp];
  const int fny = (int)f.ny;
  const int16_t* fb = reinterpret_cast<const int16_t*>(f.m);
  const bool seg0 = fc < f.nx && fc < f.ld, seg1 = fc + 8 < f.nx && fc + 8 < f.ld;
  const bool hok = lane == 31 && fc + 16 < f.nx;
  const int64_t pdelta = (int64_t)fny * f.ld;    // one fine plane
  // the next fine row to issue: jf of planes 2K, 2K+1, 2K+2 (planes 2K + 2 <= 2 nz_c < nz_f always exist)
  int jf = 2 * J0;
  int64_t of = ((int64_t)2 * K * fny + jf) * f.ld + fc;
  auto issue = [&](int slot) {
    const bool in = (unsigned)jf < (unsigned)fny;
    const bool i0 = in && seg0, i1 = in && seg1, hk = hok && in;
#pragma unroll
    for (int pl = 0; pl < 3; ++pl) {
      const int64_t o = of + pl * pdelta;
      cp16(&S.f[slot][pl][4 + 8 * lane], fb + (i0 ? o : 0), i0 ? 16u : 0u);
      cp16(&S.f[slot][pl][8 + 8 * lane], fb + (i1 ? o + 8 : 0), i1 ? 16u : 0u);
      cp4_if(lane == 31, &S.f[slot][pl][kRRowWords - 4], fb + (hk ? o + 16 : 0), hk ? 4u : 0u);
    }
    of += f.ld;
    ++jf;
  };
  // h_k = v[2c] + 2 v[2c+1] + v[2c+2] (c = c0 + k) of the plane-combined fine row in `slot`
  auto hrow = [&](int slot, int32_t (&h)[8]) {
    int32_t v[17];
#pragma unroll
    for (int pl = 0; pl < 3; ++pl) {
      const uint4 a = *reinterpret_cast<const uint4*>(&S.f[slot][pl][4 + 8 * lane]);
      const uint4 b = *reinterpret_cast<const uint4*>(&S.f[slot][pl][8 + 8 * lane]);
      uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
      if (fpartial) {
#pragma unroll
        for (int i = 0; i < 8; ++i) w[i] &= fmask[i];
      }
      const int32_t nxt = reinterpret_cast<const int16_t*>(&S.f[slot][pl][0])[8 + 16 * (lane + 1)];
      const int32_t m = pl == 1 ? 2 : 1;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int32_t lo = (int32_t)(int16_t)(w[i] & 0xffffu), hi = (int32_t)w[i] >> 16;
        v[2 * i] = pl == 0 ? lo : v[2 * i] + m * lo;
        v[2 * i + 1] = pl == 0 ? hi : v[2 * i + 1] + m * hi;
      }
      v[16] = pl == 0 ? nxt : v[16] + m * nxt;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) h[k] = v[2 * k] + 2 * v[2 * k + 1] + v[2 * k + 2];
  };

  uint32_t vmax = 0, vmin = 0, redo_rows = 0;
  uint64_t ormag = 0;
  bool any = false;
  if (!PASS1 && p.narrow) {
    for (int J = J0; J < J1; ++J)
      if (act) narrowv<8>(reinterpret_cast<const int32_t*>(q.tmp), p, out, crow0 + J, c0, red);
  } else if (J0 < J1) {
    auto walk = [&](auto v32tag, auto foldtag) {
      constexpr bool V32 = decltype(v32tag)::value, FOLD = decltype(foldtag)::value;
      // prologue: fine rows 2 J0 .. 2 J0 + 3 in two groups of two (ring slot = (row - 2 J0) mod 6)
      issue(0);
      issue(1);
      cp_commit();
      issue(2);
      issue(3);
      cp_commit();
      cp_wait<1>();
      __syncwarp();
      int32_t hp[8];
      hrow(0, hp);
      int b = 0;                                 // slot of fine row 2J
      for (int J = J0; J < J1; ++J) {
        const int i = J - J0;
        auto sl = [&](int d) { return b + d >= kR3Slots ? b + d - kR3Slots : b + d; };
        __syncwarp();                            // every lane is done with the slots of rows 2J-2, 2J-1
        issue(sl(4));                            // fine rows 2J + 4, 2J + 5
        issue(sl(5));
        cp_commit();
        cp_wait<1>();                            // fine rows <= 2J + 3 have landed
        __syncwarp();
        int32_t hm[8], hn[8];
        hrow(sl(1), hm);
        hrow(sl(2), hn);
        int32_t H[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) { H[k] = hp[k] + 2 * hm[k] + hn[k]; hp[k] = hn[k]; }
        if (act) {
          bool redo = !ec.fast;
          if (ec.fast)
            redo = emit8<PASS1, V32, FOLD>(ec, fq, H, H, false, nvalid, partial, out, tmp, crow0 + J, c0, ormag,
                                           vmax, vmin);
          if (redo) redo_rows |= 1u << i;
          any = any || nvalid > 0;
        }
        b = sl(2);
      }
      cp_wait<0>();
    };
    if (ec.fold) {
      if (ec.v32) walk(std::true_type{}, std::true_type{});
      else walk(std::false_type{}, std::true_type{});
    } else {
      if (ec.v32) walk(std::true_type{}, std::false_type{});
      else walk(std::false_type{}, std::false_type{});
    }
    for (uint32_t m = redo_rows; m != 0u; m &= m - 1u) {
      const int J = J0 + __ffs(m) - 1;
      if (act) restrict3_slow<PASS1>(f, p, out, tmp, J, K, c0, red);
    }
  }
  if (PASS1) fold_key(red, ormag, any && ec.fast);
  else red.nrm = max(red.nrm, packed_norm(vmax, vmin, out.is32 != 0));
  block_commit(red, q.meta_out, q.stats, PASS1);
  if (!PASS1) op_epilogue(q, p);
}

// ---------------------------------------------------------------------------
// Interpolation: y' = y - P d (CORR) or P d.  A lane owns 8 fine columns c0..
// (coarse columns C = c0/2 .. C+3 and C-1 from the previous lane); a stage is
// coarse row P (lane slots of 8 bytes after the west halo pair) and fine rows
// 2P, 2P+1 of y.  In 3D the CTAs of fine plane k stage coarse row P of the
// planes that plane interpolates from: Q for k = 2Q + 1 (weight 2), Q - 1 and Q
// for k = 2Q (weight 1 each), combined before the horizontal interpolation.
// ---------------------------------------------------------------------------
constexpr int kPStages = 4;
constexpr int kPRowWords = 4 + 64;
template <int ND>
struct __align__(16) StageP {
  uint32_t d[kPStages][ND == 3 ? 2 : 1][kPRowWords];
  uint4 y[kPStages][2][32];
};

// H (= P_m d) and L (= y) of fine row j of plane kf from global memory (general path; mantissas of type T)
template <bool CORR, int ND, class T = int16_t, int NV = 8>
__device__ __forceinline__ void prolong_hl_global(const VIn& d, const VIn& y, int64_t j, int64_t kf, int64_t c0,
                                                  int32_t (&H)[NV], int32_t (&L)[NV]) {
  const int64_t cny = d.ny;
  auto gx = [&](int64_t Q, int64_t J, int64_t i) -> int32_t {   // coarse row J of plane Q at fine column i
    if (J < 0 || J >= cny || Q < 0 || Q >= d.nz) return 0;
    const int64_t row = Q * cny + J;
    return (i & 1) ? 2 * ld1_t<T>(d, row, (i - 1) >> 1) : ld1_t<T>(d, row, (i >> 1) - 1) + ld1_t<T>(d, row, i >> 1);
  };
  auto gyx = [&](int64_t Q, int64_t i) -> int32_t {            // interpolation in y, then x, on plane Q
    return (j & 1) ? 2 * gx(Q, (j - 1) >> 1, i) : gx(Q, (j >> 1) - 1, i) + gx(Q, j >> 1, i);
  };
  const int64_t frow = kf * y.ny + j;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const int64_t i = c0 + k;
    int32_t pd;
    if (ND == 3) pd = (kf & 1) ? 2 * gyx((kf - 1) >> 1, i) : gyx((kf >> 1) - 1, i) + gyx(kf >> 1, i);
    else pd = gyx(0, i);
    H[k] = CORR ? -pd : pd;
    L[k] = CORR ? ld1_t<T>(y, frow, i) : 0;
  }
}

template <bool CORR, bool PASS1, int ND, class T = int16_t, int NV = 8>
__device__ __noinline__ void prolong_slow(const VIn& d, const VIn& y, const Plan& p, const VOut& out, int32_t* tmp,
                                          int64_t j, int64_t kf, int64_t c0, Red& red) {
  int32_t H[NV], L[NV];
  prolong_hl_global<CORR, ND, T, NV>(d, y, j, kf, c0, H, L);
  slow_hlv<PASS1, NV>(H, L, p, out, tmp, kf * out.ny + j, c0, red);
}

// grid: (fine column chunks of 32 lanes x NV, strips of 4 * rs row pairs, fine planes).  T: the mantissas
// of d and y, int16 (8 fine columns per lane, 4 coarse) or int32 (4 fine, 2 coarse; 2D, d of at most 29
// bits so that P_m d is exact in int32).
template <bool CORR, bool PASS1, int ND, bool B = false, class T = int16_t>
__global__ void __launch_bounds__(128, 6) k_prolong16(const __grid_constant__ TransferP Pv,
                                                      const TransferP* __restrict__ Pb) {
  static_assert(!B || ND == 2, "batched launches are 2D");
  constexpr bool W32 = sizeof(T) == 4;
  static_assert(!W32 || ND == 2, "int32 mantissas: 2D");
  constexpr int NV = W32 ? 4 : 8;      // fine columns per lane
  constexpr int NC = NV / 2;           // coarse columns per lane
  pdl_wait();
  const TransferP& P = B ? Pb[blockIdx.z] : Pv;
  const VIn& d = P.f;
  const VIn& y = P.y;
  const QDesc& q = P.q;
  const VOut& out = P.out;
  const int rs = P.rs;
  __shared__ Plan sp;
  __shared__ StageP<ND> stg[4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * (32 * NV) + lane * NV;
  const int64_t C = c0 >> 1;                     // first coarse column of this lane (multiple of NC)
  const int ny = (int)out.ny;                    // fine rows (of one plane)
  const int kf = ND == 3 ? (int)blockIdx.z : 0;  // fine plane
  const int64_t frow0 = (int64_t)kf * ny;        // global row of the plane's fine row 0
  const int P0 = (int)(((int64_t)blockIdx.y * 4 + warp) * rs);   // first row pair (fine rows 2P0, 2P0+1)
  const int P1 = min(P0 + rs, (ny + 1) / 2);
  const bool act = c0 < out.ld;
  const int nvalid = (int)(out.nx - c0 < NV ? (out.nx - c0 < 0 ? 0 : out.nx - c0) : NV);
  const bool partial = nvalid < NV;
  // coarse columns C + m (m < NC) beyond d.nx, fine y columns beyond nx: 0 (partial chunks only)
  const int cvalid = (int)(d.nx - C < NC ? (d.nx - C < 0 ? 0 : d.nx - C) : NC);
  const uint32_t cm0 = W32 ? ((0 < cvalid) ? 0xffffffffu : 0u) : (((0 < cvalid) ? 0xffffu : 0u) | ((1 < cvalid) ? 0xffff0000u : 0u));
  const uint32_t cm1 = W32 ? ((1 < cvalid) ? 0xffffffffu : 0u) : (((2 < cvalid) ? 0xffffu : 0u) | ((3 < cvalid) ? 0xffff0000u : 0u));
  uint32_t ymask[4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
    ymask[i] = W32 ? ((i < nvalid) ? 0xffffffffu : 0u)
                   : (((2 * i < nvalid) ? 0xffffu : 0u) | ((2 * i + 1 < nvalid) ? 0xffff0000u : 0u));

  StageP<ND>& S = stg[warp];
  const int ncr = (int)d.ny, nyr = CORR ? ny : 1;   // rows per plane
  const T* db = reinterpret_cast<const T*>(d.m);
  const T* yb = CORR ? reinterpret_cast<const T*>(y.m) : nullptr;
  const bool dseg = C < d.nx && C < d.ld;
  // west halo word: lane 0 copies coarse (C-2, C-1) (int16) or C-1 (int32)
  constexpr int kHw = W32 ? 1 : 2;
  const bool hok = lane == 0 && C >= kHw && C - 1 < d.nx;
  const bool yseg = CORR && c0 < y.nx && c0 < y.ld;
  // coarse planes: qa (and qb = qa + 1 on even fine planes of a 3D grid); a plane outside the grid reads 0
  const bool odd = ND == 3 && (kf & 1);
  const int qa = ND == 3 ? (odd ? (kf - 1) >> 1 : (kf >> 1) - 1) : 0;
  const bool qaok = (unsigned)qa < (unsigned)d.nz, qbok = ND == 3 && !odd && (unsigned)(qa + 1) < (unsigned)d.nz;
  const int64_t qdelta = (int64_t)ncr * d.ld;    // plane qb - plane qa
  // the next stage: coarse row jc (stage s holds coarse row P0 - 1 + s, y rows 2 jc, 2 jc + 1)
  int jc = P0 - 1;
  int64_t od = ((int64_t)qa * ncr + jc) * d.ld + C, oy = CORR ? (frow0 + 2 * jc) * y.ld + c0 : 0;
  auto issue = [&](int slot, bool with_y) {
    const bool in = (unsigned)jc < (unsigned)ncr;
    const bool ia = in && qaok;
    cp8(&S.d[slot][0][4 + 2 * lane], db + ((ia && dseg) ? od : 0), (ia && dseg) ? 8u : 0u);
    const bool hk = hok && ia;
    cp4_if(lane == 0, &S.d[slot][0][3], db + (hk ? od - kHw : 0), hk ? 4u : 0u);
    if (ND == 3 && !odd) {
      const int pb = ND == 3 ? 1 : 0;
      const bool ib = in && qbok;
      cp8(&S.d[slot][pb][4 + 2 * lane], db + ((ib && dseg) ? od + qdelta : 0), (ib && dseg) ? 8u : 0u);
      const bool hb = hok && ib;
      cp4_if(lane == 0, &S.d[slot][pb][3], db + (hb ? od + qdelta - kHw : 0), hb ? 4u : 0u);
    }
    if (CORR && with_y) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const bool yin = yseg && (unsigned)(2 * jc + h) < (unsigned)nyr;
        cp16(&S.y[slot][h][lane], yb + (yin ? oy + h * y.ld : 0), yin ? 16u : 0u);
      }
    }
    od += d.ld;
    if (CORR) oy += 2 * y.ld;
    ++jc;
    cp_commit();
  };
  // the first three stages do not depend on the plan: issued before it is built (nnqcomp and qcomp's
  // first pass)
  auto prologue = [&]() {
    issue(0, false);                           // coarse row P0 - 1 only
    issue(1, true);
    issue(2, true);
  };
  const bool early = (PASS1 || q.mode == kNnqcomp) && P0 < P1;
  const bool with_mu = !PASS1 && q.mode == kQcomp;
  const MetaIn mi = threadIdx.x == 0 ? load_meta(q, with_mu) : MetaIn{0, 0, 0, 0, 0};
  if (early) prologue();
  if (threadIdx.x == 0) build_plan_m(q, mi, with_mu, sp);
  __syncthreads();
  const Plan& p = sp;
  const Fast fq = make_fast(p, PASS1);
  const EmitC ec = make_emit(fq, q, CORR ? -1 : 1, PASS1);
  Red red = {0, 0, 0};
  int32_t* tmp = (PASS1 && p.use_tmp && !p.guarded) ? reinterpret_cast<int32_t*>(q.tmp) : nullptr;
  // coarse columns C - 1 .. C + NC - 1 of the staged row of plane slot pl
  auto dvals = [&](int slot, int pl, int32_t (&dv)[NC + 1]) {
    const uint2 u = *reinterpret_cast<const uint2*>(&S.d[slot][pl][4 + 2 * lane]);
    const uint32_t u0 = u.x & cm0, u1 = u.y & cm1;
    if constexpr (W32) {
      dv[0] = reinterpret_cast<const int32_t*>(&S.d[slot][pl][0])[3 + 2 * lane];   // coarse column C - 1
      dv[1] = (int32_t)u0;
      dv[NC] = (int32_t)u1;
    } else {
      dv[0] = reinterpret_cast<const int16_t*>(&S.d[slot][pl][0])[7 + 4 * lane];   // coarse column C - 1
      dv[1] = (int32_t)(int16_t)(u0 & 0xffffu); dv[2] = (int32_t)u0 >> 16;
      dv[NC > 2 ? 3 : 1] = (int32_t)(int16_t)(u1 & 0xffffu); dv[NC] = (int32_t)u1 >> 16;
    }
  };
  // g_k: horizontal interpolation of the (plane-combined) coarse row in `slot` at fine columns c0 + k
  auto grow = [&](int slot, int32_t (&g)[NV]) {
    int32_t dv[NC + 1];
    dvals(slot, 0, dv);
    if (ND == 3) {
      if (odd) {
#pragma unroll
        for (int m = 0; m <= NC; ++m) dv[m] *= 2;
      } else {
        int32_t db5[NC + 1];
        dvals(slot, ND == 3 ? 1 : 0, db5);
#pragma unroll
        for (int m = 0; m <= NC; ++m) dv[m] += db5[m];
      }
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) g[k] = (k & 1) ? 2 * dv[(k + 1) / 2] : dv[k / 2] + dv[k / 2 + 1];
  };

  uint32_t vmax = 0, vmin = 0, redo_rows = 0;
  uint64_t ormag = 0;
  bool any = false;
  if (!PASS1 && p.narrow) {
    for (int j = 2 * P0; j < 2 * P1 && j < ny; ++j)
      if (act) narrowv<NV>(reinterpret_cast<const int32_t*>(q.tmp), p, out, frow0 + j, c0, red);
  } else if (P0 < P1) {
    auto walk = [&](auto v32tag, auto foldtag) {
      constexpr bool V32 = decltype(v32tag)::value, FOLD = decltype(foldtag)::value;
      if (!early) prologue();
      cp_wait<2>();
      __syncwarp();
      int32_t gm[NV];
      grow(0, gm);
      for (int P = P0; P < P1; ++P) {
        const int i = P - P0;
        issue((i + 3) & (kPStages - 1), true);   // stage i + 3 into the slot of stage i - 1
        cp_wait<2>();                            // stage i + 1 (coarse row P, y rows 2P, 2P+1) has landed
        __syncwarp();
        const int slot = (i + 1) & (kPStages - 1);
        int32_t gc[NV];
        grow(slot, gc);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = 2 * P + h;
          if (j >= ny) break;
          int32_t H[NV], L[NV];
          if (CORR) {
            uint4 u = S.y[slot][h][lane];
            if (partial) { u.x &= ymask[0]; u.y &= ymask[1]; u.z &= ymask[2]; u.w &= ymask[3]; }
            if constexpr (W32) {
              L[0] = (int32_t)u.x; L[1] = (int32_t)u.y; L[NV > 2 ? 2 : 0] = (int32_t)u.z; L[NV - 1] = (int32_t)u.w;
            } else {
              int32_t l8[8];
              unpack8(u, l8);
#pragma unroll
              for (int k = 0; k < NV; ++k) L[k] = l8[k];
            }
          } else {
#pragma unroll
            for (int k = 0; k < NV; ++k) L[k] = 0;
          }
#pragma unroll
          for (int k = 0; k < NV; ++k) H[k] = h == 0 ? gm[k] + gc[k] : 2 * gc[k];
          if (act) {
            bool redo = !ec.fast;
            if (ec.fast)
              redo = emit8<PASS1, V32, FOLD, NV>(ec, fq, H, L, CORR, nvalid, partial, out, tmp, frow0 + j, c0, ormag,
                                                 vmax, vmin);
            if (redo) redo_rows |= 1u << (2 * i + h);
            any = any || nvalid > 0;
          }
        }
#pragma unroll
        for (int k = 0; k < NV; ++k) gm[k] = gc[k];
      }
      cp_wait<0>();
    };
    if (ec.fold) {
      if (ec.v32) walk(std::true_type{}, std::true_type{});
      else walk(std::false_type{}, std::true_type{});
    } else {
      if (ec.v32) walk(std::true_type{}, std::false_type{});
      else walk(std::false_type{}, std::false_type{});
    }
    for (uint32_t m = redo_rows; m != 0u; m &= m - 1u) {
      const int j = 2 * P0 + __ffs(m) - 1;
      if (act) prolong_slow<CORR, PASS1, ND, T, NV>(d, y, p, out, tmp, j, kf, c0, red);
    }
  }
  if (PASS1) fold_key(red, ormag, any && ec.fast);
  else red.nrm = max(red.nrm, packed_norm(vmax, vmin, out.is32 != 0));
  pdl_trigger();
  block_commit(red, q.meta_out, q.stats, PASS1);
  if (!PASS1) op_epilogue(q, p, blockIdx.x == 0 && blockIdx.y == 0 && (B || blockIdx.z == 0));
}

}  // namespace bfp
