// bfp_device.cuh -- device arithmetic shared by the BFP kernels.
//
// Integer primitives of Sec. 2 (signed bit width, floor shift, narrowing),
// the per-op quantisation plan (the "setup-func" of Alg. qcomp / nnqcomp run
// once per CTA from the device meta blocks), and the per-element finishing
// step that turns an exact result into a w_out-bit mantissa.
//
// Exact results.  An op's exact value is z* = H * 2^Eh + L * 2^El (one or two
// exponent groups; App. B setup rules give e* = min(Eh, El)).  H and L are
// exact 64-bit integers (their msb is bounded on the host, <= 62).  The two
// groups are combined at the exponent Ez:
//   d = |Eh - El| <= 64 : Z = (T << d) + B exactly, Ez = e*;
//   d  > 64             : Z = (T << 64) + floor(B / 2^(d-64)), Ez = E_top - 64,
// where T / B are the groups with the larger / smaller exponent.  In the
// second case Z = floor(z* / 2^Ez) exactly, and since |T << 64| dwarfs B, every
// element with T != 0 has msb(Z) >= 64 while elements with T == 0 are exact in
// B; the normalised exponent and all outputs at or above Ez are therefore
// exact.
#pragma once

#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

namespace bfp {

typedef __int128 i128;
typedef unsigned __int128 u128;

constexpr int kMetaMu = 2;     // meta word of qcomp's atomic max (mu* key)
constexpr int kGuard = 64;     // group alignment beyond which the bottom group is floor-shifted
constexpr int kVec = 8;        // mantissas per thread per row

// ---------------------------------------------------------------------------
// Sec. 2 primitives
// ---------------------------------------------------------------------------

// Signed bit width min{v >= 1 : z in X_v}; msb(0) = 1, msb(23) = 6 (Fig. 2).
__host__ __device__ __forceinline__ int msb64(int64_t z) {
  uint64_t v = (uint64_t)(z ^ (z >> 63));
#ifdef __CUDA_ARCH__
  return 65 - __clzll((long long)v);
#else
  int b = 0;
  while (v) { ++b; v >>= 1; }
  return b + 1;
#endif
}

__host__ __device__ __forceinline__ int bitlen_u128(u128 v) {
  uint64_t hi = (uint64_t)(v >> 64), lo = (uint64_t)v;
#ifdef __CUDA_ARCH__
  return hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);
#else
  int b = 0;
  while (v) { ++b; v >>= 1; }
  return b;
#endif
}

__host__ __device__ __forceinline__ int msb128(i128 z) {
  u128 v = (u128)(z ^ (z >> 127));
  return bitlen_u128(v) + 1;
}

__device__ __forceinline__ int msb_acc(int64_t z) { return msb64(z); }
__device__ __forceinline__ int msb_acc(i128 z) { return msb128(z); }

// floor(z / 2^t) for t >= 0
__device__ __forceinline__ int64_t shr_floor(int64_t z, int64_t t) { return z >> (t > 63 ? 63 : t); }
__device__ __forceinline__ i128 shr_floor(i128 z, int64_t t) { return z >> (t > 127 ? 127 : t); }

// exact z << k for k >= 0 through unsigned arithmetic (caller guarantees the fit)
__device__ __forceinline__ int64_t shl_exact(int64_t z, int k) { return (int64_t)((uint64_t)z << k); }
__device__ __forceinline__ i128 shl_exact(i128 z, int k) { return (i128)((u128)z << k); }

// decr(): the low `width` bits as a two's-complement integer (width <= 32)
__device__ __forceinline__ int32_t wrap_bits(uint64_t low, int width) {
  int s = 64 - width;
  return (int32_t)((int64_t)(low << s) >> s);
}

// low 64 bits of floor(z * 2^-t) for any t (the window store of Alg. qcomp)
__device__ __forceinline__ uint64_t low_shift(int64_t z, int64_t t) {
  if (t >= 0) return (uint64_t)shr_floor(z, t);
  return (-t) >= 64 ? 0ull : ((uint64_t)z << (-t));
}
__device__ __forceinline__ uint64_t low_shift(i128 z, int64_t t) {
  if (t >= 0) return (uint64_t)shr_floor(z, t);
  return (-t) >= 128 ? 0ull : (uint64_t)((u128)z << (-t));
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while the previous kernel in the stream finishes;
// pdl_wait() returns once that kernel has completed and its writes are
// visible (at once when there is no such kernel), so every kernel calls it
// before its first global memory access.  pdl_trigger() lets the next kernel
// be scheduled; the kernels call it after their main loop.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------------------
// BFP mantissa -> FP64 (the IR update x + m 2^e)
// ---------------------------------------------------------------------------

// The rare case kept out of line, so that the FP64 pipe is not used speculatively.
static __device__ __noinline__ double ldexp_slow(int32_t m, int64_t e) {
  return ldexp((double)m, (int)(e > 4000 ? 4000 : (e < -4000 ? -4000 : e)));
}

// m * 2^e as a double, exact for |m| < 2^31 whenever the result is normal
// (built from its bits); otherwise ldexp.
__device__ __forceinline__ double mant_pow2(int32_t m, int64_t e) {
  if (m == 0) return 0.0;
  const uint64_t sign = m < 0 ? (1ull << 63) : 0ull;
  const uint32_t a = m < 0 ? (uint32_t)(-(int64_t)m) : (uint32_t)m;
  const int lz = __clz(a);                                  // a has 32 - lz significant bits
  const int64_t be = e + (31 - lz) + 1023;                   // biased exponent of the leading bit
  if (be >= 1 && be <= 2046) {
    const uint64_t frac = (((uint64_t)a << (lz + 1)) & 0xffffffffull) << 20;   // bits below the leading one
    return __longlong_as_double((long long)(sign | ((uint64_t)be << 52) | frac));
  }
  return ldexp_slow(m, e);
}

// ---------------------------------------------------------------------------
// Quantisation plan
// ---------------------------------------------------------------------------

enum Mode : int32_t { kQcomp = 0, kNnqcomp = 1 };

// Host-side description of one quantised op (everything that does not depend
// on device-resident exponents or norms).
struct QDesc {
  const int64_t* meta_a;  // first vector input (or null)
  const int64_t* meta_b;  // second vector input (or null)
  int64_t* meta_out;
  uint64_t* stats;        // bfp_stats counters or null
  void* tmp;              // qcomp window scratch (int32) or null
  // exponent groups: E = c + ea * e_a + eb * e_b
  int64_t ch, cl;
  int32_t ha, hb, la, lb;
  int32_t two;            // 1 when the L group exists
  int32_t hbits, lbits;   // bounds on msb(H), msb(L)
  // gamma rule: sum_k gm[k] * norm(v_k) * 2^(ge[k] + e(v_k)), v_k = a (0) or b (1)
  int32_t ng;
  int32_t gv[2];
  uint64_t gm[2];
  int64_t ge[2];
  int32_t has_gamma;
  int64_t gamma_m, gamma_e;
  int32_t mode, w_out, w_tmp, use_tmp;
};

// Per-CTA plan built from a QDesc and the input meta blocks.
struct Plan {
  int64_t Ez;       // exponent of the combined integer Z
  int64_t Eb;       // exponent of the bottom group (exact fallback)
  int64_t e_star;   // App. B e*
  int64_t Gam;      // msb(gamma_m) + e_gamma (e* + 1 for gamma = 0)
  int64_t e_out;    // result exponent (nnqcomp: from gamma; qcomp pass 2: from mu*)
  int64_t e_tmp;    // exponent of the qcomp window
  int32_t two, top_is_h, s_top, s_bot, guarded, wide;
  int32_t mode, w_out, w_tmp, use_tmp;
  int32_t overflow, underflow, narrow;   // qcomp pass 2 decisions
};

__device__ __forceinline__ int64_t group_exp(int64_t c, int32_t ka, int32_t kb, int64_t ea, int64_t eb) {
  return c + (ka ? ea : 0) + (kb ? eb : 0);
}

// bitlen(a1 2^diff + a2) + 1 + e2 for 0 <= diff < 64 in 128-bit arithmetic (out of line: the sums
// that do not fit 63 bits)
static __device__ __noinline__ int64_t gamma_msb_wide(uint64_t a1, uint64_t a2, int64_t diff, int64_t e2) {
  const u128 s = ((u128)a1 << diff) + (u128)a2;
  return (int64_t)bitlen_u128(s) + 1 + e2;
}

// msb(gamma_m) + e_gamma for gamma = sum of two non-negative dyadics (exact).  The terms are
// ordered so that the first is non-zero and the second is zero or has the lower exponent; a second
// term below 2^e1 (gap >= 64) cannot change the bit length; otherwise the aligned sum is taken in
// 64 bits when it stays below 2^63, else in 128 bits.
__device__ __forceinline__ bool gamma_msb(uint64_t a1, int64_t e1, uint64_t a2, int64_t e2, int64_t* out) {
  const bool swp = a1 == 0 || (a2 != 0 && e1 < e2);
  const uint64_t A = swp ? a2 : a1, Bv = swp ? a1 : a2;
  const int64_t EA = swp ? e2 : e1, EB = swp ? e1 : e2;
  if (A == 0) return false;
  const int64_t diff = EA - EB;
  if (Bv == 0 || diff >= 64) { *out = (int64_t)(65 - __clzll((long long)A)) + EA; return true; }
  if (diff <= 62 && (A >> (62 - diff)) == 0 && (Bv >> 62) == 0) {
    *out = (int64_t)(65 - __clzll((long long)((A << diff) + Bv))) + EB;
    return true;
  }
  *out = gamma_msb_wide(A, Bv, diff, EB);
  return true;
}

// Plan from the input exponents (ea, eb) and max-|m| norms (na, nb).
__device__ __forceinline__ void build_plan_v(const QDesc& q, int64_t ea, int64_t na, int64_t eb, int64_t nb, Plan& p) {
  int64_t Eh = group_exp(q.ch, q.ha, q.hb, ea, eb);
  p.two = q.two;
  p.mode = q.mode;
  p.w_out = q.w_out;
  p.w_tmp = q.w_tmp;
  p.use_tmp = q.use_tmp;
  p.overflow = p.underflow = p.narrow = 0;
  if (q.two) {
    int64_t El = group_exp(q.cl, q.la, q.lb, ea, eb);
    int64_t d = Eh - El;
    p.top_is_h = d >= 0;
    int64_t D = d >= 0 ? d : -d;
    int64_t Etop = d >= 0 ? Eh : El, Ebot = d >= 0 ? El : Eh;
    int topbits = d >= 0 ? q.hbits : q.lbits;
    p.e_star = Ebot;
    p.Eb = Ebot;
    if (D <= kGuard) {
      p.s_top = (int32_t)D; p.s_bot = 0; p.Ez = Ebot; p.guarded = 0;
      p.wide = (topbits + (int)D > 62) ? 1 : 0;
    } else {
      int64_t sb = D - kGuard;
      p.s_top = kGuard; p.s_bot = (int32_t)(sb > 63 ? 63 : sb); p.Ez = Etop - kGuard;
      p.guarded = 1; p.wide = 1;
    }
  } else {
    p.top_is_h = 1; p.s_top = 0; p.s_bot = 0; p.Ez = Eh; p.Eb = Eh; p.e_star = Eh;
    p.guarded = 0; p.wide = 0;
  }
  // gamma (Table tab:estimates rules or the caller's bound)
  int64_t G;
  bool nz;
  if (q.has_gamma) {
    nz = gamma_msb(q.gamma_m < 0 ? (uint64_t)(-q.gamma_m) : (uint64_t)q.gamma_m, q.gamma_e, 0, 0, &G);
  } else {
    uint64_t a[2] = {0, 0};
    int64_t e[2] = {0, 0};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (k < q.ng) {
        uint64_t nrm = (uint64_t)(q.gv[k] == 0 ? na : nb);
        int64_t ev = q.gv[k] == 0 ? ea : eb;
        a[k] = q.gm[k] * nrm;
        e[k] = q.ge[k] + ev;
      }
    }
    nz = gamma_msb(a[0], e[0], a[1], e[1], &G);
  }
  p.Gam = nz ? G : p.e_star + 1;   // gamma = 0 read as the zero scalar with exponent e*
  p.e_out = p.Gam - q.w_out;       // Alg. nnqcomp: lambda_out = mu_out - w_out
  p.e_tmp = p.Gam - q.w_tmp;       // Alg. qcomp: lambda_tmp = mu_tmp - w_tmp
}

__device__ __forceinline__ void build_plan(const QDesc& q, Plan& p) {
  build_plan_v(q, q.meta_a ? q.meta_a[0] : 0, q.meta_a ? q.meta_a[1] : 0, q.meta_b ? q.meta_b[0] : 0,
               q.meta_b ? q.meta_b[1] : 0, p);
}

// Completes the plan of qcomp's second pass from mu* (the atomic max key).
__device__ __forceinline__ void plan_from_mu(Plan& p, int64_t key) {
  // key 0: no element (empty block) -> mu* = 1 at e* (the initial value of Alg. qcomp)
  int64_t mu_abs = key >= 256 ? p.Ez + (key - 256) : (key > 0 ? p.Eb + key : p.e_star + 1);
  p.e_out = mu_abs - p.w_out;
  p.overflow = p.Gam < mu_abs;                           // mu_tmp < mu*
  p.underflow = (mu_abs - p.w_out) < (p.Gam - p.w_tmp);  // lambda_out < lambda_tmp
  p.narrow = p.use_tmp && !p.guarded && !p.overflow && !p.underflow;
}

// The meta words a plan reads: exponent and max |m| of each input, and the first pass's mu* key for
// qcomp's second pass (absent inputs read 0).  Loaded by one thread with loads that stay where they
// are written: the staged kernels issue them ahead of their ring's first copies, so the round trip
// overlaps those copies instead of following them.
struct MetaIn {
  int64_t ea, na, eb, nb, mu;
};
__device__ __forceinline__ int64_t ld_meta(const int64_t* p) {
  int64_t v;
  asm volatile("ld.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ MetaIn load_meta(const QDesc& q, bool with_mu) {
  MetaIn m = {0, 0, 0, 0, 0};
  if (q.meta_a) { m.ea = ld_meta(q.meta_a); m.na = ld_meta(q.meta_a + 1); }
  if (q.meta_b) { m.eb = ld_meta(q.meta_b); m.nb = ld_meta(q.meta_b + 1); }
  if (with_mu) m.mu = ld_meta(q.meta_out + kMetaMu);
  return m;
}
// build_plan from preloaded meta words, then plan_from_mu for qcomp's second pass
__device__ __forceinline__ void build_plan_m(const QDesc& q, const MetaIn& m, bool with_mu, Plan& p) {
  build_plan_v(q, m.ea, m.na, m.eb, m.nb, p);
  if (with_mu) plan_from_mu(p, m.mu);
}

// Register-resident fast path of one op: valid when the exact integer
// Z = (H << dh) + (L << dl) fits in int64 (no wide / guarded combine) and the
// output (or window) exponent is at or above Ez, so every element needs only
// shifts by uniform amounts, a clamp and a bit width.
struct Fast {
  int32_t ok;           // fast path usable
  int32_t dh, dl;       // left shifts of H and L into Z (one of them is 0)
  int32_t t;            // Z >> t gives the result (pass 2 / nnqcomp) or the window (pass 1)
  int32_t tl;           // pass 1 with the window below Ez: the window is the low w bits of Z << tl (t = 0)
  int32_t w;            // width that result / window is reduced to
  int32_t clamp;        // nnqcomp saturation (qcomp results fit by construction)
};

__device__ __forceinline__ Fast make_fast(const Plan& p, bool pass1) {
  Fast f;
  const int64_t t = pass1 ? (p.e_tmp - p.Ez) : (p.e_out - p.Ez);
  // qcomp's first pass keeps decr(w_tmp, z* >> lambda_tmp); when lambda_tmp is below the exact result's
  // exponent that is a left shift, whose low w_tmp bits come from the low bits of Z alone
  const bool left = pass1 && p.use_tmp && t < 0 && t >= -31;
  f.ok = (!p.wide && !p.guarded && (t >= 0 || left || (pass1 && !p.use_tmp))) ? 1 : 0;
  f.tl = left ? (int32_t)(-t) : 0;
  f.dh = (p.two && p.top_is_h) ? p.s_top : 0;
  f.dl = (p.two && !p.top_is_h) ? p.s_top : 0;
  f.t = (int32_t)(t < 0 ? 0 : (t > 63 ? 63 : t));
  f.w = pass1 ? p.w_tmp : p.w_out;
  f.clamp = (!pass1 && p.mode == kNnqcomp) ? 1 : 0;
  return f;
}

// ---------------------------------------------------------------------------
// Per-element steps
// ---------------------------------------------------------------------------

template <class Acc>
__device__ __forceinline__ Acc combine(int64_t H, int64_t L, const Plan& p) {
  if (!p.two) return (Acc)H;
  int64_t T = p.top_is_h ? H : L, B = p.top_is_h ? L : H;
  return shl_exact((Acc)T, p.s_top) + (Acc)(B >> p.s_bot);
}

// Key for the block maximum of qcomp's first pass (one atomic-max per CTA).
template <class Acc>
__device__ __forceinline__ int mu_key(Acc Z, int64_t H, int64_t L, const Plan& p) {
  if (!p.guarded) return 256 + msb_acc(Z);
  int64_t T = p.top_is_h ? H : L, B = p.top_is_h ? L : H;
  return T != 0 ? 256 + msb_acc(Z) : msb64(B);
}

// floor(Z * 2^-t) narrowed to X_w (saturating); sat set when clamped.
// (R: the mantissa type, int32_t, or int64_t for outputs of 33..62 bits.)
template <class Acc, class R = int32_t>
__device__ __forceinline__ R narrow_sat(Acc Z, int64_t t, int w, int& sat) {
  const int64_t hi = (1ll << (w - 1)) - 1, lo = -(1ll << (w - 1));
  if (t >= 0) {
    Acc v = shr_floor(Z, t);
    if (v > (Acc)hi) { ++sat; return (R)hi; }
    if (v < (Acc)lo) { ++sat; return (R)lo; }
    return (R)v;
  }
  if (Z == 0) return 0;
  int64_t k = -t;
  if (k >= 64 || msb_acc(Z) + k > w) { ++sat; return Z < 0 ? (R)lo : (R)hi; }
  return (R)((int64_t)Z << k);
}

// Output mantissa at the plan's e_out (nnqcomp, or qcomp recompute).
template <class Acc, class R = int32_t>
__device__ __forceinline__ R finish(Acc Z, int64_t H, int64_t L, const Plan& p, int& sat) {
  int64_t t = p.e_out - p.Ez;
  if (!p.guarded || t >= 0) return narrow_sat<Acc, R>(Z, t, p.w_out, sat);
  int64_t T = p.top_is_h ? H : L, B = p.top_is_h ? L : H;
  if (T != 0) {  // |z*| >= 2^(Ez+63) > 2^(e_out + w_out): saturates
    ++sat;
    return T < 0 ? (R)(-(1ll << (p.w_out - 1))) : (R)((1ll << (p.w_out - 1)) - 1);
  }
  return narrow_sat<int64_t, R>((int64_t)B, p.e_out - p.Eb, p.w_out, sat);
}

// qcomp window value decr(w* - w_tmp, z* >> lambda_tmp) at exponent e_tmp.
template <class Acc>
__device__ __forceinline__ int32_t window(Acc Z, const Plan& p) {
  return wrap_bits(low_shift(Z, p.e_tmp - p.Ez), p.w_tmp);
}

// ---------------------------------------------------------------------------
// Block reductions and the epilogue shared by all quantised kernels
// ---------------------------------------------------------------------------

struct Red {
  long long key;      // max mu key (pass 1)
  long long nrm;      // max |m_out|
  long long sat;      // saturated count
};

__device__ __forceinline__ long long warp_max(long long v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ long long warp_sum(long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reduces (key, nrm, sat) over the block and commits them with one atomic each.
// Must be called by every thread of the block.
__device__ __forceinline__ void block_commit(Red r, int64_t* meta_out, uint64_t* stats, bool pass1) {
  __shared__ long long s_key[32], s_nrm[32], s_sat[32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  r.key = warp_max(r.key);
  r.nrm = warp_max(r.nrm);
  r.sat = warp_sum(r.sat);
  if (lane == 0) { s_key[wid] = r.key; s_nrm[wid] = r.nrm; s_sat[wid] = r.sat; }
  __syncthreads();
  if (wid == 0) {
    long long k = lane < nw ? s_key[lane] : LLONG_MIN;
    long long n = lane < nw ? s_nrm[lane] : 0;
    long long s = lane < nw ? s_sat[lane] : 0;
    k = warp_max(k); n = warp_max(n); s = warp_sum(s);
    if (lane == 0) {
      if (pass1) {
        atomicMax((long long*)&meta_out[kMetaMu], k);
      } else {
        if (n > 0) atomicMax((long long*)&meta_out[1], n);
        if (s > 0 && stats) atomicAdd((unsigned long long*)&stats[4], (unsigned long long)s);
      }
    }
  }
}

}  // namespace bfp
