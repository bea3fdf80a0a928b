// bfp_coarse.cuh -- the coarse end of the V-cycle on one SM.
//
// Below a few hundred thousand points a level's ops are dominated by launch
// and round-trip latency, and the coarsest level's 32 sweeps would be 32
// launches.  One CTA instead runs every level from n_c (<= 127) down to 3 in
// shared memory: the host flattens the recursive schedule of Alg. v-cycle
// (exactly the order the global driver uses) into a list of ops; the CTA
// executes the list.  Each op builds its plan from the same QDesc the C ABI op
// would use and quantises through the same device arithmetic (combine /
// mu_key / finish), so the result is bit-identical to running the ops one by
// one.  qcomp's second pass always recomputes (the window is only a cache);
// its overflow / underflow counts are still those of Alg. qcomp.
//
// Synchronisation: every thread plans each op in registers, so an nnqcomp op
// costs one block barrier (qcomp two).  Ops on levels with n <= 15 run on warp
// 0 alone with warp reductions while the other warps wait at the next
// full-block op.
//
// Buffers are stored with a zero halo: point (i, j) of an n x n level sits at
// (j + 1)(n + 2) + i + 1, so no neighbour, restriction or interpolation read
// needs a bounds test.
#pragma once

#include <type_traits>

#include "bfp_host.h"

namespace bfp {

enum CoarseKind : int32_t { cJac0 = 0, cJac = 1, cRes = 2, cRestrict = 3, cProlong = 4,
                            cVarJac0 = 5, cVarJac = 6,   // these two: the coarsest-level run only
                            cCheb = 7 };   // host side only: built as a cJac op (T r, reading r for y)

struct CoarseOp {
  int32_t kind;
  int32_t a, b, out;     // buffer ids (-1: none)
  int32_t solo;          // run by warp 0 alone
  int32_t sync_before;   // first full-block op after a run of solo ops
  int32_t run;           // on the op at CoarseArgs::run_k: the number of identical solo sweeps (on a
                         // level of <= 32 points, alternating between buffers a and out) it starts
  int64_t c, nb, mw;     // stencil / smoother coefficients
  // the folded multipliers k0, k1, k2 of the int16 register path (set by set_fold_consts): k_i =
  // fc[i] 2^dl when bit i of fsel is set, else fc[i] 2^dh; valid while that shift is <= flim[i]
  int32_t fc[3], flim[3], fsel;
  QDesc q;               // static description (meta pointers unused)
};

// Host: the folded-multiplier constants of an op from its kind and coefficients.  A coefficient c
// shifted left by sh stays exact in int32 up to flim = the largest sh <= 30 with (c 2^sh) >> sh == c
// (the bound only grows down to sh = 0); c = 0 folds at any shift.
inline void set_fold_consts(CoarseOp& op) {
  const int32_t c = (int32_t)op.c, nb = (int32_t)op.nb, mw = (int32_t)op.mw;
  int32_t fc[3] = {0, 0, 0}, fsel = 0;
  switch (op.kind) {
    case cJac0: fc[0] = mw; break;
    case cJac: fc[0] = c; fc[1] = nb; fc[2] = mw; fsel = 4; break;
    case cRes: fc[0] = c; fc[1] = nb; fc[2] = -1; fsel = 4; break;
    case cRestrict: fc[0] = 1; break;
    default: fc[0] = -1; fc[2] = 1; fsel = 4; break;   // prolongation with correction
  }
  for (int i = 0; i < 3; ++i) {
    int lim = 0x7fffffff;
    if (fc[i] != 0) {
      lim = 0;
      for (int sh = 1; sh <= 30; ++sh) {
        if ((int32_t)((uint32_t)fc[i] << sh) >> sh != fc[i]) break;
        lim = sh;
      }
    }
    op.fc[i] = fc[i];
    op.flim[i] = lim;
  }
  op.fsel = fsel;
}

struct CoarseBuf {
  int32_t off;           // byte offset of the (n + 2)^2 padded buffer in dynamic shared memory
  int32_t n;             // points per side
};

struct CoarseArgs {
  const CoarseOp* ops;
  const CoarseBuf* bufs;
  int32_t nops, nbufs;
  int32_t run_k;         // first op of the coarsest level's sweep run (nops: none)
  int32_t meta_off;      // byte offsets in dynamic shared memory: meta blocks,
  int32_t ops_off;       // the op list (copied in at start),
  int32_t bufs_off;      // the buffer table
  int32_t data_off;      // and the mantissa buffers (up to smem_bytes)
  int32_t smem_bytes;
  VIn rin;               // level n_c right-hand side (global) ...
  const int64_t* rin_meta;
  int32_t rin_buf;       // ... and the buffer it is loaded into
  VOut yout;             // level n_c result (global) ...
  int64_t* yout_meta;
  int32_t yout_buf;      // ... read from this buffer (set by the schedule)
  uint64_t* stats;
};

// W: a type wide enough for sums of 16 mantissas of T
template <class T>
struct CoarseView {
  using W = typename std::conditional<sizeof(T) == 2, int32_t, int64_t>::type;
  T* p;
  int s;                 // row stride n + 2
  __device__ __forceinline__ W operator()(int i, int j) const { return (W)p[(j + 1) * s + i + 1]; }
  __device__ __forceinline__ void put(int i, int j, int32_t v) const { p[(j + 1) * s + i + 1] = (T)v; }
};

template <class T>
__device__ __forceinline__ CoarseView<T> cview(unsigned char* sm, const CoarseBuf& b) {
  return CoarseView<T>{reinterpret_cast<T*>(sm + b.off), b.n + 2};
}

// General (wide / guarded / below-Ez) quantisation of one element, out of line.
__device__ __noinline__ long long coarse_key_general(int64_t H, int64_t L, const Plan* pp) {
  const Plan& p = *pp;
  if (p.wide) {
    const i128 Z = combine<i128>(H, L, p);
    return mu_key<i128>(Z, H, L, p);
  }
  const int64_t Z = combine<int64_t>(H, L, p);
  return mu_key<int64_t>(Z, H, L, p);
}

// value in the low 32 bits, saturation count above
__device__ __noinline__ int64_t coarse_val_general(int64_t H, int64_t L, const Plan* pp) {
  const Plan& p = *pp;
  int sat = 0;
  int32_t v;
  if (p.wide) {
    const i128 Z = combine<i128>(H, L, p);
    v = finish<i128>(Z, H, L, p, sat);
  } else {
    const int64_t Z = combine<int64_t>(H, L, p);
    v = finish<int64_t>(Z, H, L, p, sat);
  }
  return (int64_t)(uint32_t)v | ((int64_t)sat << 32);
}

// int16 register path: Z is a sum of at most three products k_s * P_s of int32
// multipliers (the op's coefficients with the group shifts dh / dl folded in)
// and int32 partial sums P_s of mantissas, each one mul.wide; the result is
// the low word of Z >> t, saturated through one range test on Z.
struct CoarseMul {
  int32_t ok;
  int32_t k0, k1, k2;   // multipliers of the partial sums (see coarse_pass16)
  int32_t t;            // Z >> t gives the result
  int32_t clamp;        // nnqcomp saturation test active
  int32_t vlo, vhi;     // X_w bounds
  int64_t zmin;         // vlo 2^t
  uint64_t zrange;      // 2^(w + t): Z in range iff Z - zmin < zrange (unsigned)
};

__device__ __forceinline__ CoarseMul make_mul(const Fast& f, const CoarseOp& op) {
  CoarseMul m;
  m.k0 = m.k1 = m.k2 = 0;
  m.t = f.t;
  const int32_t w = f.w > 32 ? 32 : f.w;
  m.vhi = (int32_t)((1u << (w - 1)) - 1u);
  m.vlo = -m.vhi - 1;
  const int32_t e = f.w + f.t;                // the range is [vlo 2^t, (vhi + 1) 2^t)
  m.clamp = f.clamp && e <= 63;               // beyond that every int64 Z is in range
  const uint32_t lo = e < 32 ? (1u << (e & 31)) : 0u, hi = e < 32 ? 0u : (1u << ((e - 32) & 31));
  m.zrange = m.clamp ? (((uint64_t)hi << 32) | lo) : 0;
  m.zmin = -(int64_t)(m.zrange >> 1);
  const int32_t s0 = (op.fsel & 1) ? f.dl : f.dh, s1 = (op.fsel & 2) ? f.dl : f.dh, s2 = (op.fsel & 4) ? f.dl : f.dh;
  m.k0 = (int32_t)((uint32_t)op.fc[0] << (s0 & 31));
  m.k1 = (int32_t)((uint32_t)op.fc[1] << (s1 & 31));
  m.k2 = (int32_t)((uint32_t)op.fc[2] << (s2 & 31));
  const bool ok = s0 <= op.flim[0] && s1 <= op.flim[1] && s2 <= op.flim[2];
  m.ok = (ok && f.ok && f.w <= 32) ? 1 : 0;
  return m;
}

// What every thread needs to run one pass of an op (built once per pass by one thread).
struct CoarseExec {
  Fast f;
  CoarseMul m;
};

// Columns per thread and row: n <= 127 with 32 lanes, or n <= 15 with 16.
constexpr int kCoarseCols = 4;
constexpr int kCoarseThreads = 512;

struct CoarseRes {
  long long key, nrm;
  int sat;
};

// The general pass (any storage type, any plan), kept out of line: it runs only
// for int32 storage or when the int16 register path does not apply.
template <class T, int KIND, bool PASS1>
__device__ __noinline__ CoarseRes coarse_pass_any(unsigned char* sm, const CoarseOp& op, const CoarseBuf bo,
                                                  const CoarseBuf* bufs, const Fast f, const Plan* pp, int i0,
                                                  int istep, int j0, int jstep) {
  long long key = 0, nrm = 0;
  int sat = 0;
  const int n = bo.n;
  const CoarseView<T> O = cview<T>(sm, bo);
  const CoarseView<T> A = cview<T>(sm, bufs[op.a >= 0 ? op.a : op.out]);
  const CoarseView<T> B = cview<T>(sm, bufs[op.b >= 0 ? op.b : op.out]);
  const int64_t c = op.c, nbc = op.nb, mw = op.mw;
  const int64_t hi = (1ll << (f.w - 1)) - 1, lo = -(1ll << (f.w - 1));
  using W = typename CoarseView<T>::W;
  for (int j = j0; j < n; j += jstep) {
    for (int u = 0; u < kCoarseCols; ++u) {
      const int i = i0 + u * istep;
      if (i >= n) break;
      int64_t H, L;
      if (KIND == cJac0) {
        H = mw * B(i, j);
        L = 0;
      } else if (KIND == cJac || KIND == cRes) {
        const int64_t ns = (int64_t)(A(i - 1, j) + A(i + 1, j)) + (A(i, j - 1) + A(i, j + 1));
        H = c * A(i, j) + nbc * ns;
        L = KIND == cJac ? mw * B(i, j) : -(int64_t)B(i, j);
      } else if (KIND == cRestrict) {
        const int fi = 2 * i + 1, fj = 2 * j + 1;
        const W r0 = A(fi - 1, fj - 1) + 2 * A(fi, fj - 1) + A(fi + 1, fj - 1);
        const W r1 = A(fi - 1, fj) + 2 * A(fi, fj) + A(fi + 1, fj);
        const W r2 = A(fi - 1, fj + 1) + 2 * A(fi, fj + 1) + A(fi + 1, fj + 1);
        H = (int64_t)r0 + 2 * (int64_t)r1 + r2;
        L = 0;
      } else {
        auto g = [&](int J) -> W {
          return (i & 1) ? 2 * A((i - 1) >> 1, J) : A((i >> 1) - 1, J) + A(i >> 1, J);
        };
        const W pd = (j & 1) ? 2 * g((j - 1) >> 1) : g((j >> 1) - 1) + g(j >> 1);
        H = -(int64_t)pd;
        L = B(i, j);
      }
      if (f.ok) {
        const int64_t Z = (int64_t)((uint64_t)H << f.dh) + (int64_t)((uint64_t)L << f.dl);
        if (PASS1) {
          key = max(key, (long long)(256 + msb64(Z)));
        } else {
          int64_t t = Z >> f.t;
          if (f.clamp) {
            if (t > hi) { t = hi; ++sat; } else if (t < lo) { t = lo; ++sat; }
          }
          O.put(i, j, (int32_t)t);
          nrm = max(nrm, (long long)(t < 0 ? -t : t));
        }
      } else if (PASS1) {
        key = max(key, coarse_key_general(H, L, pp));
      } else {
        const int64_t r = coarse_val_general(H, L, pp);
        const int32_t v = (int32_t)(uint32_t)r;
        sat += (int)(r >> 32);
        O.put(i, j, v);
        nrm = max(nrm, (long long)(v < 0 ? -(long long)v : (long long)v));
      }
    }
  }
  return CoarseRes{key, nrm, sat};
}

// One pass of one op over points (i0 + istep u, j0 + jstep v), u < kCoarseCols.
template <class T, int KIND, bool PASS1>
__device__ __forceinline__ void coarse_pass(unsigned char* sm, const CoarseOp& op, const CoarseBuf* bufs,
                                            const CoarseExec& ex, const Plan* pp, int i0, int istep, int j0,
                                            int jstep, long long& key, long long& nrm, int& sat) {
  const CoarseBuf bo = bufs[op.out];
  const int n = bo.n;
  if (sizeof(T) == 2 && ex.m.ok) {
    const CoarseMul& m = ex.m;
    const CoarseView<int16_t> O = cview<int16_t>(sm, bo);
    const CoarseView<int16_t> A = cview<int16_t>(sm, bufs[op.a >= 0 ? op.a : op.out]);
    const CoarseView<int16_t> B = cview<int16_t>(sm, bufs[op.b >= 0 ? op.b : op.out]);
    uint64_t ormag = 0;
    bool any = false;
    uint32_t nr = 0;
    for (int j = j0; j < n; j += jstep) {
#pragma unroll
      for (int u = 0; u < kCoarseCols; ++u) {
        const int i = i0 + u * istep;
        if (i >= n) break;
        int64_t z;
        if (KIND == cJac0) {
          z = (int64_t)m.k0 * B(i, j);
        } else if (KIND == cJac || KIND == cRes) {
          const int32_t ns = (A(i - 1, j) + A(i + 1, j)) + (A(i, j - 1) + A(i, j + 1));
          z = (int64_t)m.k0 * A(i, j) + (int64_t)m.k1 * ns + (int64_t)m.k2 * B(i, j);
        } else if (KIND == cRestrict) {
          // coarse (i, j) gathers fine (2i+1+dx, 2j+1+dy) with weights (2-|dx|)(2-|dy|)
          const int fi = 2 * i + 1, fj = 2 * j + 1;
          const int32_t r0 = A(fi - 1, fj - 1) + 2 * A(fi, fj - 1) + A(fi + 1, fj - 1);
          const int32_t r1 = A(fi - 1, fj) + 2 * A(fi, fj) + A(fi + 1, fj);
          const int32_t r2 = A(fi - 1, fj + 1) + 2 * A(fi, fj + 1) + A(fi + 1, fj + 1);
          z = (int64_t)m.k0 * (r0 + 2 * r1 + r2);
        } else {  // cProlong with correction: Z = -P_m d 2^dh + y 2^dl
          // fine i odd sits on coarse (i-1)/2 (weight 2); even i between i/2-1 and i/2
          auto g = [&](int J) -> int32_t {
            return (i & 1) ? 2 * A((i - 1) >> 1, J) : A((i >> 1) - 1, J) + A(i >> 1, J);
          };
          const int32_t pd = (j & 1) ? 2 * g((j - 1) >> 1) : g((j >> 1) - 1) + g(j >> 1);
          z = (int64_t)m.k0 * pd + (int64_t)m.k2 * B(i, j);
        }
        if (PASS1) {
          ormag |= (uint64_t)(z ^ (z >> 63));
          any = true;
        } else {
          const uint32_t zl = (uint32_t)z, zh = (uint32_t)((uint64_t)z >> 32);
          int32_t v = m.t < 32 ? (int32_t)__funnelshift_r(zl, zh, m.t) : ((int32_t)zh >> (m.t - 32));
          if (m.clamp && (uint64_t)(z - m.zmin) >= m.zrange) {
            v = z < 0 ? m.vlo : m.vhi;
            ++sat;
          }
          O.put(i, j, v);
          const uint32_t a = (uint32_t)(v < 0 ? -v : v);
          nr = a > nr ? a : nr;
        }
      }
    }
    if (PASS1 && any) key = max(key, (long long)(256 + (64 - __clzll((long long)ormag)) + 1));
    nrm = max(nrm, (long long)nr);
    return;
  }
  const CoarseRes r = coarse_pass_any<T, KIND, PASS1>(sm, op, bo, bufs, ex.f, pp, i0, istep, j0, jstep);
  key = max(key, r.key);
  nrm = max(nrm, r.nrm);
  sat += r.sat;
}

template <class T, bool PASS1>
__device__ __forceinline__ void coarse_dispatch(unsigned char* sm, const CoarseOp& op, const CoarseBuf* bufs,
                                                const CoarseExec& ex, const Plan* pp, int i0, int istep, int j0,
                                                int jstep, long long& key, long long& nrm, int& sat) {
  switch (op.kind) {
    case cJac0: coarse_pass<T, cJac0, PASS1>(sm, op, bufs, ex, pp, i0, istep, j0, jstep, key, nrm, sat); break;
    case cJac: coarse_pass<T, cJac, PASS1>(sm, op, bufs, ex, pp, i0, istep, j0, jstep, key, nrm, sat); break;
    case cRes: coarse_pass<T, cRes, PASS1>(sm, op, bufs, ex, pp, i0, istep, j0, jstep, key, nrm, sat); break;
    case cRestrict: coarse_pass<T, cRestrict, PASS1>(sm, op, bufs, ex, pp, i0, istep, j0, jstep, key, nrm, sat); break;
    default: coarse_pass<T, cProlong, PASS1>(sm, op, bufs, ex, pp, i0, istep, j0, jstep, key, nrm, sat); break;
  }
}

// Register plan of one op for the fast paths: the part of the full Plan that
// the passes and the meta block need, computed by every thread that runs the
// op (no shared-memory round trip, no barrier).  Exponents are handled in
// int32 (inputs within +-2^28).  Whenever the full plan would not take the
// fast path (wide or guarded groups, a result exponent below Ez) lean_first /
// lean_second return false and the op runs from the full Plan instead.
struct CoarseLean {
  int32_t Ez, Gam, e_out;
  int32_t D, top, two;
  int32_t ov, un;               // qcomp overflow / underflow of the second pass
};

__device__ __forceinline__ void lean_exec(const CoarseOp& op, const CoarseLean& L, int32_t t, int32_t w, bool pass1,
                                          bool clamp, CoarseExec& ex) {
  ex.f.ok = 1;
  ex.f.dh = (L.two && L.top) ? L.D : 0;
  ex.f.dl = (L.two && !L.top) ? L.D : 0;
  ex.f.t = t < 0 ? 0 : (t > 63 ? 63 : t);
  ex.f.tl = 0;                  // the on-chip cycle keeps no qcomp window
  ex.f.w = w;
  ex.f.clamp = (!pass1 && clamp) ? 1 : 0;
  ex.m = make_mul(ex.f, op);
}

__device__ __forceinline__ bool lean_first(const CoarseOp& op, int64_t ea64, int64_t na, int64_t eb64, int64_t nb,
                                           CoarseLean& L, CoarseExec& ex) {
  const QDesc& q = op.q;
  const int64_t lim = 1ll << 28;
  if (ea64 <= -lim || ea64 >= lim || eb64 <= -lim || eb64 >= lim) return false;
  const int32_t ea = (int32_t)ea64, eb = (int32_t)eb64;
  const int32_t Eh = (int32_t)q.ch + (q.ha ? ea : 0) + (q.hb ? eb : 0);
  const int32_t El = (int32_t)q.cl + (q.la ? ea : 0) + (q.lb ? eb : 0);
  L.two = q.two;
  const int32_t d = q.two ? Eh - El : 0;
  L.top = d >= 0;
  L.D = d >= 0 ? d : -d;
  L.Ez = (q.two && d > 0) ? El : Eh;
  const bool wide = q.two && ((L.top ? q.hbits : q.lbits) + L.D > 62);
  // gamma (Table tab:estimates rule) exactly as build_plan_v
  const uint64_t a0 = q.gm[0] * (uint64_t)(q.gv[0] == 0 ? na : nb);
  const int64_t e0 = q.ge[0] + (q.gv[0] == 0 ? ea : eb);
  uint64_t a1 = 0;
  int64_t e1 = 0;
  if (q.ng > 1) {
    a1 = q.gm[1] * (uint64_t)(q.gv[1] == 0 ? na : nb);
    e1 = q.ge[1] + (q.gv[1] == 0 ? ea : eb);
  }
  int64_t G = 0;
  const bool nz = gamma_msb(a0, e0, a1, e1, &G);
  L.Gam = nz ? (int32_t)G : L.Ez + 1;
  L.e_out = L.Gam - q.w_out;
  L.ov = L.un = 0;
  const bool qc = q.mode == kQcomp;
  const int32_t t = qc ? (L.Gam - q.w_tmp) - L.Ez : L.e_out - L.Ez;
  if (wide || (!qc && t < 0) || q.has_gamma || q.use_tmp) return false;
  lean_exec(op, L, t, qc ? q.w_tmp : q.w_out, qc, q.mode == kNnqcomp, ex);
  return true;
}

// qcomp: the second pass from the block maximum key (plan_from_mu with Eb = e* = Ez)
__device__ __forceinline__ bool lean_second(const CoarseOp& op, int32_t key, CoarseLean& L, CoarseExec& ex) {
  const QDesc& q = op.q;
  const int32_t mu = key >= 256 ? L.Ez + (key - 256) : (key > 0 ? L.Ez + key : L.Ez + 1);
  L.e_out = mu - q.w_out;
  L.ov = L.Gam < mu;
  L.un = L.e_out < L.Gam - q.w_tmp;
  const int32_t t = L.e_out - L.Ez;
  if (t < 0) return false;
  lean_exec(op, L, t, q.w_out, false, false, ex);
  return true;
}

struct CoarseCounts {
  unsigned long long calls, recomputed, overflow, underflow;
  __device__ __forceinline__ void add(bool ov, bool un, bool qc) {
    calls += 1;
    if (qc) {
      if (ov || un) recomputed += 1;
      if (ov) overflow += 1;
      if (un) underflow += 1;
    }
  }
};

// A run of damped-Jacobi sweeps on a level of n x n <= 32 points, on warp 0
// with the grid in registers (lane l holds point (l mod n, l / n); neighbours
// by shuffles).  Every sweep plans and quantises exactly as the general loop's
// int16 register path (lean plan, Z = k0 y + k1 (W + E + S + N) + k2 r, one
// shift, the nnqcomp range test, qcomp's block-maximum key); the meta block is
// written once, for the run's last output.  A sweep whose plan leaves that
// path stops the run: its input goes to shared memory and the general loop
// takes over from it.  Out of line (and with results returned by value): the
// main loop keeps its own register allocation.
struct CoarseRun {
  int32_t done;          // sweeps done
  int32_t prev;          // buffer holding their result (the next op's input), meta in (pe, pn)
  int64_t pe, pn;
  int32_t sat;           // this lane's saturated elements
  CoarseCounts cnt;      // thread 0: the sweeps' counters
};

__device__ __noinline__ CoarseRun coarse_sweep_run(unsigned char* sm, const CoarseOp* op0, const CoarseBuf* bufs,
                                                   int64_t* metas, int64_t ea, int64_t na, int64_t eb, int64_t nb) {
  CoarseRun res;
  res.done = 0; res.prev = -1; res.pe = 0; res.pn = 0; res.sat = 0;
  res.cnt = CoarseCounts{0, 0, 0, 0};
  CoarseCounts& cnt = res.cnt;
  int sat = 0;
  const CoarseOp op = *op0;                      // register copy: every sweep has the same descriptor
  const int lane = threadIdx.x & 31;
  const int n = bufs[op.out].n;
  const bool act = lane < n * n;
  const int i = act ? lane % n : 0, j = act ? lane / n : 0;
  const bool hw = act && i > 0, he = act && i + 1 < n, hs = act && j > 0, hn = act && j + 1 < n;
  const int32_t bv = act ? (int32_t)cview<int16_t>(sm, bufs[op.b])(i, j) : 0;
  int32_t y = act ? (int32_t)cview<int16_t>(sm, bufs[op.a])(i, j) : 0;
  const bool qc = op.q.mode == kQcomp;
  int bin = op.a, bout = op.out;
  int r = 0;
  for (; r < op.run; ++r) {
    CoarseLean L;
    CoarseExec ex;
    if (!lean_first(op, ea, na, eb, nb, L, ex) || !ex.m.ok) break;
    const int32_t wv = __shfl_sync(0xffffffffu, y, hw ? lane - 1 : lane);
    const int32_t ev = __shfl_sync(0xffffffffu, y, he ? lane + 1 : lane);
    const int32_t sv = __shfl_sync(0xffffffffu, y, hs ? lane - n : lane);
    const int32_t nv = __shfl_sync(0xffffffffu, y, hn ? lane + n : lane);
    const int32_t ns = ((hw ? wv : 0) + (he ? ev : 0)) + ((hs ? sv : 0) + (hn ? nv : 0));
    if (qc) {
      const int64_t z1 = (int64_t)ex.m.k0 * y + (int64_t)ex.m.k1 * ns + (int64_t)ex.m.k2 * bv;
      const uint64_t om = (uint64_t)(z1 ^ (z1 >> 63));
      const unsigned key = act ? (unsigned)(256 + (64 - __clzll((long long)om)) + 1) : 0u;
      const unsigned kk = __reduce_max_sync(0xffffffffu, key);
      if (!lean_second(op, (int32_t)kk, L, ex) || !ex.m.ok) break;
    }
    const CoarseMul& m = ex.m;
    const int64_t z = (int64_t)m.k0 * y + (int64_t)m.k1 * ns + (int64_t)m.k2 * bv;
    const uint32_t zl = (uint32_t)z, zh = (uint32_t)((uint64_t)z >> 32);
    int32_t v = m.t < 32 ? (int32_t)__funnelshift_r(zl, zh, m.t) : ((int32_t)zh >> (m.t - 32));
    const bool out = m.clamp && (uint64_t)(z - m.zmin) >= m.zrange;
    v = out ? (z < 0 ? m.vlo : m.vhi) : v;
    sat += (out && act) ? 1 : 0;
    v = act ? v : 0;
    const unsigned nn = __reduce_max_sync(0xffffffffu, (unsigned)(v < 0 ? -v : v));
    y = v;
    cnt.add(L.ov != 0, L.un != 0, qc);           // every lane (thread 0's copy is the one kept)
    ea = L.e_out;
    na = (int64_t)nn;
    const int t = bin;
    bin = bout;
    bout = t;
  }
  // y is the input of sweep r (the output of sweep r - 1, or the run's input when r == 0)
  if (r > 0) {
    if (act) cview<int16_t>(sm, bufs[bin]).put(i, j, y);
    if (threadIdx.x == 0) {
      metas[bin * BFP_META_WORDS] = ea;
      metas[bin * BFP_META_WORDS + 1] = na;
    }
    __syncwarp();
  }
  res.done = r;
  res.prev = bin;
  res.pe = ea;
  res.pn = na;
  res.sat = sat;
  return res;
}

// The smoothing of a coarsest level with n^d <= 32 points (int16 mantissas)
// when it runs from global memory (3D, or 2D without the on-chip cycle): the
// level's first sweep from y = 0 and its remaining sweeps in one launch of one
// warp, the grid in registers (lane l holds point (l mod n, (l / n) mod n,
// l / n^2)).  Each sweep follows the on-chip schedule's ops exactly: the lean
// plan and folded multipliers when they apply, else the full plan and the
// general per-element quantiser; qcomp's second pass recomputes.  Only the last
// result, its meta block (e, max |m|) and the counters are written.
struct SweepRunArgs {
  CoarseOp op0, op1;     // damped Jacobi from y = 0, and from y
  int32_t sweeps, n, nd;
  int32_t var;           // variable coefficients (2D): per-point faces kf and weights kq, H = y 2^s - q A'y
  int32_t s;
  VIn kf[4], kq;
  VIn r;                 // right-hand side of the level
  const int64_t* r_meta;
  VOut y;                // result (padding columns written as 0)
  int64_t* y_meta;
  uint64_t* stats;
};

template <bool B>
__global__ void __launch_bounds__(32) k_sweep_run(const __grid_constant__ SweepRunArgs A1,
                                                  const SweepRunArgs* __restrict__ Ab) {
  pdl_wait();
  const SweepRunArgs& a = B ? Ab[blockIdx.z] : A1;
  const int lane = threadIdx.x;
  const int n = a.n, nn = n * n, np = a.nd == 3 ? nn * n : nn;
  const bool act = lane < np;
  const int i = act ? lane % n : 0, j = act ? (lane / n) % n : 0, k = act ? lane / nn : 0;
  const bool hw = act && i > 0, he = act && i + 1 < n, hs = act && j > 0, hn = act && j + 1 < n;
  const bool hb = act && a.nd == 3 && k > 0, ht = act && a.nd == 3 && k + 1 < n;
  const int64_t row = (int64_t)j + (int64_t)n * k;
  const int32_t bv = act ? (int32_t)reinterpret_cast<const int16_t*>(a.r.m)[row * a.r.ld + i] : 0;
  auto kld = [&](const VIn& v) -> int32_t {
    return (a.var && act) ? (int32_t)reinterpret_cast<const int16_t*>(v.m)[row * v.ld + i] : 0;
  };
  const int32_t fw = kld(a.kf[0]), fe = kld(a.kf[1]), fs = kld(a.kf[2]), fn = kld(a.kf[3]), qv = kld(a.kq);
  const int64_t eb = a.r_meta[0], nb = a.r_meta[1];
  int64_t ea = 0, na = 0;
  int32_t y = 0;
  int sat = 0;
  CoarseCounts cnt = {0, 0, 0, 0};
  for (int sw = 0; sw < a.sweeps; ++sw) {
    const CoarseOp& op = sw == 0 ? a.op0 : a.op1;
    const bool qc = op.q.mode == kQcomp;
    // neighbour sum of y (the first sweep has no y)
    const int32_t wv = __shfl_sync(0xffffffffu, y, hw ? lane - 1 : lane);
    const int32_t ev = __shfl_sync(0xffffffffu, y, he ? lane + 1 : lane);
    const int32_t sv = __shfl_sync(0xffffffffu, y, hs ? lane - n : lane);
    const int32_t nv = __shfl_sync(0xffffffffu, y, hn ? lane + n : lane);
    const int32_t bz = __shfl_sync(0xffffffffu, y, hb ? lane - nn : lane);
    const int32_t tz = __shfl_sync(0xffffffffu, y, ht ? lane + nn : lane);
    const int32_t ns = (((hw ? wv : 0) + (he ? ev : 0)) + ((hs ? sv : 0) + (hn ? nv : 0))) +
                       ((hb ? bz : 0) + (ht ? tz : 0));
    int64_t H, Lg;
    if (a.var) {       // y 2^s - q (c y - sum k_f y_f) and q r (q r alone on the first sweep)
      const int64_t ay = ((int64_t)fw + fe + fs + fn) * y -
                         ((int64_t)fw * (hw ? wv : 0) + (int64_t)fe * (he ? ev : 0) + (int64_t)fs * (hs ? sv : 0) +
                          (int64_t)fn * (hn ? nv : 0));
      H = sw == 0 ? (int64_t)qv * bv : (int64_t)((uint64_t)(int64_t)y << a.s) - (int64_t)qv * ay;
      Lg = sw == 0 ? 0 : (int64_t)qv * bv;
    } else {
      H = sw == 0 ? op.mw * (int64_t)bv : op.c * (int64_t)y + op.nb * (int64_t)ns;
      Lg = sw == 0 ? 0 : op.mw * (int64_t)bv;
    }
    CoarseLean L;
    CoarseExec ex;
    Plan P;
    const bool lean0 = lean_first(op, ea, na, eb, nb, L, ex);
    bool lean = lean0;
    if (!lean) {
      build_plan_v(op.q, ea, na, eb, nb, P);
      ex.f = make_fast(P, qc);
      ex.m = make_mul(ex.f, op);
    }
    if (a.var) ex.m.ok = 0;   // folded multipliers need constant coefficients
    // Z on the register path (folded multipliers: the same value as (H << dh) + (L << dl))
    auto zreg = [&](const CoarseMul& m) -> int64_t {
      return sw == 0 ? (int64_t)m.k0 * bv : (int64_t)m.k0 * y + (int64_t)m.k1 * ns + (int64_t)m.k2 * bv;
    };
    if (qc) {
      long long key = 0;
      if (act) {
        if (ex.m.ok) {
          const int64_t z = zreg(ex.m);
          key = 256 + (64 - __clzll((long long)(uint64_t)(z ^ (z >> 63)))) + 1;
        } else if (ex.f.ok) {
          const int64_t Z = (int64_t)((uint64_t)H << ex.f.dh) + (int64_t)((uint64_t)Lg << ex.f.dl);
          key = 256 + msb64(Z);
        } else {
          key = coarse_key_general(H, Lg, &P);
        }
      }
      const unsigned kk = __reduce_max_sync(0xffffffffu, (unsigned)key);
      if (lean) lean = lean_second(op, (int32_t)kk, L, ex);
      if (!lean) {
        if (lean0) build_plan_v(op.q, ea, na, eb, nb, P);
        plan_from_mu(P, (int64_t)kk);
        ex.f = make_fast(P, false);
        ex.m = make_mul(ex.f, op);
      }
      if (a.var) ex.m.ok = 0;
    }
    int32_t v = 0;
    if (act) {
      if (ex.m.ok) {
        const CoarseMul& m = ex.m;
        const int64_t z = zreg(m);
        const uint32_t zl = (uint32_t)z, zh = (uint32_t)((uint64_t)z >> 32);
        v = m.t < 32 ? (int32_t)__funnelshift_r(zl, zh, m.t) : ((int32_t)zh >> (m.t - 32));
        if (m.clamp && (uint64_t)(z - m.zmin) >= m.zrange) {
          v = z < 0 ? m.vlo : m.vhi;
          ++sat;
        }
      } else if (ex.f.ok) {
        const int64_t Z = (int64_t)((uint64_t)H << ex.f.dh) + (int64_t)((uint64_t)Lg << ex.f.dl);
        const int64_t hi = (1ll << (ex.f.w - 1)) - 1, lo = -(1ll << (ex.f.w - 1));
        int64_t t = Z >> ex.f.t;
        if (ex.f.clamp) {
          if (t > hi) { t = hi; ++sat; } else if (t < lo) { t = lo; ++sat; }
        }
        v = (int32_t)t;
      } else {
        const int64_t rr = coarse_val_general(H, Lg, &P);
        v = (int32_t)(uint32_t)rr;
        sat += (int)(rr >> 32);
      }
    }
    const unsigned nrm = __reduce_max_sync(0xffffffffu, (unsigned)(v < 0 ? -v : v));
    cnt.add(lean ? L.ov != 0 : P.overflow != 0, lean ? L.un != 0 : P.underflow != 0, qc);
    ea = lean ? (int64_t)L.e_out : P.e_out;
    na = (int64_t)nrm;
    y = v;
  }
  // the result with its padding columns, the meta block, the counters
  const int rows = a.nd == 3 ? nn : n;
  const int64_t ld = a.y.ld, total = (int64_t)rows * ld;
  for (int64_t base = 0; base < total; base += 32) {
    const int64_t idx = base + lane;
    const int64_t rr = idx / ld, cc = idx - rr * ld;
    const int src = (int)(rr * n + (cc < n ? cc : 0));
    const int32_t val = __shfl_sync(0xffffffffu, y, src < 32 ? src : 0);
    if (idx < total) reinterpret_cast<int16_t*>(a.y.m)[idx] = (int16_t)(cc < n ? val : 0);
  }
  const long long sats = warp_sum((long long)sat);
  if (lane < BFP_META_WORDS) a.y_meta[lane] = lane == 0 ? ea : (lane == 1 ? na : 0);
  if (lane == 0 && a.stats) {
    const unsigned long long cc[5] = {cnt.calls, cnt.recomputed, cnt.overflow, cnt.underflow,
                                      (unsigned long long)sats};
    for (int t = 0; t < 5; ++t)
      if (cc[t]) atomicAdd((unsigned long long*)&a.stats[t], cc[t]);
  }
}

// Every thread that runs an op plans it in registers; a full-block op then
// costs one barrier (qcomp two) for its block maximum, a solo op (warp 0
// alone) only warp reductions.  Thread 0 writes every meta block; the output
// meta of the previous op stays in registers (prev / pe / pn) until then.
// Block maxima rotate over three slots (full-block op c uses slot c mod 3 and
// clears slot c + 1 before its first barrier).
// B: a batched launch, grid z the instance, arguments Ab[z]
template <class T, bool B>
__global__ void __launch_bounds__(kCoarseThreads, 1) k_coarse_vcycle(const __grid_constant__ CoarseArgs A1,
                                                                      const CoarseArgs* __restrict__ Ab) {
  pdl_wait();
  const CoarseArgs& a = B ? Ab[blockIdx.z] : A1;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ Plan s_plan[kCoarseThreads / 32];   // full plans (general path only)
  __shared__ unsigned int s_key[3], s_nrm[3];
  __shared__ unsigned long long s_sat;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nth >> 5;
  int64_t* metas = reinterpret_cast<int64_t*>(sm + a.meta_off);
  CoarseOp* ops = reinterpret_cast<CoarseOp*>(sm + a.ops_off);
  CoarseBuf* bufs = reinterpret_cast<CoarseBuf*>(sm + a.bufs_off);
  // zero the meta blocks and the buffers (halo included); copy the schedule in
  {
    int4* mz = reinterpret_cast<int4*>(sm + a.meta_off);
    for (int i = tid; i < a.nbufs * BFP_META_WORDS / 2; i += nth) mz[i] = make_int4(0, 0, 0, 0);
    int4* dz = reinterpret_cast<int4*>(sm + a.data_off);
    for (int i = tid; i < (a.smem_bytes - a.data_off) / 16; i += nth) dz[i] = make_int4(0, 0, 0, 0);
    const int n4 = (int)(a.nops * sizeof(CoarseOp) / 4);
    for (int i = tid; i < n4; i += nth) reinterpret_cast<int32_t*>(ops)[i] = reinterpret_cast<const int32_t*>(a.ops)[i];
    for (int i = tid; i < a.nbufs; i += nth) bufs[i] = a.bufs[i];
    if (tid < 3) { s_key[tid] = 0; s_nrm[tid] = 0; }
    if (tid == 0) s_sat = 0;
  }
  __syncthreads();
  // the level-n_c right-hand side and its meta
  {
    const CoarseView<T> R = cview<T>(sm, bufs[a.rin_buf]);
    const int n = bufs[a.rin_buf].n;
    for (int j = warp; j < n; j += nw)
      for (int i = lane; i < n; i += 32) R.p[(j + 1) * R.s + i + 1] = reinterpret_cast<const T*>(a.rin.m)[(int64_t)j * a.rin.ld + i];
    if (tid < BFP_META_WORDS) metas[a.rin_buf * BFP_META_WORDS + tid] = a.rin_meta[tid];
  }
  __syncthreads();
  int prev = -1;                 // output buffer of the previous op, meta in (pe, pn)
  int64_t pe = 0, pn = 0;
  int c = 0;                     // full-block ops so far
  int sat = 0;
  CoarseCounts cnt = {0, 0, 0, 0};
  Plan* pp = &s_plan[warp];
  // the op list in two ranges around the sweep run (the run's call stays out of the loop body)
  auto exec_ops = [&](int k_begin, int k_end) {
  for (int k = k_begin; k < k_end; ++k) {
    const CoarseOp& op = ops[k];
    const bool solo = op.solo != 0;
    if (solo && warp != 0) continue;
    if (op.sync_before) {
      __syncthreads();           // the solo ops' results and meta blocks
      prev = -1;
    }
    int64_t ea = 0, na = 0, eb = 0, nb = 0;
    if (op.a >= 0) {
      if (op.a == prev) { ea = pe; na = pn; }
      else { ea = metas[op.a * BFP_META_WORDS]; na = metas[op.a * BFP_META_WORDS + 1]; }
    }
    if (op.b >= 0) {
      if (op.b == prev) { eb = pe; nb = pn; }
      else { eb = metas[op.b * BFP_META_WORDS]; nb = metas[op.b * BFP_META_WORDS + 1]; }
    }
    const bool qc = op.q.mode == kQcomp;
    CoarseLean L;
    CoarseExec ex;
    bool lean = lean_first(op, ea, na, eb, nb, L, ex);
    bool built = false;
    if (!lean) {                 // full plan (uniform decision)
      __syncwarp();
      if (lane == 0) {
        Plan p;
        build_plan_v(op.q, ea, na, eb, nb, p);
        *pp = p;
      }
      __syncwarp();
      built = true;
      ex.f = make_fast(*pp, qc);
      ex.m = make_mul(ex.f, op);
    }
    const int i0 = solo ? (lane & 15) : lane, istep = solo ? 16 : 32;
    const int j0 = solo ? (lane >> 4) : warp, jstep = solo ? 2 : nw;
    const int slot = c % 3;
    if (!solo && tid == 0) {
      s_key[(c + 1) % 3] = 0u;
      s_nrm[(c + 1) % 3] = 0u;
    }
    long long key = 0, nrm = 0;
    if (qc) {
      coarse_dispatch<T, true>(sm, op, bufs, ex, pp, i0, istep, j0, jstep, key, nrm, sat);
      unsigned kk = __reduce_max_sync(0xffffffffu, (unsigned)key);
      if (!solo) {
        if (lane == 0) atomicMax(&s_key[slot], kk);
        __syncthreads();
        kk = s_key[slot];
      }
      if (lean) lean = lean_second(op, (int32_t)kk, L, ex);
      if (!lean) {
        __syncwarp();
        if (lane == 0) {
          Plan p;
          if (built) p = *pp;
          else build_plan_v(op.q, ea, na, eb, nb, p);
          plan_from_mu(p, (int64_t)kk);
          *pp = p;
        }
        __syncwarp();
        ex.f = make_fast(*pp, false);
        ex.m = make_mul(ex.f, op);
      }
    }
    coarse_dispatch<T, false>(sm, op, bufs, ex, pp, i0, istep, j0, jstep, key, nrm, sat);
    unsigned nn = __reduce_max_sync(0xffffffffu, (unsigned)nrm);
    if (!solo) {
      if (lane == 0) atomicMax(&s_nrm[slot], nn);
      __syncthreads();
      nn = s_nrm[slot];
      ++c;
    } else {
      __syncwarp();              // this op's results before the next op reads them
    }
    const int64_t eo = lean ? (int64_t)L.e_out : pp->e_out;
    prev = op.out;
    pe = eo;
    pn = (int64_t)nn;
    if (tid == 0) {
      metas[op.out * BFP_META_WORDS] = eo;
      metas[op.out * BFP_META_WORDS + 1] = (int64_t)nn;
      cnt.add(lean ? L.ov != 0 : pp->overflow != 0, lean ? L.un != 0 : pp->underflow != 0, qc);
    }
  }
  };
  const int kr = a.run_k < a.nops ? a.run_k : a.nops;
  exec_ops(0, kr);
  int k_next = kr;
  if (sizeof(T) == 2 && kr < a.nops && warp == 0) {
    // the sweep run (warp 0; the other warps pass its solo ops and wait at the next full-block op)
    const CoarseOp& op = ops[kr];
    const int64_t ea = op.a == prev ? pe : metas[op.a * BFP_META_WORDS];
    const int64_t na = op.a == prev ? pn : metas[op.a * BFP_META_WORDS + 1];
    const int64_t eb = op.b == prev ? pe : metas[op.b * BFP_META_WORDS];
    const int64_t nb = op.b == prev ? pn : metas[op.b * BFP_META_WORDS + 1];
    const CoarseRun run = coarse_sweep_run(sm, &op, bufs, metas, ea, na, eb, nb);
    if (run.done > 0) {
      prev = run.prev;
      pe = run.pe;
      pn = run.pn;
      sat += run.sat;
      cnt.calls += run.cnt.calls;
      cnt.recomputed += run.cnt.recomputed;
      cnt.overflow += run.cnt.overflow;
      cnt.underflow += run.cnt.underflow;
    }
    k_next = kr + run.done;      // the general loop resumes at the first sweep not done
  }
  exec_ops(k_next, a.nops);
  {
    const long long s = warp_sum((long long)sat);
    if (lane == 0 && s) atomicAdd(&s_sat, (unsigned long long)s);
  }
  __syncthreads();
  // the level-n_c result back to global memory (padding columns written as 0)
  {
    const CoarseBuf yb = bufs[a.yout_buf];
    const CoarseView<T> Y = cview<T>(sm, yb);
    const int64_t ld = a.yout.ld;
    T* dst = reinterpret_cast<T*>(a.yout.m);
    for (int j = warp; j < yb.n; j += nw)
      for (int64_t i = lane; i < ld; i += 32) dst[(int64_t)j * ld + i] = (T)(i < yb.n ? Y((int)i, j) : 0);
    if (tid < BFP_META_WORDS) a.yout_meta[tid] = metas[a.yout_buf * BFP_META_WORDS + tid];
    if (tid == 0 && a.stats) {
      const unsigned long long cc[5] = {cnt.calls, cnt.recomputed, cnt.overflow, cnt.underflow, s_sat};
      for (int t = 0; t < 5; ++t)
        if (cc[t]) atomicAdd((unsigned long long*)&a.stats[t], cc[t]);
    }
  }
}

}  // namespace bfp
