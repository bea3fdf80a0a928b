// bfp_coarse.cuh -- the coarse end of the V-cycle on one SM.
//
// Below a few hundred thousand points a level's ops are dominated by launch
// and round-trip latency, and the coarsest level's 32 sweeps would be 32
// launches.  One CTA instead runs every level from n_c (<= 127) down to 3 in
// shared memory: the host flattens the recursive schedule of Alg. v-cycle
// (exactly the order the global driver uses) into a list of ops; the CTA
// executes the list with __syncthreads between passes.  Each op builds its
// plan from the same QDesc the C ABI op would use and quantises through the
// same device arithmetic (combine / mu_key / finish), so the result is
// bit-identical to running the ops one by one.  qcomp's second pass always
// recomputes (the window is only a cache); its overflow / underflow counts
// are still those of Alg. qcomp.
#pragma once

#include "bfp_host.h"

namespace bfp {

enum CoarseKind : int32_t { cJac0 = 0, cJac = 1, cRes = 2, cRestrict = 3, cProlong = 4 };

struct CoarseOp {
  int32_t kind;
  int32_t a, b, out;     // buffer ids (-1: none)
  int64_t c, nb, mw;     // stencil / smoother coefficients
  QDesc q;               // static description; meta pointers are set on the device
};

struct CoarseBuf {
  int32_t off;           // byte offset of the mantissas in dynamic shared memory
  int32_t n;             // points per side
};

struct CoarseArgs {
  const CoarseOp* ops;
  const CoarseBuf* bufs;
  int32_t nops, nbufs;
  int32_t is32;          // mantissa storage: int32 (else int16)
  int32_t meta_off;      // byte offsets in dynamic shared memory: meta blocks,
  int32_t ops_off;       // the op list (copied in at start) and
  int32_t bufs_off;      // the buffer table
  VIn rin;               // level n_c right-hand side (global) ...
  const int64_t* rin_meta;
  int32_t rin_buf;       // ... and the buffer it is loaded into
  VOut yout;             // level n_c result (global) ...
  int64_t* yout_meta;
  int32_t yout_buf;      // ... read from this buffer (set by the schedule)
  uint64_t* stats;
};

struct CoarseMem {
  unsigned char* base;
  int32_t is32;
  __device__ __forceinline__ int32_t get(const CoarseBuf& b, int i, int j) const {
    if (i < 0 || j < 0 || i >= b.n || j >= b.n) return 0;
    const int idx = j * b.n + i;
    return is32 ? reinterpret_cast<const int32_t*>(base + b.off)[idx]
                : (int32_t)reinterpret_cast<const int16_t*>(base + b.off)[idx];
  }
  __device__ __forceinline__ void put(const CoarseBuf& b, int idx, int32_t v) const {
    if (is32) reinterpret_cast<int32_t*>(base + b.off)[idx] = v;
    else reinterpret_cast<int16_t*>(base + b.off)[idx] = (int16_t)v;
  }
};

// exact groups (H, L) of one output element of a coarse op
__device__ __forceinline__ void coarse_elem(const CoarseOp& op, const CoarseMem& m, const CoarseBuf& ba,
                                            const CoarseBuf& bb, int i, int j, int64_t& H, int64_t& L) {
  switch (op.kind) {
    case cJac0:
      H = op.mw * (int64_t)m.get(bb, i, j);
      L = 0;
      break;
    case cJac:
    case cRes: {
      const int64_t ns = (int64_t)m.get(ba, i - 1, j) + m.get(ba, i + 1, j) + m.get(ba, i, j - 1) + m.get(ba, i, j + 1);
      H = op.c * (int64_t)m.get(ba, i, j) + op.nb * ns;
      const int64_t rv = m.get(bb, i, j);
      L = op.kind == cJac ? op.mw * rv : -rv;
      break;
    }
    case cRestrict: {
      // coarse (i, j) gathers fine (2i+1+dx, 2j+1+dy) with weights (2-|dx|)(2-|dy|)
      int64_t acc = 0;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx)
          acc += (int64_t)((2 - (dx < 0 ? -dx : dx)) * (2 - (dy < 0 ? -dy : dy))) *
                 m.get(ba, 2 * i + 1 + dx, 2 * j + 1 + dy);
      H = acc;
      L = 0;
      break;
    }
    default: {  // cProlong with correction: H = -P_m d, L = y
      int64_t acc = 0;
      int Jy[2], wy[2], ny = 0, Ix[2], wx[2], nx = 0;
      if (j & 1) { Jy[0] = (j - 1) / 2; wy[0] = 2; ny = 1; } else { Jy[0] = j / 2 - 1; wy[0] = 1; Jy[1] = j / 2; wy[1] = 1; ny = 2; }
      if (i & 1) { Ix[0] = (i - 1) / 2; wx[0] = 2; nx = 1; } else { Ix[0] = i / 2 - 1; wx[0] = 1; Ix[1] = i / 2; wx[1] = 1; nx = 2; }
      for (int u = 0; u < ny; ++u)
        for (int v = 0; v < nx; ++v) acc += (int64_t)(wy[u] * wx[v]) * m.get(ba, Ix[v], Jy[u]);
      H = -acc;
      L = m.get(bb, i, j);
      break;
    }
  }
}

// One element's result in the register fast path (see Fast) or the general path.
template <bool PASS1>
__device__ __forceinline__ void coarse_quant(int64_t H, int64_t L, const Plan& p, const Fast& f, long long& key,
                                             int32_t& v, int& sat) {
  if (f.ok) {
    const int64_t Z = (int64_t)((uint64_t)H << f.dh) + (int64_t)((uint64_t)L << f.dl);
    if (PASS1) {
      key = max(key, (long long)(256 + msb64(Z)));
    } else {
      int64_t t = Z >> f.t;
      if (f.clamp) {
        const int64_t hi = (1ll << (f.w - 1)) - 1, lo = -(1ll << (f.w - 1));
        if (t > hi) { t = hi; ++sat; } else if (t < lo) { t = lo; ++sat; }
      }
      v = (int32_t)t;
    }
    return;
  }
  if (p.wide) {
    const i128 Z = combine<i128>(H, L, p);
    if (PASS1) key = max(key, (long long)mu_key<i128>(Z, H, L, p));
    else v = finish<i128>(Z, H, L, p, sat);
  } else {
    const int64_t Z = combine<int64_t>(H, L, p);
    if (PASS1) key = max(key, (long long)mu_key<int64_t>(Z, H, L, p));
    else v = finish<int64_t>(Z, H, L, p, sat);
  }
}

__global__ void __launch_bounds__(1024, 1) k_coarse_vcycle(const CoarseArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ Plan sp;
  __shared__ Fast sf;
  __shared__ long long s_key, s_nrm, s_sat;
  __shared__ unsigned long long s_cnt[5];
  const int tid = threadIdx.x, nth = blockDim.x;
  const CoarseMem m{sm, a.is32};
  int64_t* metas = reinterpret_cast<int64_t*>(sm + a.meta_off);
  // the schedule and buffer table live in shared memory for the whole cycle
  CoarseOp* ops = reinterpret_cast<CoarseOp*>(sm + a.ops_off);
  CoarseBuf* bufs = reinterpret_cast<CoarseBuf*>(sm + a.bufs_off);
  {
    const int n4 = (int)(a.nops * sizeof(CoarseOp) / 4);
    for (int i = tid; i < n4; i += nth) reinterpret_cast<int32_t*>(ops)[i] = reinterpret_cast<const int32_t*>(a.ops)[i];
    for (int i = tid; i < a.nbufs; i += nth) bufs[i] = a.bufs[i];
  }
  if (tid < 5) s_cnt[tid] = 0;
  __syncthreads();
  // load the level-n_c right-hand side and its meta
  {
    const CoarseBuf rb = bufs[a.rin_buf];
    const int tot = rb.n * rb.n;
    for (int idx = tid; idx < tot; idx += nth) {
      const int i = idx % rb.n, j = idx / rb.n;
      const int64_t off = (int64_t)j * a.rin.ld + i;
      const int32_t v = a.is32 ? reinterpret_cast<const int32_t*>(a.rin.m)[off]
                               : (int32_t)reinterpret_cast<const int16_t*>(a.rin.m)[off];
      m.put(rb, idx, v);
    }
    if (tid < BFP_META_WORDS) metas[a.rin_buf * BFP_META_WORDS + tid] = a.rin_meta[tid];
  }
  __syncthreads();
  for (int oi = 0; oi < a.nops; ++oi) {
    const CoarseOp& op = ops[oi];
    const CoarseBuf bo = bufs[op.out];
    const CoarseBuf ba = op.a >= 0 ? bufs[op.a] : bo;
    const CoarseBuf bb = op.b >= 0 ? bufs[op.b] : bo;
    const bool qc = op.q.mode == kQcomp;
    if (tid == 0) {
      QDesc q = op.q;
      q.meta_a = op.a >= 0 ? metas + op.a * BFP_META_WORDS : nullptr;
      q.meta_b = op.b >= 0 ? metas + op.b * BFP_META_WORDS : nullptr;
      q.meta_out = metas + op.out * BFP_META_WORDS;
      build_plan(q, sp);
      sf = make_fast(sp, qc);
      s_key = 0;
      s_nrm = 0;
      s_sat = 0;
    }
    __syncthreads();
    const int tot = bo.n * bo.n;
    if (qc) {
      long long key = 0;
      const Fast f = sf;
      for (int idx = tid; idx < tot; idx += nth) {
        int64_t H, L;
        coarse_elem(op, m, ba, bb, idx % bo.n, idx / bo.n, H, L);
        int32_t v;
        int s = 0;
        coarse_quant<true>(H, L, sp, f, key, v, s);
      }
      key = warp_max(key);
      if ((tid & 31) == 0) atomicMax(&s_key, key);
      __syncthreads();
      if (tid == 0) {
        plan_from_mu(sp, s_key);
        sf = make_fast(sp, false);
      }
      __syncthreads();
    }
    long long nrm = 0, sat = 0;
    {
      const Fast f = sf;
      long long key = 0;
      for (int idx = tid; idx < tot; idx += nth) {
        int64_t H, L;
        coarse_elem(op, m, ba, bb, idx % bo.n, idx / bo.n, H, L);
        int s = 0;
        int32_t v = 0;
        coarse_quant<false>(H, L, sp, f, key, v, s);
        m.put(bo, idx, v);
        nrm = max(nrm, (long long)(v < 0 ? -(long long)v : (long long)v));
        sat += s;
      }
    }
    nrm = warp_max(nrm);
    sat = warp_sum(sat);
    if ((tid & 31) == 0) {
      atomicMax(&s_nrm, nrm);
      if (sat) atomicAdd((unsigned long long*)&s_sat, (unsigned long long)sat);
    }
    __syncthreads();
    if (tid == 0) {
      int64_t* mo = metas + op.out * BFP_META_WORDS;
      mo[0] = sp.e_out;
      mo[1] = s_nrm;
      s_cnt[0] += 1;
      if (qc) {
        if (sp.overflow || sp.underflow) s_cnt[1] += 1;
        if (sp.overflow) s_cnt[2] += 1;
        if (sp.underflow) s_cnt[3] += 1;
      }
      s_cnt[4] += (unsigned long long)s_sat;
    }
    __syncthreads();
  }
  // the level-n_c result back to global memory (padding columns written as 0)
  {
    const CoarseBuf yb = bufs[a.yout_buf];
    const int64_t rows = yb.n, ld = a.yout.ld;
    for (int64_t idx = tid; idx < rows * ld; idx += nth) {
      const int64_t j = idx / ld, i = idx - j * ld;
      const int32_t v = i < yb.n ? m.get(yb, (int)i, (int)j) : 0;
      if (a.yout.is32) reinterpret_cast<int32_t*>(a.yout.m)[idx] = v;
      else reinterpret_cast<int16_t*>(a.yout.m)[idx] = (int16_t)v;
    }
    if (tid < BFP_META_WORDS) a.yout_meta[tid] = metas[a.yout_buf * BFP_META_WORDS + tid];
    if (tid < 5 && a.stats && s_cnt[tid]) atomicAdd((unsigned long long*)&a.stats[tid], s_cnt[tid]);
  }
}

}  // namespace bfp
