// bfp_desc.h -- the host-side "setup-func" of each BFP op: exponent groups,
// exact-width bounds (App. B setup rules) and the gamma rule (Table
// tab:estimates; damped-Jacobi rows are this library's reading).  Shared by
// the C ABI functions and the on-chip coarse V-cycle so both describe an op
// identically.  Each returns the op's default w_add through *w_add_rule.
#pragma once

#include "bfp_host.h"

namespace bfp {

inline int64_t iabs64(int64_t v) { return v < 0 ? -v : v; }

inline int stencil_width(const bfp_stencil* A) {
  return hmsb(A->center) > hmsb(A->nbr) ? hmsb(A->center) : hmsb(A->nbr);
}

// z = A x (Alg. espmv-setup): H = c x + n sum(nbrs) at e_A + e_x
inline int32_t desc_apply(const bfp_stencil* A, int wx, QDesc& d, int* w_add_rule) {
  const int mA = 2 * A->ndim + 1;
  d.ch = A->e; d.ha = 1; d.two = 0;
  d.hbits = stencil_width(A) + wx + clog2(mA);
  d.ng = 1; d.gv[0] = 0;                               // gamma = ||A||_inf ||x||
  d.gm[0] = (uint64_t)(iabs64(A->center) + 2 * A->ndim * iabs64(A->nbr)); d.ge[0] = A->e;
  *w_add_rule = 2;
  return BFP_OK;
}

// r_v = A y - r (Alg. egemv, alpha = 1, beta = -1): H = A y at e_A + e_y, L = -r at e_r
inline int32_t desc_residual(const bfp_stencil* A, int wy, int wr, QDesc& d, int* w_add_rule) {
  const int mA = 2 * A->ndim + 1;
  d.ch = A->e; d.ha = 1;
  d.cl = 0; d.lb = 1;
  d.two = 1;
  d.hbits = stencil_width(A) + wy + clog2(mA);
  d.lbits = wr + 1;
  // gamma = 1/4 (2 c1 + 1) ||r|| with c1 = 2 omega  ->  (|omega| + 1/4) ||r||
  const int64_t om = iabs64(A->omega.m), oe = A->omega.e;
  uint64_t cm;
  int64_t ce;
  if (oe <= -2) { cm = (uint64_t)om + (1ull << (-2 - oe)); ce = oe; }
  else {
    if (oe + 2 > 30) return BFP_ERR_ARG;
    cm = ((uint64_t)om << (oe + 2)) + 1ull; ce = -2;
  }
  if (cm >= (1ull << 32)) return BFP_ERR_ARG;
  d.ng = 1; d.gv[0] = 1; d.gm[0] = cm; d.ge[0] = ce;
  *w_add_rule = 4;                                     // V residual row
  return BFP_OK;
}

// Jacobi coefficients: S = I - omega A as one BFP block (e_S = min(0, e_omega + e_A))
inline int32_t jacobi_operator(const bfp_stencil* A, int64_t* Sc, int64_t* Sn, int64_t* eS) {
  const int64_t mw = A->omega.m, ew = A->omega.e;
  *eS = (ew + A->e) < 0 ? (ew + A->e) : 0;
  const int64_t k = ew + A->e - *eS;
  if (-*eS > 40 || k > 40) return BFP_ERR_ARG;
  *Sc = ((int64_t)1 << (-*eS)) - ((mw * A->center) << k);
  *Sn = -((mw * A->nbr) << k);
  if (*Sc >= (1ll << 31) || *Sc < -(1ll << 31) || *Sn >= (1ll << 31) || *Sn < -(1ll << 31)) return BFP_ERR_WIDTH;
  return BFP_OK;
}

// y' = S y + omega r (Alg. egemv(S, y, r, 1, omega)); wy == 0: zero guess, y' = omega r
inline int32_t desc_jacobi(const bfp_stencil* A, int wy, int wr, QDesc& d, int* w_add_rule) {
  const int64_t mw = A->omega.m, ew = A->omega.e;
  const int mA = 2 * A->ndim + 1;
  *w_add_rule = 2;                                     // relaxation row
  if (wy == 0) {
    d.ch = ew; d.hb = 1; d.two = 0;                    // omega r at e_omega + e_r
    d.hbits = hmsb(mw) + wr;
    d.ng = 1; d.gv[0] = 1; d.gm[0] = (uint64_t)iabs64(mw); d.ge[0] = ew;
    return BFP_OK;
  }
  int64_t Sc, Sn, eS;
  int32_t rc = jacobi_operator(A, &Sc, &Sn, &eS);
  if (rc) return rc;
  const int wS = hmsb(Sc) > hmsb(Sn) ? hmsb(Sc) : hmsb(Sn);
  d.ch = eS; d.ha = 1;                                 // S y at e_S + e_y
  d.cl = ew; d.lb = 1;                                 // omega r at e_omega + e_r
  d.two = 1;
  d.hbits = wS + wy + clog2(mA);
  d.lbits = hmsb(mw) + wr;
  d.ng = 2;                                            // gamma = ||S||_inf ||y|| + |omega| ||r||
  d.gv[0] = 0; d.gm[0] = (uint64_t)(iabs64(Sc) + 2 * A->ndim * iabs64(Sn)); d.ge[0] = eS;
  d.gv[1] = 1; d.gm[1] = (uint64_t)iabs64(mw); d.ge[1] = ew;
  return BFP_OK;
}

// Two Chebyshev steps from y = 0 as one stencil (Alg. v-cycle relaxation line,
// qgemv(A, r, r, c2, c1) = c2 A r + c1 r): T = c1 I + c2 A exactly, one block at
// e_T = min(e_c1, e_c2 + e_A); BFP_ERR_WIDTH when a coefficient passes 31 bits.
inline int32_t cheby_operator(const bfp_stencil* A, bfp_scalar c1, bfp_scalar c2, int64_t* Tc, int64_t* Tn,
                              int64_t* eT) {
  if (c1.m >= (1ll << 31) || c1.m < -(1ll << 31) || c2.m >= (1ll << 31) || c2.m < -(1ll << 31)) return BFP_ERR_ARG;
  const int64_t e2 = c2.e + A->e;
  *eT = c1.e < e2 ? c1.e : e2;
  auto shl = [](int64_t v, int64_t s, int64_t* o) {
    if (v == 0) { *o = 0; return true; }
    if (s < 0 || hmsb(v) + s > 40) return false;
    *o = (int64_t)((uint64_t)v << s);
    return true;
  };
  int64_t a, b, n;
  if (!shl(c1.m, c1.e - *eT, &a) || !shl(c2.m * A->center, e2 - *eT, &b) || !shl(c2.m * A->nbr, e2 - *eT, &n))
    return BFP_ERR_WIDTH;
  *Tc = a + b;
  *Tn = n;
  if (*Tc >= (1ll << 31) || *Tc < -(1ll << 31) || *Tn >= (1ll << 31) || *Tn < -(1ll << 31)) return BFP_ERR_WIDTH;
  return BFP_OK;
}

// y = T r: H = T r at e_T + e_r; gamma c1 ||r|| (relaxation row, w_add 2)
inline int32_t desc_cheby(const bfp_stencil* A, bfp_scalar c1, bfp_scalar c2, int wr, QDesc& d, int* w_add_rule,
                          int64_t* Tc, int64_t* Tn) {
  int64_t eT;
  const int32_t rc = cheby_operator(A, c1, c2, Tc, Tn, &eT);
  if (rc) return rc;
  const int mA = 2 * A->ndim + 1;
  const int wT = hmsb(*Tc) > hmsb(*Tn) ? hmsb(*Tc) : hmsb(*Tn);
  d.ch = eT; d.ha = 1; d.two = 0;
  d.hbits = wT + wr + clog2(mA);
  d.ng = 1; d.gv[0] = 0; d.gm[0] = (uint64_t)iabs64(c1.m); d.ge[0] = c1.e;
  *w_add_rule = 2;
  return BFP_OK;
}

// r_c = R~ r_f (full weighting, m_R = 3^d; R~ = P^T in 2D, P^T/2 in 3D)
inline int32_t desc_restrict(int nd, int wf, QDesc& d, int* w_add_rule) {
  const int64_t eR = nd == 2 ? -2 : -4;
  int mR = 1;
  for (int i = 0; i < nd; ++i) mR *= 3;
  d.ch = eR; d.ha = 1; d.two = 0;
  d.hbits = hmsb(1ll << nd) + wf + clog2(mR);
  d.ng = 1; d.gv[0] = 0;                               // gamma = ||R~||_inf ||r_v||  (= 4 ||r_v||)
  d.gm[0] = nd == 2 ? 16 : 64; d.ge[0] = eR;
  *w_add_rule = 6;                                     // restriction row
  return BFP_OK;
}

// y' = y - P d (wy > 0) or P d (wy == 0): H = -P_m d (or +P_m d) at e_P + e_d, L = y at e_y
inline int32_t desc_prolong(int nd, int wd, int wy, QDesc& d, int* w_add_rule) {
  const int64_t eP = -nd;
  d.ch = eP; d.ha = 1;
  d.hbits = hmsb(1ll << nd) + wd + nd + 1;
  if (wy > 0) {
    d.cl = 0; d.lb = 1; d.two = 1;
    d.lbits = wy + 1;
    d.ng = 2;                                          // gamma = ||y|| + ||P|| ||d||
    d.gv[0] = 1; d.gm[0] = 1; d.ge[0] = 0;
    d.gv[1] = 0; d.gm[1] = 1ull << nd; d.ge[1] = eP;
    *w_add_rule = 1;                                   // correction row
  } else {
    d.two = 0;
    d.ng = 1;                                          // gamma = ||P|| ||x||
    d.gv[0] = 0; d.gm[0] = 1ull << nd; d.ge[0] = eP;
    *w_add_rule = 0;                                   // FMG interpolation row
  }
  return BFP_OK;
}

// ---- variable coefficients (bfp_varstencil): the exponent groups, width bounds and gamma rules
// of bfp_var_apply / bfp_var_residual / bfp_var_jacobi (shared with the coarsest-level run) ----

// A'x: H = A'x at e_k + e_x; gamma ||A'|| ||x||
inline int32_t desc_var_apply(const bfp_varstencil* A, int wx, QDesc& d, int* w_add_rule) {
  d.ch = A->e_k; d.ha = 1; d.two = 0;
  d.hbits = hmsb(A->a_norm) + wx + 1;
  d.ng = 1; d.gv[0] = 0; d.gm[0] = (uint64_t)A->a_norm; d.ge[0] = A->e_k;
  *w_add_rule = 2;
  return BFP_OK;
}

// r_v = A'y - r: H = A'y at e_k + e_y, L = -r at e_r; gamma (omega + 1/4) ||r|| (V residual row)
inline int32_t desc_var_residual(const bfp_varstencil* A, int wy, int wr, QDesc& d, int* w_add_rule) {
  d.ch = A->e_k; d.ha = 1;
  d.cl = 0; d.lb = 1;
  d.two = 1;
  d.hbits = hmsb(A->a_norm) + wy + 1;
  d.lbits = wr + 1;
  const int64_t om = iabs64(A->omega.m), oe = A->omega.e;
  uint64_t cm;
  int64_t ce;
  if (oe <= -2) { cm = (uint64_t)om + (1ull << (-2 - oe)); ce = oe; }
  else {
    if (oe + 2 > 30) return BFP_ERR_ARG;
    cm = ((uint64_t)om << (oe + 2)) + 1ull; ce = -2;
  }
  if (cm >= (1ull << 32)) return BFP_ERR_ARG;
  d.ng = 1; d.gv[0] = 1; d.gm[0] = cm; d.ge[0] = ce;
  *w_add_rule = 4;
  return BFP_OK;
}

// y' = y + Q (r - A'y): H = y 2^s - q A'y at e_q + e_k + e_y (s = -(e_q + e_k)), L = q r at e_q + e_r;
// gamma ||y|| + ||q|| ||r||.  wy == 0: y' = Q r (H = q r at e_q + e_r; gamma ||q|| ||r||).
inline int32_t desc_var_jacobi(const bfp_varstencil* A, int wy, int wr, QDesc& d, int* w_add_rule, int32_t* s_out) {
  const int qb = hmsb(A->q_norm);
  *w_add_rule = 2;
  *s_out = 0;
  if (wy == 0) {
    d.ch = A->e_q; d.hb = 1; d.two = 0;
    d.hbits = qb + wr + 1;
    d.ng = 1; d.gv[0] = 1; d.gm[0] = (uint64_t)A->q_norm; d.ge[0] = A->e_q;
    return BFP_OK;
  }
  const int64_t s = -(A->e_q + A->e_k);
  if (s < 0 || s > 40) return BFP_ERR_ARG;
  d.ch = A->e_q + A->e_k; d.ha = 1;
  d.cl = A->e_q; d.lb = 1;
  d.two = 1;
  const int hb1 = wy + (int)s, hb2 = qb + hmsb(A->a_norm) + wy;
  d.hbits = (hb1 > hb2 ? hb1 : hb2) + 2;
  d.lbits = qb + wr + 1;
  d.ng = 2;
  d.gv[0] = 0; d.gm[0] = 1; d.ge[0] = 0;
  d.gv[1] = 1; d.gm[1] = (uint64_t)A->q_norm; d.ge[1] = A->e_q;
  *s_out = (int32_t)s;
  return BFP_OK;
}

}  // namespace bfp
