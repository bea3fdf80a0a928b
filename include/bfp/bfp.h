/*
 * bfp.h -- C ABI of the GB300 block-floating-point multigrid library.
 *
 * Method: Kohl, McCormick, Tamstorf, "Multigrid methods using Block Floating
 * Point Arithmetic" (arXiv:2307.00124).  A BFP block is x = 2^e * m with
 * integer mantissas m in X_w = [-2^(w-1), 2^(w-1)-1] sharing one exponent e
 * (Sec. 2).  Every op computes its exact result z* with the App. B setup
 * rules and quantises it to w_out bits, either normalised (Alg. qcomp) or
 * saturated and truncated from a bound gamma (Alg. nnqcomp).
 *
 * General conventions
 *  - Every pointer named "device" is CUDA device memory owned by the caller.
 *  - Every call is asynchronous on the given stream (a cudaStream_t; NULL is
 *    the legacy default stream).  Argument errors are returned synchronously;
 *    nothing is read back from the device inside an op.
 *  - Exponents and norms live on the device in the vector's meta block, so a
 *    sequence of ops never synchronises with the host.
 *  - Inputs and outputs of one call must not alias (mantissas or meta).
 *  - Return value: a bfp_status (0 = BFP_OK).
 */
#ifndef BFP_BFP_H
#define BFP_BFP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void* bfp_stream; /* cudaStream_t */

typedef enum {
  BFP_OK = 0,
  BFP_ERR_ARG = -1,       /* null pointer, bad width, aliasing, bad scalar */
  BFP_ERR_SHAPE = -2,     /* sizes, leading dimension or alignment */
  BFP_ERR_WIDTH = -3,     /* an exact intermediate would exceed 62 bits per group */
  BFP_ERR_CUDA = -4,      /* a CUDA runtime call failed */
  BFP_ERR_NONFINITE = -5, /* NaN or Inf in an FP64 input (reported via meta) */
  BFP_ERR_TIMEOUT = -6,   /* a bounded device wait gave up */
  BFP_ERR_NOCONV = -7,    /* ir_solve reached its iteration limit */
  BFP_ERR_CAPACITY = -8   /* larger than a fixed-size static scratch area */
} bfp_status;

/* Words in a vector's device meta block. */
#define BFP_META_WORDS 8
/* meta[0]: shared exponent e.  meta[1]: max_i |m_i| (written by the producer).
 * meta[2..7]: scratch of the op that writes this vector (mu*, flags). */
#define BFP_META_EXP 0
#define BFP_META_NORM 1
#define BFP_META_MU 2
#define BFP_META_FLAGS 3

/* One BFP block (Sec. 2: tuple (e, m, w, d)).
 *   mant : device, int16_t when 1 <= w <= 16, int32_t when 17 <= w <= 32;
 *          16-byte aligned.  int64_t when 33 <= w <= 62 is accepted by
 *          bfp_normalize, bfp_from_f64, bfp_to_f64, bfp_axpy, bfp_residual
 *          (y and r) and bfp_ir_iterate_bfp; every other op returns
 *          BFP_ERR_ARG for it.
 *   meta : device, BFP_META_WORDS int64 (see above), 8-byte aligned.
 *   n    : points per dimension, x fastest; unused dimensions are 1.
 *   ld   : elements between consecutive x-lines (rows); ld >= n[0] and
 *          ld % 8 == 0.  Row r = y + n[1]*z starts at mant + r*ld.  Elements
 *          in [n[0], ld) are ignored on input and written as 0 on output.
 */
typedef struct {
  void* mant;
  int64_t* meta;
  int32_t w;
  int32_t ndim;
  int64_t n[3];
  int64_t ld;
} bfp_vec;

/* An exact dyadic scalar 2^e * m (a BFP block of one element), |m| < 2^31. */
typedef struct {
  int64_t m;
  int64_t e;
} bfp_scalar;

typedef enum {
  BFP_QCOMP = 0,  /* Alg. qcomp: exact up to w_out bits, normalised result */
  BFP_NNQCOMP = 1 /* Alg. nnqcomp: window from gamma, saturate, no normalisation */
} bfp_mode;

/* Quantisation request of one op.
 *   w_out     : result width, 1..32 (must equal the output vector's w).
 *   w_add     : w_tmp - w_out for Alg. qcomp; < 0 selects the op's value
 *               from Table tab:estimates.
 *   mode      : bfp_mode.
 *   has_gamma : 0 -> gamma from the op's rule (Table tab:estimates; the
 *               damped-Jacobi rows are this library's reading), 1 -> gamma.
 *   gamma     : the bound on ||z||_inf used when has_gamma = 1 (>= 0).
 *   tmp       : device int32 scratch with the output's layout (rows * ld
 *               elements) holding the w_tmp-bit window of Alg. qcomp; NULL
 *               makes qcomp recompute every element in its second pass (the
 *               result is identical).  Ignored by nnqcomp.
 */
typedef struct {
  int32_t w_out;
  int32_t w_add;
  int32_t mode;
  int32_t has_gamma;
  bfp_scalar gamma;
  void* tmp;
} bfp_q;

/* Optional device counters (uint64[8]) accumulated with atomics:
 * [0] quantised ops, [1] qcomp recomputations (overflow or underflow),
 * [2] overflows, [3] underflows, [4] saturated elements (nnqcomp). */
typedef struct {
  uint64_t* counters;
} bfp_stats;

/* Constant-coefficient star stencil (2*ndim+1 points) as one BFP block, plus
 * the damped-Jacobi weight paired with it.
 *   center, nbr : mantissas (|.| < 2^15), e : shared exponent.
 *   omega       : smoother weight (bfp_jacobi; also the residual gamma rule).
 * Laplacian of the model problem after setup S (Alg. solver-setup):
 *   2D: center 4, nbr -1, e -2 (A' = D^-1 A_h); 3D: center 6, nbr -1, e -3
 *   (A' = h^2/8 A_h; the diagonal 3/4 is folded into omega). */
typedef struct {
  int32_t ndim;
  int32_t reserved;
  int64_t center;
  int64_t nbr;
  int64_t e;
  bfp_scalar omega;
} bfp_stencil;

/* ---- helpers --------------------------------------------------------------- */

/* Text for a status code.  Never NULL. */
const char* bfp_status_str(int32_t status);
/* Library version (major*10000 + minor*100 + patch). */
int32_t bfp_version(void);
/* Number of kernels this library has enqueued in this process so far
 * (launched directly or recorded into a captured graph). */
int64_t bfp_kernel_launches(void);
/* Smallest valid ld for rows of n0 elements. */
int64_t bfp_pitch(int64_t n0);
/* Floor-quantise a double to a normalised BFP scalar of w bits (quant(),
 * read as floor; Alg. ir / v-cycle / fmg).  Host only. */
int32_t bfp_scalar_from_double(double x, int32_t w, bfp_scalar* out);
/* The model-problem Laplacian of ndim (2 or 3) with Jacobi weight omega
 * (for A_h's diagonal) floor-quantised to w_omega bits.  Host only. */
int32_t bfp_laplace_stencil(int32_t ndim, double omega, int32_t w_omega, bfp_stencil* out);

/* ---- BFP ops (Sec. 4, App. B) ------------------------------------------------ */

/* out = quantisation of x to q->w_out bits (exact z* = x; Sec. 2 normalised
 * representation).  out has x's shape; either may hold int64 mantissas. */
int32_t bfp_normalize(const bfp_vec* x, const bfp_vec* out, const bfp_q* q,
                      const bfp_stats* st, bfp_stream stream);

/* out = floor-quantised normalised BFP of the doubles x (device, dense,
 * n[0]*n[1]*n[2] values, x fastest) at out->w bits (1..62).  The doubles are read as
 * one exact block with e* = -1074; the result is Alg. qcomp's (quant() of
 * Alg. ir).  A NaN or Inf sets meta[BFP_META_FLAGS] bit 0 and out is
 * unspecified. */
int32_t bfp_from_f64(const double* x, const bfp_vec* out, bfp_stream stream);

/* out (device, dense doubles) = m * 2^e, exact when representable (|m| < 2^53;
 * wider mantissas are rounded to nearest). */
int32_t bfp_to_f64(const bfp_vec* x, double* out, bfp_stream stream);

/* meta[1] of x = max_i |m_i| over the block's n[0]*n[1]*n[2] mantissas
 * (padding columns ignored): the norm word every gamma rule reads (Table
 * tab:estimates norms are max |m| * 2^e; the max-|mantissa| reduction of
 * Alg. qcomp's first loop).  For blocks whose mantissas were written by the
 * caller; the exponent word is left as it is.  Any storage (w <= 62). */
int32_t bfp_block_norm(const bfp_vec* x, bfp_stream stream);

/* z = a*x + b*y (Alg. eaxpby-setup / eaxpby-row, then qcomp or nnqcomp); x, y
 * and z may differ in width and storage (int16 / int32 / int64; z up to 62
 * bits).  BFP_ERR_WIDTH when msb(a) + w_x or msb(b) + w_y passes 62. */
int32_t bfp_axpy(bfp_scalar a, const bfp_vec* x, bfp_scalar b, const bfp_vec* y,
                 const bfp_vec* z, const bfp_q* q, const bfp_stats* st, bfp_stream stream);

/* out = sum_i x_i y_i exactly (Sec. 2 remark on BFP dot products; 128-bit
 * accumulator), normalised to w_out bits (1..62).  out: device int64[8],
 * out[0] = mantissa, out[1] = exponent, out[2..7] scratch. */
int32_t bfp_dot(const bfp_vec* x, const bfp_vec* y, int32_t w_out, int64_t* out,
                bfp_stream stream);

/* z = A x (Alg. espmv-setup / espmv-row with m_A = 2*ndim+1; qspmv). */
int32_t bfp_stencil_apply(const bfp_stencil* A, const bfp_vec* x, const bfp_vec* z,
                          const bfp_q* q, const bfp_stats* st, bfp_stream stream);

/* rv = A y - r (Alg. egemv with alpha = 1, beta = -1; the V-cycle residual
 * line of Alg. v-cycle, with the paper's sign).  y and r may differ in
 * storage, int64 included (rv: w <= 32). */
int32_t bfp_residual(const bfp_stencil* A, const bfp_vec* y, const bfp_vec* r,
                     const bfp_vec* rv, const bfp_q* q, const bfp_stats* st,
                     bfp_stream stream);

/* Two Chebyshev steps from y = 0 in one call (Alg. v-cycle relaxation line,
 * qgemv(A, r, r, c2, c1)): y_out = c2 A r + c1 r, computed exactly as the
 * stencil T = c1 I + c2 A (one block at e_T = min(e_c1, e_c2 + e_A)) applied
 * to r, then quantised.  gamma = |c1| ||r||_inf (Table tab:estimates
 * relaxation row), w_add 2.  BFP_ERR_WIDTH when a coefficient of T passes
 * 31 bits. */
int32_t bfp_cheby(const bfp_stencil* A, bfp_scalar c1, bfp_scalar c2, const bfp_vec* r,
                  const bfp_vec* y_out, const bfp_q* q, const bfp_stats* st, bfp_stream stream);

/* y_out = y + omega (r - A y) = S y + omega r with S = I - omega A (damped
 * Jacobi in the relaxation slot of Alg. v-cycle; egemv(S, y, r, 1, omega)).
 * y == NULL means a zero initial guess: y_out = omega r. */
int32_t bfp_jacobi(const bfp_stencil* A, const bfp_vec* y, const bfp_vec* r,
                   const bfp_vec* y_out, const bfp_q* q, const bfp_stats* st,
                   bfp_stream stream);

/* r_c = R~ r_f, full weighting R~ = D_c^-1 R_FW D_f (P^T in 2D, P^T/2 in 3D):
 * the restriction line of Alg. v-cycle (qspmv with m_R = 3^d).
 * r_f has n = 2*n_c + 1 points per dimension. */
int32_t bfp_restrict(const bfp_vec* r_f, const bfp_vec* r_c, const bfp_q* q,
                     const bfp_stats* st, bfp_stream stream);

/* y_out = y - P d (Alg. v-cycle correction line: qgemv(P, d, y, -1, 1)), or
 * y_out = P d when y == NULL (Alg. fmg interpolation line: qspmv(P, x)).
 * P is bilinear (2D) / trilinear (3D) interpolation. */
int32_t bfp_prolong(const bfp_vec* d, const bfp_vec* y, const bfp_vec* y_out,
                    const bfp_q* q, const bfp_stats* st, bfp_stream stream);

/* ---- variable coefficients (2D -div(k grad u), a workload not in the paper) ---- */

/* The 5-point operator of -div(k grad u) with harmonic-mean face coefficients,
 * scaled by h^2 (A' = h^2 A_h): row i has c_i = k_W + k_E + k_S + k_N on the
 * diagonal and -k_f for its faces W, E, S, N.  The four face arrays are one
 * BFP block (int16 mantissas, or int32 for a high-precision copy used only
 * by apply / residual; one exponent e_k); the centre is their exact integer
 * sum.  Damped Jacobi uses per-point weights q_i 2^e_q ~ omega / c_i.
 *   n     : interior points (x, y); every array is n[1] rows of pitch ld
 *           (ld >= n[0], ld % 8 == 0), device memory, 16-byte aligned;
 *   k     : face mantissas W, E, S, N (k[f][j ld + i]);   e_k : their exponent;
 *   q, e_q: smoother weights (int16; may be NULL for apply / residual);
 *   a_norm: max_i 2 c_i (||A'||_inf = a_norm 2^e_k), < 2^20 for int16 faces,
 *           < 2^34 for int32 faces;  q_norm: max_i q_i;
 *   omega : the damping, used by the residual's gamma rule;
 *   k_storage : 16 (or 0) = int16 faces, 32 = int32 faces (bfp_var_jacobi
 *           needs 16).
 * The arrays are owned by the caller, or by a hierarchy
 * (bfp_hierarchy_var_level). */
typedef struct {
  int64_t n[2];
  int64_t ld;
  const void* k[4];
  int64_t e_k;
  const int16_t* q;
  int64_t e_q;
  int64_t a_norm;
  int64_t q_norm;
  bfp_scalar omega;
  int32_t k_storage;
  int32_t reserved;
} bfp_varstencil;

/* z = A' x (exact, then q).  gamma rule ||A'||_inf ||x||_inf, w_add 2. */
int32_t bfp_var_apply(const bfp_varstencil* A, const bfp_vec* x, const bfp_vec* z, const bfp_q* q,
                      const bfp_stats* st, bfp_stream stream);
/* rv = A' y - r (the paper's residual sign).  gamma (omega + 1/4) ||r||_inf
 * (Table tab:estimates, V residual row), w_add 4. */
int32_t bfp_var_residual(const bfp_varstencil* A, const bfp_vec* y, const bfp_vec* r, const bfp_vec* rv,
                         const bfp_q* q, const bfp_stats* st, bfp_stream stream);
/* y_out = y + Q (r - A' y), Q = diag(q 2^e_q); y == NULL: y_out = Q r.  gamma
 * ||y|| + ||q|| ||r|| (||I - Q A'||_inf = 1 when q_i c_i 2^(e_q+e_k) <= 1),
 * w_add 2.  Requires -40 <= e_q + e_k <= 0. */
int32_t bfp_var_jacobi(const bfp_varstencil* A, const bfp_vec* y, const bfp_vec* r, const bfp_vec* y_out,
                       const bfp_q* q, const bfp_stats* st, bfp_stream stream);
/* All three: 2D vectors of shape n, 1 <= w <= 32 for apply / residual and
 * w <= 24 for jacobi (y and r of one storage class); BFP_ERR_SHAPE on a shape
 * mismatch, BFP_ERR_WIDTH when the exact width would pass 62 bits, BFP_ERR_ARG
 * for null arrays or aliasing. */

/* ---- no-allocation variant ---------------------------------------------------- */

/* bfp_jacobi for callers that cannot allocate device memory at the call site
 * (inside a host callback or another context where CUDA allocation calls are
 * not allowed, under a device-memory budget owned by another framework, or
 * where the implicit device synchronisation of cudaMalloc / cudaFree is not
 * acceptable).  The paper has no counterpart: this is a deployment variant.
 * Same arguments and result as bfp_jacobi; q->tmp is ignored.  In qcomp mode
 * with w_tmp = w_out + w_add <= 32 (w_add < 0: the relaxation row's 2) the
 * w_tmp-bit window lives in a static device array of
 * bfp_noalloc_window_capacity() int32 entries (16 MiB on every GPU that
 * loads the library, held until exit); nothing is allocated.  nnqcomp, and
 * qcomp with a wider w_tmp, use no scratch and take any size.
 *  - qcomp outputs that use the window with rows * ld larger than the
 *    capacity: BFP_ERR_CAPACITY.
 *  - Each call looks up the array's device address on the current device
 *    (so a device reset in the process is harmless); the first lookup on a
 *    device may load the module, so make the first call before any stream
 *    capture.
 *  - All calls on a device share the array; calls that overlap on the GPU
 *    (unordered streams) race on it. */
int64_t bfp_noalloc_window_capacity(void);
int32_t bfp_jacobi_noalloc(const bfp_stencil* A, const bfp_vec* y, const bfp_vec* r,
                           const bfp_vec* y_out, const bfp_q* q, const bfp_stats* st,
                           bfp_stream stream);

/* ---- multigrid (Alg. v-cycle, fmg, ir) ---------------------------------------- */

typedef struct bfp_hierarchy bfp_hierarchy;

/* Solver set-up for -Laplace u = f on the unit square/cube, zero Dirichlet
 * boundary, n = 2^J - 1 interior points per side (finite differences). */
typedef struct {
  int32_t ndim;          /* 2 or 3 */
  int32_t w;             /* one mantissa width for all BFP vectors, 1..32 */
  int64_t n;             /* finest interior points per side, 2^J - 1 >= 3 */
  int32_t mode;          /* bfp_mode for every op inside the V-cycle */
  int32_t nu1, nu2;      /* pre- and post-smoothing sweeps (>= 1, >= 0) */
  int32_t coarse_sweeps; /* Jacobi sweeps on the coarsest level (n = 3) */
  int32_t n_fmg;         /* N of Alg. fmg: IR-V steps per level */
  double omega;          /* Jacobi weight for A_h's diagonal (4/5 in 2D, 6/7 in 3D) */
  int32_t w_omega;       /* storage width of the quantised weight */
  int32_t use_tmp;       /* 1: qcomp keeps the w_tmp window (Alg. qcomp); 0: recompute */
  int32_t use_graph;     /* 1: replay IR steps from a captured CUDA graph */
  int32_t coarse_onchip; /* 2D: the levels from the first with n <= N run as one shared-memory
                            kernel; N = 127 for 1, N = min(value, 127) for values > 1, 0: off
                            (default 63) */
  int32_t arith;         /* bfp_arith: the V-cycle's vectors and arithmetic (default BFP) */
  int32_t tile_rows;     /* rows per warp strip of the row-walking kernels for this solver's
                            ops (0: the launchers' size heuristic); set by an autotuner */
  int32_t w_step;        /* progressive precision (Sec. 4, eq. width-bounds: the inner width grows
                            by m = 1 bit per refinement): level k (0 = finest) gives its ops'
                            results, the restriction to level k+1 and the IR residual on level k
                            included, w_k = max(w - k w_step, 2) bits; 0: w on every level
                            (default).  Each level's vectors take the storage of their width
                            (int32 fine levels, int16 coarse ones when w > 16).  w_step > 0
                            needs arith BFP, and w <= 16 for variable coefficients */
  int32_t smoother;      /* bfp_smoother (default BFP_SMOOTH_JACOBI) */
  double cheby_eta;      /* BFP_SMOOTH_CHEBY: the part [eta rho, rho] of the spectrum the two
                            Chebyshev steps target, 0 < eta < 1 (default 0.15: the i/100 that
                            minimises the FP64 V(1,0) convergence factor on level 5, 2D and 3D) */
  int32_t w_add_max;     /* cap on the Table tab:estimates w_add of every op the solver enqueues:
                            w_tmp = w_out + min(w_add*, w_add_max) (Table tab:recomputation's
                            experiment); < 0: no cap (default -1) */
} bfp_solver_opts;

/* Relaxation of the V-cycle.
 *   BFP_SMOOTH_JACOBI: V(nu1, nu2) with damped Jacobi (omega), coarse_sweeps
 *     sweeps on the coarsest level (the default).
 *   BFP_SMOOTH_CHEBY: the paper's V(1,0) (Alg. v-cycle): one bfp_cheby
 *     relaxation from y = 0, then residual, restriction, coarse correction; no
 *     post-smoothing; the coarsest level gets the relaxation alone.  c1, c2
 *     come from Alg. cheby-nodes with rho = 1 + cos(pi/32) (the largest
 *     eigenvalue of D^-1 A on level 5, Alg. solver-setup's bound taken exactly)
 *     and cheby_eta, scaled for A's diagonal d (c1/d, c2/d^2) and
 *     floor-quantised to w_omega bits; the V residual's gamma uses c1
 *     ((2 c1 + 1)/4 ||r||).  nu1, nu2, coarse_sweeps and omega are unused.
 *     Constant coefficients and arith BFP only. */
typedef enum { BFP_SMOOTH_JACOBI = 0, BFP_SMOOTH_CHEBY = 1 } bfp_smoother;

/* BFP_ARITH_BFP is the paper's method; FP32 and BF16 (storage, with FP32
 * arithmetic) are float baselines of the same schedule for comparison. */
typedef enum { BFP_ARITH_BFP = 0, BFP_ARITH_FP32 = 1, BFP_ARITH_BF16 = 2 } bfp_arith;

/* Fill opts with the defaults of the 2D/3D model problem. */
int32_t bfp_solver_opts_default(int32_t ndim, int64_t n, int32_t w, bfp_solver_opts* o);

/* Allocate the level hierarchy on the current CUDA device (cudaMalloc; the
 * hierarchy owns every buffer it allocates). */
int32_t bfp_hierarchy_create(const bfp_solver_opts* o, bfp_hierarchy** h);
void bfp_hierarchy_destroy(bfp_hierarchy* h);

/* Copies the hierarchy's device counters (bfp_stats layout, uint64[8], plus
 * [5] FP64 IR residual quantisations and [6] of those that recomputed the
 * residual because the Alg. qcomp window missed; the window's gamma is the
 * previous IR residual's norm with w_add 4, or on an FMG level's first step
 * the coarser level's last one with w_add 5, Table tab:estimates) to host
 * memory; synchronises the stream.  bfp_hierarchy_reset_stats zeroes them
 * (asynchronously). */
int32_t bfp_hierarchy_read_stats(bfp_hierarchy* h, uint64_t* host8, bfp_stream stream);
/* The same counters for the finest level's separately launched ops alone
 * (its V-cycle ops, FMG interpolation, IR residual and, for
 * bfp_ir_iterate_bfp, the IR residual and update; not the on-chip coarse
 * cycle). */
int32_t bfp_hierarchy_read_finest_stats(bfp_hierarchy* h, uint64_t* host8, bfp_stream stream);
int32_t bfp_hierarchy_reset_stats(bfp_hierarchy* h, bfp_stream stream);

/* y = V(nu1,nu2)(r) on the finest level: approximate solution of A' y = r
 * (Alg. v-cycle correction scheme with damped Jacobi, or the paper's V(1,0)
 * with the Chebyshev relaxation when opts.smoother says so).  r and y use the
 * hierarchy's width and finest shape. */
int32_t bfp_vcycle(bfp_hierarchy* h, const bfp_vec* r, const bfp_vec* y, bfp_stream stream);

/* The FP64 halves of one IR step on the finest level (Alg. ir residual and
 * correction lines, in FP64 with the signs flipped):
 *   bfp_ir_residual: r = quant(b' - A' x) at r->w bits, normalised, with
 *     b' = (h^2/2^p) f; the residual is evaluated in a fixed order with
 *     correctly rounded operations; f, x: device dense doubles (n^d).
 *   bfp_ir_update:   x = x + y (y dequantised exactly, one rounding). */
int32_t bfp_ir_residual(bfp_hierarchy* h, const double* f, const double* x, const bfp_vec* r,
                        bfp_stream stream);
int32_t bfp_ir_update(double* x, const bfp_vec* y, bfp_stream stream);

/* FP64 iterative refinement (Alg. ir with FP64 residual and update):
 * k steps of  r = b' - A' x,  y = V(quant(r)),  x = x + y  on the finest level,
 * where b' = (h^2 / 2^p) f.  f, x: device dense doubles (n^d).  No host sync.
 * With opts.arith FP32 / BF16, quant(r) is r rounded to FP32 (then to BF16)
 * and V is the float V-cycle; bfp_fmg and ir_solve follow the same rule. */
int32_t bfp_ir_iterate(bfp_hierarchy* h, const double* f, double* x, int32_t k,
                       bfp_stream stream);

/* IR with x and b held as BFP blocks (Alg. ir as printed, no FP64 pass):
 * k steps of
 *   r = qgemv(A', x, b, 1, -1)  quantised by Alg. qcomp to the finest level's
 *                               width (qcomp on every IR residual),
 *   y = V(r)                    (the hierarchy's V-cycle, as bfp_vcycle),
 *   x = qsub(x, y)              quantised by Alg. qcomp to x->w bits.
 * b: the scaled right-hand side b' = s f (s from bfp_hierarchy_rhs_scale),
 * quantised by the caller (e.g. bfp_from_f64) to b->w bits.  x: the iterate,
 * updated in place; x->w is the working width (1..62; int64 storage above
 * 32 bits, BFP_ERR_WIDTH when A'x would pass the 62-bit group bound).  x and
 * b have the finest shape, any storage (b->w <= 62) and do not overlap.
 * Variable-coefficient hierarchies (x and b of one storage class, at most
 * 32 bits) use their finest
 * operator with 26-bit faces (bfp_hierarchy_var_ir_operator: Alg. ir
 * quantises A to the input width, finer than the inner solver's 16-bit
 * faces).  A scratch copy of x is allocated on the first call (and again
 * when x's storage changes).  With opts.use_graph and a
 * non-default stream two steps are captured once per (b, x, stream) and
 * replayed.  Float hierarchies: BFP_ERR_ARG.  No host sync. */
int32_t bfp_ir_iterate_bfp(bfp_hierarchy* h, const bfp_vec* b, const bfp_vec* x, int32_t k,
                           bfp_stream stream);
/* s with b' = s f for this hierarchy's finest level: h^2 for variable
 * coefficients, h^2 / 2^p for the model problem (p = 2 in 2D, 3 in 3D). */
int32_t bfp_hierarchy_rhs_scale(const bfp_hierarchy* h, double* out);

/* Full multigrid (Alg. fmg) from x = 0: on each level from the coarsest,
 * interpolate the coarser solution at width w (bfp_prolong) and run n_fmg
 * IR-V steps; the coarse right-hand sides are full-weighting restrictions of
 * b'.  x: device dense doubles (n^d) receiving the finest solution. */
int32_t bfp_fmg(bfp_hierarchy* h, const double* f, double* x, bfp_stream stream);

typedef struct {
  int32_t max_iter;   /* IR steps at most */
  int32_t fmg_start;  /* 1: start from FMG, 0: from the given x */
  double tol;         /* stop when ||b' - A'x||_inf <= tol * ||b'||_inf (checked on the host) */
  int32_t stall_fallback; /* 1: the safety mechanism of Sec. 5 (see ir_solve); 0: off */
  int32_t reserved;
} bfp_ir_opts;

typedef struct {
  int32_t iterations;
  int32_t converged;
  double res_inf;     /* final ||b' - A'x||_inf */
  double res0_inf;    /* ||b'||_inf */
  int32_t fallback_at; /* the IR step from which the V-cycle ran with qcomp, -1: never */
  int32_t reserved;
} bfp_ir_report;

/* IR to a tolerance (Alg. ir): synchronises with the host once per step to
 * read the residual norm.  Returns BFP_ERR_NOCONV when max_iter is reached.
 * Safety mechanism (Sec. 5, closing the discussion of skipping
 * normalisation): with stall_fallback set and an nnqcomp hierarchy, once the
 * residual norm after step i is above half the norm two steps earlier (the
 * convergence stalls), every later step runs the separately launched V-cycle
 * ops with qcomp (the on-chip coarse cycle keeps its mode). */
int32_t ir_solve(bfp_hierarchy* h, const double* f, double* x, const bfp_ir_opts* o,
                 bfp_ir_report* rep, bfp_stream stream);

/* Hierarchy of the variable-coefficient problem -div(k grad u) = f (2D):
 * k_nodes are k at the (n+2) x (n+2) grid nodes, boundary included, host
 * doubles row-major [y][x].  Each level's operator comes from the node values
 * injected to that level (coarse node c = fine node 2c), set up on the host:
 * harmonic-mean faces ((2 a) b) / (a + b) in FP64, floor-quantised to 16-bit
 * mantissas with one exponent (the largest face gets 15 significant bits), and
 * weights q_i = floor(omega_m 2^s / c_i) with the largest s that keeps q in 16
 * bits.  opts: ndim 2, arith BFP, w <= 24 (coarse_onchip is ignored).  The
 * solver calls (bfp_vcycle, bfp_fmg, bfp_ir_iterate, ir_solve,
 * bfp_ir_residual) then use these operators, b' = h^2 f, and the FP64 IR
 * residual b' - (c x - (((k_W x_W + k_E x_E) + k_S x_S) + k_N x_N)) with the
 * unquantised FP64 faces, c = ((k_W + k_E) + k_S) + k_N. */
int32_t bfp_hierarchy_create_var(const bfp_solver_opts* o, const double* k_nodes, bfp_hierarchy** h);
/* Level l's operator (device arrays owned by the hierarchy; 0 = finest).
 * BFP_ERR_ARG for a constant-coefficient hierarchy or a bad level. */
int32_t bfp_hierarchy_var_level(const bfp_hierarchy* h, int32_t level, bfp_varstencil* out);
/* The finest operator of the IR residual in bfp_ir_iterate_bfp: the same
 * faces floor-quantised to 26-bit int32 mantissas (the largest face gets 25
 * significant bits, so A'x stays within 62 bits for x up to 32 bits); q NULL,
 * k_storage 32.  BFP_ERR_ARG for a constant-coefficient hierarchy. */
int32_t bfp_hierarchy_var_ir_operator(const bfp_hierarchy* h, bfp_varstencil* out);

/* ---- batched solves (many independent instances, one graph launch) ------------ */
/* count independent hierarchies (opts[i]: size, width, mode, schedule of
 * instance i), solved together: bfp_batch_solve captures [FMG] +
 * ir_steps[i] IR-V steps of every instance into one CUDA graph (re-captured
 * only when the arguments change) and launches it once on stream (which must
 * not be the legacy default stream).  Instances with equal options form a
 * group that runs on one graph branch: each op of the shared schedule is ONE
 * launch over all the group's instances still running at that point (grid z =
 * instance), with the same per-instance results as a single-instance solve; a
 * group whose schedule uses an op without a batched form (3D, int32 storage,
 * variable coefficients, float baselines) runs its instances on branches of
 * their own.  f[i], x[i]: device dense doubles of instance i (x[i] is the
 * initial iterate when fmg == 0).  bfp_batch_times waits for the last launch
 * and writes, per instance, the ms from the launch start to the end of that
 * instance's last op. */
typedef struct bfp_batch bfp_batch;
int32_t bfp_batch_create(const bfp_solver_opts* opts, int32_t count, bfp_batch** out);
int32_t bfp_batch_solve(bfp_batch* b, const double* const* f, double* const* x, const int32_t* ir_steps,
                        int32_t fmg, bfp_stream stream);
/* The same work for instance i alone, as its own graph launch (the comparison
 * the batched launch is measured against). */
int32_t bfp_batch_solve_one(bfp_batch* b, int32_t i, const double* f, double* x, int32_t ir_steps, int32_t fmg,
                            bfp_stream stream);
int32_t bfp_batch_times(bfp_batch* b, float* ms);
/* Of the last captured solve: groups run as merged launches, and instances on
 * branches of their own. */
int32_t bfp_batch_info(const bfp_batch* b, int32_t* merged_groups, int32_t* separate_instances);
void bfp_batch_destroy(bfp_batch* b);

/* ---- float baselines (not in the paper) ------------------------------------------ */
/* FP32 and BF16-storage / FP32-arithmetic versions of the V-cycle ops, for the
 * comparison the paper's method is measured against.  Arithmetic is FP32 with
 * round-to-nearest and no contraction, in the order stated per op; BF16
 * vectors hold the upper half of an FP32 value (loads widen exactly, stores
 * round to nearest-even).  The coefficients come from a bfp_stencil:
 * c = center 2^e, nb = nbr 2^e, om = omega.m 2^omega.e (dyadic, exact in FP32).
 * Neighbours outside the grid are 0; padding columns of outputs are written
 * as 0.  Status codes and stream behaviour as for the BFP ops. */
typedef enum { FLT_F32 = 0, FLT_BF16 = 1 } flt_dtype;

typedef struct {
  void* data;          /* device pointer (float, or BF16 bit patterns as uint16), 16-byte aligned */
  int32_t dtype;       /* flt_dtype */
  int32_t ndim;        /* 2 or 3 */
  int64_t n[3];        /* points per dimension, x fastest (unused dimensions 1) */
  int64_t ld;          /* row stride in elements: >= n[0], multiple of 8 */
} flt_vec;

/* out = y + om (r - a), a = c y + nb s, s = (W + E) + (S + N) [+ (B + T)];
 * y == NULL: out = om r.  y, r, out: same shape and dtype, out distinct. */
int32_t flt_jacobi(const bfp_stencil* A, const flt_vec* y, const flt_vec* r, const flt_vec* out,
                   bfp_stream stream);
/* out = a - r (the V-cycle residual r_v = A'y - r). */
int32_t flt_residual(const bfp_stencil* A, const flt_vec* y, const flt_vec* r, const flt_vec* out,
                     bfp_stream stream);
/* Full weighting r_c = R~ r_f (coarse n_c = (n_f - 1)/2): along x (f0 + 2 f1) + f2
 * with fine index 2I + 1 of coarse I in the middle, then the same along y [and z],
 * times 2^-2 (2D) or 2^-4 (3D). */
int32_t flt_restrict(const flt_vec* r_f, const flt_vec* r_c, bfp_stream stream);
/* out = y - P d (y != NULL) or P d: interpolation along x, then y [then z];
 * on a coarse point its value, between two coarse points 0.5 a + 0.5 b. */
int32_t flt_prolong(const flt_vec* d, const flt_vec* y, const flt_vec* out, bfp_stream stream);
/* y = V(nu1,nu2)(r) on the finest level of a hierarchy created with
 * opts.arith FP32 (dtype F32) or BF16 (dtype BF16). */
int32_t flt_vcycle(bfp_hierarchy* h, const flt_vec* r, const flt_vec* y, bfp_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* BFP_BFP_H */
