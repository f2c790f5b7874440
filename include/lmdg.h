/* liblmdg -- low-memory discrete-ordinates discontinuous Galerkin transport sweeps on one GB300.
 *
 * C ABI for the hot path of Sun & Hauck, "Low-memory, discrete ordinates, discontinuous Galerkin methods
 * for radiative transport" (arXiv 1907.01027): the upwind transport sweep of the standard Q1 S_N-DG scheme
 * and of the two low-memory schemes, the angular reduction fused into the sweep, GMRES on the
 * sweep-reduced systems, mixed-precision iterative refinement and the adjoint sweep.
 *
 * Problem (eq-main, Section 1): on a uniform Cartesian mesh of nx x ny square cells (Section 2.1),
 *   Omega . grad Psi + (sigma_s/eps + eps sigma_a) Psi = (sigma_s/eps) Psi_bar + eps q,  Psi = alpha on inflow,
 * discretised by S_N collocation (eq:sn) and upwind DG with the Legendre Q1 basis (1, xi, eta, xi*eta) per
 * cell (eq-Ljk, eq-sndg-scheme).
 *
 * Conventions for every entry point:
 *   - Cell (i, j) (i < nx along x, j < ny along y) has index p = j*nx + i.  Per-cell vectors are [nx*ny][4]
 *     doubles in the Legendre basis above ("moments"), cell-major.  Below, N = nx*ny is the number of cells.
 *   - Return value: 0 on success, a negative LMDG_ERR_* code otherwise; lmdg_strerror() describes it.
 *   - Vectors passed to lmdg_sweep / lmdg_solve / lmdg_adjoint are DEVICE pointers (cudaMalloc'd memory of
 *     the context's device) unless LMDG_HOST_PTRS is set in flags, in which case they are host pointers and
 *     the call copies through its own device buffers.  The caller owns every buffer it passes.
 *   - stream is a cudaStream_t (NULL = the legacy default stream).  Calls on a context are not thread safe;
 *     use one context per host thread.  Device-pointer calls are asynchronous with respect to the host except
 *     where stated; lmdg_solve and lmdg_adjoint synchronise the stream (they read residual norms).
 *   - No entry point throws; CUDA failures are reported as LMDG_ERR_CUDA.
 */
#ifndef LMDG_H
#define LMDG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lmdg_ctx lmdg_ctx;

/* Scheme: standard S_N-DG with the full Q1 space V_h (eq-sndg-scheme); low-memory LMDG with
 * V_h^lm = V_{h,0} + D_{h,1} (eq-gene-scheme, Section 3.2); reconstructed RLMDG (eq-rlmdg-vari,
 * Section 3.3); P0-DG, the S_N-DG scheme on the piecewise constants V_{h,0} (the comparison scheme of
 * Section 3.1: first order, without the diffusion limit).  For P0-DG the reduced vector keeps the [N][4]
 * layout; its unknown is the cell average (entry 0) and entries 1..3 are carried by the identity. */
enum { LMDG_STD = 0, LMDG_LM = 1, LMDG_RLM = 2, LMDG_P0 = 3 };

/* Arithmetic of the sweeps inside lmdg_solve.  FP64: everything in double.  FP32: sweeps in float inside an
 * FP64 iterative-refinement loop (residuals, GMRES orthogonalisation and least squares stay FP64).
 * FP32_BF16STORE: as FP32, and the angular unknowns written by storing sweeps are bfloat16. */
enum { LMDG_FP64 = 0, LMDG_FP32 = 1, LMDG_FP32_BF16STORE = 2 };

/* Arithmetic of the residual sweeps of the FP32 modes (lmdg_options.resid).  FP64: double.  F32X2: float-float
 * -- each value the unevaluated sum of two floats (48 significant bits, relative error of each operation a few
 * 2^-48 of its operands, float's exponent range), on the FP32 pipe.  The refinement itself (the update of x,
 * the residual norms, GMRES) stays FP64 in both. */
enum { LMDG_RESID_FP64 = 0, LMDG_RESID_F32X2 = 1 };

/* lmdg_sweep flags */
enum {
  LMDG_SWEEP_SOURCE = 1,   /* y = K x - b (affine map whose zero solves the reduced system) instead of y = K x */
  LMDG_SWEEP_FP32 = 2,     /* run the sweep in float (x, y stay double) */
  LMDG_SWEEP_STORE = 4,    /* also store the angular unknowns of this sweep in the context (see lmdg_get_psi) */
  LMDG_HOST_PTRS = 8,      /* x, y (and other vectors of the call) are host pointers */
  LMDG_SWEEP_F32X2 = 16,   /* run the sweep in float-float (see LMDG_RESID_F32X2); not with LMDG_SWEEP_FP32 or
                              LMDG_SWEEP_STORE */
  LMDG_SOLVE_EXACT_REF = 32 /* lmdg_solve, FP32 modes started from zero: take b and the tolerance reference ||b||
                              from a sweep in the residual arithmetic instead of an FP32 sweep (see lmdg_solve) */
};

/* Errors */
enum {
  LMDG_OK = 0,
  LMDG_ERR_ARG = -1,        /* invalid argument (sizes, NULL, eps <= 0, negative cross sections, ...) */
  LMDG_ERR_QUAD = -2,       /* quadrature: sum w != 1, a direction on an axis, or n_Omega not 4 * k */
  LMDG_ERR_NOMEM = -3,      /* device allocation failed */
  LMDG_ERR_CUDA = -4,       /* a CUDA call failed */
  LMDG_ERR_NOTCONV = -5,    /* iteration limit reached before the tolerance (the output still holds the
                               last iterate) */
  LMDG_ERR_TIMEOUT = -6,    /* a sweep kernel gave up waiting for an upstream tile (spin limit); the
                               kernel exits cleanly and the context stays usable */
  LMDG_ERR_BREAKDOWN = -7,  /* non-finite residual or Krylov breakdown */
  LMDG_ERR_STATE = -8       /* call out of order (e.g. lmdg_get_psi before a storing sweep) */
};

typedef struct {
  int nx, ny;          /* cells along x and along y (each >= 1, nx * ny <= 2^30) */
  double x0, y0;       /* lower-left corner */
  double h;            /* cell side (> 0): the domain is [x0, x0 + nx h] x [y0, y0 + ny h] */
} lmdg_mesh;

typedef struct {
  int n;               /* number of directions n_Omega: a multiple of 4, at most 1024 */
  const double *ox;    /* host [n] Omega_x, none zero, |Omega| < 1 (projection of the unit sphere) */
  const double *oy;    /* host [n] Omega_y, none zero */
  const double *w;     /* host [n] positive weights summing to 1 (eq-polyquad (i)) */
} lmdg_quadrature;

typedef struct {
  int precision;       /* LMDG_FP64 (default), LMDG_FP32 or LMDG_FP32_BF16STORE: sweeps inside lmdg_solve */
  int restart;         /* GMRES restart length m (default 30, at most 120) */
  int max_iters;       /* cap on the total number of GMRES iterations (default 5000) */
  double tol;          /* relative residual target ||r_k|| <= tol ||r_0|| (default 1e-8) */
  double inner_tol;    /* FP32 modes: relative tolerance of each inner GMRES solve (default 1e-4) */
  int max_refine;      /* FP32 modes: cap on outer refinement steps (default 50) */
  int precond;         /* right preconditioner of GMRES: 1 (default) diag(I, diag(B11))^-1 for LMDG/RLMDG (the
                          identity for Q1-DG); 0 none; 2 the same followed by the vertex diffusion correction
                          (lmdg_precond_apply) for the diffusive regime; 3 the correction added to the cell-block
                          Jacobi step (optically thick cells) -- 2 and 3 not for LMDG_P0 (LMDG_ERR_ARG) */
  long long spin_limit;/* polls of a readiness flag before a sweep reports LMDG_ERR_TIMEOUT (default 2^26) */
  int device;          /* CUDA device ordinal (default 0) */
  int suppress;        /* LMDG_RLM only, 1: no reconstruction across an interior face where sigma_s or sigma_a
                          changes (the remedy of Section 4 for the kinks at a cross-section discontinuity: the
                          upwind difference across such a face is zero); default 0 */
  int recon;           /* LMDG_RLM only, 1: RLMDG* -- from the third cell on, the reconstructed slope is the centre
                          slope of the quadratic through the cell averages of the cell and its two upwind
                          neighbours, (3 u_i - 4 u_{i-1} + u_{i-2}) / (2h) (the three-cell reconstruction of
                          Section 4.1); not combined with suppress; default 0 (two-cell, Section 3.3.1).  Its
                          sweep amplifies along rays through optically thin cells (sigma_t h below about 0.01 over
                          hundreds of cells), where round-off then dominates.  2: the Q1-type reconstruction
                          (Section 3.3.1 names it without a formula): the two-cell slopes and the xi eta coefficient
                          (h/2)^2 delta_xy, delta_xy the upwind y-difference of the reconstructed x-slopes (over h,
                          and over h/2 against 2 a1 / h, the inflow data's derivative along the y-inflow face);
                          exact for bilinear angular fluxes; not combined with suppress */
  int resid;           /* FP32 modes: arithmetic of the residual sweeps, LMDG_RESID_FP64 (default) or
                          LMDG_RESID_F32X2 */
} lmdg_options;

typedef struct {
  int iters;           /* GMRES iterations (all restarts, all refinement steps) */
  int refinements;     /* outer FP64 refinement steps (FP32 modes), 0 for FP64 */
  int sweeps_fp64;     /* full transport sweeps run in FP64 */
  int sweeps_fp32;     /* full transport sweeps run in FP32 */
  double resid0;       /* tolerance reference ||b - K x0|| (||b|| when starting from zero): from a sweep in the
                          residual arithmetic, or from an FP32 sweep in the FP32 modes started from zero without
                          LMDG_SOLVE_EXACT_REF */
  double resid;        /* final ||b - K x|| from a residual sweep (FP64, or float-float with LMDG_RESID_F32X2) */
  double time_ms;      /* wall time of the call (host clock) */
  double sweep_ms_fp64;/* device time inside FP64 sweep kernels (CUDA events around each launch) */
  double sweep_ms_fp32;/* device time inside FP32 sweep kernels */
  long long launches;  /* kernels launched by the call */
  int sweeps_f32x2;    /* full transport sweeps run in float-float */
  double sweep_ms_f32x2; /* device time inside float-float sweep kernels */
  double kappa_est;    /* largest condition number of a GMRES cycle's Hessenberg matrix (the right-preconditioned
                          operator K M restricted to the cycle's Krylov space: a lower estimate of cond(K M), exact
                          as the space fills).  Two solutions with relative residuals r1, r2 differ relatively by
                          at most about cond (r1 + r2): with this estimate, the error bound the solve states. */
} lmdg_stats;

/* Fill *opt with the defaults listed above. */
int lmdg_default_options(lmdg_options *opt);

/* Create a problem context (setup step: Section 2.1 data).  All inputs are host pointers and are copied.
 *   sigma_s, sigma_a : [N] per-cell cross sections, sigma_s >= 0, sigma_a >= 0, sigma_t > 0 everywhere.
 *   q                : source as Legendre moments; q_layout 0: [N] cell constants; 1: [N][4];
 *                      2: [n_Omega][N][4] angle dependent (Section 4.1 allows q to depend on angle).
 *   alpha            : inflow data (the boundary condition Psi = alpha on the inflow boundary, eq-main), NULL for
 *                      vacuum.  alpha_layout 0: alpha points to one value, the same constant on every inflow face
 *                      for every direction.  alpha_layout 1: [n_Omega][2 ny + 2 nx][2]: per direction the
 *                      boundary faces of the west side (x = x0, ny faces by row j), the east side (ny), the south
 *                      side (y = y0, nx faces by column i) and the north side (nx), each with the coefficients
 *                      (a0, a1) of alpha = a0 + a1 t along the face, t in [-1, 1] increasing with the global
 *                      coordinate.  Only inflow faces are read.  The reconstruction of RLMDG uses a0 as the
 *                      face-midpoint value of alpha (Section 3.3.1).  Other layouts return LMDG_ERR_ARG.
 *   eps              : scaling parameter epsilon > 0 of eq-main.
 *   variant          : LMDG_STD, LMDG_LM, LMDG_RLM or LMDG_P0.
 *   opt              : NULL for defaults.
 * Device memory: O(n_Omega * N) for the angular-flux store, O(N) for the rest. */
int lmdg_setup(lmdg_ctx **out, const lmdg_mesh *mesh, const lmdg_quadrature *quad,
               const double *sigma_s, const double *sigma_a, const double *q, int q_layout,
               const double *alpha, int alpha_layout, double eps, int variant, const lmdg_options *opt);

/* One application of the sweep-reduced operator (one transport sweep over all directions with the angular
 * reduction fused into it), on vectors of [N][4] doubles:
 *   LMDG_STD : K x = x - P L^-1 M x  (eq-sndg-phi), x = Phi, the scalar-flux moments;
 *              b = P L^-1 Q.
 *   LMDG_LM  : K [X0; X1] of eq-lmdg-reducemat, evaluated as in eq-nonrec-block; x = (X0, X1) per cell;
 *              b = the right-hand side of eq-lmdg-reducemat minus K [0; z], z = B11^-1 Sigma Q1.
 *   LMDG_RLM : the reduced RLMDG operator of Section 3.3.2 with the second block row
 *              G' = Sigma Ltilde10 + B11 P1 R (with X1 = (B11^-1 Sigma Ltilde10 + P1 R) Psi0 the printed row
 *              Sigma Ltilde10 leaves a B11 P1 R Psi0 term unclosed);
 *              b = its right-hand side minus K [0; z], z = B11^-1 Sigma Qtilde1.
 * With LMDG_SWEEP_SOURCE the call returns y = K x - b, so that the solution of lmdg_solve zeroes it (for the
 * low-memory variants this is the paper's system written for the shifted unknown X1 - z, i.e. GMRES started
 * from X1 = z).  LMDG_SWEEP_STORE keeps this sweep's angular unknowns: psi [n_Omega][N][4] for LMDG_STD,
 * psi0 [n_Omega][N] for the low-memory variants (bfloat16 for an FP32 sweep when the context's precision is
 * LMDG_FP32_BF16STORE).  LMDG_SWEEP_FP32 / LMDG_SWEEP_F32X2 run the sweep in float /
 * float-float (x and y stay double); LMDG_SWEEP_F32X2 with LMDG_SWEEP_FP32 or LMDG_SWEEP_STORE returns
 * LMDG_ERR_ARG.  Asynchronous on stream for device pointers. */
int lmdg_sweep(lmdg_ctx *ctx, const double *x, double *y, int flags, void *stream);

/* Solve the reduced system with restarted GMRES (right-preconditioned, see lmdg_options.precond), then run
 * the recovery sweep (eq-sndg-final-sweep, eq-lm-step4 and its RLMDG analogue), storing the angular unknowns.
 * FP32 modes: the first iterate comes from FP32 sweeps alone (an FP32 right-hand side and one FP32 GMRES
 * cycle); every later step computes the residual b - K x with a sweep in the residual arithmetic (FP64, or
 * float-float with LMDG_RESID_F32X2), runs FP32-sweep GMRES on it and updates x in FP64 (iterative
 * refinement).  Convergence is ||b - K x|| <= tol ||b||, the residual in the residual arithmetic.  The reference
 * ||b||: from x0 = 0 in the FP32 modes it is the norm of the FP32 right-hand side, which differs from the exact
 * ||b|| by the FP32 sweep's normwise relative error (below 1e-5 on the tested problems), so the relative residual
 * reached is tol (1 + that error); with LMDG_SOLVE_EXACT_REF in flags b comes from a residual-arithmetic sweep
 * instead (one such sweep in place of an FP32 one) and the bound is tol itself.  With x0 given, or in FP64, the
 * reference is ||b - K x0|| from a residual-arithmetic sweep.
 *   x0  : initial guess [N][4] (NULL = zero), in the unknowns of lmdg_sweep with LMDG_SWEEP_SOURCE.
 *   x   : output [N][4], the converged unknowns (may be NULL).
 *   phi : output [N][4], the scalar-flux moments sum_l w_l psi_l of the discrete solution (may be NULL).
 *   stats: may be NULL.
 * Returns LMDG_ERR_NOTCONV (with outputs written) if max_iters is reached. */
int lmdg_solve(lmdg_ctx *ctx, const double *x0, double *x, double *phi, lmdg_stats *stats, int flags,
               void *stream);

/* Copy the angular unknowns kept by the last storing sweep (lmdg_solve always stores) to psi:
 * LMDG_STD [n_Omega][N][4], low-memory variants [n_Omega][N] (cell averages psi0; the isotropic slopes
 * are the phi output of lmdg_solve).  Directions in the order given to lmdg_setup. */
int lmdg_get_psi(lmdg_ctx *ctx, double *psi, int flags, void *stream);

/* Adjoint sensitivities of the detector functional J = sum_K g_K int_K Psi_bar dx (g: [N] weights) with
 * respect to the per-cell sigma_s, sigma_a and the per-cell constant source q (no counterpart in the paper:
 * the discrete adjoint of its schemes), for LMDG_STD and LMDG_LM with q_layout 0 or 1.  Requires a centrally
 * symmetric quadrature (LMDG_ERR_QUAD otherwise): then the transpose of each direction's upwind block is the
 * block of the opposite direction, so the adjoint system is the forward reduced system with the detector
 * response as source; the forward angular flux is stored (FP64) and correlated cell by cell with the adjoint one
 * in a final sweep.  Outputs [N] each (any may be NULL) and J.  RLMDG (a Petrov-Galerkin scheme whose adjoint
 * has reconstructed test functions) returns LMDG_ERR_ARG. */
int lmdg_adjoint(lmdg_ctx *ctx, const double *g, double *dJ_dsigma_s, double *dJ_dsigma_a,
                 double *dJ_dq, double *J, lmdg_stats *stats, int flags, void *stream);

/* B11 = Sigma L11 Sigma^T - Sigma M1 of eq-lmdg-psi1 (the isotropic-slope block) applied to x [N][3]:
 * y [N][3].  Provided for the paper-literal reduced right-hand side and for checking. */
int lmdg_b11_apply(lmdg_ctx *ctx, const double *x, double *y, int flags, void *stream);

/* Solve B11 z = r by conjugate gradients (B11 is SPD for centrally symmetric quadratures, Theorem
 * lem-B11) to relative residual tol; iters (may be NULL) receives the iteration count. */
int lmdg_b11_solve(lmdg_ctx *ctx, const double *r, double *z, double tol, int *iters, int flags,
                   void *stream);

/* y = Minv x: the right preconditioner that lmdg_solve applies before every sweep, on [N][4] vectors (no
 * counterpart in the paper, which leaves preconditioning to future work).  precond 1: the Jacobi scaling
 * diag(I, diag(B11))^-1 of the low-memory schemes (identity for Q1-DG).  precond 2: that scaling, then the
 * vertex diffusion correction u -> u + I_h D_a^-1 R_h (sigma_s/eps) u: K ~ D_t^-1 D_a on the slowly converging
 * modes of the diffusive regime (D_t = -div D grad + sigma_t, D_a = -div D grad + eps sigma_a, D = 1/(3 sigma_t)),
 * so K^-1 ~ I + D_a^-1 (sigma_s/eps).  D_a is each scheme's diffusion limit on the continuous Q1 functions of
 * the (nx+1) x (ny+1) vertices (Section 3.1): int D grad d . grad v for Q1-DG (eq-lmdg-cg), int D Pi_0(grad d) .
 * Pi_0(grad v) for LMDG and RLMDG (eq-difflimPF), plus int eps sigma_a d v and the vacuum boundary term
 * sum over sides of A_n int d v (A_n = sum_{Omega.n > 0} w Omega.n); R_h tests the cell function against the
 * vertex hat functions, I_h takes the bilinear interpolant's Legendre moments; for the low-memory schemes u
 * holds (X0, X1) and the scalar-flux slopes are -X1.  D_a^-1 is one geometric multigrid V-cycle (bilinear
 * prolongation, two components per coarse vertex below the finest level of the cell-average operator, Galerkin
 * coarse operators, two damped block-Jacobi steps (omega = 0.7) before and after, dense coarsest solve up to
 * 1156 unknowns, else 50 Jacobi steps; levels halve nx and ny while both are even and above 2), built by
 * lmdg_setup.  precond 3: y = B^-1 x + C(J x), C the correction above, J the scaling of precond 1 and B the
 * cell-diagonal blocks of K (one 4 x 4 block per cell: the part of K e_(K,r) in cell K, found by lmdg_setup with
 * four FP64 sweeps in which no cell sees upwind data, and inverted per cell; LMDG_ERR_BREAKDOWN from lmdg_setup if
 * a block has no usable pivot).  In optically thick cells most slow modes of the iteration change from cell to
 * cell and no vertex function carries them; on these K acts through its diagonal blocks to leading order.
 * x and y distinct; asynchronous on stream for device pointers. */
int lmdg_precond_apply(lmdg_ctx *ctx, const double *x, double *y, int flags, void *stream);

/* Operator application that allocates nothing (no counterpart in the paper: it is a deployment variant of
 * lmdg_sweep's homogeneous mode, y = K x, for callers that cannot call cudaMalloc -- e.g. a host framework
 * that owns all device memory through its own pool, a latency-critical loop that cannot take cudaMalloc's
 * implicit device synchronisation, or an embedding runtime that hands over only input and output buffers).
 *   variant          : LMDG_STD, LMDG_LM or LMDG_RLM.
 *   n, h             : n x n cells of side h.
 *   n_omega, ox, oy, w : DEVICE arrays [n_omega] of directions and weights, grouped by quadrant in the order
 *                      (+,+), (-,+), (-,-), (+,-) with n_omega/4 directions each; n_omega a multiple of 4, at
 *                      most 1024.  The grouping is checked on the device before the sweep: a direction whose
 *                      signs do not match its quadrant slot, or that lies on an axis, returns LMDG_ERR_QUAD.
 *   sigma_t          : DEVICE [n*n] sigma_s/eps + eps sigma_a;  sigma_s_over_eps : DEVICE [n*n] sigma_s/eps.
 *   x, y             : DEVICE [n*n][4] doubles, 16-byte aligned (x: input, y: output, distinct).
 *   spin_limit       : polls of a readiness flag before giving up with LMDG_ERR_TIMEOUT.
 * The sweep's scratch (strip traces, partial reductions, control words) is a fixed 16 MiB device array
 * reserved on every GPU that loads the library until the process exits; problems whose scratch does not fit
 * (roughly n*n*(136 to 232) + n_omega*n^2*0.75 bytes) are rejected with LMDG_ERR_ARG.  The first call on a
 * device (with that device current) looks the array up and initialises it: make that call before any stream
 * capture.  Calls share the array; calls whose kernels overlap on the GPU race and must be serialised.  The
 * call synchronises the stream to read the sweep's error word. */
int lmdg_sweep_noalloc(int variant, int n, double h, int n_omega, const double *ox, const double *oy,
                       const double *w, const double *sigma_t, const double *sigma_s_over_eps,
                       const double *x, double *y, long long spin_limit, void *stream);

/* ---- Angle sharding (Section 2.1.1: L is block diagonal over the directions, so every direction's sweep is
 * independent and only the angular reduction couples them).  A sweep's reduction is formed from "partial sets":
 * one per (quadrant, direction group) of the launch shape, each an [N][NR] array (NR reduced values per cell) in
 * the sweep's arithmetic (double; float for LMDG_SWEEP_FP32; a pair of floats, 8 bytes, for LMDG_SWEEP_F32X2),
 * summed by the epilogue in a fixed order.  Sharding splits the sets into nshards contiguous chunks of chunk_sets
 * sets; shard r sweeps the directions of chunk r over the whole mesh (on its own GPU, with its own context of the
 * same problem), the chunks are gathered into one buffer (an all-gather between the GPUs), and lmdg_sweep_combine
 * then gives a result bitwise equal to lmdg_sweep.  A partial buffer holds nshards * chunk_sets sets (chunk r at
 * byte offset r * chunk_bytes; sets past the last one are padding).  Contexts of one problem set up with the same
 * arguments (and the same LMDG_SWEEP_GEOM environment) have the same layout. */

/* Layout of the partial sets for the arithmetic of flags (LMDG_SWEEP_FP32 / LMDG_SWEEP_F32X2 / neither) split
 * into nshards chunks (1 <= nshards <= 4096): the number of sets, the sets per chunk and the bytes per chunk (any
 * pointer may be NULL). */
int lmdg_shard_layout(const lmdg_ctx *ctx, int flags, int nshards, int *sets, int *chunk_sets, size_t *chunk_bytes);

/* Sweep the directions of chunk `shard` of nshards at x (DEVICE [N][4]) and write their partial sets into chunk
 * `shard` of parts (DEVICE, nshards * chunk_bytes bytes, 16-byte aligned; the other chunks are not touched).
 * flags: LMDG_SWEEP_SOURCE, LMDG_SWEEP_FP32 or LMDG_SWEEP_F32X2, LMDG_SWEEP_STORE (stores this shard's directions
 * only: lmdg_get_psi then returns them, the other directions' entries being whatever the context held before);
 * LMDG_HOST_PTRS returns LMDG_ERR_ARG, and so does float-float with FP32 or with storing.  Errors: LMDG_ERR_ARG
 * (NULL pointers, shard outside [0, nshards), nshards outside [1, 4096]), LMDG_ERR_TIMEOUT, LMDG_ERR_CUDA,
 * LMDG_ERR_NOMEM (the stored unknowns).  Synchronises the stream (reads the sweep's error word). */
int lmdg_sweep_shard(lmdg_ctx *ctx, const double *x, void *parts, int shard, int nshards, int flags,
                     void *stream);

/* The epilogue of lmdg_sweep from a complete partial buffer (every chunk written by lmdg_sweep_shard, here or on
 * other GPUs): y = K x, or K x - b with LMDG_SWEEP_SOURCE, as lmdg_sweep gives for the same flags; x, parts, y
 * DEVICE pointers (parts as laid out by lmdg_shard_layout for these flags; a chunk not written holds whatever the
 * buffer held).  LMDG_ERR_ARG for NULL pointers, host pointers, LMDG_SWEEP_STORE, or float-float with FP32.
 * Asynchronous on stream. */
int lmdg_sweep_combine(lmdg_ctx *ctx, const double *x, const void *parts, double *y, int flags, void *stream);

/* Problem sizes of a context: cells along x and y, n_Omega, variant (any pointer may be NULL). */
int lmdg_info(const lmdg_ctx *ctx, int *nx, int *ny, int *n_omega, int *variant);

/* Free every device buffer of the context.  NULL is ignored. */
void lmdg_destroy(lmdg_ctx *ctx);

/* Static description of an error code. */
const char *lmdg_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* LMDG_H */
