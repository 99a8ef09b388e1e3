/*
 * ssd.h -- C ABI of libssd: regularized boundary integrals for the coupled
 * Stokes-Darcy problem solved by Dirichlet-Neumann domain decomposition
 * (Tlupova, "A domain decomposition solution of the Stokes-Darcy system in
 * 3D based on boundary integrals", arXiv 2110.10749).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every call returns an int status (enum ssd_status).  On failure the
 *   context keeps a one-line message, read with ssd_ctx_last_error().
 * - n is the outward unit normal of the porous body, i.e. it points into the
 *   fluid (the paper's n_D on the interface; n_S = -n).  yhat = y - x for a
 *   target y and a source x, r = |yhat|, rho = r / delta.
 * - Point sets and densities are structure-of-arrays in FP64:
 *   xyz[3][n] = x row, y row, z row; a vector density u[3][n] likewise.
 * - Buffers passed to ssd_* calls are DEVICE pointers owned by the caller,
 *   unless a parameter is marked "host".  The library owns the context, its
 *   workspace and the prepared layouts; it never frees caller memory.
 * - Operator calls (ssd_laplace_*, ssd_stokes_* without _solve) are
 *   asynchronous on the given stream.  Quadrature, solver and layout calls
 *   synchronise the stream before they return, because they report counts
 *   or iteration results to the host.
 * - prec selects the arithmetic of the pair sums: SSD_FP64 (plain double) or
 *   SSD_FP32C (single precision pair terms, compensated two-float
 *   accumulation per target, FP64 epilogue).  Krylov and interface
 *   arithmetic is always FP64.
 * - Non-finite scalar arguments, n <= 0, delta <= 0, mu <= 0, kappa <= 0,
 *   theta outside (0,1] and NULL required pointers give SSD_EINVAL before any
 *   work is enqueued.
 * - A context is used by one host thread at a time.  Its workspace is a
 *   cache of device blocks handed out again as soon as a call has enqueued
 *   its work, so the work of one context must stay in one stream order: use
 *   one stream per context, or order the streams yourself (an event from the
 *   previous call's stream) before a call on another stream.
 */
#ifndef SSD_H
#define SSD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ssd_ctx ssd_ctx;
typedef struct ssd_layout ssd_layout;
/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *ssd_stream;

enum ssd_status {
    SSD_OK = 0,
    SSD_EINVAL = 1,    /* invalid argument */
    SSD_ENOMEM = 2,    /* device or pinned allocation failed */
    SSD_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
    SSD_ENOTCONV = 4,  /* iteration limit reached; outputs hold the last iterate */
    SSD_ENUMERIC = 5   /* NaN or Inf appeared in a residual */
};

enum ssd_precision { SSD_FP64 = 0, SSD_FP32C = 1 };

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` (which becomes current for the
 * calling thread).  *ctx receives the handle.
 *
 * Tuning read from the environment at creation (all optional):
 *   SSD_PAIR_SYM=0      no symmetric far-block plans: every operator on a
 *                       prepared layout runs the direct kernels, whose split
 *                       sums are added in a fixed order (results reproducible
 *                       bit for bit); with the plans (default) the far block
 *                       pairs of the four layer operators are evaluated once
 *                       for both directions and summed by FP64 atomic adds,
 *                       so results vary in the last bits of an FP64 sum
 *   SSD_PAIR_LPT=0      direct FP32C/FP64 grids in plain (tile, split) order
 *                       instead of near-first order
 *   SSD_PAIR_WAVES=k    FP32C direct grid sized for k (1..64) waves of resident CTAs
 *   SSD_PAIR_WAVES64=k  the same for the FP64 direct grid */
int ssd_ctx_create(ssd_ctx **ctx, int device);
/* Free the context, its workspace and layouts.  NULL is accepted. */
int ssd_ctx_destroy(ssd_ctx *ctx);
/* Static text of a status code. */
const char *ssd_status_string(int status);
/* Message of the last failure on this context ("" if none). */
const char *ssd_ctx_last_error(const ssd_ctx *ctx);

/* Kernel timing.  When enabled, the library brackets every pair-sum launch
 * with CUDA events on the launching stream.  Statistics per kernel class
 * (enum ssd_kernel_class) accumulate until reset; reading them synchronises
 * the recorded events.  pairs counts ordered (target, source) pairs. */
enum ssd_kernel_class {
    SSD_K_LAPLACE_SL = 0, SSD_K_LAPLACE_DL = 1, SSD_K_STOKES_SL = 2,
    SSD_K_STOKES_DL = 3, SSD_K_STOKES_SLDL = 4, SSD_K_LAPLACE_SLDL = 5,
    SSD_K_LAPLACE_DL_T = 6, SSD_K_STOKES_DL_T = 7,
    SSD_K_COUNT = 8
};
typedef struct {
    int64_t launches;  /* pair-sum kernel launches */
    double ms;         /* summed device time of those launches */
    double pairs;      /* ordered pairs evaluated */
} ssd_kernel_stats;
int ssd_ctx_set_timing(ssd_ctx *ctx, int enable);
int ssd_ctx_kernel_stats(ssd_ctx *ctx, int kernel_class, int precision, ssd_kernel_stats *out /* host */);
int ssd_ctx_reset_stats(ssd_ctx *ctx);
/* Total kernel launches the library issued since the context was created
 * (every kernel of the library, not only the pair sums). */
int ssd_ctx_launch_count(const ssd_ctx *ctx, int64_t *out /* host */);
/* Wait for the work queued on `stream` (on the whole device when stream is
 * NULL) and report failures of asynchronous calls: the operator, row-block,
 * batched-application and field calls return once their kernels are queued,
 * so a kernel that fails there surfaces here as SSD_ECUDA (SSD_ENOMEM for an
 * allocation), with the CUDA error text in ssd_ctx_last_error.  SSD_EINVAL
 * when the calling thread's current device is not the context's. */
int ssd_sync(ssd_ctx *ctx, ssd_stream stream);
/* Measurement aid (the paper has no counterpart): the FP32 FMA rate this
 * device reaches, in TFLOP/s (FMA = 2 flops), from a kernel that keeps 16
 * independent FMA chains per thread on every SM (packed = 1: as f32x2
 * FFMA2 instructions, the form the pair kernels use; 0: scalar FFMA).
 * Synchronises the device's legacy stream. */
int ssd_fp32_fma_rate(ssd_ctx *ctx, int packed, double *tflops /* host */);

/* ------------------------------------------------------------- quadrature */

/* Surfaces: level sets phi = 0 with phi > 0 outside.  SPHERE and ELLIPSOID
 * are eqs. Sphere and Ellipsoid of Section 5.4 (SPHERE uses abc[0] as the
 * radius).  STAR is the star-shaped surface |x - c| = r(xi),
 * r(xi) = 1 + sum_{l<=4} sum_{m=-l..l} c_lm Y_lm(xi), xi = (x - c)/|x - c|,
 * with real orthonormal spherical harmonics (Condon-Shortley phase removed:
 * Y_l,m = sqrt(2) (-1)^m Re Y_l^m for m > 0, sqrt(2) (-1)^m Im Y_l^|m| for
 * m < 0) and clm[k], k = l^2 + l + m, 25 coefficients; phi = (|x - c| - 1) -
 * sum_k c_k Y_k(xi).  The sum of |c_lm| sqrt((2l+1)/(4 pi)) must be < 1.
 * The paper's own examples are the sphere and the ellipsoid; star surfaces
 * are smooth test shapes of the same construction. */
enum ssd_surface_kind { SSD_SPHERE = 0, SSD_ELLIPSOID = 1, SSD_STAR = 2, SSD_MOLECULE = 3 };
/* SSD_MOLECULE is the four-atom molecule of eq. Molecule, centres
 * (sqrt3/3, 0, -sqrt6/12), (-sqrt3/6, +-1/2, -sqrt6/12), (0, 0, sqrt6/4) shifted by
 * center, sum_k exp(-|x - x_k|^2/r^2) = c with r = abc[0], c = abc[1] (0 selects the
 * paper's r = 0.5, c = 0.6).  Its roots follow the star surfaces' sampling and
 * bisection on [min_k x_k,i - D, max_k x_k,i + D], D = 1.0625 r sqrt(log(4/c)). */
typedef struct {
    int kind;
    double center[3];
    double abc[3];       /* semi-axes (ELLIPSOID); abc[0] = R (SPHERE) */
    const double *clm;   /* host [25] (STAR only; may be NULL otherwise) */
} ssd_surface;

/*
 * Quadrature points of Section 5.4 (eq. Quadrature).  For each axis e_i the
 * grid lines of spacing h anchored at the origin, through (j1 h, j2 h) in the
 * other two coordinates, are intersected with the surface; an intersection x
 * is kept when |n(x) . e_i| >= cos(angle_deg) and gets the weight
 * psi_i(n) h^2 / |n_i|, with psi_i = b(acos|n_i|/theta) / sum_j b(acos|n_j|/theta),
 * b(r) = exp(r^2/(r^2-1)) for |r| < 1 (theta = angle_deg in radians).
 * Order: axis 0,1,2; j1 ascending; j2 ascending; smaller root first.
 * meta[4][n] = (axis, j1, j2, ordinal of the crossing along its line).
 * Sphere and ellipsoid roots are closed forms.  Star-surface roots follow a
 * fixed procedure: with Rb = 1 + sum |c_k| sqrt((2l+1)/(4 pi)), phi is sampled
 * at t_k = t_lo + k dt, t_lo = c_i - 1.0625 Rb, dt = ((c_i + 1.0625 Rb) - t_lo)/K,
 * K = ceil(2.125 Rb * 64); each sign change (phi > 0 against not) is bisected
 * (mid = 0.5 (lo + hi)) until the midpoint equals an end point, and the end
 * point with the smaller |phi| is the root.  More than 8 kept crossings on
 * one line is an error (SSD_EINVAL).
 * Pass xyz == NULL to query the count only (*n_out).  Otherwise capacity
 * must be >= the count (else SSD_EINVAL with *n_out set to the count).
 * Points and normals are computed with correctly rounded +,-,*,/,sqrt only.
 * Synchronises `stream`.
 */
int ssd_quadrature_points(ssd_ctx *ctx, const ssd_surface *surf /* host */, double h,
                          double angle_deg, int64_t capacity, int64_t *n_out /* host */,
                          double *xyz, double *nrm, double *w, int32_t *meta,
                          ssd_stream stream);

/*
 * Shape derivatives of a STAR surface's quadrature set with respect to its 25
 * coefficients c_k, at fixed h and angle: dxyz[k][3][n], dnrm[k][3][n],
 * dw[k][n] (device), in the order of ssd_quadrature_points; n must equal its
 * point count.  A point moves along its grid line (dx = e_i dt); normals and
 * weights follow from the normal formula and the partition of unity.  The
 * set itself is held fixed: a point entering or leaving it does so with zero
 * weight, so sums over the set stay differentiable.  The paper states no
 * shape derivatives; these are derivatives of its quadrature rule.
 * Synchronises `stream`.
 */
int ssd_quadrature_jacobian(ssd_ctx *ctx, const ssd_surface *surf /* host */, double h,
                            double angle_deg, int64_t n, double *dxyz, double *dnrm, double *dw,
                            ssd_stream stream);

/* ----------------------------------------------------------------- points */

typedef struct {
    int64_t n;
    const double *xyz;   /* [3][n] device */
    const double *nrm;   /* [3][n] device, unit outward normals */
    const double *w;     /* [n] device, quadrature weights */
    ssd_layout *layout;  /* optional: from ssd_points_prepare(); NULL = per-call packing */
} ssd_points;

/* Build a device layout of the point set for the pair kernels: FP32 copies
 * of positions, weighted normals and weights in a spatially sorted order,
 * and per-tile bounding boxes for the near/far split.  Stores the handle in
 * pts->layout.  The layout refers to the point data by value: it must be
 * rebuilt if the points change.  Synchronises `stream`. */
int ssd_points_prepare(ssd_ctx *ctx, ssd_points *pts /* host struct */, ssd_stream stream);
/* Release a layout built by ssd_points_prepare and clear pts->layout. */
int ssd_points_release(ssd_ctx *ctx, ssd_points *pts /* host struct */);

/* ---------------------------------------------------------- layer operators
 * All four follow Sections 5.1-5.3 with the smoothed kernels of Section 5.3:
 *   s1 = erf(rho) - 2/(3 sqrt(pi)) rho (2 rho^2 - 5) e^{-rho^2}
 *   s2 = erf(rho) + 2/(3 sqrt(pi)) rho (2 rho^2 - 3) e^{-rho^2}
 *   s3 = erf(rho) - 2/(3 sqrt(pi)) rho (4 rho^4 - 14 rho^2 + 3) e^{-rho^2}
 *   s4 = erf(rho) - 2/(9 sqrt(pi)) rho (8 rho^6 - 36 rho^4 + 6 rho^2 + 9) e^{-rho^2}
 * summed over every quadrature point x_j (weight w_j) for every target
 * y_i = x_i, the self pair included at its finite limit.
 */

/* (L g)(y) = sum_x w g G^delta,  G^delta = -s1(rho) / (4 pi r)  (Section 5.1, 5.3). */
int ssd_laplace_SL(ssd_ctx *ctx, const ssd_points *pts, double delta, const double *g,
                   double *out, int prec, ssd_stream stream);
/* (D^L p)(y) = sum_x w [p(x) - p(y)] dG^delta/dn_x,
 * dG^delta/dn_x = -(yhat . n_x) s2(rho) / (4 pi r^3).  D^L = H - I/2 (eq. H_subtr). */
int ssd_laplace_DL(ssd_ctx *ctx, const ssd_points *pts, double delta, const double *p,
                   double *out, int prec, ssd_stream stream);
/* (M f)(y) = 1/(8 pi mu) sum_x w S^delta f,
 * S^delta_ab = delta_ab s1/r + yhat_a yhat_b s3/r^3  (Section 5.2, 5.3).  f, out [3][n]. */
int ssd_stokes_SL(ssd_ctx *ctx, const ssd_points *pts, double delta, double mu,
                  const double *f, double *out, int prec, ssd_stream stream);
/* (D^S u)(y) = -1/(8 pi) sum_x w [u(x) - u(y)]_a T^delta_abc n_c(x),
 * T^delta_abc = -6 yhat_a yhat_b yhat_c s4/r^5.  D^S = K + I/2 (eq. K_subtr).  u, out [3][n]. */
int ssd_stokes_DL(ssd_ctx *ctx, const ssd_points *pts, double delta, const double *u,
                  double *out, int prec, ssd_stream stream);
/* The Stokes double layer of ssd_stokes_DL in FP32C, without any device
 * allocation.  The paper has no counterpart: this call is for callers that
 * cannot call cudaMalloc at this point, for example code whose device memory
 * is reserved up front by another allocator (so a new allocation can fail),
 * or code that must not trigger the device-wide synchronisation a cudaFree
 * implies.  Inputs and output are the caller's (pts->layout is ignored; the
 * points are used in caller order).  Scratch: one file-scope device array of
 * 16 MiB, held on every device that loads the library until the process
 * exits.  Limit: n rounded up to a multiple of 512 must not exceed 32768
 * (larger sets give SSD_EINVAL before any work).  The context's device must
 * be the current device (SSD_EINVAL otherwise).  The first call with a given
 * ssd_ctx looks up the array's device address and keeps it in the ssd_ctx;
 * make that call before any stream capture.  Like all of an ssd_ctx's device
 * state, the address belongs to the CUDA context current when it was taken:
 * use the ssd_ctx under that CUDA context only, and destroy it before a
 * cudaDeviceReset.  All calls share the array: calls whose work can overlap
 * on the GPU (other streams, other host threads) race and must be serialised
 * by the caller.  Asynchronous on `stream`. */
int ssd_stokes_DL_noalloc(ssd_ctx *ctx, const ssd_points *pts, double delta, const double *u,
                          double *out, ssd_stream stream);
/* Row blocks of the four operators, for splitting one application over
 * several devices (each holds the whole point set and density and computes
 * its own rows; one gather of the results per application).  Rows are
 * positions in the point set's spatial order (the layout order that
 * ssd_points_prepare builds, or an equal temporary one): row k is caller
 * point order[k] of ssd_points_order.  Computes out[c][order[k]] for
 * row_begin <= k < row_end only (the other entries of out are not written),
 * with the direct kernels and the whole application's splits, so bit-identical
 * to the same entries of the whole application whenever that runs the direct
 * kernels too (SSD_PAIR_SYM=0, or a layout below the symmetric plans' share of
 * far block pairs); where the whole application runs a symmetric plan the two
 * agree to the rounding of the precision.  op: 0 = L
 * (ssd_laplace_SL), 1 = D^L (ssd_laplace_DL), 2 = M (ssd_stokes_SL, mu
 * used), 3 = D^S (ssd_stokes_DL); dens, out as for that call.  SSD_EINVAL
 * unless 0 <= row_begin < row_end <= n.  Asynchronous on `stream`. */
int ssd_apply_rows(ssd_ctx *ctx, const ssd_points *pts, int op, double delta, double mu,
                   const double *dens, int64_t row_begin, int64_t row_end, double *out,
                   int prec, ssd_stream stream);
/* The spatial order of a point set: order[k] (host, [n]) = caller index of
 * row k.  Synchronises `stream`. */
int ssd_points_order(ssd_ctx *ctx, const ssd_points *pts, int32_t *order, ssd_stream stream);
/* One pass sharing r, erf and exp between both layers:
 * out = alpha (M f) + beta (D^S u)   [Stokes],   out = alpha (L g) + beta (D^L p)   [Laplace].
 * Used for the right-hand sides and residuals b - A x of the local solves. */
int ssd_stokes_SLDL(ssd_ctx *ctx, const ssd_points *pts, double delta, double mu,
                    const double *f, const double *u, double alpha, double beta,
                    double *out, int prec, ssd_stream stream);
int ssd_laplace_SLDL(ssd_ctx *ctx, const ssd_points *pts, double delta, const double *g,
                     const double *p, double alpha, double beta, double *out, int prec,
                     ssd_stream stream);

/*
 * Transposes of the discrete operators, for adjoint (reverse-mode) solves.
 * With A the matrix that ssd_laplace_SL / _DL / ssd_stokes_SL / _DL apply
 * (op = enum ssd_operator, SL or DL only), out = A^T dens:
 *   single layers: A = S W with S symmetric, so A^T v = W S v (w at the target);
 *   Laplace DL:  (A^T v)_i = 1/(4 pi) sum_j s2/r^3 [(yhat.w_i n_i) v_j + (yhat.w_j n_j) v_i];
 *   Stokes DL:   (A^T v)_i = -3/(4 pi) sum_j s4/r^5 yhat [(yhat.w_i n_i)(yhat.v_j) + (yhat.w_j n_j)(yhat.v_i)],
 * yhat = x_i - x_j (the second terms are the transposed subtraction).
 * mu is used by the Stokes single layer only.  Asynchronous on `stream`.
 */
int ssd_apply_transpose(ssd_ctx *ctx, const ssd_points *pts, int op, double delta, double mu,
                        const double *dens, double *out, int prec, ssd_stream stream);

/* ------------------------------------------------------------ local solves */

typedef struct {
    double tol;    /* stop when ||b - A x|| <= tol ||b|| (GMRES estimate) or, for SA,
                      when ||x_k - x_{k-1}|| <= tol ||x_k|| */
    int maxit;     /* total iteration limit */
    int restart;   /* GMRES restart length m (1..512; batched solves 1..256) */
    int use_sa;    /* 1: successive approximations (eqs. Darcy_BIEM_iter,
                      Stokes_BIEM_iter) instead of GMRES */
    int prec;      /* enum ssd_precision of the pair sums */
    int deflate;   /* Stokes solves: 1 adds n (w . (u.n))/sum(w) to the operator.  The
                      continuous I/2 - K has the normal field in its null space, so
                      I - D^S has a near-null vector (eigenvalue O(h^5)) that amplifies
                      rounding, most of all in FP32C; the rank-one term removes it and
                      selects the zero-net-flux solution (int u.n dS = 0, the Darcy
                      compatibility condition).  0 = the operator as printed. */
    int warm;      /* 1: start from a previous solution instead of 0.  In relaxed D-N
                      sweeps (outer_gmres = 0) each local solve starts from the previous
                      sweep's solution; ssd_darcy_solve / ssd_stokes_solve start from
                      the values already in their output array.  Ignored by the
                      interface GMRES's sweeps and by batched solves. */
} ssd_krylov;

/*
 * Darcy pressure on the interface (eq. Darcy_final): 1/2 p = H p + b_D with
 * b_D = (mu/kappa) L q, q = u_D . n the normal Darcy velocity.  Solved as
 * -D^L p + (w . p)/sum(w) = b_D: the operator annihilates constants and the
 * rank-one term fixes the gauge without changing the solution of a
 * consistent system.  p_out has zero quadrature-weighted mean.
 * iters, relres: host.  Synchronises `stream`.
 */
int ssd_darcy_solve(ssd_ctx *ctx, const ssd_points *pts, double delta, double mu,
                    double kappa, const double *q, double *p_out, const ssd_krylov *kr,
                    int *iters, double *relres, ssd_stream stream);
/*
 * Stokes velocity on the interface (eq. Stokes_final): 1/2 u = K u + b_S with
 * b_S = U_inf - M f, solved as (I - D^S) u = b_S.  f, u_out [3][n];
 * uinf, iters, relres: host.  Synchronises `stream`.
 */
int ssd_stokes_solve(ssd_ctx *ctx, const ssd_points *pts, double delta, double mu,
                     const double *f, const double uinf[3], double *u_out,
                     const ssd_krylov *kr, int *iters, double *relres, ssd_stream stream);

/* ------------------------------------------------- Dirichlet-Neumann solve */

enum ssd_traction_mode {
    SSD_TRACTION_BJS = 0,         /* f = -p_D n + s (gamma/sqrt(kappa)) (u - (u.n) n), eq. f */
    SSD_TRACTION_JOSEPH_TAO = 1   /* porous-sphere benchmark of Section 7.3 (eqs. f_r, f_theta) */
};

typedef struct {
    double mu, kappa, gamma;   /* viscosity, permeability, BJS coefficient */
    double uinf[3];            /* far-field velocity */
    double delta;              /* smoothing radius (the paper uses 3h) */
    double theta;              /* relaxation (eq. q_update), in (0,1] */
    double tol_outer;          /* DDM residual (SA) or interface GMRES tolerance */
    int maxit_outer;
    int outer_gmres;           /* 0: relaxed sweeps (SA); 1: GMRES on the interface */
    int traction_mode;         /* enum ssd_traction_mode */
    int bjs_implicit;          /* BJS mode: 0 = slip term from the previous sweep's
                                  velocity (Section 3, step 2, as printed); 1 = slip
                                  term at the Stokes step's own velocity, i.e.
                                  (I - D^S) u + s (gamma/sqrt(kappa)) M(u - (u.n) n)
                                  = U_inf + M(p_D n), one fused SL+DL pass per
                                  matvec; the interface state is then q alone */
    double bjs_sign;           /* s in the BJS traction: +1 (default) or -1 */
    double radius;             /* sphere radius R (JOSEPH_TAO mode; sphere centred at 0) */
    ssd_krylov inner;          /* local solves; inner.tol applies to both */
    int refine;                /* FP32C interface GMRES only: up to this many refinement
                                  steps, each taking the true residual F(z) - z from one
                                  FP64 sweep (whose local systems are solved by iterative
                                  refinement: FP64 residual, FP32C correction) and solving
                                  D (I - G) e = D r for the correction with FP32C sweeps;
                                  the returned fields are those of the last FP64 sweep.
                                  0 = off */
} ssd_ddm_params;

/*
 * Dirichlet-Neumann iteration of Sections 3 and 6.  From q = 0, u_prev = 0,
 * each sweep: b_D = (mu/kappa) L q; Darcy solve for p_D; traction f from p_D
 * (and u_prev in BJS mode); b_S = U_inf - M f; Stokes solve for u_S;
 * q <- (1 - theta) q + theta u_S . n.
 * outer_gmres = 0: sweeps until ||q_k - q_{k-1}|| <= tol ||q_k|| (eq. DDM_residual).
 * outer_gmres = 1: GMRES on the affine interface map z -> G z + c,
 *   z = q (JOSEPH_TAO mode, gamma = 0, or bjs_implicit) or z = (q, u_prev) (lagged BJS),
 *   solving D (I - G) z = D c where D divides the q rows of the stacked form
 *   by theta (the unrelaxed map: theta (q - u.n) / theta; D = I for z = q),
 *   then one sweep from the solution gives the returned fields.
 * Outputs (device): q[n], p_D[n], u_S[3][n], f_S[3][n] (any may be NULL).
 * Host outputs: drag[3] = sum_x w f (eq. drag_int), *outer_its,
 *   inner_its[2 * max(maxit_outer + 2, 1)] = (Darcy, Stokes) iterations per sweep,
 *   res_hist[maxit_outer] = DDM residual per sweep (SA) or the interface
 *   GMRES residual estimate ||D (c - (I - G) z_k)|| / ||D c|| after each step k
 *   (GMRES; one cycle of up to min(maxit_outer, 512) steps, then restarts),
 *   followed, with refine, by the FP64 residual ||D (F(z) - z)|| / ||D c|| of
 *   each refinement step; an entry of -1 ends the history when it is shorter
 *   than maxit_outer.  Host pointers may be NULL.
 * Synchronises `stream`.
 */
int ssd_ddm_solve(ssd_ctx *ctx, const ssd_points *pts, const ssd_ddm_params *prm,
                  double *q, double *p_D, double *u_S, double *f_S, double drag[3],
                  int *outer_its, int *inner_its, double *res_hist, ssd_stream stream);

/*
 * One Dirichlet-Neumann sweep (Section 3, steps 1-3; Section 6, steps
 * (a)-(f)) from the interface state (q, u_prev): b_D = (mu/kappa) L q, Darcy
 * solve for p_D, traction f from p_D (and u_prev: the lagged slip of BJS mode
 * with bjs_implicit = 0; ignored otherwise), b_S = U_inf - M f, Stokes solve
 * for u_S, q_out = (1 - theta) q + theta u_S . n.  Local solves start from 0
 * (prm->inner.warm is ignored); prm->outer_gmres, tol_outer and maxit_outer
 * are ignored.  At a fixed point of the sweep, (q_out, u_S) = (q, u_prev).
 * Device arrays: q[n] and q_out[n] (required, may not overlap), u_prev[3][n]
 * (NULL = zero), outputs p_D[n], u_S[3][n], f_S[3][n] (any may be NULL).
 * inner_its[2] (host, may be NULL) = (Darcy, Stokes) GMRES steps.
 * Returns SSD_ENOTCONV (outputs filled) when a local solve reached its
 * limit.  Synchronises `stream`.
 */
int ssd_ddm_sweep(ssd_ctx *ctx, const ssd_points *pts, const ssd_ddm_params *prm,
                  const double *q, const double *u_prev, double *q_out, double *p_D,
                  double *u_S, double *f_S, int inner_its[2], ssd_stream stream);

/*
 * Same solve with HOST buffers: copies xyz[3][n], nrm[3][n], w[n] to the
 * device, prepares the layout, solves, and copies q, p_D, u_S, f_S back
 * (host outputs may be NULL).  Pinned host memory gives the fastest copies.
 */
int ssd_ddm_solve_host(ssd_ctx *ctx, int64_t n, const double *xyz, const double *nrm,
                       const double *w, const ssd_ddm_params *prm, double *q, double *p_D,
                       double *u_S, double *f_S, double drag[3], int *outer_its,
                       int *inner_its, double *res_hist, ssd_stream stream);

/*
 * Columns of the discrete iteration matrix of the D-N sweeps (eq. A_mat,
 * Section 6) assembled by its definition: column j of A~ is F(e_j) - F(0),
 * F one sweep on the interface variable q (u_inf and the traction's constant
 * part cancel in the difference).  Computes columns col0 .. col0 + ncol - 1
 * into A (device, column-major n x ncol: A[k n + i] = (A~ e_{col0+k})_i).
 * One sweep per column, in the precision of prm->inner.  The interface state
 * must be q alone (SSD_EINVAL for the lagged slip with gamma != 0).
 * Synchronises `stream`; SSD_ENOTCONV if a local solve reached its limit.
 */
int ssd_ddm_iteration_matrix(ssd_ctx *ctx, const ssd_points *pts, const ssd_ddm_params *prm,
                             int64_t col0, int64_t ncol, double *A, ssd_stream stream);

/*
 * Spectrum of the discrete iteration matrix of the D-N sweeps (eq. A_mat,
 * Section 6; Fig. 5): m Arnoldi steps (Gram-Schmidt twice) on
 * A~ v = F(v) - F(0), F one relaxed sweep with prm's theta, from the start
 * vector v_i = frac(0.6180339887498949 i) - 1/2 (all modes present), then the
 * eigenvalues of the m x m Hessenberg block by the double-shifted QR
 * iteration on the host.  Stops early (invariant subspace) when a new
 * vector's norm falls below 1e-12 of its column.  Outputs (host):
 * *m_out steps taken, ritz_re/ritz_im[m] (first *m_out valid), H[(m+1) * m]
 * column-major (may be NULL).  m in 1..512; the lagged BJS slip with
 * gamma != 0 is not supported (its iteration acts on (q, u)).  Synchronises
 * `stream`.
 */
int ssd_ddm_spectrum(ssd_ctx *ctx, const ssd_points *pts, const ssd_ddm_params *prm, int m,
                     int *m_out, double *ritz_re, double *ritz_im, double *H, ssd_stream stream);

/*
 * The host step of ssd_ddm_spectrum on its own: eigenvalues of an upper
 * Hessenberg matrix by the double-shifted QR iteration (Francis shifts from
 * the trailing 2 x 2 block, exceptional shifts every tenth sweep, deflation
 * when a subdiagonal entry is negligible against its diagonal neighbours or
 * by the Ahues-Tisseur test).  Lets a caller take the Ritz values of a
 * leading block of the H that ssd_ddm_spectrum returns.
 * h: host, column-major, n x n with leading dimension ldh >= n; entries below
 * the subdiagonal are ignored; h is not modified.  wr, wi: host [n], the
 * eigenvalues by diagonal position at deflation, a complex pair in adjacent
 * entries with the positive imaginary part first.  Runs on the host only (no
 * context, no device).  SSD_EINVAL: n outside 1..4096, ldh < n, NULL pointer
 * or a non-finite entry; SSD_ENUMERIC: no convergence within 100 n sweeps.
 */
int ssd_hessenberg_eigenvalues(int n, const double *h /* host */, int ldh, double *wr /* host */,
                               double *wi /* host */);

/* ------------------------------------------------------ off-surface fields
 * Field values away from the surface from the boundary data of a D-N solve
 * (FP64, bare kernels; accurate for field points a few grid spacings from
 * the surface: the paper gives no near-surface correction).  Field points
 * targets[3][nt] and outputs are device arrays; nt may be 0.
 *
 * Darcy pressure inside the body, Green's representation (eq. Greens) with
 * dp/dn = -(mu/kappa) q (Darcy's law, the interface flux q = u . n):
 *   p_D(y) = (mu/kappa) sum_j w_j q_j G(y, x_j) + sum_j w_j p_j dG/dn(x_j),
 *   G = -1/(4 pi r), dG/dn = -(y - x) . n / (4 pi r^3);  out[nt].
 * Stokes velocity outside, eq. Stokes with n_S = -n and 1/(8 pi mu):
 *   u_S(y) = U_inf - 1/(8 pi mu) sum_j w_j S(y - x_j) f_j
 *            + 6/(8 pi) sum_j w_j (u_j . yh)(yh . n_j) yh / r^5;  out[3][nt].
 * Stokes pressure outside (the paper prints the velocity representation only;
 * these are the pressures that go with its two kernels, the Stokeslet's
 * 2 yh / r^3 and the stresslet's 4 (-I / r^3 + 3 yh yh / r^5), far-field
 * pressure 0):
 *   p_S(y) = -1/(8 pi) sum_j w_j 2 (yh . f_j) / r^3
 *            - mu/(8 pi) sum_j w_j 4 [-(u_j . n_S) / r^3 + 3 (yh . u_j)(yh . n_S) / r^5];
 *   out[nt].
 * q, p_D, f, u are the outputs of ssd_ddm_solve.  Asynchronous on `stream`.
 */
int ssd_darcy_pressure_field(ssd_ctx *ctx, const ssd_points *pts, double mu, double kappa,
                             const double *q, const double *p_D, int64_t nt, const double *targets,
                             double *out, ssd_stream stream);
int ssd_stokes_velocity_field(ssd_ctx *ctx, const ssd_points *pts, double mu,
                              const double uinf[3] /* host */, const double *f, const double *u,
                              int64_t nt, const double *targets, double *out, ssd_stream stream);
int ssd_stokes_pressure_field(ssd_ctx *ctx, const ssd_points *pts, double mu, const double *f,
                              const double *u, int64_t nt, const double *targets, double *out,
                              ssd_stream stream);

/* ---------------------------------------------------------------- adjoint
 * Derivatives of a scalar output of the Dirichlet-Neumann solve with respect
 * to the two physical parameters of Sections 2 and 7, log(kappa) and gamma,
 * by the discrete adjoint of the computed map (the paper reports drag against
 * kappa and gamma in Section 7 and Tables 1-2; it computes no derivatives).
 * Functionals, e = U_inf / |U_inf| (e = z when U_inf = 0):
 *   SSD_FUNC_DRAG: J = e . sum_x w f           (drag along the flow, eq. drag_int)
 *   SSD_FUNC_FLUX: J = sum_x w q (e . x)       (first moment of the interface flux)
 * Requirements: outer_gmres = 1, inner.use_sa = 0, and in BJS mode with
 * gamma != 0 bjs_implicit = 1 (the lagged slip has no fixed-point map in q
 * alone).  Cost: one forward solve, one transposed interface GMRES (each
 * matvec one transposed Stokes and one transposed Darcy solve) and, for the
 * drag with BJS slip, one more transposed Stokes solve.
 * Host outputs: *value = J (may be NULL), grad[0] = dJ/dlog(kappa),
 * grad[1] = dJ/dgamma (0 in JOSEPH_TAO mode, where gamma does not enter).
 * Returns SSD_ENOTCONV (with the values filled) when a forward or adjoint
 * solve hit its iteration limit.  Synchronises `stream`.
 */
enum ssd_functional { SSD_FUNC_DRAG = 0, SSD_FUNC_FLUX = 1 };
int ssd_ddm_gradient(ssd_ctx *ctx, const ssd_points *pts, const ssd_ddm_params *prm,
                     int functional, double *value, double grad[2], ssd_stream stream);

/*
 * Geometric gradients.  For the scalar outputs of ssd_ddm_gradient, also the
 * derivatives of J with respect to every point's data: gx[3][n] = dJ/dx_k,
 * gn[3][n] = dJ/dn_k, gw[n] = dJ/dw_k (device, overwritten), with the point
 * data treated as independent inputs of the discrete solve.  BJS traction
 * only.  Contract them with ssd_quadrature_jacobian's outputs
 * (ssd_shape_contract) for derivatives in shape coefficients.  Costs one more
 * transposed Darcy solve, one Darcy solve and four FP64 pair passes of the
 * geometric kernels below.  Synchronises `stream`.
 */
int ssd_ddm_gradient_geometry(ssd_ctx *ctx, const ssd_points *pts, const ssd_ddm_params *prm,
                              int functional, double *value, double grad[2], double *gx,
                              double *gn, double *gw, ssd_stream stream);

/*
 * Derivatives of the bilinear form B(a, b) = sum_i a_i . (K b)_i in the point
 * data, K the pair sum of op (SSD_OP_LAPLACE_SL, _DL, SSD_OP_STOKES_SL, _DL;
 * Sections 5.1-5.3, double layers with their subtraction, single layers with
 * their self term): adds alpha dB/dx_k to gx[3][n], alpha dB/dn_k to gn[3][n]
 * and alpha dB/dw_k to gw[n] (device, accumulated).  a and b are [c][n]
 * (c = 1 Laplace, 3 Stokes).  FP64, derivatives of the smoothed kernels in
 * closed form (Taylor series below rho = 0.5).  Asynchronous on `stream`.
 */
int ssd_geometry_gradient(ssd_ctx *ctx, const ssd_points *pts, int op, double delta, double mu,
                          double alpha, const double *a, const double *b, double *gx, double *gn,
                          double *gw, ssd_stream stream);

/*
 * out[k] = sum_i dxyz[k][.][i] . gx[.][i] + dnrm[k][.][i] . gn[.][i] + dw[k][i] gw[i]
 * for k < ncoef (1..512): the chain rule from point data to shape
 * coefficients.  Device inputs, host output.  Synchronises `stream`.
 */
int ssd_shape_contract(ssd_ctx *ctx, int64_t n, int ncoef, const double *dxyz, const double *dnrm,
                       const double *dw, const double *gx, const double *gn, const double *gw,
                       double *out, ssd_stream stream);

/* ------------------------------------------------------------------ batches
 * Many independent surfaces (uneven point counts, one smoothing radius each)
 * handled in one launch per operator application.  The caller concatenates
 * the surfaces' point sets: surface s owns indices [offsets[s], offsets[s+1])
 * of xyz[3][n_total], nrm[3][n_total], w[n_total].  Densities of a batched
 * call are [nrhs][c][n_total] (c = 1 scalar, 3 vector): right-hand side r
 * applies every surface's operator to its own part of block r.  The
 * operators are those of the single-surface calls above, evaluated surface
 * by surface; nothing couples two surfaces.
 */
typedef struct ssd_batch_layout ssd_batch_layout;
typedef struct {
    int32_t nsurf;
    const int64_t *offsets;   /* host [nsurf + 1], offsets[0] = 0, increasing */
    const double *delta;      /* host [nsurf], smoothing radius per surface */
    const double *xyz;        /* device [3][n_total] */
    const double *nrm;        /* device [3][n_total] */
    const double *w;          /* device [n_total] */
    ssd_batch_layout *layout; /* from ssd_batch_prepare (required by batched calls) */
} ssd_batch;

/* Build the batched layout: per-surface Morton order, padding to 512, FP32
 * and FP64 copies, per-surface constants and the work-item tables of both
 * precisions.  Synchronises `stream`. */
int ssd_batch_prepare(ssd_ctx *ctx, ssd_batch *b /* host struct */, ssd_stream stream);
int ssd_batch_release(ssd_ctx *ctx, ssd_batch *b /* host struct */);

enum ssd_operator {
    SSD_OP_LAPLACE_SL = 0, SSD_OP_LAPLACE_DL = 1, SSD_OP_STOKES_SL = 2,
    SSD_OP_STOKES_DL = 3, SSD_OP_STOKES_SLDL = 4, SSD_OP_LAPLACE_SLDL = 5
};
/* One launch for every (surface, right-hand side): out = op(dens0[, dens1]).
 * op: enum ssd_operator; for the fused operators dens0 is the double-layer
 * density and dens1 the single-layer one, weighted alpha (SL) and beta (DL).
 * nrhs in 1..16.  Asynchronous on `stream`. */
int ssd_batch_apply(ssd_ctx *ctx, const ssd_batch *b, int op, int nrhs, double mu, double alpha,
                    double beta, const double *dens0, const double *dens1, double *out, int prec,
                    ssd_stream stream);

/* Dirichlet-Neumann solves of every (surface, right-hand side), all advanced
 * together: every operator application of the sweep is one batched launch,
 * and the local and interface GMRES run per system (own Hessenberg matrix,
 * Givens rotations and stopping test; converged systems are frozen) in one
 * Krylov cycle (restart = maxit, at most 256).  prm->delta is ignored (the
 * batch gives one per surface); prm->uinf is ignored (uinf[r] is the
 * far-field velocity of right-hand side r).  Supported: interface GMRES
 * (outer_gmres = 1) with JOSEPH_TAO traction, or BJS traction with gamma = 0
 * or bjs_implicit = 1.  Outputs (device, [nrhs][c][n_total]): q, p_D (c = 1),
 * u_S, f_S (c = 3); any may be NULL.  Host outputs [nrhs][nsurf]: outer
 * iterations, final interface residual; drag [nrhs][nsurf][3].
 * Synchronises `stream`. */
int ssd_batch_ddm_solve(ssd_ctx *ctx, const ssd_batch *b, const ssd_ddm_params *prm, int nrhs,
                        const double *uinf /* host [nrhs][3] */, double *q, double *p_D,
                        double *u_S, double *f_S, double *drag, int *outer_its, double *relres,
                        ssd_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* SSD_H */
