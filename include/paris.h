/*
 * paris.h -- C ABI of the GB300 (sm_103a) one-fluid pressure projection.
 *
 * The library computes one projection step of the PARIS one-fluid method
 * (arXiv 2012.11744, Sec. 3.2 Eqs. fotm, cont-eq1 and poisson; Sec. 3.7 and
 * 3.8) on a single GPU:
 *
 *   1. beta_f = 1/rho_f, rho = rho1 C + rho2 (1 - C) (Eq. muH), face density
 *      the mean of the two cells, beta = 0 on wall faces      paris_face_coeffs
 *   2. b = (grad^h . u*)/dt (Eqs. cont2, incompdisc3), mean removed
 *                                                           paris_divergence
 *   3. solve grad^h . (beta grad^h p) = b, mean(p) = 0      paris_poisson_solve
 *   4. u = u* - dt beta_f (grad^h p)_f (Eq. fotm)            paris_project
 *
 * GRID AND LAYOUT.  A regular grid of nx*ny*nz cubic cells of edge h
 * (Sec. 3.1: the VOF routines are limited to cubic cells).  Cell (i,j,k) is
 * stored at (k*ny + j)*nx + i (x fastest).  Each axis is either periodic or
 * bounded by walls (no-slip/no-penetration: zero normal velocity, homogeneous
 * Neumann condition for p, Sec. 3.8).  Face arrays (u, beta_x on x-faces etc.)
 * store face "i-1/2" of cell i at index i and have the cell layout with the
 * face axis extended by one when that axis has walls:
 *   x-faces: nz * ny * (nx + wall_x)     index (k*ny + j)*(nx+wall_x) + i
 *   y-faces: nz * (ny + wall_y) * nx     index (k*(ny+wall_y) + j)*nx + i
 *   z-faces: (nz + wall_z) * ny * nx     index (k*ny + j)*nx + i
 * Along a wall axis the entries 0 and n are the wall faces.
 *
 * MEMORY.  Unless a name ends in _host, every array argument is a DEVICE
 * pointer to IEEE double, owned by the caller, contiguous in the layout above
 * and 8-byte aligned.  The context owns its workspace (multigrid hierarchy,
 * Krylov vectors, reduction scratch), allocated in paris_create and released in
 * paris_destroy; the compute calls allocate nothing.
 *
 * STREAMS.  Every call is enqueued on the context's CUDA stream (given to
 * paris_create as a cudaStream_t cast to void*; NULL = the legacy default
 * stream).  Calls returning only a status are asynchronous; calls that fill a
 * host struct (paris_stats, the mean removed) synchronise the stream first.
 * paris_poisson_solve always synchronises: the number of iterations it runs is
 * decided from device-side residual norms.
 *
 * ERRORS.  Every call returns a paris_status; nothing is thrown across the ABI.
 * Arguments are validated before any work is enqueued.  A CUDA error is
 * reported as PARIS_ERR_CUDA and leaves the context unusable (destroy it).
 */
#ifndef PARIS_H
#define PARIS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PARIS_OK = 0,
    PARIS_ERR_INVALID_ARG = 1,   /* bad size, spacing, density, time step, null pointer */
    PARIS_ERR_CUDA = 2,          /* a CUDA call failed (allocation, launch, copy) */
    PARIS_ERR_NOT_CONVERGED = 3, /* solve hit max_iter; p holds the best iterate */
    PARIS_ERR_NONFINITE = 4,     /* a NaN/Inf appeared in the right-hand side or the residual */
    PARIS_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
    PARIS_ERR_NO_MEMORY = 6      /* device allocation failed in paris_create */
} paris_status;

typedef enum { PARIS_PERIODIC = 0, PARIS_WALL = 1 } paris_bc;

typedef enum {
    PARIS_FP64 = 0,  /* FP64 multigrid-preconditioned CG, FP64 V-cycles */
    PARIS_MIXED = 1  /* FP64 iterative refinement around FP32 V-cycle-preconditioned
                        flexible CG; residuals, solution, dot products, mean removal
                        and the coarsest solve in FP64 */
} paris_precision;

typedef enum {
    PARIS_SMOOTH_RBGS = 0,       /* red-black Gauss-Seidel with over-relaxation (Sec. 3.7.1),
                                    both colours fused into one pass over memory */
    PARIS_SMOOTH_JACOBI = 1,     /* damped Jacobi, the paper's GPU iteration (Sec. 3.7.4) */
    PARIS_SMOOTH_RBGS_2PASS = 2  /* the same red-black iteration as two in-place colour
                                    passes (bit-identical to PARIS_SMOOTH_RBGS when every
                                    periodic axis has even length) */
} paris_smoother;

typedef struct {
    int nx, ny, nz;  /* cells per axis, each >= 2 */
    double h;        /* cell edge, > 0 */
    int bc[3];       /* paris_bc for the x, y, z axes */
} paris_grid;

typedef struct {
    double tol;           /* stop when ||r||_2/||b||_2 <= tol AND ||r||_inf/||b||_inf <= tol (1e-10) */
    int max_iter;         /* cap on preconditioned iterations (V-cycles) per solve (200) */
    int precision;        /* paris_precision (PARIS_MIXED) */
    int nu1, nu2;         /* pre/post smoothing sweeps per level (2, 2) */
    double omega;         /* over-relaxation factor of the smoother (1.15; Jacobi: 0.8) */
    int smoother;         /* paris_smoother (PARIS_SMOOTH_RBGS_2PASS) */
    int coarse_max_cells; /* coarsen until the coarsest grid has at most this many cells (8) */
    double inner_tol;     /* MIXED: relative residual reduction of each FP32 inner solve (1e-5) */
    int fallback;         /* MIXED: on failure redo the solve in FP64 (1) */
    int slab_planes;      /* two-pass red-black: run each colour pass in z-slabs of this
                             many planes so the second colour finds the slab in L2
                             (0 = whole-grid passes) (0) */
    int half_coefficients; /* MIXED: the finest-level V-cycle passes read FP16 copies of
                              beta (the FP32 inner operator and the FP64 residual keep full
                              precision, so this changes speed, not the converged p) (0) */
    int level0_density;   /* MIXED, paris_projection_step only: the finest level's FP32
                             operator (colour passes, residual restriction, inner CG
                             product, level-1 coefficients) is rebuilt in registers from an
                             FP32 array of rho/2 (Eq. muH) instead of being read from three
                             FP32 face arrays: 4 instead of 12 bytes per cell and pass.  Used
                             when nx, ny, nz are even, the second level halves every axis,
                             the smoother is PARIS_SMOOTH_RBGS_2PASS and half_coefficients is
                             0; otherwise ignored.  The FP64 residual, the converged p and
                             the projection keep the FP64 beta (1) */
    int level0_tiles;     /* with level0_density: the finest level's colour passes run on
                             plane tiles staged in shared memory by bulk asynchronous (TMA)
                             copies when nx is a multiple of 8 and ny of 8 (2), or on plane
                             tiles read straight into registers, two pairs of cells per
                             thread, when nx/2 is even (1); the inner CG product and the
                             residual restriction run on the register plane tiles for 1 and
                             2.  0: always the kernels that walk z-columns one pair per
                             thread.  The colour passes give identical results in all three;
                             the product's dot products differ in summation order only (1) */
    int level0_half_rho;  /* with level0_density and level0_tiles 1: the V-cycle's finest
                             colour passes and residual restriction read rho/2 in FP16 (2
                             instead of 4 bytes per cell and pass; 11 bits of rho are
                             plenty for a preconditioner), when rho1/2 and rho2/2 lie in
                             [1e-4, 6e4]; the inner CG product, the refinement step and the
                             projection keep full precision, so this changes the V-cycle,
                             not the converged p (1) */
    int coarse_tail;      /* the small levels of the V-cycle (two-pass red-black smoother,
                             dense coarsest level): 1 the levels of at most 4096 cells, down
                             to the coarsest and back, in one launch of one block; 0 one
                             launch per step and level.  The same arithmetic in the same
                             order in both: identical results (1) */
} paris_opts;

typedef struct {
    int iters;             /* preconditioned iterations (V-cycles) in total */
    int outer_iters;       /* MIXED: FP64 refinement steps; FP64: equals iters */
    double rel_res_l2;     /* ||b - L p||_2 / ||b||_2 of the returned p, computed in FP64 */
    double rel_res_linf;   /* ||b - L p||_inf / ||b||_inf */
    double mean_b_removed; /* mean of the right-hand side removed before the solve */
    int fell_back;         /* MIXED: 1 if the FP64 fallback produced the result */
    int converged;         /* 1 if both tolerances were met */
    int levels;            /* multigrid levels used */
} paris_stats;

typedef struct paris_ctx paris_ctx;

/* Fill *o with the defaults listed above. */
void paris_default_opts(paris_opts* o);

/* Create a context for one grid: validates g (n >= 2 per axis, h > 0, bc in
 * {0,1}) and o, builds the multigrid level plan and allocates all device
 * workspace on the current device.  stream: a cudaStream_t (may be NULL).
 * Errors: INVALID_ARG, NO_MEMORY, CUDA.  On error *ctx is NULL. */
paris_status paris_create(paris_ctx** ctx, const paris_grid* g, const paris_opts* o, void* stream);

/* Release the context and its device workspace (synchronises its stream). */
paris_status paris_destroy(paris_ctx* ctx);

/* Replace the options (same grid); no reallocation unless the level plan changes. */
paris_status paris_set_opts(paris_ctx* ctx, const paris_opts* o);

/* Step 1 -- Eq. muH and Sec. 3.7.1: from the cell volume fraction C (cells,
 * values normally in [0,1]) and the densities rho1 (fluid C=1), rho2 (C=0),
 * both > 0, write beta_f = 2/(rho_L + rho_R) on every face, 0 on wall faces
 * (Sec. 3.8 coefficient zeroing).  beta_x/y/z: face arrays (see layout).
 * Errors: INVALID_ARG (null pointer, rho <= 0). */
paris_status paris_face_coeffs(paris_ctx* ctx, const double* C, double rho1, double rho2,
                               double* beta_x, double* beta_y, double* beta_z);

/* Step 2 -- Eqs. cont2/incompdisc3: rhs_c = sum over the axes of
 * (u_{+face} - u_{-face})/(h dt); wall faces contribute no flux whatever they
 * hold.  The mean of rhs is then removed (the compatibility condition of the
 * singular Neumann/periodic problem) and returned in *mean_removed when that
 * pointer (host) is not NULL, which synchronises the stream.
 * Errors: INVALID_ARG (null pointer, dt <= 0). */
paris_status paris_divergence(paris_ctx* ctx, const double* u, const double* v, const double* w,
                              double dt, double* rhs, double* mean_removed);

/* Step 2 without a context, for callers that cannot allocate device memory
 * (for example a solver embedded in an application whose own allocator owns
 * all device memory, or a time loop held to a fixed memory budget).  The
 * paper has no counterpart: this is an interface variant of paris_divergence
 * with the same result.  g describes the grid; u, v, w (face arrays), rhs
 * (cells, output) and mean_removed (one double, output, may be NULL) are
 * DEVICE pointers owned by the caller; work is enqueued on `stream` and the
 * call returns without synchronising.  No device memory is allocated: the
 * block partial sums live in one static device array of 128 KB (16384 blocks
 * of 32x8x8 cells) that every GPU loading the library holds until the process
 * exits.  Grids needing more blocks than that (beyond 512x256x256 cells, i.e.
 * ceil(nx/32)*ceil(ny/8)*ceil(nz/8) > 16384) are rejected with
 * PARIS_ERR_INVALID_ARG before any work is enqueued.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  The
 * address is kept for the life of the process: after cudaDeviceReset (or any
 * other teardown of the device's primary context) it is stale, so this entry
 * point must not be called again in that process.  An error left pending by
 * an unrelated earlier CUDA call is cleared on entry; one that persists (a
 * sticky error of the device context) is returned as PARIS_ERR_CUDA before
 * anything is enqueued.  The call does not synchronise, so it reports launch
 * errors only; a NaN or Inf in u, v or w passes into rhs.  Every call
 * overwrites the whole scratch it reads, so nothing needs clearing, but all
 * calls share the one array: calls that overlap on the GPU (other streams,
 * other threads) race and must be serialised by the caller. */
paris_status paris_divergence_noalloc(const paris_grid* g, const double* u, const double* v,
                                      const double* w, double dt, double* rhs,
                                      double* mean_removed, void* stream);

/* Step 3 -- Eq. poisson with tau folded into b: solve
 *   sum_f beta_f (p_nb - p_c)/h^2 = rhs_c
 * (the paper's A1..A7 form of Sec. 3.7.1 divided by -tau) for p with
 * mean(p) = 0.  rhs is read only; its mean is removed internally.  p: in =
 * initial guess, out = solution.  Multigrid-preconditioned CG (FP64 form) or
 * FP64 iterative refinement around FP32 multigrid-preconditioned flexible CG
 * (MIXED), per the context options; st (host, optional) receives the stats.
 * Errors: INVALID_ARG, NOT_CONVERGED (p holds the last iterate), NONFINITE
 * (NaN/Inf in rhs or during the solve), CUDA. */
paris_status paris_poisson_solve(paris_ctx* ctx, const double* beta_x, const double* beta_y,
                                 const double* beta_z, const double* rhs, double* p,
                                 paris_stats* st);

/* Step 4 -- Eq. fotm: on every non-wall face u_f <- u_f - dt beta_f (p_R - p_L)/h,
 * in place on u, v, w (in: u*, out: u); wall faces are set to 0 (Sec. 3.8 velocity
 * blocking).  Errors: INVALID_ARG (null pointer, dt <= 0). */
paris_status paris_project(paris_ctx* ctx, const double* beta_x, const double* beta_y,
                           const double* beta_z, const double* p, double dt,
                           double* u, double* v, double* w);

/* Steps 1-4 in order on device arrays: C (cells) -> beta (context scratch),
 * b, p (in: initial guess, out: mean-free solution), u/v/w in place.
 * Errors: as the four calls. */
paris_status paris_projection_step(paris_ctx* ctx, const double* C, double rho1, double rho2,
                                   double dt, double* u, double* v, double* w, double* p,
                                   paris_stats* st);

/* paris_projection_step on HOST arrays: C_host, u/v/w_host (in: u*, out: u)
 * and p_host (in: initial guess, out: p) are copied to and from device
 * buffers the context owns (allocated on the first call of this function,
 * which should therefore not be the one being timed).  Pinned host memory
 * gives the fastest copies.  The copies run on a second stream of the
 * context, in the order the step needs the data, so that they overlap the
 * face coefficients, the divergence and the velocity correction; the call
 * synchronises both streams before returning (also on an error, so no copy
 * into or out of the caller's buffers is left running). */
paris_status paris_projection_step_host(paris_ctx* ctx, const double* C_host, double rho1,
                                        double rho2, double dt, double* u_host, double* v_host,
                                        double* w_host, double* p_host, paris_stats* st);

/* Adjoint of steps 2-4 (the paper has no adjoint; derived from Eqs. fotm and
 * poisson).  Given beta, the forward pressure p and g = dLoss/du on the faces
 * (gu, gv, gw), solve the adjoint problem L q = D (B g) with the same operator
 * and options as paris_poisson_solve (q: in = initial guess, out = mean-free
 * adjoint pressure) and write, on every face,
 *   gus   = dLoss/du*   = g - G q
 *   gbeta = dLoss/dbeta = dt (G p) (G q - g)
 * with (G x)_f = (x_R - x_L)/h; both are 0 on wall faces.  Face arrays in,
 * face arrays out (device).  st (host, optional): stats of the adjoint solve.
 * Errors: INVALID_ARG, NOT_CONVERGED (outputs still written), NONFINITE, CUDA. */
paris_status paris_project_adjoint(paris_ctx* ctx, const double* beta_x, const double* beta_y,
                                   const double* beta_z, const double* p, double dt,
                                   const double* gu, const double* gv, const double* gw,
                                   double* gus, double* gvs, double* gws, double* gbeta_x,
                                   double* gbeta_y, double* gbeta_z, double* q, paris_stats* st);

/* Adjoint of step 1: dLoss/dC_c = -(rho1 - rho2)/2 * sum over the non-wall
 * faces f of cell c of gbeta_f beta_f^2, from beta_f = 2/(rho_L + rho_R) and
 * rho = rho1 C + rho2 (1 - C).  beta and gbeta: face arrays; gC: cells.
 * Errors: INVALID_ARG (null pointer, rho <= 0). */
paris_status paris_face_coeffs_adjoint(paris_ctx* ctx, double rho1, double rho2,
                                       const double* beta_x, const double* beta_y,
                                       const double* beta_z, const double* gbeta_x,
                                       const double* gbeta_y, const double* gbeta_z, double* gC);

/* ---------------------------------------------------------------------------
 * PREDICTOR FORCING (Sec. 3.2, Eq. nonconspredictedvel; Sec. 3.6.1, Eq. csf2).
 * The capillary force in CSF form, -sigma kappa grad^h C, and gravity enter
 * the predictor as an acceleration on the faces.  On every face that is not
 * a wall face, between cells L and R along its axis a,
 *   a_f = g_a - (sigma/h) kappa_f (C_R - C_L) beta_f,   kappa_f = (kappa_L + kappa_R)/2,
 * beta_f = 2/(rho_L + rho_R) the face coefficient of paris_face_coeffs (rho
 * from Eq. muH), and u*_f = u^n_f + tau a_f; wall faces get u* = 0.  Because
 * a_f uses the projection's own beta_f, a constant kappa gives a discrete
 * gradient that the projection removes exactly (to rounding): the balance of
 * a drop at rest (Laplace pressure) and of fluid layers at rest
 * (hydrostatic pressure) is kept.  kappa follows the sign convention in
 * which a sphere of fluid 1 (C = 1) of radius R has kappa = -2/R.  The
 * advection and viscous terms of the predictor are not part of this call
 * (the viscous one is paris_viscous_solve). */

/* u, v, w (in u^n, out u*, in place) and beta_x/y/z (out, as
 * paris_face_coeffs) in one pass over the faces.  C, kappa: cells (kappa may
 * be NULL: kappa = 0, gravity only).  sigma >= 0, g = (gx, gy, gz) and
 * tau >= 0 finite.  Asynchronous.
 * Errors: INVALID_ARG (null pointer, rho <= 0, sigma < 0, a non-finite
 * sigma, g or tau, tau < 0). */
paris_status paris_predictor_forcing(paris_ctx* ctx, const double* C, const double* kappa, double rho1,
                                     double rho2, double sigma, double gx, double gy, double gz,
                                     double tau, double* u, double* v, double* w, double* beta_x,
                                     double* beta_y, double* beta_z);

/* The forcing above with tau = dt, then the projection step: u, v, w in:
 * u^n, out: u^{n+1} = P(u^n + dt a); p in: initial guess, out: the pressure.
 * Fused: the forcing is applied by the face-coefficient pass of the step.
 * Errors: as paris_projection_step and paris_predictor_forcing. */
paris_status paris_projection_step_forced(paris_ctx* ctx, const double* C, const double* kappa,
                                          double rho1, double rho2, double sigma, double gx, double gy,
                                          double gz, double dt, double* u, double* v, double* w, double* p,
                                          paris_stats* st);

/* ---------------------------------------------------------------------------
 * SOLID CELLS (Sec. 3.8, "Lego" solids).  A cell flag s, 1 outside the
 * solid and 0 inside, makes every face whose two cells are not both fluid a
 * closed link: its face coefficient is zeroed (a Neumann condition for p on
 * the solid's boundary), it carries no flux in the divergence, and the
 * velocity correction leaves u = 0 there.  (The paper's printed
 * initialisation takes a face's flag from one of its cells; its text asks
 * that the solid region and its boundary be blocked, which needs both.)
 * Solid cells have no open face, so their pressure is not determined: the
 * solve reports p = 0 there and makes p mean-free over the fluid cells.  The
 * fluid region should be connected: a region cut into parts leaves one free
 * constant per part (the paper's warning that a solid must not make the
 * system ill-posed).
 *
 * paris_set_solid(ctx, s): s is a DEVICE array of nx*ny*nz bytes owned by
 * the caller (cell layout, nonzero = fluid) that must stay valid and
 * unchanged while it is set; NULL clears it.  While set, paris_face_coeffs,
 * paris_divergence, paris_poisson_solve, paris_project and the projection
 * steps apply it; the mixed form then runs its finest level from FP32 face
 * coefficients (level0_density is not used).  paris_project_adjoint returns
 * INVALID_ARG while a solid is set.  The call counts the fluid cells and
 * synchronises the stream.  Errors: INVALID_ARG (null ctx, no fluid cell),
 * CUDA. */
paris_status paris_set_solid(paris_ctx* ctx, const unsigned char* s);

/* ---------------------------------------------------------------------------
 * MARKER FUNCTION (Sec. 3.4.2, Eq. FrontMarker3).  The front-tracking
 * method spreads the gradient of the marker function I from the front onto
 * the grid as a face field G (Eq. gradI) and integrates it by solving
 *   Lap_h I = grad^h . G
 * on the whole grid: the projection's operator with beta = 1 on every face
 * (0 on wall faces, which carry no flux of G).  I is fixed up to a constant;
 * the paper does not say how it is chosen, so the caller gives mean_I (for a
 * front: the volume it encloses over the domain's volume).  gx, gy, gz: face
 * arrays (device); I: cells, in: initial guess, out: the marker.  The
 * context's coefficient arrays are overwritten (beta = 1) and its solver
 * options apply (the mixed form runs on FP32 face coefficients).
 * Synchronises.  Errors: INVALID_ARG (null pointer, non-finite mean_I, a
 * solid set on the context), NOT_CONVERGED, NONFINITE, CUDA. */
paris_status paris_marker_function(paris_ctx* ctx, const double* gx, const double* gy, const double* gz,
                                   double mean_I, double* I, paris_stats* st);

/* ---------------------------------------------------------------------------
 * FREE-SURFACE PROJECTIONS (Sec. 3.7.5 "Free-surface flow solver", with the
 * boundary condition of Eq. free_surf_norm_bc).  Only the liquid is solved;
 * here C is the GAS volume fraction, as in that section (C = 0 in the
 * liquid), and the liquid cells are those with C < 1/2.
 *
 * paris_free_surface_step: the projection in the liquid with the liquid
 * density rho_l alone (beta = 1/rho_l).  A face between a liquid cell c and
 * a gas cell g takes the gradient of Eq. mod_branches, (p_s - p_c)/(theta h),
 * theta h the distance along the face's axis from c's node to the interface
 * (theta in (0, 1], from the height function or a plane reconstruction; the
 * caller's), and p_s the interface pressure of Eq. Laplace_num,
 *     p_s = p_gas[g] + sigma (kappa[c] + kappa[g]) / 2,
 * p_gas the gas pressure per cell (the polytropic law of Eq. polygas per gas
 * pocket; the caller's).  The step forms rhs = (div u*) / dt in the liquid (wall
 * faces carry no flux), solves the SPD system (no null space: every liquid
 * region must touch the gas) in opts.precision (the mixed form: FP64
 * refinement around the FP32 V-cycle-preconditioned CG, the diagonal excess
 * on every FP32 level; fallback to FP64 as for paris_poisson_solve), and
 * corrects u = u* - dt beta grad p
 * (Eq. fotm) on every face touching the liquid with the same gradients.
 * Faces between two gas cells keep their values (the caller extrapolates
 * them); wall faces are set to 0.  p: in, the initial guess in the liquid;
 * out, the solution in the liquid and p_gas in the gas (0 without p_gas).
 *   C, kappa, p_gas, p  cells (nx*ny*nz); kappa and p_gas may be NULL (0)
 *   theta_x/y/z         face arrays (the layout of u, v, w), read on the
 *                       liquid-gas faces only; all three NULL: theta = 1
 *   u, v, w             face arrays, in u*, out the projected velocity
 * All device pointers; the context must have no solid set.  Synchronises.
 * Errors: INVALID_ARG (null C/u/v/w/p, rho_l or dt not finite and positive,
 * sigma not finite, one or two theta arrays NULL, a solid set), NO_MEMORY
 * (the free-surface work arrays, 9 bytes per cell plus the coarse levels,
 * are allocated on the first call), NOT_CONVERGED, NONFINITE, CUDA.
 *
 * paris_phantom_projection: the second ("phantom") projection of "Ensuring
 * volume conservation".  The unknowns are the first two layers of gas cells
 * (layer 1: gas cells with a liquid face neighbour; layer 2: the other gas
 * cells with a face neighbour in layer 1); the faces to the liquid keep
 * their (solved) velocities and carry no gradient; the gas beyond the two
 * layers holds phat = 0 (a Dirichlet condition at its cell centres).  It
 * solves div grad phat = div u on the layers (no density, no dt; wall faces
 * closed) and corrects u -= grad phat on the faces between two gas cells at
 * least one of which is in the layers; every other face (wall faces
 * included) is left as it is.  phat: in, the initial guess on the layers;
 * out, phat on the layers and 0 elsewhere.  Each gas pocket must reach
 * beyond two layers (else the system has no Dirichlet cell and, in general,
 * no solution: NOT_CONVERGED).  Synchronises.  Errors: INVALID_ARG (a NULL
 * pointer, a solid set), NO_MEMORY, NOT_CONVERGED, NONFINITE, CUDA. */
paris_status paris_free_surface_step(paris_ctx* ctx, const double* C, double rho_l, double dt,
                                     const double* theta_x, const double* theta_y, const double* theta_z,
                                     const double* kappa, double sigma, const double* p_gas, double* u,
                                     double* v, double* w, double* p, paris_stats* st);
paris_status paris_phantom_projection(paris_ctx* ctx, const double* C, double* u, double* v, double* w,
                                      double* phat, paris_stats* st);

/* ---------------------------------------------------------------------------
 * IMPLICIT VISCOUS STEP (Sec. 3.2.3, Eq. muelliptic).  For one velocity
 * component, u* - tau nu_f Lap_h u* = u^n on the component's own face grid,
 * Lap_h the 7-point Laplacian with spacing h.  The unknowns are the
 * component's faces except its wall faces (where it is zero).  Beyond the
 * ends of an axis the Laplacian takes: the wrapped value (periodic axis),
 * zero (the component's own wall faces), or minus the end value (a wall
 * axis of a tangential component: no-slip, the velocity vanishes on the
 * wall, half a cell beyond the last unknown).  nu_f is the kinematic
 * viscosity at the face: the printed equation multiplies the Laplacian by
 * the dynamic viscosity, which the predictor's form of the viscous term
 * divides by the density. */

/* nu_f = (mu_L + mu_R) / (rho_L + rho_R) on every face of component comp
 * (0 = x-faces, 1 = y-faces, 2 = z-faces; face layout above), mu and rho
 * from Eq. muH in the two cells sharing the face: mu = mu1 C + mu2 (1 - C),
 * rho = rho1 C + rho2 (1 - C).  Wall faces of the component get 0.  C:
 * cells; nu: the component's face array (output).  The products and sums are
 * rounded one by one, in that order (no fused multiply-add).
 * Errors: INVALID_ARG (null pointer, comp outside 0..2, a mu or rho that is
 * not finite and > 0). */
paris_status paris_face_viscosity(paris_ctx* ctx, int comp, const double* C, double mu1, double mu2,
                                  double rho1, double rho2, double* nu);

/* Solve Eq. muelliptic for component comp in its symmetric positive definite
 * form (diag(1/(tau nu)) - Lap_h) u* = u^n / (tau nu) by conjugate gradients
 * with the Jacobi preconditioner, in FP64, from the initial guess u* = u^n.
 * nu, un (in) and us (out): the component's face arrays; entries on its wall
 * faces are not read, and us gets 0 there.  nu must be finite and > 0 on the
 * unknowns.  us must not overlap un or nu.  Stops when
 * ||b - A u*||_2 <= tol ||b||_2 and ||b - A u*||_inf <= tol ||b||_inf, with
 * b = u^n/(tau nu), checked on the true residual; max_iter bounds the CG
 * iterations.  tau = 0 returns u* = u^n.  Uses the context's Krylov
 * workspace (no allocation) and synchronises the stream.  st (host,
 * optional): iters (CG iterations), outer_iters (restarts + 1), the relative
 * residual norms of the SPD form, converged; the other fields 0.
 * Errors: INVALID_ARG (null pointer, comp outside 0..2, us equal to un or nu,
 * tau < 0 or not finite, tol outside (0,1), max_iter < 1), NONFINITE (a nu
 * that is not > 0, or a NaN/Inf in the right-hand side or the residual),
 * NOT_CONVERGED (us holds the last iterate), CUDA. */
paris_status paris_viscous_solve(paris_ctx* ctx, int comp, const double* nu, double tau,
                                 const double* un, double* us, double tol, int max_iter,
                                 paris_stats* st);

/* The same solve (same arguments, stopping test and outputs) by FP64
 * iterative refinement around FP32 flexible CG (each refinement step
 * reduces its residual by paris_opts.inner_tol, or by what the tolerance
 * still needs), preconditioned by an FP32 geometric-multigrid V-cycle of the
 * component's operator: every axis halved per level (cell-centred along
 * periodic and no-slip axes, vertex-centred along the component's own wall
 * axis, with linear interpolation and full weighting there), rediscretised
 * coarse operators with the restricted mass term 1/(tau nu), red-black
 * Gauss-Seidel with the context's nu1/nu2 sweeps and omega (damped Jacobi on
 * a level with an odd periodic extent), 8 sweeps on the coarsest level.
 * The stopping test is on the FP64 residual.  The first call on a context
 * allocates the multigrid's work arrays (about 4 x 4 x 8/7 bytes per cell
 * plus 8 per cell); later calls allocate nothing.  st->iters: FP32 inner
 * iterations; st->outer_iters: refinement steps; st->levels: the multigrid
 * levels.  Errors: as paris_viscous_solve, and NO_MEMORY on the first call. */
paris_status paris_viscous_solve_mg(paris_ctx* ctx, int comp, const double* nu, double tau,
                                    const double* un, double* us, double tol, int max_iter,
                                    paris_stats* st);

/* ---------------------------------------------------------------------------
 * BATCHED PROJECTIONS.  Many independent projection steps of uneven grid
 * sizes in one persistent cooperative launch (captured in a CUDA graph on the
 * first call and replayed afterwards).  Every instance runs the same step as
 * paris_projection_step with the mixed-precision solver, starting from p = 0,
 * on a group of CTAs sized in proportion to its cells; the groups never wait
 * for one another.  Group barriers spin with an iteration limit: if one gives
 * up (it should not, since a cooperative launch keeps every CTA resident) the
 * step returns PARIS_ERR_TIMEOUT instead of hanging.
 *
 * POOLED LAYOUT.  All instances' arrays of one kind are concatenated in
 * instance order into one device buffer: C and p (cells), u (x-faces), v
 * (y-faces), w (z-faces); paris_batch_layout returns the n+1 offsets (in
 * doubles) of each pool.  Each instance's slice uses the single-grid layout. */
typedef struct paris_batch paris_batch;

/* n grids (host array), options (precision is always mixed; smoother must be
 * PARIS_SMOOTH_RBGS or PARIS_SMOOTH_RBGS_2PASS, both run as red-black colour
 * passes here), stream.  Allocates all workspace.  INVALID_ARG also when n
 * exceeds the number of CTAs the GPU can keep resident, or when an instance
 * has (nx+1)(ny+1)(nz+1) >= 2^31 (its arrays are indexed in 32 bits). */
paris_status paris_batch_create(paris_batch** b, int n, const paris_grid* grids,
                                const paris_opts* o, void* stream);
paris_status paris_batch_destroy(paris_batch* b);
/* Offsets of the pools (host arrays of n+1 int64, in doubles). */
paris_status paris_batch_layout(const paris_batch* b, int64_t* cell_off, int64_t* xf_off,
                                int64_t* yf_off, int64_t* zf_off);
/* CTAs in the persistent launch (all co-resident). */
int paris_batch_launch_ctas(const paris_batch* b);
/* One projection step of every instance: C (cell pool), rho1/rho2/dt (host
 * arrays of n), u/v/w (face pools, in: u*, out: u), p (cell pool, out: the
 * mean-free pressure), st (host array of n, optional).  Returns the first
 * failure (NONFINITE, NOT_CONVERGED) or TIMEOUT; synchronises the stream. */
paris_status paris_batch_projection_step(paris_batch* b, const double* C, const double* rho1,
                                         const double* rho2, const double* dt, double* u,
                                         double* v, double* w, double* p, paris_stats* st);
/* Autotuner: times the step for every candidate (sweeps nu1 = nu2 in {1,2,3},
 * omega in {1.0, 1.15, 1.3}, CTAs per SM in {1,2,4,8} up to the resident
 * limit) on scratch copies of u*, v*, w* (inputs are not modified), keeps the
 * fastest converged one and appends it to cache_path (one JSON object per
 * line keyed by GPU name, instance shapes and tolerance; may be NULL).  An
 * existing entry for the same key is applied without timing.  Allocates its
 * scratch (not a hot call).  best_ms (host, optional): the winner's time. */
paris_status paris_batch_autotune(paris_batch* b, const double* C, const double* rho1,
                                  const double* rho2, const double* dt, const double* u,
                                  const double* v, const double* w, const char* cache_path,
                                  double* best_ms);
paris_status paris_batch_get_tuning(const paris_batch* b, int* nu, double* omega, int* ctas_per_sm);

/* Diagnostics on device arrays, FP64: r = rhs - L p, returning (host) the
 * relative residual norms with respect to rhs (rhs taken as given, mean not
 * removed) and the maximum absolute discrete divergence max|grad^h . u| of a
 * face field (u may be NULL to skip).  Synchronises the stream. */
paris_status paris_residual_norms(paris_ctx* ctx, const double* beta_x, const double* beta_y,
                                  const double* beta_z, const double* rhs, const double* p,
                                  double* rel_l2, double* rel_linf);
paris_status paris_max_divergence(paris_ctx* ctx, const double* u, const double* v,
                                  const double* w, double* max_abs_div);

/* Self-check of the arithmetic the kernels build from integer operations, on
 * n device values v (FP64), against the GPU's own conversion and division
 * instructions: for each value the FP64->FP32 conversion of v * 2^shift
 * (round to nearest even; results below the FP32 normal range are flushed to
 * zero and not counted), the FP32->FP64 conversion back with 2^-shift, and
 * for 0 < v in [2^-123, 2^117) the FP64 reciprocal formed by Newton-Raphson
 * (Eq. muH's 1/rho_f), which must be within one ulp of 1.0/v.  *mismatches
 * (host) receives the number of disagreements.  stream: a cudaStream_t (may
 * be NULL); the call allocates 8 bytes of device memory and synchronises it.
 * Errors: INVALID_ARG (n < 0, |shift| > 60, null pointers), CUDA. */
paris_status paris_check_arithmetic(const double* v, int64_t n, int shift, int64_t* mismatches,
                                    void* stream);

/* Streaming rates of this device (context for roofline reports; no paper
 * counterpart).  a, b, c, o: device arrays of n floats each (n a positive
 * multiple of 4, 16-byte aligned), owned by the caller; a, b, c are only
 * read, o is overwritten.  Two kernels of this library run reps + 1 times
 * each on `stream` (a cudaStream_t, may be NULL; the call synchronises it),
 * the first run of each untimed:
 *   read_gbs  = 12 n bytes / best time of a read-only pass over a, b, c;
 *   triad_gbs = 12 n bytes / best time of o = a + b/2 (8 n read, 4 n written).
 * Use vectors larger than the L2 cache for DRAM rates.
 * Errors: INVALID_ARG (null or misaligned pointers, n < 4 or not a multiple
 * of 4, reps outside [1, 1000]), CUDA. */
paris_status paris_stream_rates(const float* a, const float* b, const float* c, float* o, int64_t n, int reps,
                                double* read_gbs, double* triad_gbs, void* stream);

/* Kernel-class timing (diagnostics for roofline reports).  While enabled,
 * every launch of an instrumented level-0 kernel class is bracketed by a CUDA
 * event pair on the context's stream (a pool of 16384 pairs per enable;
 * launches beyond it are counted but not timed).  paris_profile(ctx, 1)
 * clears the counters; paris_profile_read synchronises the stream and returns
 * the launches, their summed device time and their summed algorithmic bytes
 * (each array a launch must touch read or written once, at the precision the
 * kernel ran in).  Classes: */
typedef enum {
    PARIS_K_SMOOTH0 = 0,   /* one smoother pass on the finest level */
    PARIS_K_RESTRICT0 = 1, /* residual + restriction from the finest level */
    PARIS_K_PROLONG0 = 2,  /* prolongation + correction onto the finest level */
    PARIS_K_MATVEC0 = 3,   /* Krylov operator application q = A d (+ d.q) */
    PARIS_K_RESID64 = 4,   /* FP64 true residual r = f - A p (+ norms) */
    PARIS_K_COARSE = 5,    /* the V-cycle below the finest level (one timing per V-cycle) */
    PARIS_K_FIELD = 6,     /* projection step: face coefficients and divergence */
    PARIS_K_SETUP = 7,     /* per solve: right-hand side, level coefficients, coarsest inverse */
    PARIS_K_KRYLOV = 8,    /* Krylov vector updates, dot products, reductions, scalar reads */
    PARIS_K_PROJECT = 9,   /* velocity correction and the mean removal of p */
    PARIS_K_COUNT = 10
} paris_kernel_class;

typedef struct {
    int64_t launches; /* launches recorded since paris_profile(ctx, 1) */
    int64_t timed;    /* launches that had an event pair */
    double ms;        /* summed device time of the timed launches */
    double bytes;     /* summed algorithmic bytes of the timed launches */
} paris_kernel_prof;

paris_status paris_profile(paris_ctx* ctx, int enable);
paris_status paris_profile_read(paris_ctx* ctx, int kernel_class, paris_kernel_prof* out);

/* Process-wide number of CUDA kernels this library has launched. */
int64_t paris_launch_count(void);

/* Face-array sizes (number of doubles) of the context's grid; axis 0, 1, 2. */
int64_t paris_face_count(const paris_ctx* ctx, int axis);
int64_t paris_cell_count(const paris_ctx* ctx);

/* The last CUDA error the library saw in this thread, as "name: description"
 * (static thread-local string), to explain a PARIS_ERR_CUDA. */
const char* paris_last_cuda_error(void);

/* Human-readable name of a status code (static string). */
const char* paris_status_string(paris_status s);

#ifdef __cplusplus
}
#endif

#endif /* PARIS_H */
