/*
 * ccm.h - C ABI of libccm, a GB300 (sm_103a) implementation of one projection time step of
 * the conservative Cartesian cut-cell method for the incompressible Navier-Stokes equations
 * on staggered (MAC) grids (Quiros Rodriguez, Fullana, Le Chenadec, Sayadi,
 * arXiv 2211.10698).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every call returns a ccm_status; nothing else crosses the ABI (no exceptions, no exit).
 *    On failure ccm_last_error() returns a message for the calling thread.
 *  - A case owns all of its device memory.  Host pointers passed in are read or written
 *    during the call only and never retained.  Sizes are element counts and are checked
 *    (CCM_E_INVALID on mismatch).
 *  - A case is not thread-safe; different cases may be used from different threads.
 *  - Every field crosses the ABI as a float64 array of (ny+3) x (nx+3) elements, x
 *    fastest ("padded layout"): element (j+1)*(nx+3) + (i+1) holds index (i, j), i in
 *    [-1, nx+1], j in [-1, ny+1].  Index (i, j) names the pressure cell (i, j), the x-face
 *    at x_i = x0 + i*hx (u), the y-face at y_j = y0 + j*hy (v) or the node (x_i, y_j),
 *    depending on the field (on a stretched mesh x_i and y_j are the given abscissas).  Beyond
 *    a periodic side the ring holds the images of the positions at the other end.
 *  - Box sides are W=0, E=1, S=2, N=3.  A DIRICHLET side prescribes the normal velocity
 *    component bc_un and the tangential component bc_ut (an inflow is a Dirichlet side);
 *    an OUTFLOW side has zero-gradient velocity and zero pressure (Sec. 5.1); PERIODIC pairs
 *    wrap around (a box without an outflow side has a singular Poisson system, whose
 *    iterates are kept at zero mean, end of Sec. 4.6).
 *  - The immersed body is fixed and must stay two cells away from every box side.  It is
 *    no-slip (Dirichlet data D = 0 in Eqs. divergence, diag, offdiag, convective) unless the
 *    fields CCM_F_DX / CCM_F_DY give its wall a velocity D (a rotating, sliding or porous
 *    body), steady or, through ccm_set_body_motion, scaled by a prescribed function of time.
 *  - Equations are cited by their label in the paper's source.  Numbered in the order the
 *    paper prints them: approximate (2), divergence (17), compatibility (18), diag (19),
 *    offdiag (20), divD (21), convective (22), kinetic (26), semidiscrete (27),
 *    pm_prediction (30), pm_poisson (31), pm_projection (32), pm_update (33).
 */
#ifndef CCM_H
#define CCM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CCM_VERSION 1

typedef struct ccm_case_s* ccm_case;

typedef enum {
  CCM_OK = 0,
  CCM_E_INVALID = 1,        /* bad argument, size or configuration */
  CCM_E_OOM = 2,            /* device allocation failed */
  CCM_E_CUDA = 3,           /* CUDA runtime error (message in ccm_last_error) */
  CCM_E_NOT_CONVERGED = 4,  /* a PCG reached its iteration limit; state stays usable */
  CCM_E_NONFINITE = 5,      /* NaN or Inf detected in the fields */
  CCM_E_TIMEOUT = 6,        /* a device-wide barrier gave up waiting; context still usable */
  CCM_E_STATE = 7           /* call out of order (e.g. step before set_geometry) */
} ccm_status;

enum { CCM_SIDE_W = 0, CCM_SIDE_E = 1, CCM_SIDE_S = 2, CCM_SIDE_N = 3 };
/* PERIODIC: W with E, S with N (both sides of a pair); face nx is face 0 and the cells beyond
 * one side are the cells at the other.  On a uniform mesh along that axis whose cell count is
 * a multiple of 3 (the colour probing of the Helmholtz coefficients); single cases only (not
 * in batches or the request loop). */
enum { CCM_BC_DIRICHLET = 0, CCM_BC_OUTFLOW = 1, CCM_BC_PERIODIC = 2 };
enum { CCM_FP64 = 0, CCM_MIXED = 1 };         /* MIXED: FP32 inner Poisson PCG, FP64 refinement */
enum { CCM_JACOBI = 0, CCM_CHEBYSHEV = 1 };
enum { CCM_GEOM_NONE = 0, CCM_GEOM_CIRCLE = 1, CCM_GEOM_NACA = 2, CCM_GEOM_HALFPLANE = 3 };

/* Device allocator hooks (optional).  When alloc is NULL the library uses cudaMalloc. */
typedef void* (*ccm_alloc_fn)(size_t bytes, void* ctx);
typedef void (*ccm_free_fn)(void* ptr, void* ctx);

/* Case description: the mesh of Sec. 3.1 (uniform spacing), the fluid constants of Sec. 4,
 * the time step, the box boundary data and the solver settings. */
typedef struct {
  int nx, ny;                 /* pressure cells */
  double x0, x1, y0, y1;      /* box */
  double rho, mu, dt;         /* density, dynamic viscosity, time step tau */
  int bc_type[4];             /* CCM_BC_* per side */
  double bc_un[4], bc_ut[4];  /* Dirichlet normal / tangential velocity per side */
  int precision;              /* CCM_FP64 or CCM_MIXED */
  int precond;                /* Poisson preconditioner: CCM_JACOBI or CCM_CHEBYSHEV */
  int cheb_degree;            /* Chebyshev polynomial degree (>= 1) */
  double tol_p, tol_h;        /* relative residual targets, Poisson and Helmholtz */
  double tol_inner;           /* MIXED, Chebyshev or singular: relative target of each FP32
                                 inner solve of the host-driven refinement */
  int max_iter_p, max_iter_h; /* iteration limits */
  int literal_offdiag;        /* 1: Eq. offdiag with separate W^xy, W^yx (not symmetric) */
  int pressure_update;        /* volume V in the correction of Eq. pm_update,
                                 P += Phi - (dt mu / 2 rho) V^-1 cont(M^-1 pres Phi, 0):
                                 0 the full cell hx*hy (bounded in small cut cells; the
                                 default), 1 the cell's fluid volume V_p, 2 no correction */
  double replace_drop;        /* MIXED, Jacobi, nonsingular (one-launch solve): reduction of the
                                 FP32 residual that triggers an FP64 residual replacement
                                 (0 selects 0.5) */
  int autotune;               /* 1: set_geometry times candidate launch shapes of the case's
                                 one-launch Poisson solve (FP64 Jacobi: the tile plan; MIXED: the
                                 block count) on a short scratch solve and keeps the fastest,
                                 cached per grid size for the process; 0: the built-in plan.
                                 Batched solves (ccm_batch_*) do not use it. */
  ccm_alloc_fn alloc;
  ccm_free_fn free;
  void* alloc_ctx;
  void* stream;               /* cudaStream_t for all work of the case, NULL = default */
  /* Stretched rectilinear mesh (Sec. 3.1: arbitrary abscissas), host arrays read during
   * ccm_create_case only: xf[0..nx] and yf[0..ny] the face abscissas, strictly increasing,
   * xf[0] == x0, xf[nx] == x1 (likewise y).  NULL (both) for the uniform spacing.  The
   * staggered grids of Sec. 3.4 have their cells centred on the faces, so the u-grid's lines
   * are the centres of the pressure cells; beyond the box the spacing mirrors the spacing
   * inside it.  dt is the caller's (the smallest cell sets the CFL number). */
  const double* xf;
  const double* yf;
  /* Initial guess of each step's Poisson solve: 0 (default) the previous step's Phi; L in
   * 1..32 the projection of the new solution onto the span of the last L solutions in the
   * inner product of K (Fischer 1998), which lowers the iteration count of a smoothly
   * evolving flow.  Same stopping test either way.  Needs 2 L padded FP64 arrays more (the
   * case's allocator).  Setting Phi or the step counter (ccm_set_field, as a restored
   * checkpoint does) clears the history, so the restored run repeats a fresh run bit for bit;
   * setting U, V or P keeps it (it only shortens the solves).  Batched steps (ccm_batch_*) do
   * not use it; a singular (all-wall) system ignores it. */
  int guess_history;
} ccm_config;

/* Immersed body given by a level set (Sec. 3.1).  Points on the boundary count as solid. */
typedef struct {
  int kind;                   /* CCM_GEOM_* */
  double cx, cy, r;           /* circle: solid where |x - c| <= r */
  int naca_tt;                /* NACA 00tt: thickness tt percent of chord */
  int closed_te;              /* 1: closed trailing edge (-0.1036 quartic coefficient) */
  double chord, aoa_deg, le_x, le_y;
  double hp_nx, hp_ny, hp_off;/* half plane: fluid where hp_nx*x + hp_ny*y > hp_off */
} ccm_geometry;

typedef struct {
  int iters;                  /* PCG iterations (MIXED: total inner FP32 iterations) */
  int outer;                  /* MIXED: FP64 refinement sweeps; FP64: 1 */
  double rel_res;             /* final ||b - K x|| / ||b|| in FP64 */
  int converged;
} ccm_solve_stats;

typedef struct {
  int steps;                  /* steps completed by the call */
  long long iters_p, iters_h; /* PCG iterations summed over the steps */
  int last_iters_p, last_iters_h;
  double last_res_p, last_res_h;
  double max_div;             /* max |cont(U^{n+1}, D^{n+1})| over active cells after the last step */
  double kinetic;             /* sum over velocity positions of V U^2 / 2 after the last step */
  int converged;              /* every solve of every step converged */
  double mass;                /* sum of cont(U^{n+1}, D) over the box cells: the net volume flux through the
                                 box and the body (Eq. divergence telescopes) after the last step */
  double momentum_x;          /* sum over u-positions of V u (momentum per unit density) after the last step */
  double momentum_y;          /* sum over v-positions of V v */
} ccm_step_stats;

/* Field identifiers for ccm_set_field / ccm_get_field (padded layout, float64). */
enum {
  CCM_F_U = 0,                /* x-velocity at u-faces (ghosts and Dirichlet faces included) */
  CCM_F_V = 1,                /* y-velocity at v-faces */
  CCM_F_P = 2,                /* pressure P^{n-1/2} at cells */
  CCM_F_PHI = 3,              /* pressure increment Phi^n at cells (warm start of the Poisson PCG) */
  CCM_F_CONV_U = 4,           /* conv^{n-1} at u-faces (Adams-Bashforth history) */
  CCM_F_CONV_V = 5,
  CCM_F_USTAR = 6,            /* predicted velocity U* of the last step (read only) */
  CCM_F_VSTAR = 7,
  CCM_F_DIV = 8,              /* cont(U*, D^{n+1}) of the last step (read only) */
  CCM_F_STEP = 9,             /* first element: number of steps taken (as a double) */
  CCM_F_GX = 10,              /* body acceleration g_x at u-faces, the rho V g term of Eq. pm_prediction
                                 (zero unless set; steady: it applies to every later step) */
  CCM_F_GY = 11,              /* body acceleration g_y at v-faces */
  CCM_F_DX = 12,              /* the body's Dirichlet velocity D_x, one value per u-cell (the velocity of the
                                 body on the boundary inside that u-control volume; zero: no-slip) in the
                                 heterogeneous terms of Eqs. divergence, diag/offdiag and convective.  Setting D
                                 computes those terms once (the body is fixed; they are linear in D) and gives the
                                 faces whose control volume holds no fluid the value D.  With a time law
                                 (ccm_set_body_motion) this field is D0 and the body velocity is f(t) D0.  In a
                                 box without an outflow side D must carry no net flux. */
  CCM_F_DY = 13,              /* D_y, one value per v-cell */
  CCM_F_CAP = 16              /* + 9*g + k: capacity k of grid g (read only), g: 0 p, 1 u,
                                 2 v; k: 0 V, 1 X, 2 Y, 3 Ax, 4 Ay, 5 Wx, 6 Wy, 7 Bx, 8 By
                                 (Ax/Wx at the cell's left face, Ay/Wy at its bottom face) */
};

/* Operators for ccm_apply_op.  Inputs/outputs are padded float64 arrays. */
enum {
  CCM_OP_CONT = 0,            /* in0=u, in1=v -> out0 = cont(U, 0) at cells (Eq. divergence) */
  CCM_OP_PRES = 1,            /* in0=P -> out0,out1 = pres(P) on velocity unknowns (Sec. 4.1),
                                 ghost cells of P read as 0 */
  CCM_OP_CONV = 2,            /* in0=u, in1=v -> conv(U,U,0,0) on unknowns (Eq. convective),
                                 Dirichlet faces and ghosts filled from the box data */
  CCM_OP_VISC = 3,            /* in0=u, in1=v -> visc(S(U)) on unknowns (Sec. 4.2-4.3), box data
                                 filled as for CONV, outflow rules applied */
  CCM_OP_HELMHOLTZ = 4,       /* in0=u, in1=v -> (rho/dt) M U - mu visc(S_hom(U)) on unknowns,
                                 identity on inactive faces (Eq. pm_prediction) */
  CCM_OP_POISSON = 5,         /* in0=Phi -> -cont(M^-1 pres Phi, 0) on active cells, identity on
                                 inactive cells (Eq. pm_poisson) */
  CCM_OP_POISSON_DIAG = 6,    /* -> out0 = diagonal of the POISSON operator */
  CCM_OP_HELMHOLTZ_DIAG = 7   /* -> out0,out1 = diagonal of the HELMHOLTZ operator */
};

/* Create a case: validates the configuration and allocates its device memory.  *out is
 * set only on CCM_OK.  Errors: CCM_E_INVALID, CCM_E_OOM, CCM_E_CUDA. */
ccm_status ccm_create_case(const ccm_config* cfg, ccm_case* out);

/* Device memory a case with this configuration will hold (for admission control). */
ccm_status ccm_case_bytes(const ccm_config* cfg, size_t* bytes);

/* The launch shape of the case's one-launch Poisson solve: plan[0..3] = tile width, tile
 * height, tiles per row and tiles of the one-barrier solve of the case's precision (FP64, or
 * for a mixed case the one-barrier mixed solve; 0 where it does not apply or the built-in
 * plan is used), plan[4] = blocks of the mixed solve with a barrier per Chebyshev step (0:
 * built-in), plan[5] = CTAs of the one thread-block cluster that holds a small grid's whole
 * FP64 solve (0: not used), plan[6] = 1 when the tiles (FP64 or mixed) keep their vectors
 * in shared memory for the whole solve.  Valid after set_geometry. */
ccm_status ccm_launch_plan(ccm_case c, int plan[7]);
/* Sets the launch shape (same layout; zeros select the built-in shapes).  A tile plan needs a
 * width that is a power of two in 32..512 and the tile counts it implies (and, resident, tiles
 * that fit in shared memory at once); a cluster has 2, 4, 8 or 16 CTAs, at most ny, and
 * excludes a tile plan; a mixed case's tile plan selects the one-barrier mixed solve
 * (resident or not: its tiles, bands and, resident, vectors must fit the GPU at once) and
 * excludes block counts and clusters.  CCM_E_INVALID otherwise.  Shapes apply to the single-case
 * solve of a nonsingular system: the FP64 Jacobi solve (tiles, cluster) and the mixed solve
 * (tiles or blocks). */
ccm_status ccm_set_launch_plan(ccm_case c, const int plan[7]);

/* The FP64 fused multiply-add rate of the current GPU in TFLOP/s (2 flop per FMA), measured with
 * CUDA events on independent FMA chains: the roofline denominator of the FP64-bound kernels
 * (the paper has no counterpart).  Allocates 8 bytes of device memory during the call. */
ccm_status ccm_measure_fp64_rate(double* tflops);

/* Release every resource of the case (NULL is accepted). */
ccm_status ccm_destroy_case(ccm_case c);

/* Compute the capacities of Sec. 3 (Eqs. volumefirstkind to surfacesecondkindy, staggered
 * per Sec. 3.4) in FP64 on the device for the p-, u- and v-grids from the body's level set
 * (marching squares with exact edge crossings), derive the operator coefficients, discard
 * the level set, and initialise the velocity to bc_un[W] (x) and 0 (y) on every velocity
 * position whose control volume holds fluid.  CCM_E_INVALID if the body comes within two
 * cells of a box side. */
ccm_status ccm_set_geometry(ccm_case c, const ccm_geometry* g);

/* Copy a host field into the case (U, V, P, PHI, CONV_U, CONV_V, STEP).  count must be
 * (nx+3)*(ny+3) (STEP: >= 1).  Setting U or V refills the Dirichlet faces and ghosts.
 * Errors: CCM_E_INVALID, CCM_E_STATE (before set_geometry), CCM_E_CUDA. */
ccm_status ccm_set_field(ccm_case c, int field, const double* host, size_t count);

/* Copy a field of the case to host memory (padded layout, count = (nx+3)*(ny+3); STEP:
 * count >= 1). */
ccm_status ccm_get_field(ccm_case c, int field, double* host, size_t count);

/* Device address of a field in the case's own pitched layout (row pitch in elements in
 * *pitch, origin at index (-1, -1)); valid until ccm_destroy_case. */
ccm_status ccm_field_device_ptr(ccm_case c, int field, void** dptr, int* pitch);

/* Apply one discrete operator (CCM_OP_*) to host arrays; unused pointers may be NULL. */
ccm_status ccm_apply_op(ccm_case c, int op, const double* in0, const double* in1, double* out0,
                        double* out1);

/* Advance nsteps projection steps (PmII, Sec. 4.6, Eqs. pm_prediction, pm_poisson,
 * pm_projection, pm_update) on the device-resident state.  stats may be NULL.  Returns
 * CCM_E_NOT_CONVERGED if a solve hit its iteration limit (the step is still completed),
 * CCM_E_TIMEOUT if a device barrier gave up, CCM_E_NONFINITE on NaN/Inf. */
ccm_status ccm_step(ccm_case c, int nsteps, ccm_step_stats* stats);

/* Failure detection (for tests; the paper has no counterpart).  Sets the spin budget, in
 * clock64 cycles, that every block of the case's cooperative launches (the Helmholtz and
 * Poisson solves) waits at a device-wide barrier before it gives up (0 restores the default
 * of 2e9 cycles, about one second), and makes block absent_block of each such launch skip
 * its arrivals (-1: none, the default).  With a block absent, every other block's wait runs
 * out after the budget; the blocks then leave the launch, the library reads the error flag
 * and ccm_step returns CCM_E_TIMEOUT with the context intact.  The fields of the abandoned
 * step are not meaningful: restore a checkpoint (ccm_set_field) before stepping on.  The
 * single-cluster solve of small grids (ccm_launch_plan plan[5] > 0) uses the hardware
 * cluster barrier and is not affected.  CCM_E_INVALID for budget_cycles < 0 or
 * absent_block < -1. */
ccm_status ccm_set_barrier_fault(ccm_case c, long long budget_cycles, int absent_block);

/* Test hook for the exact fixed-point dot products of the FP64 one-barrier CG (the paper has
 * no counterpart): with every = k > 0, every k-th reduction of a solve also takes the FP64
 * fallback that a value outside the fixed-point window would trigger (FP64 partials and a
 * counter barrier), so that path runs in tests; 0 (the default): only on such a value.  The
 * fallback's sums round differently, so the fields agree with the normal path to the solver
 * tolerance, not bit for bit.  CCM_E_INVALID for every < 0. */
ccm_status ccm_set_sum_fallback(ccm_case c, int every);

/* Time law of the body velocity (Sec. 4.6, Eq. pm_prediction and the boundary condition of U*
 * that follows it: conv and S^n take D^n, S* and cont(U*, D^{n+1}) of Eq. pm_poisson take the
 * next level D^{n+1}).  From the next step on the body velocity is D(t) = f(t) D0 with
 *     f(t) = a0 + a1 sin(omega t + phase),  t = n dt at step n (the CCM_F_STEP counter),
 * and D0 the field set through CCM_F_DX / CCM_F_DY (no effect while none is set).  Every
 * D-term is the steady term of D0 scaled by f (the convective bracket by f and f^2), so a step
 * costs the same as with a steady D.  The faces without fluid of the present state take f(t_n)
 * D0 now.  a0 = 1, a1 = 0 restores the steady D = D0.  CCM_E_INVALID for a non-finite
 * parameter.  A case with a time law cannot join a batch (ccm_batch_add and ccm_batch_step
 * return CCM_E_INVALID). */
ccm_status ccm_set_body_motion(ccm_case c, double a0, double a1, double omega, double phase);

/* Enqueue nsteps projection steps on the case's stream and return without waiting; the
 * statistics accumulate on the device until ccm_read_stats.  Same state rules as
 * ccm_step.  Errors detected on the host only (CCM_E_STATE, CCM_E_INVALID, CCM_E_CUDA). */
ccm_status ccm_step_async(ccm_case c, int nsteps);

/* Wait for the case's stream and report the statistics accumulated since the previous
 * ccm_step, ccm_read_stats or ccm_set_geometry call (same meaning and return codes as
 * ccm_step). */
ccm_status ccm_read_stats(ccm_case c, ccm_step_stats* stats);

/* Force of the fluid on the body at the current state (U^n and P^{n-1/2} after the last
 * step), force[4] = {Fp_x, Fp_y, Fv_x, Fv_y}: the pressure and viscous parts, in the case's
 * units (per unit depth).  The paper reports drag and lift (Sec. 5) without a discrete
 * definition; this is the body's share of the momentum that pres(P) and visc(2 mu S) give the
 * fluid (Secs. 4.1, 4.3), i.e. with A-differences across cells equal to -n |Gamma| (Eq.
 * approximate, the surface conservation law):
 *   Fp_x = sum_cells P (A^x_{i-1/2,j} - A^x_{i+1/2,j}),  Fp_y likewise with A^y in y,
 *   Fv_x = -2 mu [sum_cells S_xx (B^xx_{i-1/2} - B^xx_{i+1/2}) + sum_nodes S_xy (B^xy_{j-1/2} - B^xy_{j+1/2})],
 *   Fv_y = -2 mu [sum_cells S_yy (B^yy_{j-1/2} - B^yy_{j+1/2}) + sum_nodes S_xy (B^yx_{i-1/2} - B^yx_{i+1/2})],
 * S of Eqs. diag and offdiag with the body's D (CCM_F_DX/DY; zero for a no-slip body), which should
 * have no normal component (no flux through the body).  The terms vanish wherever the grid is
 * uncut.  force is a host array the caller owns.  Waits for the case's stream.  CCM_E_STATE
 * before ccm_set_geometry. */
ccm_status ccm_body_force(ccm_case c, double force[4]);

/* Record the body force after every step of ccm_step / ccm_step_async (a reduction enqueued
 * after the step, no host synchronisation) into a device ring of `capacity` rows of four
 * doubles, allocated with the case's allocator; 0 stops recording and frees it.  Setting a
 * capacity clears the record.  Waits for the case's stream.  CCM_E_OOM if the ring cannot be
 * allocated (recording is then off). */
ccm_status ccm_set_force_history(ccm_case c, int capacity);

/* Copy the newest min(max_rows, recorded, capacity) rows of the record, oldest first, into
 * host[rows][4]; *rows receives that count and *total (may be NULL) the number of steps
 * recorded since ccm_set_force_history.  Row k is what ccm_body_force would have returned
 * after that step.  Waits for the case's stream. */
ccm_status ccm_get_force_history(ccm_case c, double* host, int max_rows, int* rows, long long* total);

/* Per-launch timing of the dominant kernel (the Poisson PCG): when enabled, CUDA events are
 * recorded on the case's stream around every Poisson PCG launch.  ccm_kernel_timing
 * returns (and resets) the summed event time in ms, the number of PCG launches, the PCG
 * iterations those launches ran, and the number of library kernel launches enqueued by the
 * steps since the last reset.  Waits for the case's stream. */
ccm_status ccm_enable_kernel_timing(ccm_case c, int enable);
ccm_status ccm_kernel_timing(ccm_case c, double* poisson_ms, long long* poisson_launches,
                             long long* poisson_iters, long long* kernel_launches);

/* Solve the pressure Poisson system of Eq. pm_poisson, K Phi = rhs (rhs on active cells,
 * padded layout, host), starting from the case's PHI field, and store the solution in PHI.
 * With the MIXED precision setting the inner solves run in FP32 and the FP64 residual is
 * refined to tol_p. */
ccm_status ccm_solve_pressure(ccm_case c, const double* rhs_host, ccm_solve_stats* stats);

/* Maximum padded size, (ny+3) * pitch elements, that ccm_solve_pressure_noalloc accepts. */
#define CCM_NOALLOC_MAX_ELEMS 131072

/* Pressure solve for callers that cannot allocate device memory.  The paper has no
 * counterpart: this entry point exists for callers that may not call cudaMalloc, such as a
 * host framework that owns all device memory through its own pool, a process under a hard
 * device-memory cap, or latency-sensitive code that must avoid the device-wide
 * synchronisation cudaMalloc and cudaFree imply.  It solves the same system as
 * ccm_solve_pressure, in FP64 with the Jacobi preconditioner to tol_p, whatever the case's
 * precision and preconditioner settings, but allocates nothing: its scratch vectors sit in
 * one fixed file-scope device array of about 6.4 MB that every GPU loading the library keeps
 * until the process exits.
 *   rhs_dev  right-hand side, device memory in the case's pitched layout: (ny+3) rows of
 *            `pitch` doubles (pitch from ccm_field_device_ptr), origin at index (-1, -1);
 *            only active cells are read.  Not modified.
 *   phi_dev  same layout; in: warm start, out: solution (zero outside active cells).
 * Grids with (ny+3)*pitch > CCM_NOALLOC_MAX_ELEMS are rejected with CCM_E_INVALID.  All calls
 * share the one array, so calls that overlap on the GPU race; each call clears what must
 * start at zero.  The first call on a device looks the array's device address up (with that
 * device current); make it before any stream capture.  Runs on the case's stream and
 * returns when the solve has finished. */
ccm_status ccm_solve_pressure_noalloc(ccm_case c, const double* rhs_dev, double* phi_dev, ccm_solve_stats* stats);

/* ---- Batches: independent cases advanced together -------------------------------------
 * Serving form of the step (the paper has one case at a time).  Every case of a batch must
 * use the batch's stream and the same precision setting.  Every stage of a step is one launch
 * for all cases: the explicit stages (box data, predictor right-hand side, U* and the Poisson
 * right-hand side, projection), one cooperative launch for the CN Helmholtz solves, and one
 * for the Poisson solves (FP64 CG or the mixed solve with each case's preconditioner; with a
 * singular case, FP64 Jacobi-PCG or the FP64 refinement with batched FP32 inner solves),
 * each case on a range of blocks sized by its cells (and width, as tuned).  When every case has an outflow
 * side, steps after each case's first replay two captured CUDA graphs (one per time-level
 * parity), recaptured when the cases change.  A batch holds at most as many cases as the GPU
 * holds PCG blocks (2 per SM).  Cases keep their own state and can leave and join a batch
 * between steps. */
typedef struct ccm_batch_s* ccm_batch;
ccm_status ccm_batch_create(int max_cases, void* stream, ccm_batch* out);
ccm_status ccm_batch_destroy(ccm_batch b);
ccm_status ccm_batch_add(ccm_batch b, ccm_case c);
ccm_status ccm_batch_remove(ccm_batch b, ccm_case c);
int ccm_batch_size(ccm_batch b);
/* Advance every case of the batch nsteps steps; stats (may be NULL) receives one entry per
 * case, in the order the cases were added.  Returns the first non-OK status of any case. */
ccm_status ccm_batch_step(ccm_batch b, int nsteps, ccm_step_stats* stats);
/* Whether steps replay captured graphs (1, the default) or issue every launch (0).  Both give
 * the same fields bit for bit. */
ccm_status ccm_batch_set_graphs(ccm_batch b, int enable);
/* Steps this batch has replayed from captured graphs. */
ccm_status ccm_batch_graph_steps(ccm_batch b, long long* steps);
/* Online tuning of the Poisson launch's block split: with it on (the default), the three steps
 * after the cases' first each use one candidate split (blocks in proportion to cells x nx^a,
 * a = 0, 1/2, 1; the steps advance the cases as usual) and the one with the least Poisson time
 * per cell-iteration is kept.  When the batch's cells have changed by more than 30 % since the
 * split was tuned (cases joined or left), the next three steps tune it again.  Off: a = 0. */
ccm_status ccm_batch_set_tuning(ccm_batch b, int enable);
/* The exponent a in use and whether the tuning has finished. */
ccm_status ccm_batch_split(ccm_batch b, double* exponent, int* tuned);

/* ---- Request loop (serving) ------------------------------------------------------------
 * Flow-past-body requests wait in a FIFO queue; each round of ccm_server_run admits queued
 * requests in arrival order while their device footprint (ccm_case_bytes) fits the HBM budget
 * and a batch slot is free, advances all resident requests by one chunk of steps through a
 * batch (FP64 and mixed-precision requests in separate batches), and retires the requests
 * that reached their step count.  Requests submitted while others run join at the next
 * round (continuous batching).  Not thread-safe: submit, run and poll from one thread. */
typedef struct ccm_server_s* ccm_server;
ccm_status ccm_server_create(size_t hbm_budget_bytes, int max_batch, int chunk_steps, void* stream, ccm_server* out);
ccm_status ccm_server_destroy(ccm_server s);
/* Queue a request (the config's stream is replaced by the server's); CCM_E_OOM if it can
 * never fit the budget. */
ccm_status ccm_server_submit(ccm_server s, const ccm_config* cfg, const ccm_geometry* geo, int nsteps, long long* id);
/* Run `rounds` rounds; *active (may be NULL) receives the number of queued or running
 * requests left.  Returns the first error a batch step reported (requests continue). */
ccm_status ccm_server_run(ccm_server s, int rounds, int* active);
/* state: 0 queued, 1 running, 2 done, 3 failed; times3: submit, admit, done (seconds, one
 * monotonic clock); stats: last step's statistics, iteration counts summed over all steps. */
ccm_status ccm_server_poll(ccm_server s, long long id, int* state, double* times3, ccm_step_stats* stats);
/* Any field of a running request (as ccm_get_field); CCM_F_U, CCM_F_V or CCM_F_P of a finished
 * one, whose case was destroyed at completion after these fields were copied to host memory
 * (a finished request holds no device memory). */
ccm_status ccm_server_get_field(ccm_server s, long long id, int field, double* host, size_t count);
/* Forget a finished or queued request and free its host copies (CCM_E_STATE while it runs). */
ccm_status ccm_server_release(ccm_server s, long long id);
size_t ccm_server_bytes_in_use(ccm_server s);

/* Thread-local message of the last failure ("" if none). */
const char* ccm_last_error(void);

/* Library version (CCM_VERSION). */
int ccm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CCM_H */
