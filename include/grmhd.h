/*
 * grmhd.h -- C ABI of the GB300 GR-MHD step library (libgrmhd.so).
 *
 * The library advances the ideal GR-MHD equations of cuHARM (Begue et al.,
 * arXiv 2205.02484) on a modified-Kerr-Schild grid with the HARM-style
 * conservative scheme of its Section 2: PLM-MC reconstruction (Eqs. 16-17),
 * LLF or HLL fluxes (Eqs. 18-21), flux-CT (Eqs. 22-24), connection sources
 * (Eqs. 7, 15), the RK2 predictor-corrector (Eqs. 25-26), the CFL time step
 * (Eq. 27), Newton/Brent/entropy conserved-to-primitive inversion (Section
 * 2.3, Eqs. 28-32), failure fixups (Eq. 33), floors and ceilings (Section 2.4,
 * Eq. 34), and horizon diagnostics (Section 4.2, Eqs. 38-42).  Every step of
 * the method runs in CUDA kernels compiled for sm_103a.
 *
 * Conventions shared by all calls:
 *  - Every function returns 0 on success or a negative GRMHD_E* code; no C++
 *    exception crosses the ABI.  grmhd_last_error() returns a message for the
 *    last failure of a context (or of context creation when ctx is NULL); the
 *    string is owned by the library and valid until the next call on it.
 *  - Primitive arrays P hold 8 fields (rho, u, ut^1, ut^2, ut^3, B^1, B^2,
 *    B^3) in the paper's notation of Eq. 11; conserved arrays U hold 9 fields
 *    sqrt(-g) (rho u^t, T^t_t, T^t_1, T^t_2, T^t_3, B^1, B^2, B^3, S u^t)
 *    (Section 2.1 and Eq. 12, S = p / rho^(gam-1)).  Field-major layout:
 *    element (f, i, j, k) of an active-zone array sits at
 *    ((f * n1 + i) * n2 + j) * n3 + k, with k (phi) fastest.
 *  - Pointers are either host or device memory as the on_device argument
 *    says.  Buffers passed in are always owned by the caller; the library
 *    copies from and into them and never keeps a pointer past the call.  The
 *    context owns all of its device memory, streams and CUDA graphs.
 *  - All device work of a context is issued on its stream (the stream given
 *    in grmhd_grid_params, or a stream the library creates when that is NULL).
 *    Calls that return data to the host synchronise that stream first.
 */
#ifndef GRMHD_H
#define GRMHD_H

#ifdef __cplusplus
extern "C" {
#endif

#define GRMHD_OK 0
#define GRMHD_EINVAL (-1)     /* bad argument or parameter */
#define GRMHD_ECUDA (-2)      /* CUDA runtime error (message in grmhd_last_error) */
#define GRMHD_ENOMEM (-3)     /* device or host allocation failed */
#define GRMHD_ENONFINITE (-4) /* non-finite value found in the state */
#define GRMHD_EFIXUP (-5)     /* some failed zones could not be fixed (Eq. 33) */
#define GRMHD_EITER (-6)      /* a bounded loop ran out of iterations */
#define GRMHD_ESTATE (-7)     /* call made in the wrong order (e.g. step before init) */

/* metric kinds for grmhd_set_metric */
#define GRMHD_KERR_MKS 0   /* Kerr in modified Kerr-Schild coordinates (Section 4.1) */
#define GRMHD_MINK_CART 1  /* flat space, Cartesian box (tests) */

/* boundary kinds (used for GRMHD_MINK_CART; Kerr grids always use inflow /
 * polar reflection / periodic in X1 / X2 / X3, Section 4.1) */
#define GRMHD_BC_INFLOW 0
#define GRMHD_BC_POLAR 1
#define GRMHD_BC_PERIODIC 2
#define GRMHD_BC_OUTFLOW 3
#define GRMHD_BC_EXTERNAL 4 /* bc3 only: the X3 ghosts are written by the caller (grmhd_x3_unpack), for a
                               phi slab of a decomposed grid; on a Kerr grid the slab spans
                               [x3min, x3max) of phi, which sets dX3 */

#define GRMHD_PLM 0 /* Eqs. 16-17 */
#define GRMHD_PPM 1 /* the parabolic reconstruction of Section 2.2 */

#define GRMHD_LLF 0 /* Eq. 18 */
#define GRMHD_HLL 1 /* Eq. 21 */

#define GRMHD_FP64 0  /* every stage in FP64 */
#define GRMHD_MIXED 1 /* reconstruction, fluxes, EMFs in FP32; U and the inversion in FP64 */

/* per-zone inversion flags (grmhd_con2prim): low 3 bits = method */
#define GRMHD_C2P_NR 0           /* 2D Newton-Raphson on (W, v^2), Eqs. 29-30 */
#define GRMHD_C2P_BRENT_W 1      /* 1D Brent in W */
#define GRMHD_C2P_ENTROPY 2      /* entropy inversion (Eq. 32) as fallback */
#define GRMHD_C2P_ENTROPY_BETA 3 /* entropy inversion chosen because beta < 1e-2 */
#define GRMHD_C2P_FAIL 8         /* inversion failed: zone needs a fixup */
#define GRMHD_C2P_FAIL_D 16      /* D <= 0 or non-finite input */
#define GRMHD_C2P_FAIL_ENT 32    /* entropy inversion impossible */
#define GRMHD_C2P_LEARNED 64     /* with GRMHD_C2P_NR: Newton converged from the learned rescue start */

typedef struct grmhd_ctx grmhd_ctx;

/* Grid of n1 x n2 x n3 active zones (X1 = radius-like, X2 = polar, X3 = phi).
 * For GRMHD_KERR_MKS: r(X1) = R0 + exp(X1) inside x_b = ln(r_br - R0) and
 * R0 + exp(X1 + (X1 - x_b)^n_x) outside; theta(X2) = pi/2 (1+X2) +
 * (1-hslope)/2 sin(pi (1+X2)) with X2 in [-1, 1]; X3 = phi in [0, 2 pi)
 * (Eq. 36).  X1 spans [ln(r_in - R0), X1(r_out)].  For GRMHD_MINK_CART the
 * box [x1min, x1max] x [x2min, x2max] x [x3min, x3max] and bc1..bc3 are used. */
typedef struct {
    int n1, n2, n3;
    int metric;
    double r_in, r_out, hslope, r_br, n_x, R0;
    double x1min, x1max, x2min, x2max, x3min, x3max;
    int bc1, bc2, bc3;
    int riemann;   /* GRMHD_LLF or GRMHD_HLL */
    int precision; /* GRMHD_FP64 or GRMHD_MIXED */
    int device;    /* CUDA device ordinal */
    void *stream;  /* cudaStream_t to issue work on, or NULL */
    /* A theta slab of a decomposed grid (Sec. 3): the active X2 rows
     * [j0, j0 + n2) of a grid of n2_total rows (n2_total = 0: not a slab,
     * j0 must be 0).  The metric is built at the rows' global X2 positions
     * (dX2 from n2_total), the poles are the whole grid's, and the X2 ghost
     * rows of a side inside the grid (or of a periodic side) are written by
     * the caller (grmhd_x2_unpack).  A slab has n2 >= 4 rows, is not also a
     * phi slab (bc3 external), steps by the stage parts below and takes its
     * state from grmhd_set_state (grmhd_init_torus: GRMHD_EINVAL). */
    int j0, n2_total;
    /* Face reconstruction: GRMHD_PLM, the MC-limited linear slopes of Eqs.
     * 16-17, or GRMHD_PPM, the piecewise parabolic method Section 2.2 names as
     * its successor (Colella & Woodward 1984 for uniform zones in code
     * coordinates: interface values from MC-limited slopes, then the
     * monotonicity constraints; no contact steepening or shock flattening),
     * whose face stencil reads three zones on each side. */
    int recon;
    /* Polar cylindrification (Section 4.1, after Tchekhovskoy et al. 2011;
     * the paper prints no formula).  cyl_r <= 0: off.  Otherwise, Kerr grids
     * only, inside a band of X2 width cyl_dx2 (0 < cyl_dx2 <= 1) next to each
     * pole theta(X1, X2) = theta_MKS(X2'), X2' = pole -/+ cyl_dx2 phi(s) with
     * s = |X2 - pole| / cyl_dx2, phi(s) = s + (lambda - 1) s (1 - s^2)^3 and
     * lambda(r) = (1 + (cyl_r / r)^4)^(1/4): the rows next to the pole are
     * widened by lambda(r), which for r << cyl_r keeps them near cylinders
     * of radius cyl_r theta_MKS.  grmhd_set_metric refuses (GRMHD_EINVAL)
     * lambda > 5/2 at the innermost ghost face, where phi' would come close
     * to changing sign, and a band on a flat-space grid. */
    double cyl_r, cyl_dx2;
} grmhd_grid_params;

/* Physics constants; the paper's values are cfl 0.45 (Eq. 27), nr_tol 1e-10
 * (Section 2.3), sigma_max 50, bu_max 2500, gamma_max 50 and beta_entropy
 * 1e-2 (Section 2.4). */
typedef struct {
    double gam;
    double cfl, nr_tol, sigma_max, bu_max, gamma_max, beta_entropy;
    int nr_maxit, brent_maxit, fix_maxsweep;
} grmhd_phys_params;

/* Fishbone-Moncrief torus with inner edge r_in and pressure maximum r_max
 * (Section 5); A_phi = max(rho/rho_max - 0.2, 0) (Eq. 45) normalised so that
 * max p_g / max p_B = beta0 (beta0 <= 0: no field); internal energy
 * perturbed by a factor 1 + pert_amp (2 xi - 1) with xi from splitmix64(seed
 * XOR zone index).  kappa is the polytropic constant (it cancels after the
 * rho_max normalisation; 1e-3 if <= 0). */
typedef struct {
    double r_in, r_max, beta0, pert_amp, kappa;
    unsigned long long seed;
} grmhd_torus_params;

/* Diagnostics (Section 4.2): horizon fluxes at the first zone with r >= r_H,
 * mdot = sum sqrt(-g) rho u^1 dX2 dX3 (Eq. 38), phib = 1/2 sum |sqrt(-g) B^1|
 * dX2 dX3 (Eq. 39), edot = -sum sqrt(-g) T^1_t (Eq. 41), ldot = sum sqrt(-g)
 * T^1_3 (Eq. 40), PhiB = phib / sqrt|mdot| (Eq. 42); divb_max is the largest
 * corner divergence of Eq. 24; disk_mass / disk_eb are the initial disk
 * integrals of Section 5.  Counters accumulate over all steps since init. */
typedef struct {
    double t, dt, mdot, phib, PhiB, edot, ldot, divb_max, disk_mass, disk_eb;
    double eta; /* (edot - mdot) / |mdot| (Eqs. 38, 41); 0 when mdot = 0 */
    long long nr_iters, n_nr, n_brent, n_entropy, n_entropy_beta, n_fail, n_floor, n_ceil,
        n_gcap, n_fixed, fix_sweeps, n_steps;
    long long n_learned; /* inversions converged by Newton from the learned rescue start (grmhd_set_learned_guess) */
} grmhd_diag;

/* Create a context: validates the parameters, allocates the device state and
 * builds nothing else.  *out is set only on success.  Errors: EINVAL, ENOMEM,
 * ECUDA. */
int grmhd_init_grid(const grmhd_grid_params *grid, const grmhd_phys_params *phys,
                    grmhd_ctx **out);

/* Build the metric tables (Section 4.1, Eqs. 35-36): g_{mu nu}, g^{mu nu},
 * sqrt(-g) and the lapse at zone centres and X1/X2 face centres, and the
 * connection Gamma^l_{mu nu} at centres (exact derivatives by forward-mode
 * dual numbers).  a is the black-hole spin (ignored for flat space). */
int grmhd_set_metric(grmhd_ctx *ctx, double a, int kind);

/* Set the torus initial state (needs grmhd_set_metric with GRMHD_KERR_MKS),
 * fill the ghosts and compute the first time step from a flux sweep. */
int grmhd_init_torus(grmhd_ctx *ctx, const grmhd_torus_params *torus);

/* Copy a full active-zone state in (P: 8 fields, U: 9 fields) with the time
 * t and the next step dt; ghosts are refilled from the boundary conditions.
 * In GRMHD_MIXED mode P is rounded to FP32.  A host state (on_device = 0)
 * is copied in four byte ranges on four internal streams (several copy
 * engines), ordered after the work already on the context stream; the call
 * returns when the state is on the device.  The status word read by
 * grmhd_sync is cleared (counters keep accumulating).  If P or U holds a
 * non-finite value the call returns GRMHD_ENONFINITE and the context has no
 * state until a later grmhd_set_state or grmhd_init_torus succeeds
 * (grmhd_step: GRMHD_ESTATE). */
int grmhd_set_state(grmhd_ctx *ctx, const double *P, const double *U, double t, double dt,
                    int on_device);

/* Set the state from the conserved variables alone (U: 9 fields, FP64) with
 * the time t and the next step dt; the primitives are re-derived on the
 * device by the step's own inversion, floors, ceilings, Lorentz cap and
 * fixups (Sections 2.3-2.4, Eq. 33), Newton starting from the primitives the
 * context holds, and the ghosts refilled.  U passes through unchanged except
 * where a floor or a fixup acts (then, as in a step, U is recomputed from
 * the corrected primitives).  For a U that grmhd_get_state returned (P is
 * the inversion of U after every step) the primitives come back to the
 * inversion's tolerance (GRMHD_MIXED: the mixed Newton's acceptance, up to
 * ~1e-5 relative in u of cold gas), so a serving loop can move half the
 * bytes of a full state.  The inversions count in the diagnostics counters like a stage's.
 * Needs a state already (grmhd_set_state or grmhd_init_torus: GRMHD_ESTATE
 * otherwise) and a whole grid (a slab: GRMHD_EINVAL); t and dt finite,
 * dt >= 0 (GRMHD_EINVAL).  A host U is copied as in grmhd_set_state; the
 * call returns when the primitives are on the device.  A non-finite value in
 * U returns GRMHD_ENONFINITE and leaves the context without a state;
 * unfixable inversion failures raise GRMHD_EFIXUP at the next grmhd_sync. */
int grmhd_set_state_u(grmhd_ctx *ctx, const double *U, double t, double dt, int on_device);

/* Copy the active-zone state out (any of P, U, t, dt may be NULL); a host
 * copy is split as in grmhd_set_state.  Returns when the copy is done. */
int grmhd_get_state(grmhd_ctx *ctx, double *P, double *U, double *t, double *dt,
                    int on_device);

/* Advance nsteps full RK2 steps (Eqs. 25-26) with the CFL time step of Eq. 27
 * (dt of step n+1 from the predictor sweep of step n).  Asynchronous on the
 * context stream; each step replays one captured CUDA graph.  Inversion
 * failures that the fixups cannot repair within fix_maxsweep Jacobi sweeps
 * (Eq. 33) raise GRMHD_EFIXUP, and a failed zone whose conserved vector is
 * not finite raises GRMHD_ENONFINITE, at the next grmhd_sync or
 * grmhd_diagnostics; the state is still stepped (the unrepaired zones keep
 * their previous primitives) and grmhd_set_state clears the status.
 * GRMHD_EINVAL for a phi slab
 * (bc3 = GRMHD_BC_EXTERNAL), whose ghost planes must be exchanged between
 * the stages (grmhd_stage), and for a theta slab (n2_total > 0), which steps
 * by the stage parts. */
int grmhd_step(grmhd_ctx *ctx, int nsteps);

/* Batched stand-alone inversion of n conserved states U (9 x n, sqrt(-g)
 * included) at the centre metric of active zones loc[n] (loc = i*n2 + j),
 * starting from and overwriting P_inout (8 x n).  flags[n] receives the
 * GRMHD_C2P_* code, iters[n] (may be NULL) the Newton iterations.  With
 * use_learned_guess = 1 Newton first starts from the loaded MLP's W and, if
 * it does not converge, again from P_inout (for callers whose P_inout is a
 * poor start); with use_learned_guess = 2 Newton starts from P_inout and, if
 * it does not converge, from the MLP's W before Brent (the step's order, see
 * grmhd_set_learned_guess; such zones are flagged GRMHD_C2P_NR |
 * GRMHD_C2P_LEARNED).  iters counts every Newton run.  Same method order
 * and tolerances as the step otherwise (Section 2.3).  The zones that leave
 * Newton (Brent, the entropy inversion) finish in a second pass over a
 * compacted list, with the same results; n < 2^31 - 1 (GRMHD_EINVAL
 * otherwise); the context keeps n + 1 ints of device scratch for the list,
 * allocated on the first call that needs more. */
int grmhd_con2prim(grmhd_ctx *ctx, const double *U, const int *loc, double *P_inout,
                   int *flags, int *iters, long n, int use_learned_guess, int on_device);

/* Diagnostics of a grid split over several contexts (the slabs of the
 * decomposition, Section 3), combined on the device.  grmhd_diag_partials
 * writes this context's GRMHD_DIAG_NPART partial values to device memory
 * out_dev (asynchronous on the context stream): its horizon-shell sums of
 * Eqs. 38-41, its largest corner divergence (Eq. 24), its Eq. 43 numerator and
 * mass sum over r_H <= r <= r_bar_max (r_bar_max <= 0 or a flat grid: 0), t,
 * dt and its counters.  grmhd_diag_combine adds nparts such vectors stored
 * one after another at parts_dev (device memory, e.g. gathered from all ranks)
 * in their order, in one device thread, so that every rank forms the same
 * bits: integrals and counters add, div B and the fixup sweep count take the
 * largest, t, dt and the step count are the first vector's; then
 * Phi_BH = phi_B / sqrt|Mdot| (Eq. 42), (Edot - Mdot)/|Mdot| and the Eq. 43
 * quotient are formed.  out receives the whole grid's diagnostics (disk_mass
 * and disk_eb from this context); bary3 (may be NULL) the barycentric radius,
 * its mass sum and numerator.  Returns the context's status like
 * grmhd_sync. */
#define GRMHD_DIAG_NPART 26
int grmhd_diag_partials(grmhd_ctx *ctx, double r_bar_max, double *out_dev);
int grmhd_diag_combine(grmhd_ctx *ctx, const double *parts_dev, int nparts, grmhd_diag *out, double *bary3);

/* Batched conserved variables of n primitive states at zones loc[n]. */
int grmhd_prim2cons(grmhd_ctx *ctx, const double *P, const int *loc, double *U, long n,
                    int on_device);

/* Riemann fluxes after flux-CT for the current primitives, active faces only:
 * out[d][c][n1+1][n2+1][n3+1] (d = direction, c = 9 components, face index
 * along d; unused slots zero).  In GRMHD_MIXED the energy component (c = 1)
 * is carried rest-mass subtracted, the energy flux plus the mass flux, as the
 * mixed update uses it.  *dt_out (may be NULL) receives the CFL step of
 * Eq. 27.  Runs the step's own flux and EMF kernels.  For tests. */
int grmhd_fluxes(grmhd_ctx *ctx, double *out, double *dt_out, int on_device);

/* Synchronise the context stream and return the device-side status
 * (GRMHD_EFIXUP / GRMHD_ENONFINITE if a step hit one) or 0. */
int grmhd_sync(grmhd_ctx *ctx);

/* Synchronise and compute the diagnostics of the current state. */
int grmhd_diagnostics(grmhd_ctx *ctx, grmhd_diag *out);

/* Release everything the context owns. NULL is allowed. */
void grmhd_destroy(grmhd_ctx *ctx);

const char *grmhd_last_error(const grmhd_ctx *ctx);

/* Number of timing slots filled by grmhd_step_profiled. */
#define GRMHD_PROF_SLOTS 16

/* Run nsteps steps without the graph, with a CUDA event on the context
 * stream before each kernel group, and accumulate the elapsed milliseconds:
 * ms_out[stage*7 + part] for stage 0 (predictor) / 1 (corrector) and part
 * 0-2 fluxes along X1..X3 (Eqs. 16-21), 3 EMFs (Eq. 22), 4 update + inversion
 * (Eqs. 25-26, Section 2.3-2.4), 5 fixups (Eq. 33), 6 boundary fill; ms_out[14]
 * the time-step finalisation (Eq. 27), ms_out[15] the whole step.  The state
 * advances exactly as with grmhd_step.  ms_out holds GRMHD_PROF_SLOTS doubles. */
int grmhd_step_profiled(grmhd_ctx *ctx, int nsteps, double *ms_out);

/* Throughput of dependent-FMA chains on device (fp64 = 1: double, 0:
 * float), in TFLOP/s (2 flops per FMA): the ALU roofline denominators for
 * kernels bound by FP64 or FP32 arithmetic.  Allocates a 8 KB buffer and
 * runs a few sub-second kernels. */
int grmhd_peak_probe(int device, int fp64, double *tflops);

/* ----------------------------------------------------------------------
 * Ensemble: many independent grids advanced together.  Every kernel class
 * of the RK2 step (face sweeps, EMFs, update + inversion, fixups, boundary
 * fill, dt) is one persistent launch that walks a ragged tile list over all
 * members, and one ensemble step is one captured CUDA graph.  Members are
 * contexts made with grmhd_init_grid / grmhd_set_metric / grmhd_init_torus
 * (or grmhd_set_state); they may differ in size, spin, adiabatic index and
 * field, but must share the device and the precision.  They keep their own
 * state, time step, counters and diagnostics (read them with the member
 * calls), must outlive the ensemble, and are stepped on the first member's
 * stream.  Each member evolves exactly as it would alone.
 * ---------------------------------------------------------------------- */
typedef struct grmhd_ens grmhd_ens;

/* Tiling of the persistent launches: elements per thread per tile and
 * persistent blocks per SM, for the face sweeps and for the update kernel. */
typedef struct {
    int items_flux, items_update, blocks_per_sm_flux, blocks_per_sm_update;
    /* members with at least 2^solo_log2 active zones step with their own
     * single-grid kernels, on up to 16 parallel branches of the ensemble
     * graph beside the batched kernels (their flux and EMF arrays then stay
     * in L2 between the kernels of their step); 0: every member is batched.
     * Range 0 or 10-40. */
    int solo_log2;
} grmhd_ens_tiling;

/* Build an ensemble of n member contexts (each with metric and state).
 * Errors: EINVAL (mixed devices or precisions, a member that is a phi or
 * theta slab, or a member with GRMHD_PPM faces: the batched sweeps walk PLM
 * columns), ESTATE (member not ready), ENOMEM. */
int grmhd_ensemble_create(grmhd_ctx *const *members, int n, grmhd_ens **out);

/* Advance every member by nsteps RK2 steps (asynchronous; graph replay). */
int grmhd_ensemble_step(grmhd_ens *ens, int nsteps);

/* Set / read the tiling (1-16 elements per thread, 1-64 blocks per SM, the
 * solo threshold). */
int grmhd_ensemble_set_tiling(grmhd_ens *ens, const grmhd_ens_tiling *t);
int grmhd_ensemble_get_tiling(const grmhd_ens *ens, grmhd_ens_tiling *t);

/* Time trial steps over a grid of tilings (face sweeps and update timed
 * separately with CUDA events), then over solo thresholds (whole steps),
 * keep the fastest, and restore every member's state, counters and time step
 * afterwards.  best / best_ms (one step of the chosen tiling) may be NULL. */
int grmhd_ensemble_autotune(grmhd_ens *ens, int trial_steps, grmhd_ens_tiling *best, double *best_ms);

/* Synchronise and return the first member status error (GRMHD_EFIXUP ...). */
int grmhd_ensemble_sync(grmhd_ens *ens);

void grmhd_ensemble_destroy(grmhd_ens *ens);
const char *grmhd_ensemble_last_error(const grmhd_ens *ens);

/* Horizon diagnostics that allocate no device memory at all.  The paper has
 * no counterpart: this is a library convenience for callers that may not
 * call cudaMalloc -- for example a host application that has handed all
 * device memory to its own pool allocator and forbids further allocation,
 * or a monitoring hook that must not disturb a fixed memory budget between
 * steps.  It computes the same sums as grmhd_diagnostics (same kernels) but
 * keeps the reduction's partial sums in a fixed array of the library
 * (256 KiB, reserved on every device that loads the library until exit)
 * instead of the context's scratch buffer.
 *   out_dev: caller-owned device memory for 8 doubles; once the context
 *            stream has run the work, out_dev[0..4] = mdot, phib, edot, ldot,
 *            divb_max and out_dev[5..7] are zero.  The call is asynchronous
 *            on the context stream and does not synchronise it.
 * Limit: the horizon shell n2 * n3 may not exceed 2,097,152 zones
 * (GRMHD_EINVAL with a message otherwise).  The first call on a device
 * looks up the array's device address; make that first call before any
 * stream capture.  All calls on a device share the array: calls whose
 * kernels overlap on the GPU (e.g. contexts on different streams) race. */
int grmhd_diagnostics_noalloc(grmhd_ctx *ctx, double *out_dev);

/* ---------------------------------------------------------------------
 * Learned Newton start of the inversion (Section 2.3 names the Newton
 * starting point; the learned guess is this library's extension).  A 5-64-64-1
 * ReLU network maps five invariants of a conserved state to log(W/D), where
 * W = Gamma^2 (rho + u + p) and D = Gamma rho.  Newton then starts from that W,
 * with v^2 from Eq. 29.
 *
 * Features, from the Section 2.3 variables with tau = -n.Q - D, each argument
 * clamped below at 1e-30:
 *   log(tau/D), log(Qt^2/D^2), log(Bf^2/D), log((Q.Bf)^2/D^3), log(D)
 *
 * Parameter vector theta: FP32, GRMHD_MLP_NPARAM entries, in this order:
 *   W1[64][5], b1[64], W2[64][64], b2[64], W3[64], b3   (rows = output units)
 * The forward pass uses the weight matrices rounded to BF16 (ties to even)
 * and keeps inputs, biases, activations and accumulation in FP32.
 *
 * norm[GRMHD_MLP_NNORM] standardises inputs and output:
 *   feature mean[5], feature std[5], output mean, output std.
 *   x = (f - mean)/std, and prediction = s*std_y + mean_y.
 *
 * Training loss over a batch of n samples: (1/n) sum (s - t)^2, with
 * t = (y - mean_y)/std_y.  The gradient of each weight is taken at its BF16
 * value and applied to the FP32 master copy.  The optimiser is AdamW with
 * bias-corrected moments and decoupled weight decay on W1, W2, W3.
 * ------------------------------------------------------------------- */
#define GRMHD_MLP_NPARAM 4609
#define GRMHD_MLP_NNORM 12

/* Load parameters (host arrays) as the context's network; the inversion
 * entry points may then use it (use_learned_guess). */
int grmhd_mlp_load(grmhd_ctx *ctx, const float *theta, const float *norm);

/* Copy the context's network (FP32 master and norm) to host arrays. */
int grmhd_mlp_get(grmhd_ctx *ctx, float *theta, float *norm);

/* Samples first .. first+n-1 of the seeded training distribution, at
 * zone-centre metrics of this grid; needs grmhd_set_metric.  Any output may
 * be NULL.  Outputs, field-major:
 *   P (8 x n), loc (n, = i*n2 + j), U (9 x n, sqrt(-g) included),
 *   feat (5 x n, FP32), label (n, FP32 log(W/D)).
 * Sample i draws xi_k = top 53 bits of splitmix64(seed ^ (16 i + k)),
 * k = 0..9, and sets:
 *   - the zone (floor(xi_0 n1), floor(xi_1 n2));
 *   - rho = 1e-6^(1-xi_2);
 *   - u/rho = 1e-4 * 1e5^xi_3;
 *   - Gamma = 50^xi_4;
 *   - b^2/rho = 1e-3 * 1e5^xi_5;
 *   - directions (cos th, ph) = (2 xi_6 - 1, 2 pi xi_7) for the velocity and
 *     (2 xi_8 - 1, 2 pi xi_9) for the field, with components e^i/sqrt(g_ii). */
int grmhd_mlp_samples(grmhd_ctx *ctx, unsigned long long seed, long first, long n, double *P, int *loc,
                      double *U, float *feat, float *label, int on_device);

/* Predicted log(W/D) of n feature vectors (5 x n) with the loaded network. */
int grmhd_mlp_forward(grmhd_ctx *ctx, const float *feat, long n, float *y, int on_device);

/* Loss and its gradient (GRMHD_MLP_NPARAM FP32 values) over one batch of n
 * samples (n <= 262144), for the given parameters and norm. The context's
 * loaded network is left unchanged.  feat, label, grad follow on_device;
 * theta and norm are host arrays; loss (may be NULL) is a host double. */
int grmhd_mlp_loss_grad(grmhd_ctx *ctx, const float *theta, const float *norm, const float *feat,
                        const float *label, long n, float *grad, double *loss, int on_device);

/* nsteps of minibatch AdamW at a constant learning rate, from theta_inout
 * (host, FP32) with zero moments.  Step s uses samples (s*batch + b) mod n,
 * for b < batch.  theta_inout receives the result.  loss_last (may be NULL)
 * receives the mean loss of the last step, taken before its update.  The
 * loaded network is left unchanged.  batch <= 262144. */
int grmhd_mlp_train_steps(grmhd_ctx *ctx, float *theta_inout, const float *norm, const float *feat,
                          const float *label, long n, long batch, long nsteps, double lr, double beta1,
                          double beta2, double eps, double weight_decay, double *loss_last, int on_device);

typedef struct {
    long n_samples;          /* training set size (samples 0 .. n-1 of seed) */
    long n_val;              /* held-out samples n .. n+n_val-1 of the same seed */
    unsigned long long seed; /* sample seed */
    unsigned long long init_seed; /* weight initialisation seed */
    int epochs;
    int batch;               /* <= 262144 */
    double lr, lr_min;       /* cosine schedule from lr to lr_min over all steps */
    double beta1, beta2, eps, weight_decay;
} grmhd_mlp_train_params;

typedef struct {
    double loss_first, loss_last; /* mean batch loss of the first and last step */
    double val_rmse, val_maxerr;  /* error of log(W/D) on the held-out samples */
    double train_ms;              /* device time of the training steps (CUDA events) */
    double samples_per_s;         /* steps * batch / train time */
    long steps;
} grmhd_mlp_train_report;

/* Train the network on the GPU and load it as the context's network:
 *   1. generate the training and held-out samples;
 *   2. set norm from the training set's mean and std;
 *   3. initialise the weights He-uniform from init_seed;
 *   4. run epochs * n_samples / batch AdamW steps, replayed as CUDA graphs;
 *   5. evaluate the held-out error.
 * The training epochs take the set in a fresh permutation each. */
int grmhd_mlp_train(grmhd_ctx *ctx, const grmhd_mlp_train_params *tp, grmhd_mlp_train_report *rep);

/* on = 1: an inversion of grmhd_step whose Newton solves from the stage's
 * own starts (the previous primitives, and in GRMHD_MIXED first their
 * extrapolation over the previous half step) do not converge runs Newton once
 * more from the loaded network's W (v^2 of Eq. 29) before the Brent and
 * entropy fallbacks; grmhd_diag.n_learned counts the zones it converges.  The
 * previous-step start stays first because it is far closer to the root in a
 * smooth flow (1.08 Newton steps per zone at 256^3 against ~3 from the
 * network's W); the network replaces Brent where that start fails.  The
 * features are formed in FP32 from the inversion's FP64 invariants.  on = 0
 * restores the plain order.  Tolerances are unchanged.  Needs a loaded
 * network for on = 1; later loads or training runs replace the network in
 * place.  Ensemble steps always use the plain order. */
int grmhd_set_learned_guess(grmhd_ctx *ctx, int on);

/* ---------------------------------------------------------------------
 * Phi-slab decomposition (the slab layout of the paper's multi-GPU runs,
 * Section 3, split along phi).  Each slab is a context with bc3 =
 * GRMHD_BC_EXTERNAL that owns n3 consecutive phi zones.  One step of a
 * decomposed grid, on every slab:
 *   grmhd_stage(ctx, 0);  exchange the X3 ghosts of buffer 1 (P-hat);
 *   grmhd_stage(ctx, 1);  exchange the X3 ghosts of buffer 0 (P);
 *   grmhd_step_dtd(ctx, d, acc);  d = the minimum over all slabs (acc = 1
 *                                 folds a slab into d on one device; across
 *                                 devices, a MIN all-reduce of d);
 *   grmhd_finish_step(ctx, d);
 * To exchange, a slab packs its own planes with grmhd_x3_pack and unpacks its
 * neighbours' planes with grmhd_x3_unpack: side 0 takes the left
 * neighbour's side-1 pack, side 1 the right neighbour's side-0 pack, with
 * periodic wrap in phi.  The same sequence on a single context with bc3
 * periodic reproduces grmhd_step.  Every call is asynchronous on the context
 * stream and does not synchronise it.
 * ------------------------------------------------------------------- */

/* One RK2 stage (st = 0: predictor P^n -> P-hat; st = 1: corrector P-hat ->
 * P^{n+1}, Eqs. 25-26), including fixups and the X1 / X2 (and, unless
 * external, X3) boundary fill.  The predictor's faces record the
 * per-direction CFL minima of Eq. 27.  GRMHD_EINVAL for a theta slab. */
int grmhd_stage(grmhd_ctx *ctx, int st);

/* The per-direction CFL minima of the last predictor into dtd_dev (3 doubles,
 * caller-owned device memory): stored (accumulate = 0) or folded in by a
 * minimum (accumulate = 1).  Resets the context's minima. */
int grmhd_step_dtd(grmhd_ctx *ctx, double *dtd_dev, int accumulate);

/* Advance t by the current dt, then set the next dt from Eq. 27 applied to
 * dtd_dev (3 doubles of device memory: the minima over all slabs). */
int grmhd_finish_step(grmhd_ctx *ctx, const double *dtd_dev);

/* Bytes of one side's X3 planes: NG = 3 planes of all 8 primitives over the
 * ghosted (X1, X2) cross-section, layout [NG][8][n1 + 2 NG][n2 + 2 NG], element
 * type double (GRMHD_FP64) or float (GRMHD_MIXED). */
int grmhd_x3_plane_bytes(grmhd_ctx *ctx, unsigned long long *bytes);

/* Pack the two outermost active planes of buffer `which` (0 = P, 1 = P-hat)
 * on `side` (0 = low phi, k = 0, 1; 1 = high phi, k = n3-2, n3-1) into the
 * caller's device buffer. */
int grmhd_x3_pack(grmhd_ctx *ctx, int which, int side, void *buf_dev);

/* Write a neighbour's packed planes into the ghosts on `side` (0: k = -2, -1;
 * 1: k = n3, n3+1) of buffer `which`. */
int grmhd_x3_unpack(grmhd_ctx *ctx, int which, int side, const void *buf_dev);

/* ---------------------------------------------------------------------
 * Theta slabs (grid parameters j0, n2_total).  The fixups of Eq. 33 average
 * a failed zone's X1 / X2 neighbours, so on a theta slab they reach one row
 * across a slab face and each sweep must see the neighbours' current edge
 * rows.  One RK2 step of R slabs (st = 0, then 1; out = 1 for st 0, 0 for
 * st 1, the buffer the stage writes):
 *   grmhd_stage_update(ctx, st) on every slab;  (st 0:) grmhd_step_dtd;
 *   n = 0;  left = sum over slabs of grmhd_fail_count;
 *   while (left > 0 && n < fix_maxsweep):
 *       exchange kind-1 rows of buffer `out`;
 *       left = sum over slabs of grmhd_fix_sweep(ctx, st, .);  n++;
 *   grmhd_fix_end(ctx, st, n) and grmhd_stage_bc(ctx, st) on every slab;
 *   exchange kind-0 rows of buffer `out`;
 * then grmhd_finish_step with the minima over all slabs.  To exchange, a
 * slab packs its side 0 (low theta) and side 1 rows with grmhd_x2_pack and
 * unpacks its low neighbour's side-1 pack into its side 0 and its high
 * neighbour's side-0 pack into its side 1 (no neighbour across a pole).
 * Every call is asynchronous on the context stream; reading `left` on the
 * host is the caller's synchronisation.  When all slabs sit on one device,
 * grmhd_theta_ring_fix runs the whole fixup loop there instead (no host
 * read), so that a ring step can be captured in a CUDA graph.
 * ------------------------------------------------------------------- */

/* Fluxes, flux-CT, update and inversion of stage st (a stage up to its
 * fixups); the predictor's faces record the CFL minima. */
int grmhd_stage_update(grmhd_ctx *ctx, int st);

/* Add the number of zones whose inversion failed in the last
 * grmhd_stage_update to *acc_dev (one long long of device memory). */
int grmhd_fail_count(grmhd_ctx *ctx, long long *acc_dev);

/* One Jacobi sweep of the fixups (Eq. 33) over stage st's output, reading
 * the kind-1 ghost rows as the neighbours' rows; adds the number of this
 * slab's zones still failed after it to *acc_dev. */
int grmhd_fix_sweep(grmhd_ctx *ctx, int st, long long *acc_dev);

/* Close stage st's fixups: count nsweeps sweeps, mark GRMHD_EFIXUP (seen by
 * grmhd_sync) if a zone stays failed, clear the failure list. */
int grmhd_fix_end(grmhd_ctx *ctx, int st, int nsweeps);

/* The fixups (Eq. 33) of stage st of the nslab (1..16) theta slabs of one
 * grid (the decomposition of Sec. 3), all on one device and one stream,
 * given in theta order (ctxs[r]->j0 = the rows before it; together they hold
 * every row): the loop above from the fail counts through grmhd_fix_end --
 * kind-1 row exchanges between neighbouring slabs (across the periodic edge
 * of a periodic flat box too), Jacobi sweeps, the close of every slab -- run
 * by one kernel on ctxs[0]'s stream, bit for bit the host loop's result.
 * nsweeps_dev (one int of device memory, or null) receives the sweep count.
 * Errors are reported on ctxs[0] (GRMHD_EINVAL for slabs that are not such
 * a split, on another device or stream; GRMHD_ESTATE for a slab without a
 * state), and nothing is launched then. */
int grmhd_theta_ring_fix(grmhd_ctx *const *ctxs, int nslab, int st, int *nsweeps_dev);

/* Boundary fill of stage st's output (poles, X1, X3; the external X2 sides
 * are left to the exchange). */
int grmhd_stage_bc(grmhd_ctx *ctx, int st);

/* Bytes of one side's rows of an exchange, element type double
 * (GRMHD_FP64) or float (GRMHD_MIXED):
 *   kind 0: NG = 3 rows of all 8 primitives over the ghosted (X1, X3)
 *           section, layout [NG][8][n1 + 2 NG][n3 + 2 NG];
 *   kind 1: one row of the five primitives a fixup averages and the failure
 *           flag (0 or 1), over the active (X1, X3) section, layout
 *           [6][n1][n3]. */
int grmhd_x2_row_bytes(grmhd_ctx *ctx, int kind, unsigned long long *bytes);

/* Pack the outermost active rows of buffer `which` (0 = P, 1 = P-hat) on
 * `side` (0: j = 0 .. NG-1 for kind 0, j = 0 for kind 1; 1: j = n2-NG ..
 * n2-1, or j = n2-1) into the caller's device buffer. */
int grmhd_x2_pack(grmhd_ctx *ctx, int kind, int which, int side, void *buf_dev);

/* Write a neighbour's packed rows into the ghost rows on `side` (0: j = -NG
 * .. -1, or j = -1; 1: j = n2 .. n2+NG-1, or j = n2) of buffer `which`
 * (kind 1 writes the ghost rows' failure flags too). */
int grmhd_x2_unpack(grmhd_ctx *ctx, int kind, int which, int side, const void *buf_dev);

/* Barycentric radius of the disk (Sec. 4.2, Eq. 43):
 *   <r> = sum r rho sqrt(-g) dV / sum rho sqrt(-g) dV
 * over the active zones from the horizon zone (the first with centre radius
 * >= r_H, as for Eq. 38) outwards whose centre radius is <= r_bar_max;
 * sqrt(-g) dX1 dX2 dX3 of the code coordinates is the volume element of the
 * paper's integral.  out (host, 3 doubles) = (<r>, denominator, numerator);
 * <r> = 0 when the range holds no mass.  Deterministic (fixed reduction
 * order); synchronises the context stream.  Kerr grids only (GRMHD_EINVAL
 * otherwise). */
int grmhd_barycentric_radius(grmhd_ctx *ctx, double r_bar_max, double *out);

/* Library version string. */
const char *grmhd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GRMHD_H */
