/*
 * orc.h -- internal declarations of the CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This directory holds a plain, slow, FP64 CPU
 * implementation of the HARM-style conservative GR-MHD step described in
 * cuHARM (Begue et al., arXiv 2205.02484), Sections 2.1-2.4 and 4.1.  It is
 * the reference that the CUDA path is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product library never links, calls or includes anything from here, and
 * nothing here includes or calls the product library.
 *
 * Layout used throughout the oracle: every per-zone array is field-major,
 * arr[c][I][J][K] over the ghosted box (n+2*NG per direction), K fastest.
 * Metric tables are per (I, J) because the metric does not depend on phi
 * (Section 3).
 */
#ifndef ORC_H
#define ORC_H

#ifndef __cplusplus
#include <complex.h>
#endif
#include <stdint.h>

#define ORC_NG 3 /* ghost layers per side: PPM faces read zones i-3 .. i+2 */
#define ORC_NP 8 /* primitives: rho, u, ut1, ut2, ut3, B1, B2, B3 (Eq. 11) */
#define ORC_NU 9 /* conserved: the 8 of Section 2.1 plus entropy (Eq. 12) */

enum { KRHO = 0, KUU, KU1, KU2, KU3, KB1, KB2, KB3, KENT };
enum { ORC_KERR_MKS = 0, ORC_MINK_CART = 1 };
enum { ORC_BC_INFLOW = 0, ORC_BC_POLAR = 1, ORC_BC_PERIODIC = 2, ORC_BC_OUTFLOW = 3,
       ORC_BC_EXTERNAL = 4 /* X3 ghosts supplied by the caller (a phi slab of a decomposed grid) */ };
enum { ORC_LLF = 0, ORC_HLL = 1 };
enum { ORC_PLM = 0, ORC_PPM = 1 };

/* con2prim result flags: low 3 bits = method that produced the primitives,
 * bit 3 = failure (zone must be fixed by neighbour averaging, Eq. 33). */
enum { C2P_NR = 0, C2P_BRENT_W = 1, C2P_ENTROPY = 2, C2P_ENTROPY_BETA = 3 };
#define C2P_FAIL 8
#define C2P_FAIL_D 16   /* D <= 0 or non-finite input */
#define C2P_FAIL_ENT 32 /* entropy inversion impossible (S <= 0, no root) */

typedef struct {
    int n1, n2, n3;
    int metric;
    double a;
    double r_in, r_out, hslope, r_br, n_x, R0;
    double x1min, x1max, x2min, x2max, x3min, x3max;
    int bc1, bc2, bc3;
    int riemann;
    double gam, cfl, nr_tol, sigma_max, bu_max, gamma_max, beta_entropy;
    int nr_maxit, brent_maxit, fix_maxsweep;
    /* a theta slab: the active X2 rows [j0, j0 + n2) of a grid of n2_total
     * rows (n2_total = 0: the whole grid); its X2 ghost rows on a side
     * inside the grid, or on a periodic side, are supplied by the caller */
    int j0, n2_total;
    int recon; /* ORC_PLM (Eqs. 16-17) or ORC_PPM (the parabolic reconstruction Section 2.2 names) */
    /* polar cylindrification (Section 4.1): radius r_c and the X2 width of
     * the band next to each pole; cyl_r <= 0 switches it off */
    double cyl_r, cyl_dx2;
} orc_params;

typedef struct {
    double r_in, r_max, beta0, pert_amp, kappa;
    uint64_t seed;
} orc_torus_params;

typedef struct {
    double gcov[4][4], gcon[4][4], gdet, alpha;
} orc_geom;

typedef struct {
    double ucon[4], ucov[4], bcon[4], bcov[4], bsq, gamma;
} orc_state;

typedef struct {
    double t, dt, mdot, phib, PhiB, edot, ldot, divb_max, disk_mass, disk_eb, eta;
    long long nr_iters, n_nr, n_brent, n_entropy, n_entropy_beta, n_fail, n_floor, n_ceil,
        n_gcap, n_fixed, fix_sweeps, n_steps;
} orc_diag;

typedef struct orc_grid {
    orc_params p;
    int N1, N2, N3;   /* ghosted sizes */
    long nz;          /* N1*N2*N3 */
    double x1in, x2in, x3in, dx[3], xb;
    int i_h;          /* first active zone with r >= r_H */
    orc_geom *gc, *gf1, *gf2; /* centre, X1-face, X2-face metric, [N1*N2] */
    char *polar2;     /* X2-face lies on a pole (metric singular) */
    double *conn;     /* [N1*N2][4][4][4] connection at centres */
    double *rc;       /* r at centres [N1*N2] */
    double *P, *Ph, *U;
    double *F[3], *cw[3], *E[3];
    int *flag;
    double t, dt;
    double dtd[3];    /* per-direction CFL minima of the last flux sweep (Eq. 27) */
    double disk_mass, disk_eb;
    orc_diag cnt;     /* running counters (cumulative) */
} orc_grid;

/* geometry.c */
double orc_r_of_x1(const orc_grid *G, double X1);
/* theta(X2) of Eq. 36 alone (no cylindrification) */
double orc_th_of_x2(const orc_grid *G, double X2);
/* theta(X1, X2) with cylindrification; dth = (d theta/dX1, d theta/dX2) */
double orc_theta_at(const orc_grid *G, double X1, double X2, double dth[2]);
void orc_ks_gcov(double r, double th, double a, double g[4][4]);
#ifndef __cplusplus /* complex-step derivatives: C only (the op counter compiles physics as C++) */
void orc_code_gcov_c(const orc_grid *G, double complex X1, double complex X2,
                     double complex g[4][4]);
#endif
int orc_invert4(const double m[4][4], double inv[4][4], double *det);
int orc_geom_at(const orc_grid *G, double X1, double X2, orc_geom *out);
void orc_conn_at(const orc_grid *G, double X1, double X2, double conn[4][4][4]);
double orc_x1_of_r(const orc_grid *G, double r);

/* physics.c */
void orc_state_of(const double *q, const orc_geom *g, orc_state *s);
void orc_tmunu(const double *q, const orc_state *s, double gam, int mu, double T[4]);
void orc_prim_to_U(const double *q, const orc_geom *g, const orc_state *s, double gam,
                   double U[ORC_NU]);
void orc_prim_to_F(const double *q, const orc_geom *g, const orc_state *s, double gam, int d,
                   double F[ORC_NU]);
void orc_wave_speeds(const double *q, const orc_geom *g, const orc_state *s, double gam, int d,
                     double *c1, double *c2);
double orc_mc_slope(double qm, double q0, double qp);
void orc_source(const double *q, const orc_geom *g, const double conn[4][4][4],
                const orc_state *s, double gam, double S[4]);

/* con2prim.c */
int orc_con2prim(const double U[ORC_NU], const orc_geom *g, const double *guess,
                 const orc_params *p, double P[ORC_NP], int *iters, int methods);
int orc_con2prim_w(const double U[ORC_NU], const orc_geom *g, const double *guess,
                   const orc_params *p, double P[ORC_NP], int *iters, int methods, double wguess);
double orc_brent(double (*f)(double, void *), void *ctx, double a, double b, double fa,
                 double fb, double tol, int maxit, int *ok);

/* torus.c */
double orc_uniform(uint64_t seed, uint64_t idx);

/* mlp.c */
int orc_mlp_features(const double U[ORC_NU], const orc_geom *g, double feat[5]);

/* grid.c */
long orc_idx(const orc_grid *G, int i, int j, int k);
int orc_midx(const orc_grid *G, int i, int j);
void orc_bc_fill(orc_grid *G, double *P);
double orc_compute_fluxes(orc_grid *G, const double *P);
double orc_combine_dt(const double dtd[3]);
double orc_barycentric(orc_grid *G, double r_bar_max, double out[3]);
double orc_face_flux_at(orc_grid *G, int d, int i, int j, const double *q, double *Fout);
void orc_ppm_face(const double q[6], double out[2]);
void orc_flux_ct(orc_grid *G);
void orc_floors(const orc_grid *G, int i, int j, double *q, int *mod);
void orc_post_inversion_at(orc_grid *G, int i, int j, double *q, double *U, int *out);
int orc_n2_total(const orc_grid *G);
int orc_x2_external(const orc_grid *G, int side);

#endif
