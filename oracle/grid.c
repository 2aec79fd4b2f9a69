/*
 * grid.c -- oracle grid, boundary conditions, face fluxes, flux-CT, the RK2
 * step, floors/ceilings, fixups, CFL and horizon diagnostics.
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 *
 * Passages followed:
 *   finite-volume update and face fluxes ........ Section 2.2, Eqs. 13-14
 *   PLM-MC reconstruction ........................ Eqs. 16-17
 *   LLF / HLL .................................... Eqs. 18, 21
 *   wave speeds, c_max, c_min, c_w ............... Eqs. 19-20 and text after
 *   flux-CT EMFs and B-flux replacement .......... Eqs. 22-24
 *   RK2 predictor-corrector ...................... Eqs. 25-26
 *   CFL time step ................................ Eq. 27
 *   inversion, failure fixups .................... Section 2.3, Eq. 33
 *   floors, ceilings, Lorentz cap ................ Section 2.4, Eq. 34
 *   boundary conditions .......................... Section 4.1 (last paragraph)
 *   horizon fluxes ............................... Section 4.2, Eqs. 38-42
 *
 * Readings where the paper is silent (shared with the GPU path as a spec):
 *   - flux-CT edge indices printed J+3/2, K+3/2 are read J-1/2, K-1/2 (the
 *     two edges bounding the face).
 *   - sources are added with the prims of the same stage as the fluxes.
 *   - dt of step n+1 comes from the predictor sweep of step n.
 *   - X2 faces on the poles have sqrt(-g) = 0, so every flux through them is
 *     zero and their wave speed is 0 (the metric there is not evaluated).
 *   - failed-zone fixups are Jacobi sweeps: face neighbours if all four are
 *     good, else the four diagonals if all good, else the mean of all good
 *     ones among the eight; zones outside the active domain never count.
 *   - ceilings add the missing rho, u at rest in the normal (ZAMO) frame and
 *     re-invert with Newton; if that fails the prims are raised directly.
 *   - after floors, ceilings, the Lorentz cap or a fixup, U is recomputed from
 *     the final primitives.
 *   - radial boundary: primitives copied into the ghosts; where the ghost
 *     velocity points into the domain, ut^1 is reset so that u^1 = 0 at
 *     fixed ut^2, ut^3.  Polar boundary: mirror with ut^2, B^2 flipped, and
 *     ut^2 of the two zones next to each pole interpolated linearly to zero
 *     at the pole from the third zone.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "orc.h"

long orc_idx(const orc_grid *G, int i, int j, int k)
{
    return ((long)(i + ORC_NG) * G->N2 + (j + ORC_NG)) * G->N3 + (k + ORC_NG);
}

int orc_midx(const orc_grid *G, int i, int j) { return (i + ORC_NG) * G->N2 + (j + ORC_NG); }

#define AT(arr, c, z) ((arr)[(long)(c) * G->nz + (z)])

static double minf(double a, double b) { return a < b ? a : b; }
static double maxf(double a, double b) { return a > b ? a : b; }

/* ------------------------------------------------------------------ setup */

/* X2 rows of the whole grid a theta slab belongs to (n2 for a whole grid) */
int orc_n2_total(const orc_grid *G) { return G->p.n2_total > 0 ? G->p.n2_total : G->p.n2; }

/* 1 if the X2 ghost rows of a side (0 low, 1 high) come from the caller: a
 * theta slab's side inside the grid, or a periodic side of the whole grid
 * (the ghost rows then hold the far slab's edge rows) */
int orc_x2_external(const orc_grid *G, int side)
{
    const orc_params *p = &G->p;
    int n2t = orc_n2_total(G);
    if (n2t == p->n2) return 0;
    int edge = side == 0 ? p->j0 == 0 : p->j0 + p->n2 == n2t;
    if (!edge) return 1;
    return p->metric != ORC_KERR_MKS && p->bc2 == ORC_BC_PERIODIC;
}

orc_grid *orc_create(const orc_params *p)
{
    if (p->n1 < 1 || p->n2 < 1 || p->n3 < 1) return NULL;
    if (p->recon != ORC_PLM && p->recon != ORC_PPM) return NULL;
    if (p->n2_total != 0) { /* a theta slab: at least 4 rows, not also a phi slab */
        if (p->j0 < 0 || p->n2 < 4 || p->j0 + p->n2 > p->n2_total || p->bc3 == ORC_BC_EXTERNAL) return NULL;
    } else if (p->j0 != 0) {
        return NULL;
    }
    orc_grid *G = (orc_grid *)calloc(1, sizeof(orc_grid));
    G->p = *p;
    G->N1 = p->n1 + 2 * ORC_NG;
    G->N2 = p->n2 + 2 * ORC_NG;
    G->N3 = p->n3 + 2 * ORC_NG;
    G->nz = (long)G->N1 * G->N2 * G->N3;
    double x1out, x2out, x3out;
    if (p->metric == ORC_KERR_MKS) {
        G->xb = log(p->r_br - p->R0);
        G->x1in = log(p->r_in - p->R0);
        if (p->r_out <= p->r_br) {
            x1out = log(p->r_out - p->R0);
        } else {
            /* X + (X - x_b)^n_x = ln(r_out - R0) */
            double lo = G->xb, hi = log(p->r_out - p->R0);
            for (int it = 0; it < 200; it++) {
                double mid = 0.5 * (lo + hi);
                if (orc_r_of_x1(G, mid) < p->r_out) lo = mid; else hi = mid;
            }
            x1out = 0.5 * (lo + hi);
        }
        G->x2in = -1.0; x2out = 1.0;
        if (p->bc3 == ORC_BC_EXTERNAL) { /* a phi slab of the full circle, width x3max - x3min */
            G->x3in = p->x3min; x3out = p->x3max;
        } else {
            G->x3in = 0.0; x3out = 2.0 * M_PI;
        }
    } else {
        G->xb = 1e300;
        G->x1in = p->x1min; x1out = p->x1max;
        G->x2in = p->x2min; x2out = p->x2max;
        G->x3in = p->x3min; x3out = p->x3max;
    }
    G->dx[0] = (x1out - G->x1in) / p->n1;
    int n2t = p->n2_total > 0 ? p->n2_total : p->n2;
    G->dx[1] = (x2out - G->x2in) / n2t;
    G->dx[2] = (x3out - G->x3in) / p->n3;
    if (p->cyl_r > 0.0) {
        /* cylindrification on the Kerr grid only, bands that do not meet,
         * and a widening lambda(r) <= 5/2 down to the innermost ghost face
         * (lambda falls with r), which keeps the map monotone in X2 */
        double rmin = orc_r_of_x1(G, G->x1in - ORC_NG * G->dx[0]);
        double x = p->cyl_r / rmin;
        if (p->metric != ORC_KERR_MKS || !(p->cyl_dx2 > 0.0 && p->cyl_dx2 <= 1.0) || !isfinite(p->cyl_r) ||
            !(pow(1.0 + x * x * x * x, 0.25) <= 2.5)) {
            free(G);
            return NULL;
        }
    }

    long nm = (long)G->N1 * G->N2;
    G->gc = (orc_geom *)calloc(nm, sizeof(orc_geom));
    G->gf1 = (orc_geom *)calloc(nm, sizeof(orc_geom));
    G->gf2 = (orc_geom *)calloc(nm, sizeof(orc_geom));
    G->polar2 = (char *)calloc(nm, 1);
    G->conn = (double *)calloc(nm * 64, sizeof(double));
    G->rc = (double *)calloc(nm, sizeof(double));
    for (int i = -ORC_NG; i < p->n1 + ORC_NG; i++)
        for (int j = -ORC_NG; j < p->n2 + ORC_NG; j++) {
            int m = orc_midx(G, i, j);
            double X1c = G->x1in + (i + 0.5) * G->dx[0], X1f = G->x1in + i * G->dx[0];
            int jg = p->j0 + j; /* the row in the whole grid */
            double X2c = G->x2in + (jg + 0.5) * G->dx[1], X2f = G->x2in + jg * G->dx[1];
            orc_geom_at(G, X1c, X2c, &G->gc[m]);
            orc_geom_at(G, X1f, X2c, &G->gf1[m]);
            if (p->metric == ORC_KERR_MKS && (jg == 0 || jg == n2t)) {
                G->polar2[m] = 1;
            } else {
                orc_geom_at(G, X1c, X2f, &G->gf2[m]);
            }
            orc_conn_at(G, X1c, X2c, (double(*)[4][4]) & G->conn[(long)m * 64]);
            G->rc[m] = (p->metric == ORC_KERR_MKS) ? orc_r_of_x1(G, X1c) : 1.0;
        }
    G->i_h = 0;
    if (p->metric == ORC_KERR_MKS) {
        double rh = 1.0 + sqrt(1.0 - p->a * p->a);
        G->i_h = p->n1;
        for (int i = 0; i < p->n1; i++)
            if (orc_r_of_x1(G, G->x1in + (i + 0.5) * G->dx[0]) >= rh) { G->i_h = i; break; }
    }
    G->P = (double *)calloc(ORC_NP * G->nz, sizeof(double));
    G->Ph = (double *)calloc(ORC_NP * G->nz, sizeof(double));
    G->U = (double *)calloc(ORC_NU * G->nz, sizeof(double));
    for (int d = 0; d < 3; d++) {
        G->F[d] = (double *)calloc(ORC_NU * G->nz, sizeof(double));
        G->cw[d] = (double *)calloc(G->nz, sizeof(double));
        G->E[d] = (double *)calloc(G->nz, sizeof(double));
    }
    G->flag = (int *)calloc(G->nz, sizeof(int));
    return G;
}

void orc_destroy(orc_grid *G)
{
    if (!G) return;
    free(G->gc); free(G->gf1); free(G->gf2); free(G->polar2); free(G->conn); free(G->rc);
    free(G->P); free(G->Ph); free(G->U);
    for (int d = 0; d < 3; d++) { free(G->F[d]); free(G->cw[d]); free(G->E[d]); }
    free(G->flag);
    free(G);
}

/* ------------------------------------------------------- boundary fill */

static void gather(const orc_grid *G, const double *P, long z, double *q)
{
    for (int c = 0; c < ORC_NP; c++) q[c] = AT(P, c, z);
}

static void scatter(const orc_grid *G, double *P, long z, const double *q)
{
    for (int c = 0; c < ORC_NP; c++) AT(P, c, z) = q[c];
}

/* set ut^1 so that u^1 = 0, keeping ut^2, ut^3 (normal-frame components):
 * ut^1 = Gamma c with c = alpha g^{t1}, Gamma from Gamma^2 = 1 + g_ij ut^i ut^j */
static void zero_radial_velocity(const orc_geom *g, double *q)
{
    double c = g->alpha * g->gcon[0][1];
    double a2 = 1.0 - g->gcov[1][1] * c * c;
    if (!(a2 > 0.0)) return;
    double b = -2.0 * c * (g->gcov[1][2] * q[KU2] + g->gcov[1][3] * q[KU3]);
    double rest = g->gcov[2][2] * q[KU2] * q[KU2] + 2.0 * g->gcov[2][3] * q[KU2] * q[KU3] +
                  g->gcov[3][3] * q[KU3] * q[KU3];
    double cc = -(1.0 + rest);
    double disc = b * b - 4.0 * a2 * cc;
    double gam = (-b + sqrt(disc)) / (2.0 * a2);
    q[KU1] = gam * c;
}

static void inflow_check(const orc_grid *G, int i, int j, double *q, int inner)
{
    const orc_geom *g = &G->gc[orc_midx(G, i, j)];
    orc_state s;
    orc_state_of(q, g, &s);
    if ((inner && s.ucon[1] > 0.0) || (!inner && s.ucon[1] < 0.0)) zero_radial_velocity(g, q);
}

static int wrap(int k, int n) { return ((k % n) + n) % n; }

void orc_bc_fill(orc_grid *G, double *P)
{
    const orc_params *p = &G->p;
    int n1 = p->n1, n2 = p->n2, n3 = p->n3;
    double q[ORC_NP];
    int kerr = (p->metric == ORC_KERR_MKS);
    int bc1 = kerr ? ORC_BC_INFLOW : p->bc1;
    int bc2 = kerr ? ORC_BC_POLAR : p->bc2;
    int bc3 = (kerr && p->bc3 != ORC_BC_EXTERNAL) ? ORC_BC_PERIODIC : p->bc3;

    int n2t = orc_n2_total(G);
    int ext[2] = {orc_x2_external(G, 0), orc_x2_external(G, 1)};
    /* polar ut^2 interpolation in the two zones next to each pole (of the
     * whole grid: a theta slab holds a pole's three rows or none of them) */
    if (bc2 == ORC_BC_POLAR && n2t >= 6) {
        int lo = p->j0 == 0, hi = p->j0 + n2 == n2t;
        for (int i = 0; i < n1; i++)
            for (int k = 0; k < n3; k++) {
                if (lo) {
                    double u2a = AT(P, KU2, orc_idx(G, i, 2, k));
                    AT(P, KU2, orc_idx(G, i, 0, k)) = u2a * (0.5 / 2.5);
                    AT(P, KU2, orc_idx(G, i, 1, k)) = u2a * (1.5 / 2.5);
                }
                if (hi) {
                    double u2b = AT(P, KU2, orc_idx(G, i, n2 - 3, k));
                    AT(P, KU2, orc_idx(G, i, n2 - 1, k)) = u2b * (0.5 / 2.5);
                    AT(P, KU2, orc_idx(G, i, n2 - 2, k)) = u2b * (1.5 / 2.5);
                }
            }
    }
    /* X1 ghosts over active j, k */
    for (int j = 0; j < n2; j++)
        for (int k = 0; k < n3; k++)
            for (int gh = 1; gh <= ORC_NG; gh++) {
                int il = -gh, ir = n1 - 1 + gh;
                if (bc1 == ORC_BC_PERIODIC) {
                    gather(G, P, orc_idx(G, wrap(il, n1), j, k), q);
                    scatter(G, P, orc_idx(G, il, j, k), q);
                    gather(G, P, orc_idx(G, wrap(ir, n1), j, k), q);
                    scatter(G, P, orc_idx(G, ir, j, k), q);
                } else {
                    gather(G, P, orc_idx(G, 0, j, k), q);
                    if (bc1 == ORC_BC_INFLOW) inflow_check(G, il, j, q, 1);
                    scatter(G, P, orc_idx(G, il, j, k), q);
                    gather(G, P, orc_idx(G, n1 - 1, j, k), q);
                    if (bc1 == ORC_BC_INFLOW) inflow_check(G, ir, j, q, 0);
                    scatter(G, P, orc_idx(G, ir, j, k), q);
                }
            }
    /* X2 ghosts over all i, active k (a theta slab's inner sides come from
     * its neighbours) */
    for (int i = -ORC_NG; i < n1 + ORC_NG; i++)
        for (int k = 0; k < n3; k++)
            for (int gh = 1; gh <= ORC_NG; gh++) {
                int jl = -gh, jr = n2 - 1 + gh;
                if (bc2 == ORC_BC_POLAR) {
                    if (!ext[0]) {
                        gather(G, P, orc_idx(G, i, gh - 1, k), q);
                        q[KU2] = -q[KU2]; q[KB2] = -q[KB2];
                        scatter(G, P, orc_idx(G, i, jl, k), q);
                    }
                    if (!ext[1]) {
                        gather(G, P, orc_idx(G, i, n2 - gh, k), q);
                        q[KU2] = -q[KU2]; q[KB2] = -q[KB2];
                        scatter(G, P, orc_idx(G, i, jr, k), q);
                    }
                } else if (bc2 == ORC_BC_PERIODIC) {
                    if (!ext[0]) {
                        gather(G, P, orc_idx(G, i, wrap(jl, n2), k), q);
                        scatter(G, P, orc_idx(G, i, jl, k), q);
                    }
                    if (!ext[1]) {
                        gather(G, P, orc_idx(G, i, wrap(jr, n2), k), q);
                        scatter(G, P, orc_idx(G, i, jr, k), q);
                    }
                } else {
                    if (!ext[0]) {
                        gather(G, P, orc_idx(G, i, 0, k), q);
                        scatter(G, P, orc_idx(G, i, jl, k), q);
                    }
                    if (!ext[1]) {
                        gather(G, P, orc_idx(G, i, n2 - 1, k), q);
                        scatter(G, P, orc_idx(G, i, jr, k), q);
                    }
                }
            }
    /* X3 ghosts over all i, j (a slab's come from its neighbours) */
    if (bc3 == ORC_BC_EXTERNAL) return;
    for (int i = -ORC_NG; i < n1 + ORC_NG; i++)
        for (int j = -ORC_NG; j < n2 + ORC_NG; j++)
            for (int gh = 1; gh <= ORC_NG; gh++) {
                int kl = -gh, kr = n3 - 1 + gh;
                if (bc3 == ORC_BC_PERIODIC) {
                    gather(G, P, orc_idx(G, i, j, wrap(kl, n3)), q);
                    scatter(G, P, orc_idx(G, i, j, kl), q);
                    gather(G, P, orc_idx(G, i, j, wrap(kr, n3)), q);
                    scatter(G, P, orc_idx(G, i, j, kr), q);
                } else {
                    gather(G, P, orc_idx(G, i, j, 0), q);
                    scatter(G, P, orc_idx(G, i, j, kl), q);
                    gather(G, P, orc_idx(G, i, j, n3 - 1), q);
                    scatter(G, P, orc_idx(G, i, j, kr), q);
                }
            }
}

/* ----------------------------------------------------------- face fluxes */

static const orc_geom *face_geom(const orc_grid *G, int d, int i, int j)
{
    int m = orc_midx(G, i, j);
    return d == 0 ? &G->gf1[m] : (d == 1 ? &G->gf2[m] : &G->gc[m]);
}

/* The Riemann flux (Eqs. 18-21) of one face of direction d at metric record
 * (i, j) from its left and right states ql, qr: LLF or HLL.  Polar X2 faces
 * carry no flux. */
static void face_flux_lr(orc_grid *G, int d, int i, int j, const double *ql, const double *qr, double *Fout,
                         double *cwout)
{
    const orc_params *p = &G->p;
    if (d == 1 && G->polar2[orc_midx(G, i, j)]) {
        for (int c = 0; c < ORC_NU; c++) Fout[c] = 0.0;
        *cwout = 0.0;
        return;
    }
    const orc_geom *g = face_geom(G, d, i, j);
    orc_state sl, sr;
    orc_state_of(ql, g, &sl);
    orc_state_of(qr, g, &sr);
    double Ul[ORC_NU], Ur[ORC_NU], Fl[ORC_NU], Fr[ORC_NU];
    orc_prim_to_U(ql, g, &sl, p->gam, Ul);
    orc_prim_to_U(qr, g, &sr, p->gam, Ur);
    orc_prim_to_F(ql, g, &sl, p->gam, d + 1, Fl);
    orc_prim_to_F(qr, g, &sr, p->gam, d + 1, Fr);
    double c1l, c2l, c1r, c2r;
    orc_wave_speeds(ql, g, &sl, p->gam, d + 1, &c1l, &c2l);
    orc_wave_speeds(qr, g, &sr, p->gam, d + 1, &c1r, &c2r);
    double cmax = fabs(maxf(0.0, maxf(c1r, c1l)));
    double cmin = fabs(maxf(0.0, maxf(-c2r, -c2l)));
    double cw = maxf(cmax, cmin);
    if (p->riemann == ORC_HLL && cmax + cmin > 0.0) {
        for (int c = 0; c < ORC_NU; c++)
            Fout[c] = (cmax * Fl[c] + cmin * Fr[c] - cmax * cmin * (Ur[c] - Ul[c])) / (cmax + cmin);
    } else if (p->riemann == ORC_HLL) {
        for (int c = 0; c < ORC_NU; c++) Fout[c] = 0.5 * (Fl[c] + Fr[c]);
    } else {
        for (int c = 0; c < ORC_NU; c++) Fout[c] = 0.5 * (Fl[c] + Fr[c] - cw * (Ur[c] - Ul[c]));
    }
    *cwout = cw;
}

/* PLM-MC face states (Eqs. 16-17) from the four zone states along d around
 * the face (zones idx-2 .. idx+1), then the Riemann flux. */
static void face_flux_states(orc_grid *G, int d, int i, int j, const double *qm2, const double *qm1,
                             const double *q0, const double *qp1, double *Fout, double *cwout)
{
    double ql[ORC_NP], qr[ORC_NP];
    for (int c = 0; c < ORC_NP; c++) {
        ql[c] = qm1[c] + 0.5 * orc_mc_slope(qm2[c], qm1[c], q0[c]);
        qr[c] = q0[c] - 0.5 * orc_mc_slope(qm1[c], q0[c], qp1[c]);
    }
    face_flux_lr(G, d, i, j, ql, qr, Fout, cwout);
}

/* PPM face states from the six zone states along d around the face (zones
 * idx-3 .. idx+2, q6[m * ORC_NP + c]), then the Riemann flux. */
static void face_flux_states_ppm(orc_grid *G, int d, int i, int j, const double *q6, double *Fout,
                                 double *cwout)
{
    double ql[ORC_NP], qr[ORC_NP];
    for (int c = 0; c < ORC_NP; c++) {
        double z[6], lr[2];
        for (int m = 0; m < 6; m++) z[m] = q6[m * ORC_NP + c];
        orc_ppm_face(z, lr);
        ql[c] = lr[0];
        qr[c] = lr[1];
    }
    face_flux_lr(G, d, i, j, ql, qr, Fout, cwout);
}

/* One face of the grid: index (i,j,k) along direction d denotes the face
 * between zones (.., idx-1, ..) and (.., idx, ..). */
static void face_flux(orc_grid *G, const double *P, int d, int i, int j, int k, double *Fout,
                      double *cwout)
{
    int di = d == 0, dj = d == 1, dk = d == 2;
    if (G->p.recon == ORC_PPM) {
        double q6[6 * ORC_NP];
        for (int m = 0; m < 6; m++)
            gather(G, P, orc_idx(G, i + (m - 3) * di, j + (m - 3) * dj, k + (m - 3) * dk), q6 + m * ORC_NP);
        face_flux_states_ppm(G, d, i, j, q6, Fout, cwout);
        return;
    }
    double qm2[ORC_NP], qm1[ORC_NP], q0[ORC_NP], qp1[ORC_NP];
    gather(G, P, orc_idx(G, i - 2 * di, j - 2 * dj, k - 2 * dk), qm2);
    gather(G, P, orc_idx(G, i - di, j - dj, k - dk), qm1);
    gather(G, P, orc_idx(G, i, j, k), q0);
    gather(G, P, orc_idx(G, i + di, j + dj, k + dk), qp1);
    face_flux_states(G, d, i, j, qm2, qm1, q0, qp1, Fout, cwout);
}

/* The same Riemann flux for caller-given zone states along d: q[4][8] (zones
 * idx-2 .. idx+1) with PLM, q[6][8] (zones idx-3 .. idx+2) with PPM, at the
 * face metric record (i, j), i in [0, n1], j in [0, n2] for its direction;
 * returns c_w.  Lets a test check single faces of a grid too large for the
 * oracle to sweep. */
double orc_face_flux_at(orc_grid *G, int d, int i, int j, const double *q, double *Fout)
{
    double cw = 0.0;
    if (G->p.recon == ORC_PPM) face_flux_states_ppm(G, d, i, j, q, Fout, &cw); /* q: six zones */
    else face_flux_states(G, d, i, j, q, q + ORC_NP, q + 2 * ORC_NP, q + 3 * ORC_NP, Fout, &cw);
    return cw;
}

/* Fills F[d] over the boxes flux-CT needs and returns the CFL time step of
 * Eq. 27 from the active faces. */
double orc_compute_fluxes(orc_grid *G, const double *P)
{
    const orc_params *p = &G->p;
    int n[3] = {p->n1, p->n2, p->n3};
    double dtd[3] = {INFINITY, INFINITY, INFINITY};
    double Fl[ORC_NU], cw;
    for (int d = 0; d < 3; d++) {
        int lo[3], hi[3];
        for (int e = 0; e < 3; e++) {
            lo[e] = (e == d) ? 0 : -1;
            hi[e] = n[e]; /* inclusive */
        }
        for (int i = lo[0]; i <= hi[0]; i++)
            for (int j = lo[1]; j <= hi[1]; j++)
                for (int k = lo[2]; k <= hi[2]; k++) {
                    long z = orc_idx(G, i, j, k);
                    face_flux(G, P, d, i, j, k, Fl, &cw);
                    for (int c = 0; c < ORC_NU; c++) AT(G->F[d], c, z) = Fl[c];
                    G->cw[d][z] = cw;
                    int act = 1;
                    int ix[3] = {i, j, k};
                    for (int e = 0; e < 3; e++) {
                        if (e == d) act &= (ix[e] >= 0 && ix[e] <= n[e]);
                        else act &= (ix[e] >= 0 && ix[e] < n[e]);
                    }
                    if (act && cw > 0.0) dtd[d] = minf(dtd[d], p->cfl * G->dx[d] / cw);
                }
    }
    for (int d = 0; d < 3; d++) G->dtd[d] = dtd[d];
    return orc_combine_dt(dtd);
}

/* Eq. 27: 1/dt = sum over directions of 1/dt^l, each dt^l the minimum over
 * the faces of that direction */
double orc_combine_dt(const double dtd[3])
{
    double inv = 0.0;
    for (int d = 0; d < 3; d++)
        if (isfinite(dtd[d])) inv += 1.0 / dtd[d];
    return inv > 0.0 ? 1.0 / inv : INFINITY;
}

/* the per-direction minima of the grid's last flux sweep */
void orc_last_dtd(const orc_grid *G, double out[3])
{
    for (int d = 0; d < 3; d++) out[d] = G->dtd[d];
}

/* Flux-CT of Eqs. 22-23: edge EMFs from the Riemann B-fluxes, then the
 * B-fluxes replaced by edge averages. */
void orc_flux_ct(orc_grid *G)
{
    const orc_params *p = &G->p;
    int n1 = p->n1, n2 = p->n2, n3 = p->n3;
    double *F1 = G->F[0], *F2 = G->F[1], *F3 = G->F[2];
    double *E1 = G->E[0], *E2 = G->E[1], *E3 = G->E[2];
#define I3(i, j, k) orc_idx(G, i, j, k)
    for (int i = 0; i <= n1; i++)
        for (int j = 0; j <= n2; j++)
            for (int k = 0; k < n3; k++)
                E3[I3(i, j, k)] = 0.25 * (AT(F1, KB2, I3(i, j, k)) + AT(F1, KB2, I3(i, j - 1, k)) -
                                          AT(F2, KB1, I3(i, j, k)) - AT(F2, KB1, I3(i - 1, j, k)));
    for (int i = 0; i < n1; i++)
        for (int j = 0; j <= n2; j++)
            for (int k = 0; k <= n3; k++)
                E1[I3(i, j, k)] = 0.25 * (AT(F2, KB3, I3(i, j, k)) + AT(F2, KB3, I3(i, j, k - 1)) -
                                          AT(F3, KB2, I3(i, j, k)) - AT(F3, KB2, I3(i, j - 1, k)));
    for (int i = 0; i <= n1; i++)
        for (int j = 0; j < n2; j++)
            for (int k = 0; k <= n3; k++)
                E2[I3(i, j, k)] = 0.25 * (AT(F3, KB1, I3(i, j, k)) + AT(F3, KB1, I3(i - 1, j, k)) -
                                          AT(F1, KB3, I3(i, j, k)) - AT(F1, KB3, I3(i, j, k - 1)));
    for (int i = 0; i <= n1; i++)
        for (int j = 0; j < n2; j++)
            for (int k = 0; k < n3; k++) {
                long z = I3(i, j, k);
                AT(F1, KB1, z) = 0.0;
                AT(F1, KB2, z) = 0.5 * (E3[I3(i, j + 1, k)] + E3[z]);
                AT(F1, KB3, z) = -0.5 * (E2[I3(i, j, k + 1)] + E2[z]);
            }
    for (int i = 0; i < n1; i++)
        for (int j = 0; j <= n2; j++)
            for (int k = 0; k < n3; k++) {
                long z = I3(i, j, k);
                AT(F2, KB2, z) = 0.0;
                AT(F2, KB1, z) = -0.5 * (E3[I3(i + 1, j, k)] + E3[z]);
                AT(F2, KB3, z) = 0.5 * (E1[I3(i, j, k + 1)] + E1[z]);
            }
    for (int i = 0; i < n1; i++)
        for (int j = 0; j < n2; j++)
            for (int k = 0; k <= n3; k++) {
                long z = I3(i, j, k);
                AT(F3, KB3, z) = 0.0;
                AT(F3, KB1, z) = 0.5 * (E2[I3(i + 1, j, k)] + E2[z]);
                AT(F3, KB2, z) = -0.5 * (E1[I3(i, j + 1, k)] + E1[z]);
            }
#undef I3
}

/* ------------------------------------------------- floors and ceilings */

/* Density and internal-energy floors of Eq. 34 (r in units of M). */
void orc_floors(const orc_grid *G, int i, int j, double *q, int *mod)
{
    double rfl = 1e-20, ufl = 1e-20;
    if (G->p.metric == ORC_KERR_MKS) {
        double r = G->rc[orc_midx(G, i, j)];
        rfl = maxf(rfl, 1e-5 * pow(r, -0.5));
        ufl = maxf(ufl, (1e-5 / 3.0) * pow(r, -2.5));
    }
    if (q[KRHO] < rfl) { q[KRHO] = rfl; *mod = 1; }
    if (q[KUU] < ufl) { q[KUU] = ufl; *mod = 1; }
}

static void gamma_cap(const orc_grid *G, const orc_geom *g, double *q, int *mod)
{
    double usq = 0.0;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) usq += g->gcov[a + 1][b + 1] * q[KU1 + a] * q[KU1 + b];
    double gmax = G->p.gamma_max;
    if (1.0 + usq > gmax * gmax) {
        double f = sqrt((gmax * gmax - 1.0) / usq);
        q[KU1] *= f; q[KU2] *= f; q[KU3] *= f;
        *mod = 1;
    }
}

/* Floors, magnetisation ceilings and the Lorentz cap for a zone whose
 * inversion succeeded.  U is the zone's conserved state after the update. */
static void post_inversion(orc_grid *G, int i, int j, double *q, double *U, int *mod)
{
    const orc_params *p = &G->p;
    const orc_geom *g = &G->gc[orc_midx(G, i, j)];
    orc_floors(G, i, j, q, mod);
    orc_state s;
    orc_state_of(q, g, &s);
    double drho = maxf(0.0, s.bsq / p->sigma_max - q[KRHO]);
    double du = maxf(0.0, s.bsq / p->bu_max - q[KUU]);
    if (drho > 0.0 || du > 0.0) {
        G->cnt.n_ceil++;
        double dq[ORC_NP] = {drho, du, 0, 0, 0, 0, 0, 0}, dU[ORC_NU];
        orc_state ds;
        orc_state_of(dq, g, &ds);
        orc_prim_to_U(dq, g, &ds, p->gam, dU);
        double Un[ORC_NU], guess[ORC_NP], qn[ORC_NP];
        for (int c = 0; c < ORC_NU; c++) Un[c] = U[c];
        for (int c = 0; c < 5; c++) Un[c] += dU[c];
        for (int c = 0; c < ORC_NP; c++) guess[c] = q[c];
        guess[KRHO] += drho;
        guess[KUU] += du;
        int it;
        int fl = orc_con2prim(Un, g, guess, p, qn, &it, 1);
        if (fl == C2P_NR) {
            for (int c = 0; c < ORC_NP; c++) q[c] = qn[c];
        } else {
            q[KRHO] += drho;
            q[KUU] += du;
        }
        *mod = 1;
    }
    int capped = 0;
    gamma_cap(G, g, q, &capped);
    if (capped) {
        G->cnt.n_gcap++;
        *mod = 1;
    }
}

/* direct version for fixed-up zones (no second inversion) */
static void post_fixup(orc_grid *G, int i, int j, double *q)
{
    const orc_params *p = &G->p;
    const orc_geom *g = &G->gc[orc_midx(G, i, j)];
    int mod = 0;
    orc_floors(G, i, j, q, &mod);
    orc_state s;
    orc_state_of(q, g, &s);
    q[KRHO] = maxf(q[KRHO], s.bsq / p->sigma_max);
    q[KUU] = maxf(q[KUU], s.bsq / p->bu_max);
    gamma_cap(G, g, q, &mod);
}

/* ------------------------------------------------------------- fixups */

static long count_failed(const orc_grid *G)
{
    const orc_params *p = &G->p;
    long nfail = 0;
    for (int i = 0; i < p->n1; i++)
        for (int j = 0; j < p->n2; j++)
            for (int k = 0; k < p->n3; k++) nfail += (G->flag[orc_idx(G, i, j, k)] != 0);
    return nfail;
}

/* a fixup neighbour (ii, jj) of Eq. 33 must be an active zone of the whole
 * grid; a theta slab reads the rows jj = -1 and n2 next to its inner sides
 * from its ghost rows, which the caller fills with the neighbour slab's
 * current edge rows (primitives and flags) before each sweep */
static int fix_inside(const orc_grid *G, int ii, int jj)
{
    int jg = G->p.j0 + jj;
    return ii >= 0 && ii < G->p.n1 && jg >= 0 && jg < orc_n2_total(G);
}

/* One Jacobi sweep of the fixups (Eq. 33) over P: every failed zone whose
 * four face neighbours are good takes their average, else whose four
 * corner neighbours are good takes theirs, else the average of all its good
 * neighbours; the averages are all formed from the state at the start of the
 * sweep, then written.  Returns the number of zones still failed. */
static long fix_sweep(orc_grid *G, double *P, int corr)
{
    const orc_params *p = &G->p;
    int n1 = p->n1, n2 = p->n2, n3 = p->n3;
    static const int fo[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
    static const int dg[4][2] = {{1, 1}, {1, -1}, {-1, 1}, {-1, -1}};
    int *newflag = (int *)malloc(sizeof(int) * G->nz);
    double *newq = (double *)malloc(sizeof(double) * 5 * G->nz);
    memcpy(newflag, G->flag, sizeof(int) * G->nz);
    for (int i = 0; i < n1; i++)
        for (int j = 0; j < n2; j++)
            for (int k = 0; k < n3; k++) {
                long z = orc_idx(G, i, j, k);
                if (!G->flag[z]) continue;
                const int(*sets[2])[2] = {fo, dg};
                int done = 0;
                for (int s = 0; s < 2 && !done; s++) {
                    int allgood = 1;
                    for (int m = 0; m < 4; m++) {
                        int ii = i + sets[s][m][0], jj = j + sets[s][m][1];
                        if (!fix_inside(G, ii, jj) || G->flag[orc_idx(G, ii, jj, k)]) allgood = 0;
                    }
                    if (allgood) {
                        for (int c = 0; c < 5; c++) {
                            double acc = 0.0;
                            for (int m = 0; m < 4; m++)
                                acc += AT(P, c, orc_idx(G, i + sets[s][m][0], j + sets[s][m][1], k));
                            newq[(long)c * G->nz + z] = 0.25 * acc;
                        }
                        done = 1;
                    }
                }
                if (!done) {
                    int cnt = 0;
                    double acc[5] = {0, 0, 0, 0, 0};
                    for (int s = 0; s < 2; s++)
                        for (int m = 0; m < 4; m++) {
                            int ii = i + (s ? dg : fo)[m][0], jj = j + (s ? dg : fo)[m][1];
                            if (!fix_inside(G, ii, jj)) continue;
                            long zz = orc_idx(G, ii, jj, k);
                            if (G->flag[zz]) continue;
                            for (int c = 0; c < 5; c++) acc[c] += AT(P, c, zz);
                            cnt++;
                        }
                    if (cnt > 0) {
                        for (int c = 0; c < 5; c++) newq[(long)c * G->nz + z] = acc[c] / cnt;
                        done = 1;
                    }
                }
                if (done) newflag[z] = -1; /* fixed this sweep */
            }
    long left = 0;
    for (int i = 0; i < n1; i++)
        for (int j = 0; j < n2; j++)
            for (int k = 0; k < n3; k++) {
                long z = orc_idx(G, i, j, k);
                if (newflag[z] == -1) {
                    double q[ORC_NP];
                    gather(G, P, z, q);
                    for (int c = 0; c < 5; c++) q[c] = newq[(long)c * G->nz + z];
                    post_fixup(G, i, j, q);
                    scatter(G, P, z, q);
                    if (corr) {
                        const orc_geom *g = &G->gc[orc_midx(G, i, j)];
                        orc_state s;
                        orc_state_of(q, g, &s);
                        double Uz[ORC_NU];
                        orc_prim_to_U(q, g, &s, p->gam, Uz);
                        for (int c = 0; c < ORC_NU; c++) AT(G->U, c, z) = Uz[c];
                    }
                    G->flag[z] = 0;
                    G->cnt.n_fixed++;
                } else if (G->flag[z]) {
                    left++;
                }
            }
    free(newflag);
    free(newq);
    return left;
}

/* the fixups of a stage: sweeps until no zone is left failed, at most
 * fix_maxsweep of them; -1 if some zone stays failed */
static int fixups(orc_grid *G, double *P, int corr)
{
    long nfail = count_failed(G);
    int sweep = 0;
    for (; sweep < G->p.fix_maxsweep && nfail > 0; sweep++) nfail = fix_sweep(G, P, corr);
    G->cnt.fix_sweeps += sweep;
    return nfail > 0 ? -1 : 0;
}

/* con2prim of one zone followed by floors, ceilings and the Lorentz cap;
 * sets the zone's failure flag and recomputes Un where P was modified. */
static void invert_zone(orc_grid *G, int i, int j, long z, double *Un, const double *guess,
                        double *qn)
{
    const orc_params *p = &G->p;
    const orc_geom *g = &G->gc[orc_midx(G, i, j)];
    int it;
    int fl = orc_con2prim(Un, g, guess, p, qn, &it, 15);
    G->cnt.nr_iters += it;
    int meth = fl & 7;
    if (fl & C2P_FAIL) {
        G->cnt.n_fail++;
        G->flag[z] = 1;
        return;
    }
    G->flag[z] = 0;
    if (meth == C2P_NR) G->cnt.n_nr++;
    else if (meth == C2P_BRENT_W) G->cnt.n_brent++;
    else if (meth == C2P_ENTROPY) G->cnt.n_entropy++;
    else G->cnt.n_entropy_beta++;
    int mod = 0;
    post_inversion(G, i, j, qn, Un, &mod);
    if (mod) {
        G->cnt.n_floor++;
        orc_state sn;
        orc_state_of(qn, g, &sn);
        orc_prim_to_U(qn, g, &sn, p->gam, Un);
    }
}

/* -------------------------------------------------------------- stages */

/* fluxes, flux-CT, and the update and inversion of every zone (a stage up
 * to its fixups); returns the CFL step of the fluxes */
static double stage_update(orc_grid *G, const double *Pin, double *Pout, double dts, int corr)
{
    const orc_params *p = &G->p;
    int n1 = p->n1, n2 = p->n2, n3 = p->n3;
    double dtn = orc_compute_fluxes(G, Pin);
    orc_flux_ct(G);
    for (int i = 0; i < n1; i++)
        for (int j = 0; j < n2; j++) {
            int m = orc_midx(G, i, j);
            const orc_geom *g = &G->gc[m];
            const double(*conn)[4][4] = (const double(*)[4][4]) & G->conn[(long)m * 64];
            for (int k = 0; k < n3; k++) {
                long z = orc_idx(G, i, j, k);
                double q[ORC_NP], Un[ORC_NU], src[4];
                gather(G, Pin, z, q);
                orc_state s;
                orc_state_of(q, g, &s);
                orc_source(q, g, conn, &s, p->gam, src);
                long zi = orc_idx(G, i + 1, j, k), zj = orc_idx(G, i, j + 1, k),
                     zk = orc_idx(G, i, j, k + 1);
                for (int c = 0; c < ORC_NU; c++) {
                    double div = (AT(G->F[0], c, zi) - AT(G->F[0], c, z)) / G->dx[0] +
                                 (AT(G->F[1], c, zj) - AT(G->F[1], c, z)) / G->dx[1] +
                                 (AT(G->F[2], c, zk) - AT(G->F[2], c, z)) / G->dx[2];
                    double rhs = -div;
                    if (c >= 1 && c <= 4) rhs += src[c - 1];
                    Un[c] = AT(G->U, c, z) + dts * rhs;
                }
                double qn[ORC_NP];
                invert_zone(G, i, j, z, Un, q, qn);
                scatter(G, Pout, z, qn);
                if (corr)
                    for (int c = 0; c < ORC_NU; c++) AT(G->U, c, z) = Un[c];
            }
        }
    return dtn;
}

static double stage(orc_grid *G, const double *Pin, double *Pout, double dts, int corr,
                    int *status)
{
    double dtn = stage_update(G, Pin, Pout, dts, corr);
    if (fixups(G, Pout, corr) != 0) *status = -1;
    orc_bc_fill(G, Pout);
    return dtn;
}

/* One RK2 step (Eqs. 25-26).  Returns 0, or -1 if some zone could not be fixed. */
int orc_step(orc_grid *G)
{
    int status = 0;
    double dt = G->dt;
    double dtn = stage(G, G->P, G->Ph, 0.5 * dt, 0, &status);
    stage(G, G->Ph, G->P, dt, 1, &status);
    G->t += dt;
    G->dt = dtn;
    G->cnt.n_steps++;
    return status;
}

/* The two stages of orc_step, for a grid that is one slab of a decomposed
 * one: the caller exchanges the X3 ghost planes after each stage and sets the
 * next step's dt from the per-direction minima over the slabs of the
 * predictor's sweep (orc_last_dtd, combined by orc_combine_dt).  orc_stage0
 * returns this slab's own combination; orc_stage1 advances t.  Both return
 * the fixup status through *status (0, or -1 if some zone was not fixed). */
double orc_stage0(orc_grid *G, int *status)
{
    return stage(G, G->P, G->Ph, 0.5 * G->dt, 0, status);
}

void orc_stage1(orc_grid *G, int *status)
{
    stage(G, G->Ph, G->P, G->dt, 1, status);
    G->t += G->dt;
    G->cnt.n_steps++;
}

/* The parts of a stage (st 0: predictor into P-hat, st 1: corrector into
 * P) for a grid that is one theta slab of a decomposed one.  The fixup
 * sweeps of Eq. 33 reach one row across a slab face, so the caller runs
 *   orc_stage_update;  while some slab has failed zones (orc_fail_count)
 *   and fewer than fix_maxsweep sweeps ran: exchange the edge rows
 *   (orc_get_fixrow / orc_set_fixrow), orc_fix_sweep on every slab;
 *   orc_fix_end with the number of sweeps;  orc_stage_bc;  exchange the NG
 *   ghost rows (orc_get_yrow / orc_set_yrow).
 * orc_stage_update returns this slab's CFL step (st 0), orc_stage_bc(1)
 * advances t. */
double orc_stage_update(orc_grid *G, int st)
{
    return st == 0 ? stage_update(G, G->P, G->Ph, 0.5 * G->dt, 0) : stage_update(G, G->Ph, G->P, G->dt, 1);
}

long orc_fail_count(const orc_grid *G) { return count_failed(G); }

long orc_fix_sweep(orc_grid *G, int st) { return fix_sweep(G, st == 0 ? G->Ph : G->P, st); }

void orc_fix_end(orc_grid *G, int nsweeps) { G->cnt.fix_sweeps += nsweeps; }

void orc_stage_bc(orc_grid *G, int st)
{
    orc_bc_fill(G, st == 0 ? G->Ph : G->P);
    if (st == 1) {
        G->t += G->dt;
        G->cnt.n_steps++;
    }
}

/* the row of all 8 primitives at local X2 index j (-NG .. n2-1+NG), over
 * i = -NG .. n1-1+NG and k = -NG .. n3-1+NG (layout [8][N1][N3]), of P
 * (which = 0) or P-hat (which = 1) */
void orc_get_yrow(const orc_grid *G, int which, int j, double *out)
{
    const double *P = which ? G->Ph : G->P;
    long m = 0;
    for (int c = 0; c < ORC_NP; c++)
        for (int i = -ORC_NG; i < G->p.n1 + ORC_NG; i++)
            for (int k = -ORC_NG; k < G->p.n3 + ORC_NG; k++) out[m++] = AT(P, c, orc_idx(G, i, j, k));
}

void orc_set_yrow(orc_grid *G, int which, int j, const double *in)
{
    double *P = which ? G->Ph : G->P;
    long m = 0;
    for (int c = 0; c < ORC_NP; c++)
        for (int i = -ORC_NG; i < G->p.n1 + ORC_NG; i++)
            for (int k = -ORC_NG; k < G->p.n3 + ORC_NG; k++) AT(P, c, orc_idx(G, i, j, k)) = in[m++];
}

/* what a fixup sweep reads of row j: the five averaged primitives and the
 * failure flag (as 0 / 1) over the active i, k, layout [6][n1][n3] */
void orc_get_fixrow(const orc_grid *G, int which, int j, double *out)
{
    const double *P = which ? G->Ph : G->P;
    long m = 0;
    for (int c = 0; c < 6; c++)
        for (int i = 0; i < G->p.n1; i++)
            for (int k = 0; k < G->p.n3; k++) {
                long z = orc_idx(G, i, j, k);
                out[m++] = c < 5 ? AT(P, c, z) : (G->flag[z] != 0);
            }
}

void orc_set_fixrow(orc_grid *G, int which, int j, const double *in)
{
    double *P = which ? G->Ph : G->P;
    long m = 0;
    for (int c = 0; c < 6; c++)
        for (int i = 0; i < G->p.n1; i++)
            for (int k = 0; k < G->p.n3; k++) {
                long z = orc_idx(G, i, j, k);
                if (c < 5) AT(P, c, z) = in[m++];
                else G->flag[z] = in[m++] != 0.0;
            }
}

/* the (N1 x N2) plane of all 8 primitives at local X3 index k (-NG .. n3-1+NG,
 * ghosts of X1 and X2 included) of P (which = 0) or P-hat (which = 1) */
void orc_get_xplane(const orc_grid *G, int which, int k, double *out)
{
    const double *P = which ? G->Ph : G->P;
    long m = 0;
    for (int c = 0; c < ORC_NP; c++)
        for (int i = -ORC_NG; i < G->p.n1 + ORC_NG; i++)
            for (int j = -ORC_NG; j < G->p.n2 + ORC_NG; j++) out[m++] = AT(P, c, orc_idx(G, i, j, k));
}

void orc_set_xplane(orc_grid *G, int which, int k, const double *in)
{
    double *P = which ? G->Ph : G->P;
    long m = 0;
    for (int c = 0; c < ORC_NP; c++)
        for (int i = -ORC_NG; i < G->p.n1 + ORC_NG; i++)
            for (int j = -ORC_NG; j < G->p.n2 + ORC_NG; j++) AT(P, c, orc_idx(G, i, j, k)) = in[m++];
}


/* Invert the stored U of every active zone (guess: the stored P), apply
 * floors, ceilings, the Lorentz cap and fixups, then refill the ghosts.
 * Returns the number of zones that were flagged before the fixups, or -1 if
 * some could not be fixed. */
int orc_invert_all(orc_grid *G)
{
    const orc_params *p = &G->p;
    int nflag = 0;
    for (int i = 0; i < p->n1; i++)
        for (int j = 0; j < p->n2; j++)
            for (int k = 0; k < p->n3; k++) {
                long z = orc_idx(G, i, j, k);
                double q[ORC_NP], qn[ORC_NP], Un[ORC_NU];
                gather(G, G->P, z, q);
                for (int c = 0; c < ORC_NU; c++) Un[c] = AT(G->U, c, z);
                invert_zone(G, i, j, z, Un, q, qn);
                nflag += G->flag[z];
                scatter(G, G->P, z, qn);
                for (int c = 0; c < ORC_NU; c++) AT(G->U, c, z) = Un[c];
            }
    int st = fixups(G, G->P, 1);
    orc_bc_fill(G, G->P);
    return st != 0 ? -1 : nflag;
}

/* ---------------------------------------------------------------- state */

void orc_set_state(orc_grid *G, const double *Pa, const double *Ua, double t, double dt)
{
    const orc_params *p = &G->p;
    long na = (long)p->n1 * p->n2 * p->n3, a = 0;
    for (int i = 0; i < p->n1; i++)
        for (int j = 0; j < p->n2; j++)
            for (int k = 0; k < p->n3; k++, a++) {
                long z = orc_idx(G, i, j, k);
                for (int c = 0; c < ORC_NP; c++) AT(G->P, c, z) = Pa[c * na + a];
                for (int c = 0; c < ORC_NU; c++) AT(G->U, c, z) = Ua[c * na + a];
            }
    orc_bc_fill(G, G->P);
    G->t = t;
    G->dt = dt;
}

void orc_get_state(const orc_grid *G, double *Pa, double *Ua, double *t, double *dt)
{
    const orc_params *p = &G->p;
    long na = (long)p->n1 * p->n2 * p->n3, a = 0;
    for (int i = 0; i < p->n1; i++)
        for (int j = 0; j < p->n2; j++)
            for (int k = 0; k < p->n3; k++, a++) {
                long z = orc_idx(G, i, j, k);
                if (Pa)
                    for (int c = 0; c < ORC_NP; c++) Pa[c * na + a] = AT(G->P, c, z);
                if (Ua)
                    for (int c = 0; c < ORC_NU; c++) Ua[c * na + a] = AT(G->U, c, z);
            }
    if (t) *t = G->t;
    if (dt) *dt = G->dt;
}

void orc_set_dt(orc_grid *G, double dt) { G->dt = dt; }

/* CFL step of Eq. 27 for the current primitives (the extra sweep that
 * starts a run). */
double orc_initial_dt(orc_grid *G)
{
    G->dt = orc_compute_fluxes(G, G->P);
    return G->dt;
}

/* Face fluxes after flux-CT for the current primitives, active faces only,
 * out[d][c][n1+1][n2+1][n3+1] with face index along d (unused slots zero). */
double orc_fluxes(orc_grid *G, double *out)
{
    const orc_params *p = &G->p;
    double dtn = orc_compute_fluxes(G, G->P);
    orc_flux_ct(G);
    int m1 = p->n1 + 1, m2 = p->n2 + 1, m3 = p->n3 + 1;
    long nf = (long)m1 * m2 * m3;
    memset(out, 0, sizeof(double) * 3 * ORC_NU * nf);
    int n[3] = {p->n1, p->n2, p->n3};
    for (int d = 0; d < 3; d++)
        for (int i = 0; i < n[0] + (d == 0); i++)
            for (int j = 0; j < n[1] + (d == 1); j++)
                for (int k = 0; k < n[2] + (d == 2); k++) {
                    long z = orc_idx(G, i, j, k);
                    long o = ((long)i * m2 + j) * m3 + k;
                    for (int c = 0; c < ORC_NU; c++) out[((long)d * ORC_NU + c) * nf + o] = AT(G->F[d], c, z);
                }
    return dtn;
}

/* ---------------------------------------------------------- diagnostics */

void orc_diagnostics(orc_grid *G, orc_diag *out)
{
    const orc_params *p = &G->p;
    *out = G->cnt;
    out->t = G->t;
    out->dt = G->dt;
    double mdot = 0, phib = 0, edot = 0, ldot = 0;
    double dA = G->dx[1] * G->dx[2];
    if (p->metric == ORC_KERR_MKS && G->i_h < p->n1) {
        int i = G->i_h;
        for (int j = 0; j < p->n2; j++) {
            const orc_geom *g = &G->gc[orc_midx(G, i, j)];
            for (int k = 0; k < p->n3; k++) {
                double q[ORC_NP], T[4];
                gather(G, G->P, orc_idx(G, i, j, k), q);
                orc_state s;
                orc_state_of(q, g, &s);
                orc_tmunu(q, &s, p->gam, 1, T);
                mdot += g->gdet * q[KRHO] * s.ucon[1] * dA;
                phib += 0.5 * g->gdet * fabs(q[KB1]) * dA;
                edot += -g->gdet * T[0] * dA;
                ldot += g->gdet * T[3] * dA;
            }
        }
    }
    out->mdot = mdot;
    out->phib = phib;
    out->edot = edot;
    out->ldot = ldot;
    out->PhiB = mdot != 0.0 ? phib / sqrt(fabs(mdot)) : 0.0;
    /* (Edot - Mdot) / |Mdot| of Eqs. 38 and 41 */
    out->eta = mdot != 0.0 ? (edot - mdot) / fabs(mdot) : 0.0;
    /* corner divergence of Eq. 24, acting on the conserved sqrt(-g) B^i */
    double dmax = 0.0;
    /* a phi slab checks only the corners inside it: those on its low phi face
       need the neighbouring slab's conserved B */
    int periodic3 = p->bc3 != ORC_BC_EXTERNAL && ((p->metric == ORC_KERR_MKS) || p->bc3 == ORC_BC_PERIODIC);
    int k0 = (periodic3 || p->n3 == 1) ? 0 : 1;
    for (int i = 1; i < p->n1; i++)
        for (int j = 1; j < p->n2; j++)
            for (int k = k0; k < p->n3; k++) {
                double dv = 0.0;
                for (int l1 = 0; l1 < 2; l1++)
                    for (int l2 = 0; l2 < 2; l2++)
                        for (int l3 = 0; l3 < 2; l3++) {
                            int ii = i - 1 + l1, jj = j - 1 + l2, kk = k - 1 + l3;
                            kk = ((kk % p->n3) + p->n3) % p->n3;
                            long z = orc_idx(G, ii, jj, kk);
                            dv += (2 * l1 - 1) * AT(G->U, KB1, z) / (4.0 * G->dx[0]) +
                                  (2 * l2 - 1) * AT(G->U, KB2, z) / (4.0 * G->dx[1]) +
                                  (2 * l3 - 1) * AT(G->U, KB3, z) / (4.0 * G->dx[2]);
                        }
                dmax = maxf(dmax, fabs(dv));
            }
    out->divb_max = dmax;
    out->disk_mass = G->disk_mass;
    out->disk_eb = G->disk_eb;
}

/* Barycentric radius of Eq. 43: <r> = int r rho sqrt(-g) dV / int rho sqrt(-g) dV
   over r_H <= r <= r_bar_max, as midpoint sums over the active zones from the
   horizon zone (i_h, as for Eq. 38) outwards whose centre radius is at most
   r_bar_max.  sqrt(-g) dX1 dX2 dX3 of the code coordinates is the volume
   element sqrt(-g) dr dtheta dphi of the paper's.  out = (<r>, denominator,
   numerator); returns <r> (0 when the range holds no mass or the grid is not
   Kerr). */
double orc_barycentric(orc_grid *G, double r_bar_max, double out[3])
{
    const orc_params *p = &G->p;
    double num = 0.0, den = 0.0;
    double dV = G->dx[0] * G->dx[1] * G->dx[2];
    if (p->metric == ORC_KERR_MKS) {
        for (int i = G->i_h; i < p->n1; i++) {
            if (G->rc[orc_midx(G, i, 0)] > r_bar_max) continue;
            for (int j = 0; j < p->n2; j++) {
                int m = orc_midx(G, i, j);
                double r = G->rc[m], gdet = G->gc[m].gdet;
                for (int k = 0; k < p->n3; k++) {
                    double rho = AT(G->P, KRHO, orc_idx(G, i, j, k));
                    num += r * rho * gdet * dV;
                    den += rho * gdet * dV;
                }
            }
        }
    }
    out[0] = den > 0.0 ? num / den : 0.0;
    out[1] = den;
    out[2] = num;
    return out[0];
}

/* ---------------------------------------------- batched point operations */

/* loc[n] = active (i*n2 + j) of the zone whose centre metric is used */
static const orc_geom *loc_geom(const orc_grid *G, int loc)
{
    int i = loc / G->p.n2, j = loc % G->p.n2;
    return &G->gc[orc_midx(G, i, j)];
}

void orc_p2c_batch(const orc_grid *G, const double *P, const int *loc, double *U, long n)
{
    for (long a = 0; a < n; a++) {
        const orc_geom *g = loc_geom(G, loc[a]);
        double q[ORC_NP], Uz[ORC_NU];
        for (int c = 0; c < ORC_NP; c++) q[c] = P[c * n + a];
        orc_state s;
        orc_state_of(q, g, &s);
        orc_prim_to_U(q, g, &s, G->p.gam, Uz);
        for (int c = 0; c < ORC_NU; c++) U[c * n + a] = Uz[c];
    }
}

void orc_c2p_batch(const orc_grid *G, const double *U, const int *loc, const double *guess,
                   double *P, int *flags, int *iters, long n, int methods)
{
    for (long a = 0; a < n; a++) {
        const orc_geom *g = loc_geom(G, loc[a]);
        double Uz[ORC_NU], q0[ORC_NP], q[ORC_NP];
        for (int c = 0; c < ORC_NU; c++) Uz[c] = U[c * n + a];
        for (int c = 0; c < ORC_NP; c++) q0[c] = guess[c * n + a];
        int it;
        flags[a] = orc_con2prim(Uz, g, q0, &G->p, q, &it, methods);
        if (iters) iters[a] = it;
        for (int c = 0; c < ORC_NP; c++) P[c * n + a] = q[c];
    }
}

/* The limits of Section 2.4 applied to one zone (i, j) whose inversion
 * succeeded: floors (Eq. 34), the magnetisation ceilings by mass added at
 * rest in the normal frame, and the Lorentz cap.  q (8) is updated in place
 * from the zone's conserved vector U (9); out[0] = 1 if q was modified,
 * out[1] / out[2] = the zone's ceiling / cap counts.  Test access to the
 * same routine the step calls. */
void orc_post_inversion_at(orc_grid *G, int i, int j, double *q, double *U, int *out)
{
    long long c0 = G->cnt.n_ceil, g0 = G->cnt.n_gcap;
    int mod = 0;
    post_inversion(G, i, j, q, U, &mod);
    out[0] = mod;
    out[1] = (int)(G->cnt.n_ceil - c0);
    out[2] = (int)(G->cnt.n_gcap - g0);
}

/* --------------------------------------------------- table access (tests) */

void orc_geom_table(const orc_grid *G, int loc_kind, double *out)
{
    /* out[(i*n2a + j)*34 + ...] over the ghosted (i, j):
       gcov(16) gcon(16) gdet alpha; loc_kind 0 centre, 1 X1 face, 2 X2 face */
    long m = (long)G->N1 * G->N2;
    const orc_geom *tab = loc_kind == 0 ? G->gc : (loc_kind == 1 ? G->gf1 : G->gf2);
    for (long a = 0; a < m; a++) {
        memcpy(out + a * 34, tab[a].gcov, 16 * sizeof(double));
        memcpy(out + a * 34 + 16, tab[a].gcon, 16 * sizeof(double));
        out[a * 34 + 32] = tab[a].gdet;
        out[a * 34 + 33] = tab[a].alpha;
    }
}

void orc_conn_table(const orc_grid *G, double *out)
{
    memcpy(out, G->conn, sizeof(double) * 64 * G->N1 * G->N2);
}

void orc_grid_info(const orc_grid *G, double *out)
{
    out[0] = G->x1in; out[1] = G->x2in; out[2] = G->x3in;
    out[3] = G->dx[0]; out[4] = G->dx[1]; out[5] = G->dx[2];
    out[6] = G->i_h; out[7] = G->N1; out[8] = G->N2; out[9] = G->N3;
}

/* flags of the last stage for the active zones */
void orc_get_flags(const orc_grid *G, int *out)
{
    long a = 0;
    for (int i = 0; i < G->p.n1; i++)
        for (int j = 0; j < G->p.n2; j++)
            for (int k = 0; k < G->p.n3; k++) out[a++] = G->flag[orc_idx(G, i, j, k)];
}
