/*
 * geometry.c -- oracle geometry: Kerr metric in Kerr-Schild coordinates
 * (Section 4.1, Eq. 35), the modified-Kerr-Schild map (Section 4.1, Eq. 36),
 * the inverse metric, sqrt(-g), the lapse, and the connection used by the
 * source term of Eq. 7.
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 *
 * The connection is Gamma^l_{mn} = 1/2 g^{ls} (d_m g_{sn} + d_n g_{sm} - d_s g_{mn});
 * the paper does not say how it is evaluated.  Here the metric derivatives
 * are taken by the complex-step method, f'(x) = Im f(x + i h) / h, which is
 * exact to rounding for analytic f, so no finite-difference truncation enters.
 */
#include <math.h>
#include <string.h>
#include "orc.h"

/* r(X1) of Eq. 36: exponential inside x_b, hyper-exponential outside. */
static void mks_r_c(const orc_grid *G, double complex X1, double complex *r,
                    double complex *drdx)
{
    const orc_params *p = &G->p;
    if (creal(X1) < G->xb) {
        double complex e = cexp(X1);
        *r = p->R0 + e;
        *drdx = e;
    } else {
        double complex d = X1 - G->xb;
        double complex dn = 1.0, dn1 = 1.0;
        int n = (int)p->n_x;
        if ((double)n == p->n_x && n >= 1) {
            for (int m = 0; m < n - 1; m++) dn1 *= d;
            dn = dn1 * d;
        } else {
            dn = cpow(d, p->n_x);
            dn1 = cpow(d, p->n_x - 1.0);
        }
        double complex e = cexp(X1 + dn);
        *r = p->R0 + e;
        *drdx = e * (1.0 + p->n_x * dn1);
    }
}

/* theta(X2) of Eq. 36, read as pi/2 (1+Y) + (1-h)/2 sin(pi (1+Y)): the
 * equator-refining map (the printed argument pi(1+Y)/2 is not symmetric
 * about the equator). */
static void mks_th_c(const orc_grid *G, double complex X2, double complex *th,
                     double complex *dthdx)
{
    double h = G->p.hslope;
    double complex y = M_PI * (1.0 + X2);
    *th = 0.5 * M_PI * (1.0 + X2) + 0.5 * (1.0 - h) * csin(y);
    *dthdx = 0.5 * M_PI + 0.5 * (1.0 - h) * M_PI * ccos(y);
}

/* Polar cylindrification.  Section 4.1 "cylindrifies" the cells closest
 * to the poles after Tchekhovskoy et al. 2011 and prints no formula; this
 * is the reading used here.  Inside a band of width y_b = cyl_dx2 (in X2)
 * next to each pole, the MKS angle is taken at a moved coordinate
 *     X2' = pole -/+ y_b phi(s),   s = |X2 - pole| / y_b (negative beyond the pole),
 *     phi(s) = s + (lambda - 1) s (1 - s^2)^3,
 *     lambda(r) = (1 + (r_c / r)^4)^(1/4),   r_c = cyl_r.
 * At the pole phi'(0) = lambda: the first rows are widened by lambda(r),
 * which for r << r_c is r_c / r, so those rows keep a cylindrical radius
 * R = r sin(theta) of about r_c theta_MKS instead of shrinking with r -- the
 * cylinders of the name -- while for r >> r_c lambda -> 1 and the grid is
 * MKS.  The rows further out in the band are narrowed to make room:
 * phi(1) = 1, phi'(1) = 1, phi''(1) = 0 join the band to the MKS rows with
 * a continuous metric derivative, and phi is odd in s, so the mirror image
 * across the pole that the polar boundary uses is kept.  phi' > 0 (a
 * monotone map) needs lambda < 1 + 49/32; the grid refuses lambda > 5/2. */
static void cyl_lambda_c(const orc_grid *G, double complex r, double complex *lam,
                         double complex *dlam_dr)
{
    double complex x = G->p.cyl_r / r;
    double complex q = x * x * x * x;
    *lam = cpow(1.0 + q, 0.25);
    /* d/dr (1 + q)^(1/4) = (1/4) (1 + q)^(-3/4) dq/dr, dq/dr = -4 q / r */
    *dlam_dr = -q * cpow(1.0 + q, -0.75) / r;
}

/* theta(X1, X2) and its two partial derivatives: Eq. 36 outside the bands,
 * the cylindrified angle inside them */
static void theta_c(const orc_grid *G, double complex X1, double complex X2, double complex *th,
                    double complex *dth1, double complex *dth2)
{
    double yb = G->p.cyl_dx2;
    int lower = creal(X2) < 0.0;
    double complex s = lower ? (X2 + 1.0) / yb : (1.0 - X2) / yb;
    if (!(G->p.cyl_r > 0.0) || fabs(creal(s)) >= 1.0) {
        mks_th_c(G, X2, th, dth2);
        *dth1 = 0.0;
        return;
    }
    double complex r, drdx, lam, dlam;
    mks_r_c(G, X1, &r, &drdx);
    cyl_lambda_c(G, r, &lam, &dlam);
    double complex w = 1.0 - s * s;
    double complex w3 = w * w * w;
    double complex phi = s + (lam - 1.0) * s * w3;
    double complex dphi_ds = 1.0 + (lam - 1.0) * (w3 - 6.0 * s * s * w * w);
    double complex dphi_dlam = s * w3;
    /* X2' and its partials: lower pole -1 + yb phi, upper 1 - yb phi */
    double complex X2m, dthm;
    double complex dX2m_dX1;
    if (lower) {
        X2m = -1.0 + yb * phi;
        dX2m_dX1 = yb * dphi_dlam * dlam * drdx;
    } else {
        X2m = 1.0 - yb * phi;
        dX2m_dX1 = -yb * dphi_dlam * dlam * drdx;
    }
    mks_th_c(G, X2m, th, &dthm);
    *dth2 = dthm * dphi_ds; /* dX2'/dX2 = dphi/ds on both sides */
    *dth1 = dthm * dX2m_dX1;
}

double orc_r_of_x1(const orc_grid *G, double X1)
{
    double complex r, d;
    mks_r_c(G, X1, &r, &d);
    return creal(r);
}

double orc_th_of_x2(const orc_grid *G, double X2)
{
    double complex th, d;
    mks_th_c(G, X2, &th, &d);
    return creal(th);
}

double orc_theta_at(const orc_grid *G, double X1, double X2, double dth[2])
{
    double complex th, d1, d2;
    theta_c(G, X1, X2, &th, &d1, &d2);
    dth[0] = creal(d1);
    dth[1] = creal(d2);
    return creal(th);
}

/* inverse of r(X1) by bisection (monotone map) */
double orc_x1_of_r(const orc_grid *G, double r)
{
    double lo = -50.0, hi = 50.0;
    for (int it = 0; it < 400; it++) {
        double mid = 0.5 * (lo + hi);
        if (orc_r_of_x1(G, mid) < r) lo = mid; else hi = mid;
        if (hi - lo <= 1e-15 * fabs(mid)) break;
    }
    return 0.5 * (lo + hi);
}

/* Kerr-Schild line element of Eq. 35 (M = 1), written for complex r, theta. */
static void ks_gcov_c(double complex r, double complex th, double a, double complex g[4][4])
{
    double complex s = csin(th), c = ccos(th);
    double complex s2 = s * s, c2 = c * c;
    double complex sig = r * r + a * a * c2;
    double complex z = 2.0 * r / sig;
    memset(g, 0, sizeof(double complex) * 16);
    g[0][0] = -(1.0 - z);
    g[0][1] = g[1][0] = z;
    g[0][3] = g[3][0] = -a * z * s2;
    g[1][1] = 1.0 + z;
    g[1][3] = g[3][1] = -a * (1.0 + z) * s2;
    g[2][2] = sig;
    g[3][3] = s2 * (sig + a * a * (1.0 + z) * s2);
}

void orc_ks_gcov(double r, double th, double a, double g[4][4])
{
    double complex gc[4][4];
    ks_gcov_c(r, th, a, gc);
    for (int m = 0; m < 4; m++)
        for (int n = 0; n < 4; n++) g[m][n] = creal(gc[m][n]);
}

/* metric in the code coordinates (t, X1, X2, X3) */
void orc_code_gcov_c(const orc_grid *G, double complex X1, double complex X2,
                     double complex g[4][4])
{
    if (G->p.metric == ORC_MINK_CART) {
        memset(g, 0, sizeof(double complex) * 16);
        g[0][0] = -1.0;
        g[1][1] = g[2][2] = g[3][3] = 1.0;
        return;
    }
    double complex r, drdx, th, dth1, dth2, gks[4][4];
    mks_r_c(G, X1, &r, &drdx);
    theta_c(G, X1, X2, &th, &dth1, &dth2);
    ks_gcov_c(r, th, G->p.a, gks);
    if (!(G->p.cyl_r > 0.0)) { /* Eq. 36 alone: a diagonal Jacobian */
        double complex Jd[4] = {1.0, drdx, dth2, 1.0};
        for (int m = 0; m < 4; m++)
            for (int n = 0; n < 4; n++) g[m][n] = gks[m][n] * Jd[m] * Jd[n];
        return;
    }
    /* g_{mn} = (dx^a/dX^m) (dx^b/dX^n) g^KS_{ab}; the Kerr-Schild
     * coordinates (t, r, theta, phi) depend on (t, X1, X2, X3) through
     * r(X1) and theta(X1, X2) */
    double complex J[4][4] = {{0}}; /* J[a][m] = dx^a / dX^m */
    J[0][0] = 1.0;
    J[1][1] = drdx;
    J[2][1] = dth1;
    J[2][2] = dth2;
    J[3][3] = 1.0;
    for (int m = 0; m < 4; m++)
        for (int n = 0; n < 4; n++) {
            double complex s = 0.0;
            for (int a = 0; a < 4; a++)
                for (int b = 0; b < 4; b++) s += J[a][m] * J[b][n] * gks[a][b];
            g[m][n] = s;
        }
}

/* Gauss-Jordan inversion with partial pivoting; returns 0 if singular. */
int orc_invert4(const double m[4][4], double inv[4][4], double *det)
{
    double a[4][8];
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) {
            a[r][c] = m[r][c];
            a[r][c + 4] = (r == c) ? 1.0 : 0.0;
        }
    double d = 1.0;
    for (int c = 0; c < 4; c++) {
        int piv = c;
        for (int r = c + 1; r < 4; r++)
            if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
        if (a[piv][c] == 0.0) { *det = 0.0; return 0; }
        if (piv != c) {
            for (int k = 0; k < 8; k++) { double t = a[c][k]; a[c][k] = a[piv][k]; a[piv][k] = t; }
            d = -d;
        }
        double pv = a[c][c];
        d *= pv;
        for (int k = 0; k < 8; k++) a[c][k] /= pv;
        for (int r = 0; r < 4; r++) {
            if (r == c) continue;
            double f = a[r][c];
            if (f == 0.0) continue;
            for (int k = 0; k < 8; k++) a[r][k] -= f * a[c][k];
        }
    }
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) inv[r][c] = a[r][c + 4];
    *det = d;
    return 1;
}

/* Inverse metric, sqrt(-g) and lapse.  For Kerr the inverse of Eq. 35 is
 * written out in closed form (Kerr-Schild: g^tt = -(1+z), g^tr = z,
 * g^rr = Delta/Sigma, g^r phi = a/Sigma, g^th th = 1/Sigma,
 * g^phi phi = 1/(Sigma sin^2), z = 2r/Sigma; sqrt(-g) = Sigma |sin theta|)
 * and mapped to MKS by the diagonal Jacobian of Eq. 36.  A numerical 4x4
 * inverse loses accuracy with the condition number of the MKS metric, which
 * grows like (dr/dX1)^2 at large radius. */
int orc_geom_at(const orc_grid *G, double X1, double X2, orc_geom *out)
{
    double complex gc[4][4];
    orc_code_gcov_c(G, X1, X2, gc);
    for (int m = 0; m < 4; m++)
        for (int n = 0; n < 4; n++) out->gcov[m][n] = creal(gc[m][n]);
    if (G->p.metric == ORC_MINK_CART) {
        memset(out->gcon, 0, sizeof(out->gcon));
        out->gcon[0][0] = -1.0;
        out->gcon[1][1] = out->gcon[2][2] = out->gcon[3][3] = 1.0;
        out->gdet = 1.0;
        out->alpha = 1.0;
        return 1;
    }
    double complex rc, drc, thc, dth1c, dthc;
    mks_r_c(G, X1, &rc, &drc);
    theta_c(G, X1, X2, &thc, &dth1c, &dthc);
    double r = creal(rc), th = creal(thc), dr = creal(drc), dth = creal(dthc), a = G->p.a;
    double dth1 = creal(dth1c);
    double s = sin(th), c = cos(th);
    double sig = r * r + a * a * c * c, del = r * r - 2.0 * r + a * a, z = 2.0 * r / sig;
    if (s == 0.0) {
        memset(out, 0, sizeof(*out));
        return 0;
    }
    double gi[4][4] = {{0}};
    gi[0][0] = -(1.0 + z);
    gi[0][1] = gi[1][0] = z;
    gi[1][1] = del / sig;
    gi[1][3] = gi[3][1] = a / sig;
    gi[2][2] = 1.0 / sig;
    gi[3][3] = 1.0 / (sig * s * s);
    if (dth1 == 0.0) {
        double J[4] = {1.0, dr, dth, 1.0};
        for (int m = 0; m < 4; m++)
            for (int n = 0; n < 4; n++) out->gcon[m][n] = gi[m][n] / (J[m] * J[n]);
    } else {
        /* cylindrified: g^{mn} = (dX^m/dx^a) (dX^n/dx^b) g_KS^{ab} with the
         * inverse Jacobian dX1/dr = 1/r', dX2/dr = -theta_1 / (r' theta_2),
         * dX2/dtheta = 1/theta_2 (theta_k = d theta / dX^k) */
        double K[4][4] = {{0}}; /* K[m][a] = dX^m / dx^a */
        K[0][0] = 1.0;
        K[1][1] = 1.0 / dr;
        K[2][1] = -dth1 / (dr * dth);
        K[2][2] = 1.0 / dth;
        K[3][3] = 1.0;
        for (int m = 0; m < 4; m++)
            for (int n = 0; n < 4; n++) {
                double acc = 0.0;
                for (int p = 0; p < 4; p++)
                    for (int q = 0; q < 4; q++) acc += K[m][p] * K[n][q] * gi[p][q];
                out->gcon[m][n] = acc;
            }
    }
    /* det(dx/dX) = r' theta_2 whether or not theta depends on X1 */
    out->gdet = sig * fabs(s) * fabs(dr * dth);
    out->alpha = 1.0 / sqrt(-out->gcon[0][0]);
    return 1;
}

/* Connection coefficients conn[l][m][n] = Gamma^l_{mn} at (X1, X2). */
void orc_conn_at(const orc_grid *G, double X1, double X2, double conn[4][4][4])
{
    orc_geom g;
    orc_geom_at(G, X1, X2, &g);
    double dg[4][4][4]; /* dg[c][a][b] = d_c g_ab */
    memset(dg, 0, sizeof(dg));
    const double h = 1e-30;
    double complex gp[4][4];
    orc_code_gcov_c(G, X1 + I * h, X2, gp);
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) dg[1][a][b] = cimag(gp[a][b]) / h;
    orc_code_gcov_c(G, X1, X2 + I * h, gp);
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) dg[2][a][b] = cimag(gp[a][b]) / h;
    for (int l = 0; l < 4; l++)
        for (int m = 0; m < 4; m++)
            for (int n = 0; n < 4; n++) {
                double s = 0.0;
                for (int sg = 0; sg < 4; sg++)
                    s += g.gcon[l][sg] * (dg[m][sg][n] + dg[n][sg][m] - dg[sg][m][n]);
                conn[l][m][n] = 0.5 * s;
            }
}
