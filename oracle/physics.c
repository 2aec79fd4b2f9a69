/*
 * physics.c -- oracle pointwise physics of Section 2.1-2.2:
 *   four-velocity from the modified velocity (Eq. 11), b^mu from B^i
 *   (Section 2.1, after Eq. 5), T^mu_nu (Eq. 5), conserved variables and
 *   fluxes (Eqs. 6-8, plus the entropy density of Eq. 12), MC-limited slopes
 *   (Eq. 16), wave speeds from the simplified dispersion relation (Eq. 19),
 *   and the connection source term (Eqs. 7, 15).
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 */
#include <math.h>
#include "orc.h"

static double dot4(const double a[4], const double b[4])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3];
}

static void lower(const double g[4][4], const double v[4], double w[4])
{
    for (int m = 0; m < 4; m++) w[m] = g[m][0] * v[0] + g[m][1] * v[1] + g[m][2] * v[2] + g[m][3] * v[3];
}

/* u^mu and b^mu of primitive state q at a point with metric g. */
void orc_state_of(const double *q, const orc_geom *g, orc_state *s)
{
    double ut[3] = {q[KU1], q[KU2], q[KU3]};
    double usq = 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) usq += g->gcov[i + 1][j + 1] * ut[i] * ut[j];
    double gam = sqrt(1.0 + usq); /* Lorentz factor of Eq. 11 */
    s->gamma = gam;
    /* u^t = Gamma/alpha; u^i = ut^i - Gamma beta^i / alpha, beta^i = alpha^2 g^{ti} */
    s->ucon[0] = gam / g->alpha;
    for (int i = 0; i < 3; i++) s->ucon[i + 1] = ut[i] - gam * g->alpha * g->gcon[0][i + 1];
    lower(g->gcov, s->ucon, s->ucov);
    /* b^t = B^i u_i ; b^i = (B^i + b^t u^i) / u^t */
    double B[3] = {q[KB1], q[KB2], q[KB3]};
    s->bcon[0] = B[0] * s->ucov[1] + B[1] * s->ucov[2] + B[2] * s->ucov[3];
    for (int i = 0; i < 3; i++) s->bcon[i + 1] = (B[i] + s->bcon[0] * s->ucon[i + 1]) / s->ucon[0];
    lower(g->gcov, s->bcon, s->bcov);
    s->bsq = dot4(s->bcon, s->bcov);
}

/* ---- the piecewise parabolic method (Colella & Woodward 1984, uniform
 * zones in code coordinates), which Section 2.2 names as the more accurate
 * reconstruction after PLM.  Zone values a_j, MC-limited slopes d_j of Eq. 16
 * (the monotonised slopes of CW84), and:
 *   interface value  a_{j+1/2} = (a_j + a_{j+1})/2 - (d_{j+1} - d_j)/6;
 *   the zone's parabola takes a_L = a_{j-1/2}, a_R = a_{j+1/2} and is made
 *   monotone: flat (a_L = a_R = a_j) at a local extremum; else, where the
 *   parabola would overshoot inside the zone, the far edge value is moved so
 *   that the parabola's extremum sits on the near edge (a_L = 3 a_j - 2 a_R,
 *   or a_R = 3 a_j - 2 a_L).
 * Contact steepening and shock flattening are not used. */
static double ppm_interface(double am, double a0, double a1, double a2)
{
    double d0 = orc_mc_slope(am, a0, a1), d1 = orc_mc_slope(a0, a1, a2);
    return 0.5 * (a0 + a1) - (d1 - d0) / 6.0;
}

static void ppm_monotone(double a, double *aL, double *aR)
{
    double L = *aL, R = *aR;
    if ((R - a) * (a - L) <= 0.0) {
        L = a;
        R = a;
    } else {
        double d = R - L, m = a - 0.5 * (L + R);
        if (d * m > d * d / 6.0) L = 3.0 * a - 2.0 * R;
        else if (-d * d / 6.0 > d * m) R = 3.0 * a - 2.0 * L;
    }
    *aL = L;
    *aR = R;
}

/* The two states at the face between zones q[2] and q[3] from the six zone
 * values q[0..5] along the direction: out[0] = a_R of zone 2 (the left
 * state), out[1] = a_L of zone 3 (the right state). */
void orc_ppm_face(const double q[6], double out[2])
{
    double i01 = ppm_interface(q[0], q[1], q[2], q[3]); /* a_{3/2}, zone 2's left edge */
    double i12 = ppm_interface(q[1], q[2], q[3], q[4]); /* the face, a_{5/2} */
    double i23 = ppm_interface(q[2], q[3], q[4], q[5]); /* zone 3's right edge */
    double L2 = i01, R2 = i12, L3 = i12, R3 = i23;
    ppm_monotone(q[2], &L2, &R2);
    ppm_monotone(q[3], &L3, &R3);
    out[0] = R2;
    out[1] = L3;
}

/* Row mu of the mixed stress-energy tensor T^mu_nu, Eq. 5 with p = (gam-1) u. */
void orc_tmunu(const double *q, const orc_state *s, double gam, int mu, double T[4])
{
    double p = (gam - 1.0) * q[KUU];
    double w = q[KRHO] + q[KUU] + p;
    for (int n = 0; n < 4; n++) {
        T[n] = (w + s->bsq) * s->ucon[mu] * s->ucov[n] - s->bcon[mu] * s->bcov[n];
        if (n == mu) T[n] += p + 0.5 * s->bsq;
    }
}

static double entropy_density(const double *q, double gam)
{
    /* S = p / rho^(gam-1), Section 2.1 */
    return (gam - 1.0) * q[KUU] / pow(q[KRHO], gam - 1.0);
}

/* U = sqrt(-g) (rho u^t, T^t_t, T^t_i, B^i, S u^t), Section 2.1 + Eq. 12 */
void orc_prim_to_U(const double *q, const orc_geom *g, const orc_state *s, double gam,
                   double U[ORC_NU])
{
    double T[4];
    orc_tmunu(q, s, gam, 0, T);
    U[KRHO] = g->gdet * q[KRHO] * s->ucon[0];
    for (int n = 0; n < 4; n++) U[1 + n] = g->gdet * T[n];
    U[KB1] = g->gdet * q[KB1];
    U[KB2] = g->gdet * q[KB2];
    U[KB3] = g->gdet * q[KB3];
    U[KENT] = g->gdet * entropy_density(q, gam) * s->ucon[0];
}

/* Flux in direction d (1..3): sqrt(-g) (rho u^d, T^d_nu, b^d u^i - b^i u^d, S u^d), Eqs. 6-8 */
void orc_prim_to_F(const double *q, const orc_geom *g, const orc_state *s, double gam, int d,
                   double F[ORC_NU])
{
    double T[4];
    orc_tmunu(q, s, gam, d, T);
    F[KRHO] = g->gdet * q[KRHO] * s->ucon[d];
    for (int n = 0; n < 4; n++) F[1 + n] = g->gdet * T[n];
    for (int i = 1; i <= 3; i++)
        F[KB1 + i - 1] = g->gdet * (s->bcon[d] * s->ucon[i] - s->bcon[i] * s->ucon[d]);
    F[KENT] = g->gdet * entropy_density(q, gam) * s->ucon[d];
}

/*
 * Roots c1 >= c2 of the simplified dispersion relation of Eq. 19 for waves
 * along direction d.  With k_mu = (-v, delta_mu^d), omega = k_mu u^mu and
 * K^2 = k^2 + omega^2 (spatial projection), omega^2 = cms2 K^2 becomes
 *   (1-cms2)(u^d - v u^t)^2 = cms2 (g^tt v^2 - 2 g^td v + g^dd),
 * a quadratic A v^2 + B v + C = 0 in the coordinate wave speed v.
 */
void orc_wave_speeds(const double *q, const orc_geom *g, const orc_state *s, double gam, int d,
                     double *c1, double *c2)
{
    double p = (gam - 1.0) * q[KUU];
    double ef = q[KRHO] + q[KUU] + p;
    double va2 = s->bsq / (s->bsq + ef);
    double cs2 = gam * p / ef;
    double cms2 = va2 + cs2 * (1.0 - va2);
    double A1 = 1.0 - cms2;
    double ut = s->ucon[0], ud = s->ucon[d];
    double A = A1 * ut * ut - cms2 * g->gcon[0][0];
    double B = -2.0 * (A1 * ut * ud - cms2 * g->gcon[0][d]);
    double C = A1 * ud * ud - cms2 * g->gcon[d][d];
    double disc = B * B - 4.0 * A * C;
    if (disc < 0.0) disc = 0.0;
    double sq = sqrt(disc);
    double vp = (-B + sq) / (2.0 * A);
    double vm = (-B - sq) / (2.0 * A);
    *c1 = vp > vm ? vp : vm;
    *c2 = vp > vm ? vm : vp;
}

/*
 * Monotonized-central slope of Eq. 16.  The last branch is printed with an
 * absolute value; it is read as the signed central difference (q+ - q-)/2,
 * the value the MC limiter takes when the two one-sided slopes agree in sign.
 */
double orc_mc_slope(double qm, double q0, double qp)
{
    double dm = q0 - qm, dp = qp - q0, dc = qp - qm;
    if (dm * dp < 0.0) return 0.0;
    if (fabs(dm) < fabs(dp) && 2.0 * fabs(dm) < 0.5 * fabs(dc)) return 2.0 * dm;
    if (2.0 * fabs(dp) < 0.5 * fabs(dc)) return 2.0 * dp;
    return 0.5 * dc;
}

/* Source of Eq. 7 evaluated at the cell centre (Eq. 15):
 * S_nu = sqrt(-g) T^k_l Gamma^l_{nu k}. */
void orc_source(const double *q, const orc_geom *g, const double conn[4][4][4],
                const orc_state *s, double gam, double S[4])
{
    double T[4][4];
    for (int k = 0; k < 4; k++) orc_tmunu(q, s, gam, k, T[k]);
    for (int nu = 0; nu < 4; nu++) {
        double acc = 0.0;
        for (int k = 0; k < 4; k++)
            for (int l = 0; l < 4; l++) acc += T[k][l] * conn[l][nu][k];
        S[nu] = g->gdet * acc;
    }
}
