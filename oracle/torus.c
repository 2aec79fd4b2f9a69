/*
 * torus.c -- oracle initial state: Fishbone-Moncrief torus (Section 5, first
 * paragraphs), single-loop vector potential (Eq. 45) normalised to beta_0,
 * and the random perturbation of the internal energy.
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 *
 * The paper cites Fishbone & Moncrief (1976) without formulas.  Written here
 * in Boyer-Lindquist coordinates (M = 1) with Sigma = r^2 + a^2 cos^2,
 * Delta = r^2 - 2r + a^2, A = (r^2+a^2)^2 - Delta a^2 sin^2 and the FM
 * invariant l = u^t u_phi:
 *   X^2 = (sqrt(1 + 4 l^2 Sigma^2 Delta / (A^2 sin^2)) - 1) / 2   (ZAMO-frame u_(phi)^2)
 *   ln h = 1/2 ln((1 + sqrt(1 + 4 l^2 Sigma^2 Delta/(A^2 sin^2))) / (Sigma Delta / A))
 *          - 1/2 sqrt(1 + 4 l^2 Sigma^2 Delta/(A^2 sin^2)) - 2 a l r / A,
 * minus its value at (r_in, pi/2).  l is fixed by d(ln h)/dr = 0 at
 * (r_max, pi/2), found here by root finding.
 * rho = ((h-1)(gam-1)/(kappa gam))^(1/(gam-1)) with h - 1 = expm1(ln h),
 * u = kappa rho^gam/(gam-1),
 * then rho and u are divided by max(rho) over the zone centres.
 * Velocity: u^t = sqrt((1+X^2) A/(Sigma Delta)),
 *           u^phi = 2 a r sqrt(1+X^2)/sqrt(A Sigma Delta) + X sqrt(Sigma/A)/sin,
 * u^r = u^theta = 0, which is the same in Kerr-Schild coordinates.
 *
 * A_phi = max(rho/rho_max - 0.2, 0) at zone corners (analytic rho), B from
 * its discrete curl so that the corner divergence of Eq. 24 vanishes, then B
 * scaled so that max p_g / max (b^2/2) over the active zones equals beta_0.
 * Perturbation: u <- u (1 + delta (2 xi - 1)) in torus zones, xi from
 * splitmix64(seed XOR global zone index), top 53 bits.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "orc.h"

typedef double complex cplx;

static cplx fm_lnh_c(double a, double l, cplx r, double th)
{
    double s = sin(th), c = cos(th);
    cplx sig = r * r + a * a * c * c;
    cplx del = r * r - 2.0 * r + a * a;
    cplx A = (r * r + a * a) * (r * r + a * a) - del * a * a * s * s;
    cplx root = csqrt(1.0 + 4.0 * l * l * sig * sig * del / (A * A * s * s));
    return 0.5 * clog((1.0 + root) / (sig * del / A)) - 0.5 * root - 2.0 * a * l * r / A;
}

double orc_fm_lnh(double a, double l, double r, double th) { return creal(fm_lnh_c(a, l, r, th)); }

static double dlnh_dr(double a, double l, double r)
{
    const double h = 1e-30;
    return cimag(fm_lnh_c(a, l, r + I * h, 0.5 * M_PI)) / h;
}

/* l such that the pressure maximum sits at (r_max, pi/2) */
double orc_fm_ell(double a, double r_max)
{
    double lo = 0.5, hi = 50.0;
    double flo = dlnh_dr(a, lo, r_max);
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        double fm = dlnh_dr(a, mid, r_max);
        if ((fm > 0) == (flo > 0)) { lo = mid; flo = fm; } else hi = mid;
        if (hi - lo < 1e-15 * mid) break;
    }
    return 0.5 * (lo + hi);
}

/* Boyer-Lindquist contravariant FM velocity (u^t, 0, 0, u^phi) */
void orc_fm_ucon_bl(double a, double l, double r, double th, double u[4])
{
    double s = sin(th), c = cos(th);
    double sig = r * r + a * a * c * c;
    double del = r * r - 2.0 * r + a * a;
    double A = (r * r + a * a) * (r * r + a * a) - del * a * a * s * s;
    double X2 = 0.5 * (sqrt(1.0 + 4.0 * l * l * sig * sig * del / (A * A * s * s)) - 1.0);
    double X = sqrt(X2);
    u[0] = sqrt((1.0 + X2) * A / (sig * del));
    u[1] = 0.0;
    u[2] = 0.0;
    u[3] = 2.0 * a * r * sqrt(1.0 + X2) / sqrt(A * sig * del) + X * sqrt(sig / A) / s;
}

/* unnormalised FM density; *in = 1 inside the torus */
static double fm_rho(double a, double l, double lnh_in, double r, double th, double r_in,
                     double gam, double kappa, int *in)
{
    *in = 0;
    if (r < r_in || fabs(sin(th)) < 1e-10) return 0.0;
    double lnh = orc_fm_lnh(a, l, r, th) - lnh_in;
    if (!(lnh > 0.0)) return 0.0;
    *in = 1;
    double hm1 = expm1(lnh);
    return pow(hm1 * (gam - 1.0) / (kappa * gam), 1.0 / (gam - 1.0));
}

static uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double orc_uniform(uint64_t seed, uint64_t idx)
{
    return (double)(splitmix64(seed ^ idx) >> 11) * (1.0 / 9007199254740992.0);
}

#define AT(arr, c, z) ((arr)[(long)(c) * G->nz + (z)])

int orc_init_torus(orc_grid *G, const orc_torus_params *tp)
{
    const orc_params *p = &G->p;
    if (p->metric != ORC_KERR_MKS) return -1;
    if (p->n2_total != 0) return -1; /* a theta slab takes its state from set_state */
    int n1 = p->n1, n2 = p->n2, n3 = p->n3;
    double a = p->a, gam = p->gam, kappa = tp->kappa > 0 ? tp->kappa : 1e-3;
    double l = orc_fm_ell(a, tp->r_max);
    double lnh_in = orc_fm_lnh(a, l, tp->r_in, 0.5 * M_PI);
    char *intorus = (char *)calloc((long)n1 * n2, 1);
    double rhomax = 0.0;
    memset(G->P, 0, sizeof(double) * ORC_NP * G->nz);
    for (int i = 0; i < n1; i++)
        for (int j = 0; j < n2; j++) {
            double X1 = G->x1in + (i + 0.5) * G->dx[0], X2 = G->x2in + (j + 0.5) * G->dx[1];
            double dth[2];
            double r = orc_r_of_x1(G, X1), th = orc_theta_at(G, X1, X2, dth);
            int in;
            double rho = fm_rho(a, l, lnh_in, r, th, tp->r_in, gam, kappa, &in);
            intorus[i * n2 + j] = (char)in;
            double q[ORC_NP] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (in) {
                q[KRHO] = rho;
                q[KUU] = kappa * pow(rho, gam) / (gam - 1.0);
                double ubl[4];
                orc_fm_ucon_bl(a, l, r, th, ubl);
                const orc_geom *g = &G->gc[orc_midx(G, i, j)];
                /* u^r = 0: BL and KS contravariant components agree; MKS u^3 = u^phi */
                double gmm = g->alpha * ubl[0]; /* normal-frame Lorentz factor */
                double ucon[4] = {ubl[0], 0.0, 0.0, ubl[3]};
                for (int d = 1; d <= 3; d++) q[KU1 + d - 1] = ucon[d] + gmm * g->alpha * g->gcon[0][d];
                if (rho > rhomax) rhomax = rho;
            }
            for (int k = 0; k < n3; k++)
                for (int c = 0; c < ORC_NP; c++) AT(G->P, c, orc_idx(G, i, j, k)) = q[c];
        }
    if (!(rhomax > 0.0)) { free(intorus); return -2; }
    for (int i = 0; i < n1; i++)
        for (int j = 0; j < n2; j++)
            for (int k = 0; k < n3; k++) {
                long z = orc_idx(G, i, j, k);
                AT(G->P, KRHO, z) /= rhomax;
                AT(G->P, KUU, z) /= rhomax;
            }
    /* vector potential at corners (i-1/2, j-1/2) */
    if (tp->beta0 > 0.0) {
        double *Aph = (double *)calloc((long)(n1 + 1) * (n2 + 1), sizeof(double));
        for (int i = 0; i <= n1; i++)
            for (int j = 0; j <= n2; j++) {
                double dth[2];
                double X1 = G->x1in + i * G->dx[0];
                double r = orc_r_of_x1(G, X1);
                double th = orc_theta_at(G, X1, G->x2in + j * G->dx[1], dth);
                int in;
                double rho = fm_rho(a, l, lnh_in, r, th, tp->r_in, gam, kappa, &in);
                double v = rho / rhomax - 0.2;
                Aph[i * (n2 + 1) + j] = v > 0.0 ? v : 0.0;
            }
#define AC(i, j) Aph[(i) * (n2 + 1) + (j)]
        for (int i = 0; i < n1; i++)
            for (int j = 0; j < n2; j++) {
                double gd = G->gc[orc_midx(G, i, j)].gdet;
                double b1 = (AC(i, j + 1) + AC(i + 1, j + 1) - AC(i, j) - AC(i + 1, j)) / (2.0 * G->dx[1]);
                double b2 = -(AC(i + 1, j) + AC(i + 1, j + 1) - AC(i, j) - AC(i, j + 1)) / (2.0 * G->dx[0]);
                for (int k = 0; k < n3; k++) {
                    long z = orc_idx(G, i, j, k);
                    AT(G->P, KB1, z) = b1 / gd;
                    AT(G->P, KB2, z) = b2 / gd;
                    AT(G->P, KB3, z) = 0.0;
                }
            }
#undef AC
        free(Aph);
        double pmax = 0.0, bsqmax = 0.0;
        for (int i = 0; i < n1; i++)
            for (int j = 0; j < n2; j++) {
                const orc_geom *g = &G->gc[orc_midx(G, i, j)];
                for (int k = 0; k < n3; k++) {
                    long z = orc_idx(G, i, j, k);
                    double q[ORC_NP];
                    for (int c = 0; c < ORC_NP; c++) q[c] = AT(G->P, c, z);
                    orc_state s;
                    orc_state_of(q, g, &s);
                    double pg = (gam - 1.0) * q[KUU];
                    if (pg > pmax) pmax = pg;
                    if (s.bsq > bsqmax) bsqmax = s.bsq;
                }
            }
        if (bsqmax > 0.0) {
            double f = sqrt(pmax / (0.5 * bsqmax) / tp->beta0);
            for (long z = 0; z < G->nz; z++)
                for (int c = KB1; c <= KB3; c++) AT(G->P, c, z) *= f;
        }
    }
    /* disk mass and magnetic energy (Section 5) before the perturbation */
    double dV = G->dx[0] * G->dx[1] * G->dx[2], M = 0.0, EB = 0.0;
    for (int i = 0; i < n1; i++)
        for (int j = 0; j < n2; j++) {
            if (!intorus[i * n2 + j]) continue;
            const orc_geom *g = &G->gc[orc_midx(G, i, j)];
            for (int k = 0; k < n3; k++) {
                long z = orc_idx(G, i, j, k);
                double q[ORC_NP];
                for (int c = 0; c < ORC_NP; c++) q[c] = AT(G->P, c, z);
                orc_state s;
                orc_state_of(q, g, &s);
                M += g->gdet * q[KRHO] * dV;
                EB += g->gdet * s.bsq * dV;
            }
        }
    G->disk_mass = M;
    G->disk_eb = EB;
    /* perturbation, floors, conserved variables */
    for (int i = 0; i < n1; i++)
        for (int j = 0; j < n2; j++) {
            const orc_geom *g = &G->gc[orc_midx(G, i, j)];
            for (int k = 0; k < n3; k++) {
                long z = orc_idx(G, i, j, k);
                double q[ORC_NP], Uz[ORC_NU];
                for (int c = 0; c < ORC_NP; c++) q[c] = AT(G->P, c, z);
                if (intorus[i * n2 + j] && tp->pert_amp != 0.0) {
                    uint64_t gidx = ((uint64_t)i * n2 + j) * n3 + k;
                    double xi = orc_uniform(tp->seed, gidx);
                    q[KUU] *= 1.0 + tp->pert_amp * (2.0 * xi - 1.0);
                }
                int mod = 0;
                orc_floors(G, i, j, q, &mod);
                orc_state s;
                orc_state_of(q, g, &s);
                orc_prim_to_U(q, g, &s, gam, Uz);
                for (int c = 0; c < ORC_NP; c++) AT(G->P, c, z) = q[c];
                for (int c = 0; c < ORC_NU; c++) AT(G->U, c, z) = Uz[c];
            }
        }
    free(intorus);
    orc_bc_fill(G, G->P);
    G->t = 0.0;
    G->dt = orc_compute_fluxes(G, G->P);
    return 0;
}
