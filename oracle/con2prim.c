/*
 * con2prim.c -- oracle conserved-to-primitive inversion of Section 2.3.
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 *
 * Variables follow Noble et al. (2006) as reviewed in Section 2.3:
 *   D = Gamma rho, Q_mu = -n_nu T^nu_mu, Qt^mu = j^mu_nu Q^nu, Bf^mu = -n_nu *F^{mu nu},
 * and the two unknowns W = Gamma^2 h and v^2 solve Eqs. 29-30 with the
 * pressure of Eq. 31.  Methods, in the paper's order:
 *   (i)   2D Newton-Raphson on (W, v^2) to 1e-10;
 *   (ii)  if (i) does not converge: v^2(W) eliminated and a 1D Brent solve in W;
 *   (iii) if (ii) fails, or if (i) gives unphysical values: entropy inversion,
 *         W(v^2) from Eq. 32 put into Eq. 29 and a 1D Brent solve in v^2;
 *   and (iii) alone where beta = p_g / (b^2/2) < 1e-2 for the guess primitives.
 *
 * Readings where the text is ambiguous:
 *   - Eq. 30 is printed with +Bf^2/2 (1+v^2); the sign is taken as minus, the
 *     only sign for which a static magnetised fluid satisfies the equation.
 *   - for method (ii) the text swaps the roles of Eqs. 29 and 30; here v^2 is
 *     taken from Eq. 29, which is linear in v^2, and Eq. 30 is solved for W
 *     (the 1D method of Noble et al. that the paper cites).
 *   - S in Eq. 32 is the normal-frame entropy density Gamma p / rho^(gam-1)
 *     = alpha U_S / sqrt(-g), the analogue of D = Gamma rho.
 *   - Newton stops once |dW/W| < tol and |dv^2| < tol and then takes one more
 *     step; at most nr_maxit steps; v^2 is clamped into [0, 1-1e-16].
 *   - Brent solves run to machine precision, at most brent_maxit steps.
 */
#include <math.h>
#include <string.h>
#include "orc.h"

#define V2MAX (1.0 - 1.0e-16)

typedef struct {
    double D, Qtsq, Bsq, QB, nQ, Sent, gam;
    double Qtcon[3], Bf[3];
} c2p_in;

static double pressure_of(const c2p_in *c, double W, double v2)
{
    double s = sqrt(1.0 - v2);
    return (c->gam - 1.0) / c->gam * (W * (1.0 - v2) - c->D * s);
}

/* primitive velocities from Eq. 31 of Noble et al.: ut^i = Gamma/(W+B^2) (Qt^i + (Q.B) B^i / W) */
static void recover(const c2p_in *c, double W, double v2, double p, double *P)
{
    double gam = 1.0 / sqrt(1.0 - v2);
    P[KRHO] = c->D / gam;
    P[KUU] = p / (c->gam - 1.0);
    double f = gam / (W + c->Bsq);
    for (int i = 0; i < 3; i++) P[KU1 + i] = f * (c->Qtcon[i] + c->QB * c->Bf[i] / W);
}

static int physical(const double *P, double v2)
{
    for (int m = 0; m < 5; m++)
        if (!isfinite(P[m])) return 0;
    return P[KRHO] > 0.0 && P[KUU] > 0.0 && v2 >= 0.0 && v2 < 1.0;
}

/* ---- Brent's method (Brent 1973, Ch. 4): bracketing root finder that mixes
 * bisection with secant and inverse quadratic interpolation. ---- */
double orc_brent(double (*f)(double, void *), void *ctx, double a, double b, double fa,
                 double fb, double tol, int maxit, int *ok)
{
    const double eps = 2.220446049250313e-16;
    *ok = 0;
    if ((fa > 0.0 && fb > 0.0) || (fa < 0.0 && fb < 0.0)) return b;
    if (fa == 0.0) { *ok = 1; return a; }
    if (fb == 0.0) { *ok = 1; return b; }
    double c = a, fc = fa, d = b - a, e = d;
    for (int it = 0; it < maxit; it++) {
        if ((fb > 0.0 && fc > 0.0) || (fb < 0.0 && fc < 0.0)) {
            c = a; fc = fa; d = b - a; e = d;
        }
        if (fabs(fc) < fabs(fb)) {
            a = b; b = c; c = a;
            fa = fb; fb = fc; fc = fa;
        }
        double tol1 = 2.0 * eps * fabs(b) + 0.5 * tol;
        double xm = 0.5 * (c - b);
        if (fabs(xm) <= tol1 || fb == 0.0) { *ok = 1; return b; }
        if (fabs(e) >= tol1 && fabs(fa) > fabs(fb)) {
            double s = fb / fa, p, q;
            if (a == c) {
                p = 2.0 * xm * s;
                q = 1.0 - s;
            } else {
                double qq = fa / fc, r = fb / fc;
                p = s * (2.0 * xm * qq * (qq - r) - (b - a) * (r - 1.0));
                q = (qq - 1.0) * (r - 1.0) * (s - 1.0);
            }
            if (p > 0.0) q = -q; else p = -p;
            double m1 = 3.0 * xm * q - fabs(tol1 * q), m2 = fabs(e * q);
            if (2.0 * p < (m1 < m2 ? m1 : m2)) { e = d; d = p / q; }
            else { d = xm; e = d; }
        } else {
            d = xm; e = d;
        }
        a = b; fa = fb;
        if (fabs(d) > tol1) b += d;
        else b += (xm > 0.0 ? tol1 : -tol1);
        fb = f(b, ctx);
        if (!isfinite(fb)) return b;
    }
    return b;
}

/* ---- method (i): 2D Newton-Raphson on Eqs. 29-30 ---- */
static int newton2d(const c2p_in *c, double *Wp, double *v2p, const orc_params *prm, int *iters)
{
    double W = *Wp, v2 = *v2p;
    const double g1 = (c->gam - 1.0) / c->gam;
    const double QB2 = c->QB * c->QB;
    int extra = 0, n = 0;
    for (int it = 1; it <= prm->nr_maxit; it++) {
        n = it;
        double s = sqrt(1.0 - v2);
        double p = g1 * (W * (1.0 - v2) - c->D * s);
        double BW = c->Bsq + W;
        double W2 = W * W, W3 = W2 * W;
        double f1 = v2 * BW * BW - QB2 * (c->Bsq + 2.0 * W) / W2 - c->Qtsq;
        double f2 = -0.5 * c->Bsq * (1.0 + v2) + QB2 / (2.0 * W2) - W + p - c->nQ;
        double a11 = 2.0 * v2 * BW + 2.0 * QB2 * BW / W3;
        double a12 = BW * BW;
        double a21 = -QB2 / W3 - 1.0 + g1 * (1.0 - v2);
        double a22 = -0.5 * c->Bsq + g1 * (-W + 0.5 * c->D / s);
        double det = a11 * a22 - a12 * a21;
        if (!(fabs(det) > 0.0) || !isfinite(det)) break;
        double dW = -(a22 * f1 - a12 * f2) / det;
        double dv = -(-a21 * f1 + a11 * f2) / det;
        double Wn = W + dW;
        if (!(Wn > 0.0)) Wn = 0.5 * W;
        double vn = v2 + dv;
        if (vn < 0.0) vn = 0.0;
        if (vn > V2MAX) vn = V2MAX;
        double errW = fabs(Wn - W) / fabs(Wn), errv = fabs(vn - v2);
        W = Wn; v2 = vn;
        if (!isfinite(W) || !isfinite(v2)) break;
        if (extra) { *Wp = W; *v2p = v2; *iters = n; return 1; }
        if (errW < prm->nr_tol && errv < prm->nr_tol) extra = 1;
    }
    *iters = n;
    return 0;
}

/* ---- method (ii): Brent in W with v^2(W) from Eq. 29 ---- */
static double v2_of_W(const c2p_in *c, double W)
{
    double BW = c->Bsq + W;
    double v2 = (c->Qtsq + c->QB * c->QB * (c->Bsq + 2.0 * W) / (W * W)) / (BW * BW);
    if (v2 < 0.0) v2 = 0.0;
    if (v2 > V2MAX) v2 = V2MAX;
    return v2;
}

static double resid_W(double W, void *ctx)
{
    const c2p_in *c = (const c2p_in *)ctx;
    double v2 = v2_of_W(c, W);
    return -0.5 * c->Bsq * (1.0 + v2) + c->QB * c->QB / (2.0 * W * W) - W +
           pressure_of(c, W, v2) - c->nQ;
}

static int brent_w(const c2p_in *c, const orc_params *prm, double *P)
{
    double E = -c->nQ;
    double lo = c->D, hi = c->gam * (E > c->D ? E : c->D) * (1.0 + 1e-10);
    if (!(lo > 0.0) || !(hi > lo)) return 0;
    double flo = resid_W(lo, (void *)c), fhi = resid_W(hi, (void *)c);
    int ok;
    double W = orc_brent(resid_W, (void *)c, lo, hi, flo, fhi, 0.0, prm->brent_maxit, &ok);
    if (!ok) return 0;
    double v2 = v2_of_W(c, W);
    recover(c, W, v2, pressure_of(c, W, v2), P);
    return physical(P, v2);
}

/* ---- method (iii): entropy inversion, W(v^2) of Eq. 32 into Eq. 29 ---- */
static double W_of_v2_entropy(const c2p_in *c, double v2)
{
    double G = 1.0 / sqrt(1.0 - v2);
    double rho = c->D / G;
    return G * c->D + G * c->gam / (c->gam - 1.0) * pow(rho, c->gam - 1.0) * c->Sent;
}

static double resid_S(double v2, void *ctx)
{
    const c2p_in *c = (const c2p_in *)ctx;
    double W = W_of_v2_entropy(c, v2);
    double BW = c->Bsq + W;
    return v2 * BW * BW - c->QB * c->QB * (c->Bsq + 2.0 * W) / (W * W) - c->Qtsq;
}

static int entropy_inv(const c2p_in *c, const orc_params *prm, double *P)
{
    if (!(c->Sent > 0.0) || !(c->D > 0.0)) return 0;
    double lo = 0.0, hi = 1.0 - 1.0e-12;
    double flo = resid_S(lo, (void *)c), fhi = resid_S(hi, (void *)c);
    int ok = 1;
    double v2 = 0.0;
    /* analytically the residual at v^2 = 0 is -(Q.B)^2 (B^2+2W)/W^2 - Qt^2 <= 0;
     * a positive value there only comes from rounding and means v^2 = 0 */
    if (flo < 0.0)
        v2 = orc_brent(resid_S, (void *)c, lo, hi, flo, fhi, 1.0e-17, prm->brent_maxit, &ok);
    if (!ok) return 0;
    double G = 1.0 / sqrt(1.0 - v2);
    double rho = c->D / G;
    double p = (c->Sent / G) * pow(rho, c->gam - 1.0);
    double W = W_of_v2_entropy(c, v2);
    recover(c, W, v2, p, P);
    return physical(P, v2);
}

/*
 * Invert U (with sqrt(-g)) at a point with metric g.  guess holds the
 * previous primitives (Newton starting point and beta switch).  methods is a
 * bit mask of allowed methods (1 Newton, 2 Brent-W, 4 entropy, 8 beta switch),
 * 15 for the full procedure.  Returns the C2P_* flag.
 */
/* Inversion of one zone.  wguess > 0 replaces the Newton starting W taken
 * from the guess primitives, and v^2 then follows from Eq. 29 at that W (the
 * learned starting point); wguess <= 0 is the plain start from the guess. */
int orc_con2prim_w(const double U[ORC_NU], const orc_geom *g, const double *guess,
                   const orc_params *prm, double P[ORC_NP], int *iters, int methods, double wguess)
{
    *iters = 0;
    for (int m = 0; m < ORC_NP; m++) P[m] = guess[m];
    for (int i = 0; i < 3; i++) P[KB1 + i] = U[KB1 + i] / g->gdet;

    c2p_in c;
    c.gam = prm->gam;
    double f = g->alpha / g->gdet;
    c.D = f * U[KRHO];
    double Qcov[4] = {f * U[1], f * U[2], f * U[3], f * U[4]};
    c.Sent = f * U[KENT];
    double ncon[4] = {1.0 / g->alpha, -g->alpha * g->gcon[0][1], -g->alpha * g->gcon[0][2],
                      -g->alpha * g->gcon[0][3]};
    double Qcon[4];
    for (int m = 0; m < 4; m++) {
        Qcon[m] = 0.0;
        for (int n = 0; n < 4; n++) Qcon[m] += g->gcon[m][n] * Qcov[n];
    }
    c.nQ = 0.0;
    double Qsq = 0.0;
    for (int m = 0; m < 4; m++) {
        c.nQ += ncon[m] * Qcov[m];
        Qsq += Qcon[m] * Qcov[m];
    }
    c.Qtsq = Qsq + c.nQ * c.nQ;
    for (int i = 0; i < 3; i++) {
        c.Qtcon[i] = Qcon[i + 1] + ncon[i + 1] * c.nQ;
        c.Bf[i] = g->alpha * P[KB1 + i];
    }
    c.Bsq = 0.0;
    c.QB = 0.0;
    for (int i = 0; i < 3; i++) {
        c.QB += Qcov[i + 1] * c.Bf[i];
        for (int j = 0; j < 3; j++) c.Bsq += g->gcov[i + 1][j + 1] * c.Bf[i] * c.Bf[j];
    }

    int finite = isfinite(c.D) && isfinite(c.Qtsq) && isfinite(c.nQ) && isfinite(c.Bsq);
    if (!finite || !(c.D > 0.0)) return C2P_FAIL | C2P_FAIL_D;

    /* beta = p_g / p_b of the guess primitives (Section 2.3, Eq. 33 region) */
    if (methods & 8) {
        orc_state s;
        orc_state_of(guess, g, &s);
        double pg = (prm->gam - 1.0) * guess[KUU];
        if (s.bsq > 0.0 && pg < prm->beta_entropy * 0.5 * s.bsq) {
            if ((methods & 4) && entropy_inv(&c, prm, P)) return C2P_ENTROPY_BETA;
            return C2P_FAIL | C2P_FAIL_ENT;
        }
    }

    if (methods & 1) {
        double ut[3] = {guess[KU1], guess[KU2], guess[KU3]};
        double usq = 0.0;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) usq += g->gcov[i + 1][j + 1] * ut[i] * ut[j];
        /* a learned W is tried first; Newton from the guess primitives stays
           the fallback when it does not converge */
        int tries = wguess > 0.0 ? 2 : 1;
        for (int a = 0; a < tries; a++) {
            double v2 = usq / (1.0 + usq);
            double W = (1.0 + usq) * (guess[KRHO] + prm->gam * guess[KUU]);
            if (a == 0 && wguess > 0.0) {
                W = wguess;
                v2 = v2_of_W(&c, W);
            }
            if (!(W > 0.0) || !isfinite(W)) W = c.D;
            if (v2 > V2MAX) v2 = V2MAX;
            int it = 0;
            int ok = newton2d(&c, &W, &v2, prm, &it);
            *iters += it;
            if (ok) {
                recover(&c, W, v2, pressure_of(&c, W, v2), P);
                if (physical(P, v2)) return C2P_NR;
                /* converged to unphysical values: entropy fix */
                if ((methods & 4) && entropy_inv(&c, prm, P)) return C2P_ENTROPY;
                return C2P_FAIL | C2P_FAIL_ENT;
            }
        }
    }
    if ((methods & 2) && brent_w(&c, prm, P)) return C2P_BRENT_W;
    if ((methods & 4) && entropy_inv(&c, prm, P)) return C2P_ENTROPY;
    return C2P_FAIL | C2P_FAIL_ENT;
}

int orc_con2prim(const double U[ORC_NU], const orc_geom *g, const double *guess,
                 const orc_params *prm, double P[ORC_NP], int *iters, int methods)
{
    return orc_con2prim_w(U, g, guess, prm, P, iters, methods, 0.0);
}
