/*
 * mlp.c -- oracle of the learned Newton starting point for the inversion of
 * Section 2.3: the invariants of the conserved state that the network reads,
 * the seeded training samples, and a 5-64-64-1 ReLU network with its loss,
 * gradient and AdamW update, all in FP64.
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 *
 * Definitions shared with the CUDA path (none of them is printed in the
 * paper, which only names the Newton starting point; they are this
 * implementation's choices and are listed with the readings of the paper):
 *
 *   Features, from the Noble et al. variables of Section 2.3 (D, Q_mu, Qt^2,
 *   Bf^i, Q.Bf) with tau = -n.Q - D:
 *     f0 = log(tau/D), f1 = log(Qt^2/D^2), f2 = log(Bf^2/D),
 *     f3 = log((Q.Bf)^2/D^3), f4 = log(D);
 *   every argument clamped below at 1e-30.  f0..f3 are invariant under the
 *   scaling D, Q -> lambda D, lambda Q, Bf -> sqrt(lambda) Bf, under which
 *   W/D is invariant too (the homogeneity of Eqs. 29-31).
 *   Target: y = log(W/D) with W = Gamma^2 (rho + u + p).
 *
 *   Network (parameter vector theta, 4609 entries, in this order):
 *     W1[64][5], b1[64], W2[64][64], b2[64], W3[64], b3
 *   x = (f - mean_f)/std_f; h1 = relu(W1 x + b1); h2 = relu(W2 h1 + b2);
 *   s = W3 h2 + b3; prediction y = s*std_y + mean_y.  The weight matrices
 *   enter the forward pass rounded to BF16 (round to nearest even); biases,
 *   inputs and activations are not rounded.  norm[12] = mean_f[5], std_f[5],
 *   mean_y, std_y.
 *
 *   Loss over a batch of n: L = (1/n) sum (s - t)^2, t = (y - mean_y)/std_y.
 *   The gradient of a weight is taken with respect to its BF16 value and
 *   applied to the FP32 master copy (straight-through rounding).
 *
 *   AdamW (Kingma & Ba 2015 with the decoupled weight decay of Loshchilov &
 *   Hutter 2019), bias-corrected moments; decay on W1, W2, W3 only.
 *
 *   Samples: sample i draws xi_k = top 53 bits of splitmix64(seed ^ (16 i + k))
 *   for k = 0..9 and sets
 *     zone (i1, j1) = (floor(xi_0 n1), floor(xi_1 n2)) of the grid, centre metric;
 *     rho = 1e-6^(1 - xi_2); u/rho = 1e-4 * 1e5^xi_3; Gamma = 50^xi_4;
 *     sigma = b^2/rho = 1e-3 * 1e5^xi_5;
 *     velocity direction: cos(th) = 2 xi_6 - 1, ph = 2 pi xi_7, components
 *       e^i / sqrt(g_ii), scaled so that g_ij ut^i ut^j = Gamma^2 - 1;
 *     field direction: cos(th) = 2 xi_8 - 1, ph = 2 pi xi_9, components
 *       e^i / sqrt(g_ii), scaled so that b^2 = sigma rho.
 */
#include <math.h>
#include <string.h>
#include "orc.h"

#define MLP_H 64
#define MLP_IN 5
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + MLP_H * MLP_IN)
#define OFF_W2 (OFF_B1 + MLP_H)
#define OFF_B2 (OFF_W2 + MLP_H * MLP_H)
#define OFF_W3 (OFF_B2 + MLP_H)
#define OFF_B3 (OFF_W3 + MLP_H)
#define NPARAM (OFF_B3 + 1)

int orc_mlp_nparam(void) { return NPARAM; }

/* round to the nearest BF16 value, ties to even (IEEE 754 binary32 ->
 * the upper 16 bits); NaN stays NaN */
float orc_bf16_round(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu)) {
        u |= 0x00400000u;
    } else {
        uint32_t lsb = (u >> 16) & 1u;
        u += 0x7FFFu + lsb;
    }
    u &= 0xFFFF0000u;
    float y;
    memcpy(&y, &u, 4);
    return y;
}

static double clamp_log(double v) { return log(v > 1e-30 ? v : 1e-30); }

/* Section 2.3 variables of one conserved state (U includes sqrt(-g)) */
int orc_mlp_features(const double U[ORC_NU], const orc_geom *g, double feat[5])
{
    double f = g->alpha / g->gdet;
    double D = f * U[KRHO];
    if (!(D > 0.0) || !isfinite(D)) {
        for (int k = 0; k < 5; k++) feat[k] = 0.0;
        return -1;
    }
    double Q[4] = {f * U[1], f * U[2], f * U[3], f * U[4]};
    /* n^mu = (1/alpha, -alpha g^{ti}) */
    double ncon[4] = {1.0 / g->alpha, -g->alpha * g->gcon[0][1], -g->alpha * g->gcon[0][2],
                      -g->alpha * g->gcon[0][3]};
    double nQ = 0.0, Qsq = 0.0;
    for (int m = 0; m < 4; m++) {
        nQ += ncon[m] * Q[m];
        for (int n = 0; n < 4; n++) Qsq += g->gcon[m][n] * Q[m] * Q[n];
    }
    double Qt2 = Qsq + nQ * nQ; /* j^{mu nu} Q_mu Q_nu */
    double Bf[3];
    for (int i = 0; i < 3; i++) Bf[i] = g->alpha * U[KB1 + i] / g->gdet;
    double B2 = 0.0, QB = 0.0;
    for (int i = 0; i < 3; i++) {
        QB += Q[i + 1] * Bf[i];
        for (int j = 0; j < 3; j++) B2 += g->gcov[i + 1][j + 1] * Bf[i] * Bf[j];
    }
    double tau = -nQ - D;
    feat[0] = clamp_log(tau / D);
    feat[1] = clamp_log(Qt2 / (D * D));
    feat[2] = clamp_log(B2 / D);
    feat[3] = clamp_log(QB * QB / (D * D * D));
    feat[4] = log(D);
    return 0;
}

/* One training sample of the seeded distribution at a zone-centre metric of
 * the grid; any output may be NULL. */
int orc_mlp_sample(const orc_grid *G, uint64_t seed, long i, double P[ORC_NP], int *loc,
                   double U[ORC_NU], double feat[5], double *label)
{
    double xi[10];
    for (int k = 0; k < 10; k++) xi[k] = orc_uniform(seed, 16ull * (uint64_t)i + (uint64_t)k);
    int n1 = G->p.n1, n2 = G->p.n2;
    int i1 = (int)(xi[0] * n1), j1 = (int)(xi[1] * n2);
    if (i1 > n1 - 1) i1 = n1 - 1;
    if (j1 > n2 - 1) j1 = n2 - 1;
    const orc_geom *g = &G->gc[orc_midx(G, i1, j1)];
    double rho = exp(log(1e-6) * (1.0 - xi[2]));
    double uu = rho * 1e-4 * exp(log(1e5) * xi[3]);
    double lor = exp(log(50.0) * xi[4]);
    double sigma = 1e-3 * exp(log(1e5) * xi[5]);

    double q[ORC_NP];
    q[KRHO] = rho;
    q[KUU] = uu;
    double e[3], n2u = 0.0;
    {
        double ct = 2.0 * xi[6] - 1.0, st = sqrt(fmax(0.0, 1.0 - ct * ct)), ph = 2.0 * M_PI * xi[7];
        double d[3] = {st * cos(ph), st * sin(ph), ct};
        for (int a = 0; a < 3; a++) e[a] = d[a] / sqrt(g->gcov[a + 1][a + 1]);
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) n2u += g->gcov[a + 1][b + 1] * e[a] * e[b];
    }
    double us = sqrt(lor * lor - 1.0) / sqrt(n2u);
    for (int a = 0; a < 3; a++) q[KU1 + a] = us * e[a];
    {
        double ct = 2.0 * xi[8] - 1.0, st = sqrt(fmax(0.0, 1.0 - ct * ct)), ph = 2.0 * M_PI * xi[9];
        double d[3] = {st * cos(ph), st * sin(ph), ct};
        for (int a = 0; a < 3; a++) q[KB1 + a] = d[a] / sqrt(g->gcov[a + 1][a + 1]);
    }
    orc_state s;
    orc_state_of(q, g, &s);
    double lam = sqrt(sigma * rho / s.bsq);
    for (int a = 0; a < 3; a++) q[KB1 + a] *= lam;
    orc_state_of(q, g, &s);

    double Uz[ORC_NU], f[5];
    orc_prim_to_U(q, g, &s, G->p.gam, Uz);
    orc_mlp_features(Uz, g, f);
    double D = g->alpha * Uz[KRHO] / g->gdet;
    double W = s.gamma * s.gamma * (rho + uu + (G->p.gam - 1.0) * uu);
    if (P)
        for (int c = 0; c < ORC_NP; c++) P[c] = q[c];
    if (loc) *loc = i1 * n2 + j1;
    if (U)
        for (int c = 0; c < ORC_NU; c++) U[c] = Uz[c];
    if (feat)
        for (int k = 0; k < 5; k++) feat[k] = f[k];
    if (label) *label = log(W / D);
    return 0;
}

void orc_mlp_samples(const orc_grid *G, uint64_t seed, long first, long n, double *P, int *loc,
                     double *U, double *feat, double *label)
{
    for (long a = 0; a < n; a++) {
        double q[ORC_NP], Uz[ORC_NU], f[5], y;
        int l;
        orc_mlp_sample(G, seed, first + a, q, &l, Uz, f, &y);
        if (P)
            for (int c = 0; c < ORC_NP; c++) P[c * n + a] = q[c];
        if (loc) loc[a] = l;
        if (U)
            for (int c = 0; c < ORC_NU; c++) U[c * n + a] = Uz[c];
        if (feat)
            for (int k = 0; k < 5; k++) feat[k * n + a] = f[k];
        if (label) label[a] = y;
    }
}

/* ------------------------------------------------------------ network */

typedef struct {
    double x[MLP_IN], a1[MLP_H], h1[MLP_H], a2[MLP_H], h2[MLP_H], s;
} fwd_cache;

/* weights as the forward pass sees them: BF16-rounded matrices, FP32 biases */
static void eff_params(const float *theta, double *w)
{
    for (int k = 0; k < NPARAM; k++) {
        int is_bias = (k >= OFF_B1 && k < OFF_W2) || (k >= OFF_B2 && k < OFF_W3) || k == OFF_B3;
        w[k] = is_bias ? (double)theta[k] : (double)orc_bf16_round(theta[k]);
    }
}

static void forward(const double *w, const float *norm, const float f[5], fwd_cache *c)
{
    for (int i = 0; i < MLP_IN; i++) c->x[i] = ((double)f[i] - (double)norm[i]) / (double)norm[5 + i];
    for (int o = 0; o < MLP_H; o++) {
        double a = w[OFF_B1 + o];
        for (int i = 0; i < MLP_IN; i++) a += w[OFF_W1 + o * MLP_IN + i] * c->x[i];
        c->a1[o] = a;
        c->h1[o] = a > 0.0 ? a : 0.0;
    }
    for (int o = 0; o < MLP_H; o++) {
        double a = w[OFF_B2 + o];
        for (int i = 0; i < MLP_H; i++) a += w[OFF_W2 + o * MLP_H + i] * c->h1[i];
        c->a2[o] = a;
        c->h2[o] = a > 0.0 ? a : 0.0;
    }
    double s = w[OFF_B3];
    for (int o = 0; o < MLP_H; o++) s += w[OFF_W3 + o] * c->h2[o];
    c->s = s;
}

/* predictions y = log(W/D) of n feature vectors (feat field-major, 5 x n) */
void orc_mlp_forward(const float *theta, const float *norm, const float *feat, long n, double *y)
{
    double w[NPARAM];
    eff_params(theta, w);
    for (long a = 0; a < n; a++) {
        float f[5];
        for (int k = 0; k < 5; k++) f[k] = feat[k * n + a];
        fwd_cache c;
        forward(w, norm, f, &c);
        y[a] = c.s * (double)norm[11] + (double)norm[10];
    }
}

/* L = mean (s - t)^2 and dL/dw by reverse-mode differentiation, with the
 * weights w used as given (no rounding) */
double orc_mlp_loss_grad_d(const double *w, const float *norm, const float *feat, const float *label,
                           long n, double *grad)
{
    for (int k = 0; k < NPARAM; k++) grad[k] = 0.0;
    double loss = 0.0;
    for (long a = 0; a < n; a++) {
        float f[5];
        for (int k = 0; k < 5; k++) f[k] = feat[k * n + a];
        fwd_cache c;
        forward(w, norm, f, &c);
        double t = ((double)label[a] - (double)norm[10]) / (double)norm[11];
        double r = c.s - t;
        loss += r * r;
        double ds = 2.0 * r / (double)n;
        double d2[MLP_H], d1[MLP_H];
        grad[OFF_B3] += ds;
        for (int o = 0; o < MLP_H; o++) {
            grad[OFF_W3 + o] += ds * c.h2[o];
            d2[o] = c.a2[o] > 0.0 ? ds * w[OFF_W3 + o] : 0.0;
        }
        for (int i = 0; i < MLP_H; i++) {
            double acc = 0.0;
            for (int o = 0; o < MLP_H; o++) acc += w[OFF_W2 + o * MLP_H + i] * d2[o];
            d1[i] = c.a1[i] > 0.0 ? acc : 0.0;
        }
        for (int o = 0; o < MLP_H; o++) {
            grad[OFF_B2 + o] += d2[o];
            for (int i = 0; i < MLP_H; i++) grad[OFF_W2 + o * MLP_H + i] += d2[o] * c.h1[i];
        }
        for (int o = 0; o < MLP_H; o++) {
            grad[OFF_B1 + o] += d1[o];
            for (int i = 0; i < MLP_IN; i++) grad[OFF_W1 + o * MLP_IN + i] += d1[o] * c.x[i];
        }
    }
    return loss / (double)n;
}

/* the same with the FP32 parameters as the forward pass sees them */
double orc_mlp_loss_grad(const float *theta, const float *norm, const float *feat, const float *label,
                         long n, double *grad)
{
    double w[NPARAM];
    eff_params(theta, w);
    return orc_mlp_loss_grad_d(w, norm, feat, label, n, grad);
}

static int decayed(int k) { return (k >= OFF_W1 && k < OFF_B1) || (k >= OFF_W2 && k < OFF_B2) || (k >= OFF_W3 && k < OFF_B3); }

/* one AdamW step (step = 1, 2, ...) on theta with moments m, v */
void orc_mlp_adamw(double *theta, double *m, double *v, const double *grad, long step, double lr,
                   double beta1, double beta2, double eps, double wd)
{
    double c1 = 1.0 - pow(beta1, (double)step), c2 = 1.0 - pow(beta2, (double)step);
    for (int k = 0; k < NPARAM; k++) {
        double g = grad[k];
        m[k] = beta1 * m[k] + (1.0 - beta1) * g;
        v[k] = beta2 * v[k] + (1.0 - beta2) * g * g;
        double mh = m[k] / c1, vh = v[k] / c2;
        if (decayed(k)) theta[k] -= lr * wd * theta[k];
        theta[k] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* nsteps of minibatch AdamW at constant lr; step s uses samples
 * (s*batch + b) mod n, b < batch.  theta is read and written as FP32 (the
 * master copy), the moments start at zero. */
double orc_mlp_train_steps(float *theta, const float *norm, const float *feat, const float *label, long n,
                           long batch, long nsteps, double lr, double beta1, double beta2, double eps,
                           double wd, float *fb, float *lb, double *work)
{
    double *th = work, *m = work + NPARAM, *v = work + 2 * NPARAM, *g = work + 3 * NPARAM;
    for (int k = 0; k < NPARAM; k++) {
        th[k] = theta[k];
        m[k] = v[k] = 0.0;
    }
    double loss = 0.0;
    for (long s = 0; s < nsteps; s++) {
        for (long b = 0; b < batch; b++) {
            long a = (s * batch + b) % n;
            for (int k = 0; k < 5; k++) fb[k * batch + b] = feat[k * n + a];
            lb[b] = label[a];
        }
        float tf[NPARAM];
        for (int k = 0; k < NPARAM; k++) tf[k] = (float)th[k];
        loss = orc_mlp_loss_grad(tf, norm, fb, lb, batch, g);
        orc_mlp_adamw(th, m, v, g, s + 1, lr, beta1, beta2, eps, wd);
    }
    for (int k = 0; k < NPARAM; k++) theta[k] = (float)th[k];
    return loss;
}

/* batched inversion with an explicit Newton starting W per zone (<= 0: plain) */
void orc_c2p_batch_w(const orc_grid *G, const double *U, const int *loc, const double *guess,
                     const double *wguess, double *P, int *flags, int *iters, long n, int methods)
{
    for (long a = 0; a < n; a++) {
        int l = loc[a];
        const orc_geom *g = &G->gc[orc_midx(G, l / G->p.n2, l % G->p.n2)];
        double Uz[ORC_NU], q0[ORC_NP], q[ORC_NP];
        for (int c = 0; c < ORC_NU; c++) Uz[c] = U[c * n + a];
        for (int c = 0; c < ORC_NP; c++) q0[c] = guess[c * n + a];
        int it;
        flags[a] = orc_con2prim_w(Uz, g, q0, &G->p, q, &it, methods, wguess ? wguess[a] : 0.0);
        if (iters) iters[a] = it;
        for (int c = 0; c < ORC_NP; c++) P[c * n + a] = q[c];
    }
}
