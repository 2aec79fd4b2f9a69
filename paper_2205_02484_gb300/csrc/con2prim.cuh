// con2prim.cuh -- device conserved-to-primitive inversion, Section 2.3 of
// the paper (Noble et al. 2006 variables), always in FP64.
//
// Unknowns W = Gamma^2 h and v^2 solve
//   (Eq. 29) Qt^2 = v^2 (Bf^2 + W)^2 - (Q.Bf)^2 (Bf^2 + 2W) / W^2
//   (Eq. 30) Q.n  = -Bf^2/2 (1 + v^2) + (Q.Bf)^2 / (2 W^2) - W + p(W, v^2)
//   (Eq. 31) p    = (gam-1)/gam [W (1 - v^2) - D sqrt(1 - v^2)]
// Method order: 2D Newton (tolerance nr_tol) -> if not converged, Brent in W
// with v^2(W) from Eq. 29 -> if that fails, or if Newton gives unphysical
// values, entropy inversion (W(v^2) of Eq. 32 into Eq. 29, Brent in v^2);
// entropy alone where the guess has beta < beta_ent.  The sign of the Bf^2
// term of Eq. 30 is taken as minus (static magnetised fluid), and S of
// Eq. 32 is the normal-frame entropy density alpha U_S / sqrt(-g).
//
// Cost on GB300 is set by the FP64 pipe (1/64 of the FP32 rate), so the
// Newton step is written with three reciprocals (1/W, 1/sqrt(1-v^2), 1/det)
// instead of a division per term.  In the FP64 path Newton takes one more
// step after the tolerance is met (so that the oracle and this code stop on
// the same rounding-level root); the mixed path (c2p_newton_mixed) keeps the
// residuals in FP64 but forms the Newton step in FP32 and stops at
// sqrt(tol).
#pragma once
#include "mlp.cuh"
#include "physics.cuh"

namespace grmhd {

constexpr int C2P_NR = 0, C2P_BRENT_W = 1, C2P_ENTROPY = 2, C2P_ENTROPY_BETA = 3;
constexpr int C2P_FAIL = 8, C2P_FAIL_D = 16, C2P_FAIL_ENT = 32;
constexpr int C2P_LEARNED = 64; // with C2P_NR: Newton converged from the learned start
// internal: a first pass (pass = 1) stops where the chain would leave Newton
// and returns C2P_DEFER with the step to resume at (pass = 2, resume = that
// value): the entropy inversion of a low-beta zone, the entropy inversion
// after an unphysical Newton root (P then holds that root's primitives, as
// the whole chain leaves them), or Brent in W followed by the entropy
// inversion
constexpr int C2P_DEFER = 256, C2P_DEFER_BETA = 512, C2P_DEFER_ENT = 1024, C2P_DEFER_TAIL = 2048;
constexpr double V2MAX = 1.0 - 1.0e-16;

struct C2PIn {
    double D, Qtsq, Bsq, QB, nQ, Sent, gam, g1, igm1; // g1 = (gam-1)/gam, igm1 = 1/(gam-1)
    double Qt[3], Bf[3];
};

// solver parameters of a grid; the EOS ratios and the mixed path's Newton
// acceptance sqrt(tol) are formed once on the host
struct C2PPar {
    double gam, g1, igm1, beta_ent, tol, tol_mixed, ig; // ig = 1/gam
    int nr_maxit, brent_maxit;
    float gam_f, g1_f, beta_ent_f, tol_mixed_f; // FP32 copies for the mixed path
};

__device__ __forceinline__ C2PPar c2p_par(const Grid &g)
{
    return C2PPar{g.gam,      g.g1,          g.igm1,  g.beta_ent, g.nr_tol,   g.nr_tol_mixed, g.ig,
                  g.nr_maxit, g.brent_maxit, g.gam_f, g.g1_f,     g.beta_ent_f, g.tol_mixed_f};
}

// finite test on the high word: integer pipe instead of an FP64 compare
__device__ __forceinline__ bool finite64(double x)
{
    return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000;
}

// Newton starting W from the network for the inversion with invariants c:
// the features of mlp.cuh formed in FP32 from the FP64 D, Q.n, Qt^2, Bf^2
// and Q.Bf the inversion has already computed (tau = -Q.n - D subtracted in
// FP64: it is the small difference of two large numbers for cold gas); the
// log of a ratio is the difference of logs, clamped at log(1e-30) as the
// ratio itself would be.  0 when the features are undefined.  Out of line:
// the network's loops stay out of the register allocation of the update
// kernel, which reaches this only for the rare zones Newton did not settle.
// (Measured: with c passed by reference the mixed update runs 168.8 FP64-pipe
// warp slots per zone-stage against 185.3 with the invariants passed by
// value -- the same thread-level work, better reconvergence of the divergent
// Newton steps -- so the reference is kept.)
__device__ __forceinline__ void c2p_learned_features(const C2PIn &c, float f[MLP_IN])
{
    const float lo = -69.07755279f; // log(1e-30)
    const float lD = __logf((float)c.D);
    f[0] = fmaxf(__logf((float)(-c.nQ - c.D)) - lD, lo);
    f[1] = fmaxf(__logf((float)c.Qtsq) - 2.0f * lD, lo);
    f[2] = fmaxf(__logf((float)c.Bsq) - lD, lo);
    const float qb = (float)c.QB;
    f[3] = fmaxf(__logf(qb * qb) - 3.0f * lD, lo);
    f[4] = lD;
#pragma unroll
    for (int k = 0; k < MLP_IN; k++)
        if (!(f[k] == f[k])) f[k] = lo; // a NaN feature (negative argument) takes the clamp
}

// W = D exp(y) of a network output y, 0 where it is not a positive finite number
__device__ __forceinline__ double c2p_w_of(double D, float y)
{
    const float w = (float)D * __expf(y);
    return (w > 0.0f && w < INFINITY) ? (double)w : 0.0;
}

static __device__ __noinline__ double c2p_learned_w(const float *buf, const C2PIn &c)
{
    float f[MLP_IN];
    c2p_learned_features(c, f);
    return c2p_w_of(c.D, mlp_log_w_guess(buf, f));
}

// The invariants the features need (D, n.Q, Qt^2, Bf^2, Q.Bf), formed as the
// FP64 inversion forms them; false where D is not a positive finite number
__device__ inline bool c2p_feature_invariants(const double U[NU], const Geo<double> &g, const double gsp[6],
                                              C2PIn &c)
{
    const double f = g.aig;
    c.D = f * U[KRHO];
    const double Q0 = f * U[1], Q1 = f * U[2], Q2 = f * U[3], Q3 = f * U[4];
    c.nQ = g.ialpha * Q0 - g.alpha * (g.gcon[1] * Q1 + g.gcon[2] * Q2 + g.gcon[3] * Q3);
    const double t0 = gsp[0] * Q1 + gsp[1] * Q2 + gsp[2] * Q3;
    const double t1 = gsp[1] * Q1 + gsp[3] * Q2 + gsp[4] * Q3;
    const double t2 = gsp[2] * Q1 + gsp[4] * Q2 + gsp[5] * Q3;
    c.Qtsq = t0 * Q1 + t1 * Q2 + t2 * Q3;
    const double b0 = g.alpha * (U[KB1] * g.igdet), b1 = g.alpha * (U[KB2] * g.igdet), b2 = g.alpha * (U[KB3] * g.igdet);
    c.QB = Q1 * b0 + Q2 * b1 + Q3 * b2;
    c.Bsq = spatial_sq(g, b0, b1, b2);
    return c.D > 0.0 && finite64(c.D) && finite64(c.nQ) && finite64(c.Qtsq) && finite64(c.Bsq) && finite64(c.QB);
}

__device__ __forceinline__ double c2p_pressure(const C2PIn &c, double W, double v2)
{
    return c.g1 * (W * (1.0 - v2) - c.D * sqrt(1.0 - v2));
}

// primitives from (W, v^2) and the pressure; ut^i = Gamma/(W+B^2) (Qt^i + (Q.B) B^i / W)
__device__ __forceinline__ void c2p_recover(const C2PIn &c, double W, double v2, double p, double *P)
{
    double omv = 1.0 - v2;
    double lor = rsqrt(omv);
    P[KRHO] = c.D * (omv * lor);
    P[KUU] = p * c.igm1;
    // 1/(W + B^2) and 1/W from one reciprocal
    double WB = W + c.Bsq;
    double r = 1.0 / (W * WB);
    double f = lor * (W * r);
    double qbw = c.QB * (WB * r);
#pragma unroll
    for (int i = 0; i < 3; i++) P[KU1 + i] = f * (c.Qt[i] + qbw * c.Bf[i]);
}

// c2p_recover with the pressure of Eq. 31, sharing 1 - v^2 and its inverse
// square root: sqrt(1 - v^2) = (1 - v^2) / sqrt(1 - v^2)
__device__ __forceinline__ void c2p_recover_w(const C2PIn &c, double W, double v2, double *P)
{
    double omv = 1.0 - v2;
    double lor = rsqrt(omv);
    double s = omv * lor;
    P[KRHO] = c.D * s;
    P[KUU] = (c.g1 * (W * omv - c.D * s)) * c.igm1;
    double WB = W + c.Bsq;
    double r = 1.0 / (W * WB);
    double f = lor * (W * r);
    double qbw = c.QB * (WB * r);
#pragma unroll
    for (int i = 0; i < 3; i++) P[KU1 + i] = f * (c.Qt[i] + qbw * c.Bf[i]);
}

// c2p_recover_w for the mixed path, whose primitives are stored in FP32: rho
// and u (the difference of W (1 - v^2) and D sqrt(1 - v^2)) in FP64, the
// velocity factors Gamma / (W + B^2) and (Q.B) / W from an FP32 reciprocal
// of W (W + B^2), relative error ~1e-7 like the FP32 store itself
__device__ __forceinline__ void c2p_recover_mixed(const C2PIn &c, double W, double v2, double ig, double *P)
{
    double omv = 1.0 - v2;
    double lor = rsqrt(omv);
    double s = omv * lor;
    P[KRHO] = c.D * s;
    P[KUU] = (W * omv - c.D * s) * ig; // p / (gam - 1) = (W (1 - v^2) - D sqrt(1 - v^2)) / gam
    double WB = W + c.Bsq;
    double r = (double)(1.0f / (float)(W * WB));
    double f = lor * (W * r);
    double qbw = c.QB * (WB * r);
#pragma unroll
    for (int i = 0; i < 3; i++) P[KU1 + i] = f * (c.Qt[i] + qbw * c.Bf[i]);
}

__device__ __forceinline__ bool c2p_physical(const double *P, double v2)
{
    bool fin = finite64(P[0]) && finite64(P[1]) && finite64(P[2]) && finite64(P[3]) && finite64(P[4]);
    // finite doubles: x > 0 exactly when the signed 64-bit pattern is > 0
    // 0 <= v2 < 1 on the bit pattern: +-0, or a positive value below 1.0's bits
    const long long vb = __double_as_longlong(v2);
    const bool v2ok = (vb << 1) == 0 || (unsigned long long)vb < 0x3FF0000000000000ULL;
    return fin && __double_as_longlong(P[KRHO]) > 0 && __double_as_longlong(P[KUU]) > 0 && v2ok;
}

// Brent's bracketing root finder (Brent 1973): bisection safeguarded
// secant / inverse-quadratic steps, stopping at |bracket|/2 <= 2 eps |b| + tol/2.
template <typename Fn>
__device__ double brent_root(const Fn &f, double a, double b, double fa, double fb, double tol,
                             int maxit, bool &ok)
{
    const double eps = 2.220446049250313e-16;
    ok = false;
    if ((fa > 0.0 && fb > 0.0) || (fa < 0.0 && fb < 0.0)) return b;
    if (fa == 0.0) { ok = true; return a; }
    if (fb == 0.0) { ok = true; return b; }
    double c = a, fc = fa, d = b - a, e = d;
    for (int it = 0; it < maxit; it++) {
        if ((fb > 0.0) == (fc > 0.0) && fb != 0.0 && fc != 0.0) {
            c = a;
            fc = fa;
            d = b - a;
            e = d;
        }
        if (fabs(fc) < fabs(fb)) {
            a = b; b = c; c = a;
            fa = fb; fb = fc; fc = fa;
        }
        double tol1 = 2.0 * eps * fabs(b) + 0.5 * tol;
        double xm = 0.5 * (c - b);
        if (fabs(xm) <= tol1 || fb == 0.0) { ok = true; return b; }
        bool bisect = true;
        if (fabs(e) >= tol1 && fabs(fa) > fabs(fb)) {
            double s = fb / fa, p, q;
            if (a == c) {
                p = 2.0 * xm * s;
                q = 1.0 - s;
            } else {
                double qa = fa / fc, r = fb / fc;
                p = s * (2.0 * xm * qa * (qa - r) - (b - a) * (r - 1.0));
                q = (qa - 1.0) * (r - 1.0) * (s - 1.0);
            }
            if (p > 0.0) q = -q;
            else p = -p;
            double lim = fmin(3.0 * xm * q - fabs(tol1 * q), fabs(e * q));
            if (2.0 * p < lim) {
                e = d;
                d = p / q;
                bisect = false;
            }
        }
        if (bisect) {
            d = xm;
            e = d;
        }
        a = b;
        fa = fb;
        b += (fabs(d) > tol1) ? d : (xm > 0.0 ? tol1 : -tol1);
        fb = f(b);
        if (!isfinite(fb)) return b;
    }
    return b;
}

struct ResidW {
    const C2PIn *c;
    __device__ double v2(double W) const
    {
        double BW = c->Bsq + W;
        double v = (c->Qtsq + c->QB * c->QB * (c->Bsq + 2.0 * W) / (W * W)) / (BW * BW);
        return fmin(fmax(v, 0.0), V2MAX);
    }
    __device__ double operator()(double W) const
    {
        double v = v2(W);
        return -0.5 * c->Bsq * (1.0 + v) + c->QB * c->QB / (2.0 * W * W) - W + c2p_pressure(*c, W, v) -
               c->nQ;
    }
};

// rho^(gam - 1) of the entropy inversion: cube roots for the adiabatic
// indices 4/3, 5/3 and 13/9 (rho^(1/3), rho^(2/3), rho^(4/9) = cbrt(cbrt(rho))^4),
// a general power otherwise; the Brent iteration evaluates it once per step
__device__ __forceinline__ double rho_pow_gm1(double rho, double gam)
{
    if (gam == 4.0 / 3.0) return cbrt(rho);
    if (gam == 5.0 / 3.0) {
        const double r = cbrt(rho);
        return r * r;
    }
    if (gam == 13.0 / 9.0) {
        const double r = cbrt(cbrt(rho)), r2 = r * r;
        return r2 * r2;
    }
    return pow(rho, gam - 1.0);
}

struct ResidS {
    const C2PIn *c;
    __device__ double W(double v2) const
    {
        double lor = 1.0 / sqrt(1.0 - v2);
        double rho = c->D / lor;
        return lor * c->D + lor * c->gam * c->igm1 * rho_pow_gm1(rho, c->gam) * c->Sent;
    }
    __device__ double operator()(double v2) const
    {
        double w = W(v2);
        double BW = c->Bsq + w;
        return v2 * BW * BW - c->QB * c->QB * (c->Bsq + 2.0 * w) / (w * w) - c->Qtsq;
    }
};

template <bool EXTRA>
__device__ inline bool c2p_newton(const C2PIn &c, double &W, double &v2, double tol, int maxit,
                                  int &iters)
{
    const double g1 = c.g1;
    const double QB2 = c.QB * c.QB;
    bool extra = false;
    int n = 0;
    for (int it = 1; it <= maxit; it++) {
        n = it;
        double omv = 1.0 - v2;
        double is = rsqrt(omv); // 1 / sqrt(1 - v^2)
        double s = omv * is;
        double iW = 1.0 / W;
        double qw2 = QB2 * iW * iW; // (Q.B)^2 / W^2
        double p = g1 * (W * omv - c.D * s);
        double BW = c.Bsq + W;
        double f1 = v2 * BW * BW - qw2 * (c.Bsq + 2.0 * W) - c.Qtsq;
        double f2 = -0.5 * c.Bsq * (1.0 + v2) + 0.5 * qw2 - W + p - c.nQ;
        double a11 = 2.0 * v2 * BW + 2.0 * qw2 * iW * BW;
        double a12 = BW * BW;
        double a21 = -qw2 * iW - 1.0 + g1 * omv;
        double a22 = -0.5 * c.Bsq + g1 * (-W + 0.5 * c.D * is);
        double det = a11 * a22 - a12 * a21;
        if (!finite64(det) || (__double_as_longlong(det) << 1) == 0) break; // non-finite or +-0
        double idet = 1.0 / det;
        double dW = -(a22 * f1 - a12 * f2) * idet;
        double dv = -(-a21 * f1 + a11 * f2) * idet;
        double Wn = W + dW;
        if (!(Wn > 0.0)) Wn = 0.5 * W;
        double vn = fmin(fmax(v2 + dv, 0.0), V2MAX);
        bool conv = fabs(Wn - W) < tol * fabs(Wn) && fabs(vn - v2) < tol;
        W = Wn;
        v2 = vn;
        if (!finite64(W) || !finite64(v2)) break;
        if (extra) {
            iters = n;
            return true;
        }
        if (conv) {
            if (!EXTRA) {
                iters = n;
                return true;
            }
            extra = true;
        }
    }
    iters = n;
    return false;
}

// Newton for the mixed path: the residuals of Eqs. 29-30 in FP64 (they fix
// the root), the Jacobian, its inverse and the step in FP32 -- iterative
// refinement: the fixed point is still the FP64 root, and an FP32 Jacobian
// (relative error ~1e-7, ~1e-4 at the Lorentz cap) turns the quadratic
// convergence into a linear one of that rate, from starts already within
// ~1e-5.  Accepts once the step is below tol (sqrt(nr_tol)), tested in FP32.
// An iteration whose FP32 determinant is not a normal number takes the FP64
// step instead.
__device__ inline bool c2p_newton_mixed(const C2PIn &c, const C2PPar &par, double &W, double &v2, int &iters)
{
    const double g1 = c.g1, tol = par.tol_mixed;
    const int maxit = par.nr_maxit;
    const double QB2 = c.QB * c.QB;
    const bool has_qb = (__double_as_longlong(QB2) << 1) != 0; // Q.B != 0 (integer test)
    const float g1f = par.g1_f, Bsqf = (float)c.Bsq, Df = (float)c.D, tolf = par.tol_mixed_f;
    const float QB2f = has_qb ? (float)QB2 : 0.0f;
    const long long v2max_bits = __double_as_longlong(V2MAX);
    int n = 0;
    for (int it = 1; it <= maxit; it++) {
        n = it;
        double omv = 1.0 - v2;
        double is = rsqrt(omv); // 1 / sqrt(1 - v^2)
        double s = omv * is;
        double iW = 0.0, qw2 = 0.0; // (Q.B)^2 / W^2, no reciprocal where Q.B = 0 (no field)
        if (has_qb) {
            iW = 1.0 / W;
            qw2 = QB2 * iW * iW;
        }
        double p = g1 * (W * omv - c.D * s);
        double BW = c.Bsq + W;
        double f1 = v2 * BW * BW - qw2 * (c.Bsq + 2.0 * W) - c.Qtsq;
        double f2 = -0.5 * c.Bsq * (1.0 + v2) + 0.5 * qw2 - W + p - c.nQ;
        // the Jacobian's inputs formed in FP32 from the FP32 (W, v^2): only the
        // step's rate of convergence depends on them, not the root
        const float Wf = (float)W, v2f = (float)v2, omvf = 1.0f - v2f;
        const float isf = rsqrtf(omvf), iWf = 1.0f / Wf, BWf = Bsqf + Wf;
        const float qw2f = QB2f * iWf * iWf;
        const float a11 = 2.0f * v2f * BWf + 2.0f * qw2f * iWf * BWf;
        const float a12 = BWf * BWf;
        const float a21 = -qw2f * iWf - 1.0f + g1f * omvf;
        const float a22 = -0.5f * Bsqf + g1f * (-Wf + 0.5f * Df * isf);
        const float det = a11 * a22 - a12 * a21;
        double dW, dv;
        bool small;
        if (fabsf(det) >= 1.17549435e-38f && fabsf(det) < INFINITY) {
            const float idet = 1.0f / det, f1f = (float)f1, f2f = (float)f2;
            const float dWf = -(a22 * f1f - a12 * f2f) * idet;
            const float dvf = -(-a21 * f1f + a11 * f2f) * idet;
            dW = (double)dWf;
            dv = (double)dvf;
            small = fabsf(dWf) < tolf * fabsf(Wf + dWf) && fabsf(dvf) < tolf;
        } else {
            double b11 = 2.0 * v2 * BW + 2.0 * qw2 * iW * BW;
            double b12 = BW * BW;
            double b21 = -qw2 * iW - 1.0 + g1 * omv;
            double b22 = -0.5 * c.Bsq + g1 * (-W + 0.5 * c.D * is);
            double d64 = b11 * b22 - b12 * b21;
            if (!finite64(d64) || (__double_as_longlong(d64) << 1) == 0) break; // non-finite or +-0
            double idet = 1.0 / d64;
            dW = -(b22 * f1 - b12 * f2) * idet;
            dv = -(-b21 * f1 + b11 * f2) * idet;
            small = fabs(dW) < tol * fabs(W + dW) && fabs(dv) < tol;
        }
        // the updates' sign and range tests on the bit patterns (integer pipe)
        double Wn = W + dW;
        if (__double_as_longlong(Wn) <= 0) { // W + dW <= 0 (or a negative NaN): halve W instead
            Wn = 0.5 * W;
            small = false;
        }
        W = Wn;
        double vn = v2 + dv;
        const long long vb = __double_as_longlong(vn);
        v2 = vb < 0 ? 0.0 : (vb > v2max_bits ? V2MAX : vn); // clamp to [0, V2MAX]
        if (!finite64(W)) break;
        if (small) {
            iters = n;
            return true;
        }
    }
    iters = n;
    return false;
}

__device__ inline bool c2p_brent_w(const C2PIn &c, int maxit, double *P)
{
    double E = -c.nQ;
    double lo = c.D, hi = c.gam * fmax(E, c.D) * (1.0 + 1e-10);
    if (!(lo > 0.0) || !(hi > lo)) return false;
    ResidW f{&c};
    bool ok;
    double W = brent_root(f, lo, hi, f(lo), f(hi), 0.0, maxit, ok);
    if (!ok) return false;
    double v2 = f.v2(W);
    c2p_recover_w(c, W, v2, P);
    return c2p_physical(P, v2);
}

__device__ inline bool c2p_entropy(const C2PIn &c, int maxit, double *P)
{
    if (!(c.Sent > 0.0) || !(c.D > 0.0)) return false;
    ResidS f{&c};
    double lo = 0.0, hi = 1.0 - 1.0e-12;
    double flo = f(lo);
    bool ok = true;
    double v2 = 0.0;
    // the residual at v^2 = 0 is <= 0 analytically; > 0 only by rounding => v^2 = 0
    if (flo < 0.0) v2 = brent_root(f, lo, hi, flo, f(hi), 1.0e-17, maxit, ok);
    if (!ok) return false;
    double lor = 1.0 / sqrt(1.0 - v2);
    double rho = c.D / lor;
    double p = (c.Sent / lor) * rho_pow_gm1(rho, c.gam);
    c2p_recover(c, f.W(v2), v2, p, P);
    return c2p_physical(P, v2);
}

// Full inversion of one zone.  U includes sqrt(-g); gsp = the spatial
// inverse metric gamma^{ij} of the zone (packed 11 12 13 22 23 33).
// Returns the C2P_* flag; P[5..7] always receive B = U_B / sqrt(-g), and on
// failure P[0..4] keep the guess (the fixups repair the zone).
// methods: 1 Newton, 2 Brent-W, 4 entropy, 8 beta switch (15 = paper order).
// mlp_first (network buffer or null): Newton first starts from the network's W
// (v^2 from Eq. 29) and, if it does not converge, from the guess primitives
// (for callers without a good guess).  mlp_rescue: Newton from the network's
// W is tried after Newton from the guess (and the extrapolated start) fails
// and before Brent; a zone it converges returns C2P_NR | C2P_LEARNED.
// w_first (> 0, with mlp_first null): a network W the caller has already
// formed (the warp-level tensor-core inference), tried as mlp_first's.
// FP64 path: guess = the previous FP64 primitives, Newton takes one more step
// after the tolerance.  MIXED: guessf = the previous FP32 primitives (guess
// unused); the starting (W, v^2) and the beta switch are formed in FP32 with
// the FP32 metric record gf, and Newton stops once its step is below
// sqrt(tol) -- quadratic convergence then leaves an error of order tol.
// startf (MIXED, used where have_start): FP32 primitives to start Newton from
// before the guess primitives (the update passes the stage input
// extrapolated by the change over the previous half step); the beta switch
// keeps guessf.
template <bool MIXED = false>
__device__ inline int con2prim(const double U[NU], const Geo<double> &g, const double gsp[6],
                               const double *guess, const float *guessf, const C2PPar &par, int methods,
                               double P[NP], int &iters, const float *mlp_first = nullptr,
                               const Geo<float> *gf = nullptr, const float *startf = nullptr,
                               bool have_start = false, const float *mlp_rescue = nullptr, double w_first = 0.0,
                               int pass = 0, int resume = 0)
{
    iters = 0;
    if (!MIXED) {
#pragma unroll
        for (int m = 0; m < 5; m++) P[m] = guess[m];
    }
    auto fail = [&](int code) {
        if (MIXED) {
#pragma unroll
            for (int m = 0; m < 5; m++) P[m] = (double)guessf[m];
        }
        return code;
    };
    const double f = g.aig;
#pragma unroll
    for (int i = 0; i < 3; i++) P[KB1 + i] = U[KB1 + i] * g.igdet;
    C2PIn c;
    c.gam = par.gam;
    c.g1 = par.g1;
    c.igm1 = par.igm1;
    c.D = f * U[KRHO];
    const double Q0 = f * U[1], Q1 = f * U[2], Q2 = f * U[3], Q3 = f * U[4];
    // the entropy density, needed only by the entropy inversion, is formed there
    c.Sent = 0.0;
    auto entropy = [&]() {
        c.Sent = f * U[KENT];
        return c2p_entropy(c, par.brent_maxit, P);
    };
    // n^mu = (1/alpha, -alpha g^{ti}); the projection j^{mu nu} = g^{mu nu} +
    // n^mu n^nu has j^{t mu} = 0 and j^{ij} = gamma^{ij}, so Qt^i = gamma^{ij} Q_j
    // and Qt^2 = Qt^i Q_i (no cancellation against the energy)
    c.nQ = g.ialpha * Q0 - g.alpha * (g.gcon[1] * Q1 + g.gcon[2] * Q2 + g.gcon[3] * Q3);
    c.Qt[0] = gsp[0] * Q1 + gsp[1] * Q2 + gsp[2] * Q3;
    c.Qt[1] = gsp[1] * Q1 + gsp[3] * Q2 + gsp[4] * Q3;
    c.Qt[2] = gsp[2] * Q1 + gsp[4] * Q2 + gsp[5] * Q3;
    c.Qtsq = c.Qt[0] * Q1 + c.Qt[1] * Q2 + c.Qt[2] * Q3;
    // Bf^i = alpha B^i = (alpha / sqrt(-g)) U_B^i (the mixed path uses the tabulated ratio).
    // A zone without field (all U_B bits zero but the sign) skips the field terms.
    const bool field = ((__double_as_longlong(U[KB1]) | __double_as_longlong(U[KB2]) |
                         __double_as_longlong(U[KB3])) << 1) != 0;
    if (field) {
#pragma unroll
        for (int i = 0; i < 3; i++) c.Bf[i] = MIXED ? f * U[KB1 + i] : g.alpha * P[KB1 + i];
        c.QB = Q1 * c.Bf[0] + Q2 * c.Bf[1] + Q3 * c.Bf[2];
        c.Bsq = spatial_sq(g, c.Bf[0], c.Bf[1], c.Bf[2]);
    } else {
        c.Bf[0] = c.Bf[1] = c.Bf[2] = 0.0;
        c.QB = 0.0;
        c.Bsq = 0.0;
    }
    bool fin = finite64(c.D) && finite64(c.Qtsq) && finite64(c.nQ) && finite64(c.Bsq);
    // a finite D is > 0 exactly when its signed bit pattern is (integer test)
    if (!fin || __double_as_longlong(c.D) <= 0) return fail(C2P_FAIL | C2P_FAIL_D);
    if (!MIXED && pass == 2) {
        // the rest of the chain from the step a first pass deferred
        if (resume & C2P_DEFER_TAIL) {
            if ((methods & 2) && c2p_brent_w(c, par.brent_maxit, P)) return C2P_BRENT_W;
            if ((methods & 4) && entropy()) return C2P_ENTROPY;
            return fail(C2P_FAIL | C2P_FAIL_ENT);
        }
        if (entropy()) return (resume & C2P_DEFER_BETA) ? C2P_ENTROPY_BETA : C2P_ENTROPY;
        return fail(C2P_FAIL | C2P_FAIL_ENT);
    }

    if (methods & 8) {
        bool low_beta;
        if (MIXED) {
            St<float> s;
            get_state(guessf, *gf, s);
            float pg = (par.gam_f - 1.0f) * guessf[KUU];
            low_beta = s.bsq > 0.0f && pg < par.beta_ent_f * 0.5f * s.bsq;
        } else {
            St<double> s;
            get_state(guess, g, s);
            double pg = (par.gam - 1.0) * guess[KUU];
            low_beta = s.bsq > 0.0 && pg < par.beta_ent * 0.5 * s.bsq;
        }
        if (low_beta) {
            if (methods & 4) {
                if (!MIXED && pass == 1) return C2P_DEFER | C2P_DEFER_BETA;
                if (entropy()) return C2P_ENTROPY_BETA;
            }
            return fail(C2P_FAIL | C2P_FAIL_ENT);
        }
    }
    if (methods & 1) {
        // a learned W (mlp_first), then the extrapolated start, are tried first;
        // Newton from the guess primitives follows, then the learned rescue
#pragma unroll 1
        for (int a = 0; a < 4; a++) {
            const bool learned = a == 0 || a == 3, extrap = a == 1;
            if (a == 0 && !mlp_first && !(w_first > 0.0)) continue;
            if (a == 3 && !mlp_rescue) continue;
            if (extrap && !(MIXED && have_start)) continue;
            double W, v2;
            if (learned) {
                const double wl = (a == 0 && !mlp_first) ? w_first
                                                         : c2p_learned_w(a == 0 ? mlp_first : mlp_rescue, c);
                if (!(wl > 0.0)) continue;
                W = wl;
                v2 = fmin(ResidW{&c}.v2(wl), V2MAX);
            } else if (MIXED) {
                // (W, v^2) formed and checked in FP32 from the chosen FP32 primitives
                const float r0 = extrap ? startf[KRHO] : guessf[KRHO], e0 = extrap ? startf[KUU] : guessf[KUU];
                const float u1 = extrap ? startf[KU1] : guessf[KU1], u2 = extrap ? startf[KU2] : guessf[KU2],
                            u3 = extrap ? startf[KU3] : guessf[KU3];
                const float usq = spatial_sq(*gf, u1, u2, u3);
                const float Wf = (1.0f + usq) * (r0 + par.gam_f * e0);
                // v^2 below 1 (the largest float under 1.0): usq / (1 + usq) rounds to 1 for usq > ~1.7e7
                v2 = (double)fminf(usq / (1.0f + usq), 0.99999994f);
                W = (Wf > 0.0f && Wf < INFINITY) ? (double)Wf : c.D;
            } else {
                const double usq = spatial_sq(g, guess[KU1], guess[KU2], guess[KU3]);
                v2 = usq / (1.0 + usq);
                W = (1.0 + usq) * (guess[KRHO] + par.gam * guess[KUU]);
                if (!(W > 0.0) || !finite64(W)) W = c.D;
                v2 = fmin(v2, V2MAX);
            }
            int it;
            const bool conv = MIXED ? c2p_newton_mixed(c, par, W, v2, it)
                                    : c2p_newton<true>(c, W, v2, par.tol, par.nr_maxit, it);
            iters += it;
            if (conv) {
                if (MIXED) c2p_recover_mixed(c, W, v2, par.ig, P);
                else c2p_recover_w(c, W, v2, P);
                if (c2p_physical(P, v2)) return a == 3 ? (C2P_NR | C2P_LEARNED) : C2P_NR;
                if (methods & 4) {
                    if (!MIXED && pass == 1) return C2P_DEFER | C2P_DEFER_ENT;
                    if (entropy()) return C2P_ENTROPY;
                }
                return fail(C2P_FAIL | C2P_FAIL_ENT);
            }
        }
    }
    if (!MIXED && pass == 1 && (methods & 6)) return C2P_DEFER | C2P_DEFER_TAIL;
    if ((methods & 2) && c2p_brent_w(c, par.brent_maxit, P)) return C2P_BRENT_W;
    if ((methods & 4) && entropy()) return C2P_ENTROPY;
    return fail(C2P_FAIL | C2P_FAIL_ENT);
}

} // namespace grmhd
