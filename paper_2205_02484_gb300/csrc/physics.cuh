// physics.cuh -- pointwise GR-MHD physics of Sections 2.1-2.2, templated on
// the arithmetic type (double for the FP64 path, float for the mixed path).
//
//   u^mu from the modified velocity ut^i (Eq. 11): u^t = Gamma/alpha,
//   u^i = ut^i - Gamma alpha g^{ti}; b^t = B^i u_i, b^i = (B^i + b^t u^i)/u^t;
//   T^mu_nu = (w + b^2) u^mu u_nu + (p + b^2/2) delta - b^mu b_nu (Eq. 5);
//   U = sqrt(-g)(rho u^t, T^t_nu, B^i, S u^t), F^d likewise (Eqs. 6-8, 12);
//   wave speeds: roots of the quadratic form of Eq. 19 along direction d.
//
// In the mixed path the energy component of U and F is carried rest-mass
// subtracted (T^t_t + rho u^t, T^d_t + rho u^d), with 1 + u_t evaluated as
// (1 - alpha) - alpha (Gamma - 1) + g_{ti} ut^i so that no FP32 cancellation
// between the rest mass and the energy occurs; the update adds the mass flux
// back in FP64, so the stored energy is still sqrt(-g) T^t_t.
#pragma once
#include "common.cuh"

namespace grmhd {

template <typename R>
struct St {
    R ucon[4], ucov[4], bcon[4], bcov[4], bsq, gamma, usq;
};

template <typename R>
__device__ __forceinline__ R spatial_sq(const Geo<R> &g, R x, R y, R z)
{
    return g.gcov[4] * x * x + g.gcov[7] * y * y + g.gcov[9] * z * z +
           R(2) * (g.gcov[5] * x * y + g.gcov[6] * x * z + g.gcov[8] * y * z);
}

template <typename R>
__device__ __forceinline__ void lower4(const Geo<R> &g, const R v[4], R w[4])
{
#pragma unroll
    for (int m = 0; m < 4; m++)
        w[m] = g.gcov[sym(m, 0)] * v[0] + g.gcov[sym(m, 1)] * v[1] + g.gcov[sym(m, 2)] * v[2] +
               g.gcov[sym(m, 3)] * v[3];
}

// a / b: a division in FP64; in FP32 (the mixed path's face physics) the
// hardware reciprocal times a (2 ulp, within the FP32 rounding the face
// fluxes carry anyway; b is never near the float range's end here)
template <typename R>
__device__ __forceinline__ R divr(R a, R b) { return a / b; }
template <>
__device__ __forceinline__ float divr<float>(float a, float b) { return __fdividef(a, b); }

// square root: correctly rounded in FP64; in FP32 the hardware approximation
// (sqrt.approx, ~2 ulp, exact at 0) for the same reason
template <typename R>
__device__ __forceinline__ R sqrtr(R x) { return sqrt(x); }
template <>
__device__ __forceinline__ float sqrtr<float>(float x)
{
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <typename R>
__device__ __forceinline__ void get_state(const R q[NP], const Geo<R> &g, St<R> &s)
{
    R usq = spatial_sq(g, q[KU1], q[KU2], q[KU3]);
    R gm, iut; // Gamma and 1 / u^t = alpha / Gamma
    if constexpr (sizeof(R) == 8) {
        // FP64: both from one reciprocal square root (a division and a square
        // root are each an FP64 instruction sequence), to an ulp or two
        const R ig = rsqrt(R(1) + usq);
        gm = (R(1) + usq) * ig;
        iut = g.alpha * ig;
    } else {
        gm = sqrtr(R(1) + usq);
        iut = divr(g.alpha, gm);
    }
    s.usq = usq;
    s.gamma = gm;
    s.ucon[0] = gm * g.ialpha;
#pragma unroll
    for (int i = 1; i <= 3; i++) s.ucon[i] = q[KU1 + i - 1] - gm * g.alpha * g.gcon[sym(0, i)];
    lower4(g, s.ucon, s.ucov);
    s.bcon[0] = q[KB1] * s.ucov[1] + q[KB2] * s.ucov[2] + q[KB3] * s.ucov[3];
#pragma unroll
    for (int i = 1; i <= 3; i++) s.bcon[i] = (q[KB1 + i - 1] + s.bcon[0] * s.ucon[i]) * iut;
    lower4(g, s.bcon, s.bcov);
    s.bsq = s.bcon[0] * s.bcov[0] + s.bcon[1] * s.bcov[1] + s.bcon[2] * s.bcov[2] +
            s.bcon[3] * s.bcov[3];
}

template <typename R>
__device__ __forceinline__ R powr(R x, R y);
template <>
__device__ __forceinline__ double powr<double>(double x, double y) { return pow(x, y); }
template <>
__device__ __forceinline__ float powr<float>(float x, float y) { return powf(x, y); }

// rho^(1 - gam) of the entropy density (Eq. 12): reciprocal cube roots for
// the adiabatic indices 4/3, 5/3 and 13/9 (rho^(-1/3), rho^(-2/3),
// rho^(-4/9) = (rho^(-1/9))^4 with rho^(-1/9) = rcbrt(cbrt(rho))), a general
// power otherwise and for rho <= 0 (where it keeps pow's inf / NaN)
__device__ __forceinline__ double rcbrtr(double x) { return rcbrt(x); }
__device__ __forceinline__ float rcbrtr(float x) { return rcbrtf(x); }
__device__ __forceinline__ double cbrtr(double x) { return cbrt(x); }
__device__ __forceinline__ float cbrtr(float x) { return cbrtf(x); }

template <typename R>
__device__ __forceinline__ R rho_pow_1mg(R rho, R gam)
{
    if (rho > R(0)) {
        if (gam == R(4.0 / 3.0)) return rcbrtr(rho);
        if (gam == R(5.0 / 3.0)) {
            const R r = rcbrtr(rho);
            return r * r;
        }
        if (gam == R(13.0 / 9.0)) {
            const R r = rcbrtr(cbrtr(rho)), r2 = r * r;
            return r2 * r2;
        }
    }
    return powr(rho, R(1) - gam);
}

// Row mu of T^mu_nu.
template <typename R>
__device__ __forceinline__ void tmunu_row(const R q[NP], const St<R> &s, R gam, int mu, R T[4])
{
    R p = (gam - R(1)) * q[KUU];
    R w = q[KRHO] + q[KUU] + p;
    R wb = w + s.bsq;
#pragma unroll
    for (int n = 0; n < 4; n++) T[n] = wb * s.ucon[mu] * s.ucov[n] - s.bcon[mu] * s.bcov[n];
    T[mu] += p + R(0.5) * s.bsq;
}

// Conserved vector (d = 0) or flux along d (1..3), Eqs. 6-8 plus the entropy
// density of Eq. 12.  RMS: rest-mass-subtracted energy (mixed path).
template <typename R, bool RMS>
__device__ __forceinline__ void prim_to_UF(const R q[NP], const Geo<R> &g, const St<R> &s, R gam,
                                           int d, R out[NU])
{
    R T[4];
    tmunu_row(q, s, gam, d, T);
    R gd = g.gdet;
    R p = (gam - R(1)) * q[KUU];
    R ent = p * rho_pow_1mg(q[KRHO], gam);
    out[KRHO] = gd * q[KRHO] * s.ucon[d];
    if (RMS) {
        // T^d_t + rho u^d = rho u^d (1 + u_t) + (u + p + b^2) u^d u_t - b^d b_t (+ p + b^2/2 if d = t)
        R opu = g.oma - g.alpha * divr(s.usq, s.gamma + R(1)) +
                (g.gcov[1] * q[KU1] + g.gcov[2] * q[KU2] + g.gcov[3] * q[KU3]);
        R e = q[KRHO] * s.ucon[d] * opu + (q[KUU] + p + s.bsq) * s.ucon[d] * s.ucov[0] -
              s.bcon[d] * s.bcov[0];
        if (d == 0) e += p + R(0.5) * s.bsq;
        out[1] = gd * e;
    } else {
        out[1] = gd * T[0];
    }
    out[2] = gd * T[1];
    out[3] = gd * T[2];
    out[4] = gd * T[3];
    if (d == 0) {
        out[KB1] = gd * q[KB1];
        out[KB2] = gd * q[KB2];
        out[KB3] = gd * q[KB3];
    } else {
#pragma unroll
        for (int i = 1; i <= 3; i++) out[KB1 + i - 1] = gd * (s.bcon[d] * s.ucon[i] - s.bcon[i] * s.ucon[d]);
    }
    out[KENT] = gd * ent * s.ucon[d];
}

// Conserved vector and flux along d of one state together: the rows T^t_nu
// and T^d_nu share every factor, and the entropy density is evaluated once.
template <typename R, bool RMS>
__device__ __forceinline__ void prim_to_UF2(const R q[NP], const Geo<R> &g, const St<R> &s, R gam,
                                            int d, R U[NU], R F[NU])
{
    const R gd = g.gdet;
    const R p = (gam - R(1)) * q[KUU];
    const R wb = q[KRHO] + q[KUU] + p + s.bsq;
    const R ptot = p + R(0.5) * s.bsq;
    const R ent = gd * p * rho_pow_1mg(q[KRHO], gam);
    const R gut = gd * s.ucon[0], gud = gd * s.ucon[d];
    const R gbt = gd * s.bcon[0], gbd = gd * s.bcon[d];
    U[KRHO] = gut * q[KRHO];
    F[KRHO] = gud * q[KRHO];
#pragma unroll
    for (int n = 0; n < 4; n++) {
        U[1 + n] = wb * gut * s.ucov[n] - gbt * s.bcov[n];
        F[1 + n] = wb * gud * s.ucov[n] - gbd * s.bcov[n];
    }
    U[1] += gd * ptot;
    F[1 + d] += gd * ptot;
    if (RMS) {
        // T^mu_t + rho u^mu = rho u^mu (1 + u_t) + (u + p + b^2) u^mu u_t - b^mu b_t (+ ptot for mu = t)
        const R opu = g.oma - g.alpha * divr(s.usq, s.gamma + R(1)) +
                      (g.gcov[1] * q[KU1] + g.gcov[2] * q[KU2] + g.gcov[3] * q[KU3]);
        const R rest = q[KUU] + p + s.bsq;
        U[1] = gut * (q[KRHO] * opu + rest * s.ucov[0]) - gbt * s.bcov[0] + gd * ptot;
        F[1] = gud * (q[KRHO] * opu + rest * s.ucov[0]) - gbd * s.bcov[0];
    }
    U[KB1] = gd * q[KB1];
    U[KB2] = gd * q[KB2];
    U[KB3] = gd * q[KB3];
#pragma unroll
    for (int i = 1; i <= 3; i++) F[KB1 + i - 1] = gbd * s.ucon[i] - gd * s.bcon[i] * s.ucon[d];
    U[KENT] = ent * s.ucon[0];
    F[KENT] = ent * s.ucon[d];
}

// c1 >= c2: roots of (1 - cms2)(u^d - v u^t)^2 = cms2 (g^tt v^2 - 2 g^td v + g^dd)
template <typename R>
__device__ __forceinline__ void wave_speeds(const R q[NP], const Geo<R> &g, const St<R> &s, R gam,
                                            int d, R &c1, R &c2)
{
    R p = (gam - R(1)) * q[KUU];
    R ef = q[KRHO] + q[KUU] + p;
    R ee = s.bsq + ef;
    R inv = divr(R(1), ee * ef);
    R va2 = s.bsq * ef * inv;   // b^2 / (b^2 + rho + u + p)
    R cs2 = gam * p * ee * inv; // gam p / (rho + u + p)
    R cms2 = va2 + cs2 * (R(1) - va2);
    R A1 = R(1) - cms2;
    R ut = s.ucon[0], ud = s.ucon[d];
    R A = A1 * ut * ut - cms2 * g.gcon[0];
    R B = R(-2) * (A1 * ut * ud - cms2 * g.gcon[sym(0, d)]);
    R C = A1 * ud * ud - cms2 * g.gcon[sym(d, d)];
    R disc = B * B - R(4) * A * C;
    disc = disc < R(0) ? R(0) : disc;
    R sq = sqrtr(disc);
    R i2a = divr(R(0.5), A);
    R vp = (-B + sq) * i2a;
    R vm = (-B - sq) * i2a;
    c1 = vp > vm ? vp : vm;
    c2 = vp > vm ? vm : vp;
}

// MC-limited slope (Eq. 16, signed central branch)
template <typename R>
__device__ __forceinline__ R mc_slope(R qm, R q0, R qp)
{
    R dm = q0 - qm, dp = qp - q0, dc = qp - qm;
    if (dm * dp < R(0)) return R(0);
    if (fabs(dm) < fabs(dp) && R(2) * fabs(dm) < R(0.5) * fabs(dc)) return R(2) * dm;
    if (R(2) * fabs(dp) < R(0.5) * fabs(dc)) return R(2) * dp;
    return R(0.5) * dc;
}

// The same slope in FP64 with its three decisions taken on the bit patterns
// of the differences (integer operations: GB300 runs FP64 multiplies and
// compares at the FP64 rate, 1/64 of FP32's).  For finite differences whose
// magnitudes are zero or at least 2^-1020 (so that doubling and halving them
// is exact) they are the comparisons above:
// dm dp < 0 is opposite sign bits with both nonzero; |x| < |y| orders the
// magnitudes' bit patterns as unsigned integers; 2|x| < |dc|/2 is 4|x| < |dc|,
// the magnitude with its exponent raised by 2.  The values returned are the
// same products.
template <>
__device__ __forceinline__ double mc_slope<double>(double qm, double q0, double qp)
{
    const double dm = q0 - qm, dp = qp - q0, dc = qp - qm;
    const unsigned long long mag = 0x7fffffffffffffffULL, four = 2ULL << 52;
    const unsigned long long bm = (unsigned long long)__double_as_longlong(dm);
    const unsigned long long bp = (unsigned long long)__double_as_longlong(dp);
    const unsigned long long am = bm & mag, ap = bp & mag;
    const unsigned long long ac = (unsigned long long)__double_as_longlong(dc) & mag;
    if (((bm ^ bp) >> 63) && am != 0 && ap != 0) return 0.0;
    if (am < ap && am + four < ac) return 2.0 * dm;
    if (ap + four < ac) return 2.0 * dp;
    return 0.5 * dc;
}

// Piecewise parabolic faces (Colella & Woodward 1984 on uniform code-coordinate
// zones, the reconstruction Section 2.2 names after PLM): interface value
// (a_0 + a_1)/2 - (d_1 - d_0)/6 from the MC-limited slopes, then each zone's
// parabola (a_L, a, a_R) made monotone -- flat at a local extremum, else the
// far edge moved to 3 a - 2 (near edge) where the parabola would overshoot.
// x / 6: a correctly rounded division in FP64; in FP32 (the mixed path's
// faces) a product with the rounded 1/6, within an ulp of it and without
// the division's instruction sequence (three per variable and zone)
__device__ __forceinline__ double sixth(double x) { return x / 6.0; }
__device__ __forceinline__ float sixth(float x) { return x * (1.0f / 6.0f); }

template <typename R>
__device__ __forceinline__ R ppm_interface_s(R a0, R a1, R d0, R d1)
{
    return R(0.5) * (a0 + a1) - sixth(d1 - d0);
}

template <typename R>
__device__ __forceinline__ R ppm_interface(R am, R a0, R a1, R a2)
{
    return ppm_interface_s(a0, a1, mc_slope(am, a0, a1), mc_slope(a0, a1, a2));
}

template <typename R>
__device__ __forceinline__ void ppm_monotone(R a, R &L, R &Rt)
{
    if ((Rt - a) * (a - L) <= R(0)) {
        L = a;
        Rt = a;
    } else {
        const R d = Rt - L, m = a - R(0.5) * (L + Rt);
        const R d26 = sixth(d * d);
        if (d * m > d26) L = R(3) * a - R(2) * Rt;
        else if (-d26 > d * m) Rt = R(3) * a - R(2) * L;
    }
}

// left and right states at the face between zones q[2] and q[3] of six zone
// values q[0..5] along the face's direction
template <typename R>
__device__ __forceinline__ void ppm_face(const R q[6], R &ql, R &qr)
{
    const R i01 = ppm_interface(q[0], q[1], q[2], q[3]);
    const R i12 = ppm_interface(q[1], q[2], q[3], q[4]);
    const R i23 = ppm_interface(q[2], q[3], q[4], q[5]);
    R L2 = i01, R2 = i12, L3 = i12, R3 = i23;
    ppm_monotone(q[2], L2, R2);
    ppm_monotone(q[3], L3, R3);
    ql = R2;
    qr = L3;
}

// Source of Eq. 7 at the cell centre: S_nu = sqrt(-g) T^k_l Gamma^l_{nu k};
// conn holds Gamma^l_{mn} as conn[l*10 + sym(m,n)].
template <typename R>
__device__ __forceinline__ void source_terms(const R q[NP], const Geo<R> &g, const R *conn,
                                             const St<R> &s, R gam, R S[4])
{
    R T[4][4];
#pragma unroll
    for (int k = 0; k < 4; k++) tmunu_row(q, s, gam, k, T[k]);
#pragma unroll
    for (int nu = 0; nu < 4; nu++) {
        R acc = R(0);
#pragma unroll
        for (int k = 0; k < 4; k++)
#pragma unroll
            for (int l = 0; l < 4; l++) acc += T[k][l] * conn[l * 10 + sym(nu, k)];
        S[nu] = g.gdet * acc;
    }
}

template <typename R>
__device__ __forceinline__ void load_geo(const Geo<R> *tab, int m, Geo<R> &g)
{
    g = tab[m];
}

} // namespace grmhd
