// fixes.cuh -- floors, magnetisation ceilings and the Lorentz-factor cap of
// Section 2.4 (Eq. 34 and the limits b^2/rho < 50, b^2/u < 2500, Gamma < 50),
// applied after a successful inversion, plus the direct form used on zones
// repaired by neighbour averaging (Eq. 33).
//
// Ceilings add the missing rho, u as matter at rest in the normal (ZAMO)
// frame (ut^i = 0, B = 0) to U and re-invert with Newton; if that fails the
// primitives are raised directly.  U is recomputed from the final primitives
// of every modified zone.  The floor values of Eq. 34 are tabulated per
// (r, theta) with the metric.
#pragma once
#include "con2prim.cuh"

namespace grmhd {

__device__ __forceinline__ bool gamma_cap(const Grid &g, const Geo<double> &geo, double q[NP])
{
    double usq = spatial_sq(geo, q[KU1], q[KU2], q[KU3]);
    double gm = g.gamma_max;
    if (1.0 + usq > gm * gm) {
        double f = sqrt((gm * gm - 1.0) / usq);
        q[KU1] *= f;
        q[KU2] *= f;
        q[KU3] *= f;
        return true;
    }
    return false;
}

// returns bit 1 = modified, bit 2 = ceiling applied, bit 4 = Lorentz cap applied,
// bit 8 = density floored.
// gsp: the zone's spatial inverse metric (for the re-inversion of a ceiling).
// MIXED: b^2 and ut^2 (neither involves rho or u) come from one FP32 state of
// the record gf; the exact FP64 Lorentz test runs only where the FP32 ut^2 is
// within 1e-4 of the cap; qf receives the FP32 primitives to store.
template <bool MIXED = false>
__device__ inline int post_inversion(const Grid &g, const Geo<double> &geo, const double *gsp, double q[NP],
                                     const double Un[NU], const Geo<float> *gf = nullptr, float *qf = nullptr)
{
    int res = 0;
    double bsq;
    float usqf = 0.0f, rf = 0.0f, uf = 0.0f;
    bool ceil;
    if (MIXED) {
        // floors and ceilings decided in FP32, on the values that are stored
        rf = (float)q[KRHO];
        uf = (float)q[KUU];
        if (rf < gf->rfl) { q[KRHO] = geo.rfl; rf = gf->rfl; res |= 9; }
        if (uf < gf->ufl) { q[KUU] = geo.ufl; uf = gf->ufl; res |= 1; }
        qf[KRHO] = 0.0f;
        qf[KUU] = 0.0f;
#pragma unroll
        for (int m = KU1; m < NP; m++) qf[m] = (float)q[m];
        St<float> s;
        get_state(qf, *gf, s);
        usqf = s.usq;
        ceil = s.bsq * g.isig_f > rf || s.bsq * g.ibu_f > uf;
        bsq = ceil ? (double)s.bsq : 0.0; // widened only where a ceiling acts
    } else {
        if (q[KRHO] < geo.rfl) { q[KRHO] = geo.rfl; res |= 9; }
        if (q[KUU] < geo.ufl) { q[KUU] = geo.ufl; res |= 1; }
        St<double> s;
        get_state(q, geo, s);
        bsq = s.bsq;
        ceil = true;
    }
    bool moved = false;
    double drho = 0.0, du = 0.0;
    if (ceil) {
        drho = fmax(0.0, bsq * g.isig - q[KRHO]);
        du = fmax(0.0, bsq * g.ibu - q[KUU]);
    }
    if (drho > 0.0 || du > 0.0) {
        res |= 3;
        moved = true;
        double dq[NP] = {drho, du, 0, 0, 0, 0, 0, 0};
        St<double> ds;
        get_state(dq, geo, ds);
        double dU[NU], U2[NU], gs[NP], qn[NP];
        prim_to_UF<double, false>(dq, geo, ds, g.gam, 0, dU);
#pragma unroll
        for (int c = 0; c < NU; c++) U2[c] = Un[c] + (c < 5 ? dU[c] : 0.0);
#pragma unroll
        for (int c = 0; c < NP; c++) gs[c] = q[c];
        gs[KRHO] += drho;
        gs[KUU] += du;
        int it;
        int fl = con2prim<false>(U2, geo, gsp, gs, nullptr, c2p_par(g), 1, qn, it);
        if (fl == C2P_NR) {
#pragma unroll
            for (int c = 0; c < NP; c++) q[c] = qn[c];
        } else {
            q[KRHO] += drho;
            q[KUU] += du;
        }
    }
    bool test_cap = true;
    if (MIXED && !moved) {
        float gm = g.gamma_max_f;
        test_cap = 1.0f + usqf > gm * gm * 0.9999f;
    }
    if (test_cap && gamma_cap(g, geo, q)) {
        res |= 5;
        moved = true;
    }
    if (MIXED) {
        if (moved) {
#pragma unroll
            for (int m = KU1; m < NP; m++) qf[m] = (float)q[m];
            rf = (float)q[KRHO];
            uf = (float)q[KUU];
        }
        qf[KRHO] = rf;
        qf[KUU] = uf;
    }
    return res;
}

__device__ inline void post_fixup(const Grid &g, const Geo<double> &geo, double q[NP])
{
    if (q[KRHO] < geo.rfl) q[KRHO] = geo.rfl;
    if (q[KUU] < geo.ufl) q[KUU] = geo.ufl;
    St<double> s;
    get_state(q, geo, s);
    q[KRHO] = fmax(q[KRHO], s.bsq / g.sigma_max);
    q[KUU] = fmax(q[KUU], s.bsq / g.bu_max);
    gamma_cap(g, geo, q);
}

// FP64 conserved variables of q (Eqs. 6-8, 12).
//
// Mixed path: only the rest mass U_rho = sqrt(-g) rho u^t is formed in FP64
// (u^t = (1 + (Gamma - 1)) / alpha with Gamma - 1 = ut^2/(1 + Gamma) from
// the FP32 state); the rest-mass-subtracted energy sqrt(-g)(T^t_t + rho u^t),
// the momenta and the entropy come from the FP32 state, and
// U_E = (U_E + U_rho) - U_rho is assembled in FP64.  The inversion depends on
// E - D, which is therefore carried with FP32 relative accuracy of the
// thermal + kinetic + binding energy, not of the rest mass.
//
// qf (mixed path, may be null): the FP32 primitives of q, if the caller has them.
// keep_rho (mixed path): rho and the velocity are unchanged (only u was
// floored), so U_rho = sqrt(-g) rho u^t keeps its accumulated FP64 value.  The
// mixed path also keeps U_B, which no floor, ceiling or cap changes.
template <bool MIXED = false>
__device__ inline void cons_of(const double q[NP], const Geo<double> &geo, double gam, double U[NU],
                               const Geo<float> *gf = nullptr, const float *qfin = nullptr, float gam_f = 0.0f,
                               bool keep_rho = false)
{
    if (MIXED) {
        float qf[NP];
#pragma unroll
        for (int m = 0; m < NP; m++) qf[m] = qfin ? qfin[m] : (float)q[m];
        St<float> s;
        get_state(qf, *gf, s);
        float Uf[NU];
        prim_to_UF<float, true>(qf, *gf, s, gam_f, 0, Uf);
        if (!keep_rho) {
            double gm1 = (double)(s.usq / (s.gamma + 1.0f));
            U[KRHO] = geo.gdet * q[KRHO] * ((1.0 + gm1) * geo.ialpha);
        }
        U[1] = (double)Uf[1] - U[KRHO];
        U[2] = (double)Uf[2];
        U[3] = (double)Uf[3];
        U[4] = (double)Uf[4];
        U[KENT] = (double)Uf[KENT];
        return;
    }
    St<double> s;
    get_state(q, geo, s);
    double T[4];
    tmunu_row(q, s, gam, 0, T);
    double gd = geo.gdet;
    double p = (gam - 1.0) * q[KUU];
    U[KRHO] = gd * q[KRHO] * s.ucon[0];
    U[1] = gd * T[0];
    U[2] = gd * T[1];
    U[3] = gd * T[2];
    U[4] = gd * T[3];
    U[KB1] = gd * q[KB1];
    U[KB2] = gd * q[KB2];
    U[KB3] = gd * q[KB3];
    U[KENT] = gd * (p * rho_pow_1mg(q[KRHO], gam)) * s.ucon[0];
}

} // namespace grmhd
