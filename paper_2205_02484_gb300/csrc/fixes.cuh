// fixes.cuh -- floors, magnetisation ceilings and the Lorentz-factor cap of
// Section 2.4 (Eq. 34 and the limits b^2/rho < 50, b^2/u < 2500, Gamma < 50),
// applied after a successful inversion, plus the direct form used on zones
// repaired by neighbour averaging (Eq. 33).
//
// Ceilings add the missing rho, u as matter at rest in the normal (ZAMO)
// frame (ut^i = 0, B = 0) to U and re-invert with Newton; if that fails the
// primitives are raised directly.  U is recomputed from the final primitives
// of every modified zone.
#pragma once
#include "con2prim.cuh"

namespace grmhd {

__device__ __forceinline__ void floor_values(const Grid &g, double r, double &rfl, double &ufl)
{
    rfl = 1e-20;
    ufl = 1e-20;
    if (g.metric == KERR_MKS) {
        rfl = fmax(rfl, 1e-5 * pow(r, -0.5));
        ufl = fmax(ufl, (1e-5 / 3.0) * pow(r, -2.5));
    }
}

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

// returns bit 1 = modified, bit 2 = ceiling applied, bit 4 = Lorentz cap applied
__device__ inline int post_inversion(const Grid &g, const Geo<double> &geo, double r, double q[NP],
                                     const double Un[NU])
{
    int res = 0;
    double rfl, ufl;
    floor_values(g, r, rfl, ufl);
    if (q[KRHO] < rfl) { q[KRHO] = rfl; res |= 1; }
    if (q[KUU] < ufl) { q[KUU] = ufl; res |= 1; }
    St<double> s;
    get_state(q, geo, s);
    double drho = fmax(0.0, s.bsq / g.sigma_max - q[KRHO]);
    double du = fmax(0.0, s.bsq / g.bu_max - q[KUU]);
    if (drho > 0.0 || du > 0.0) {
        res |= 3;
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
        int fl = con2prim(U2, geo, gs, g.gam, g.beta_ent, g.nr_tol, g.nr_maxit, g.brent_maxit, 1, qn, it);
        if (fl == C2P_NR) {
#pragma unroll
            for (int c = 0; c < NP; c++) q[c] = qn[c];
        } else {
            q[KRHO] += drho;
            q[KUU] += du;
        }
    }
    if (gamma_cap(g, geo, q)) res |= 5;
    return res;
}

__device__ inline void post_fixup(const Grid &g, const Geo<double> &geo, double r, double q[NP])
{
    double rfl, ufl;
    floor_values(g, r, rfl, ufl);
    if (q[KRHO] < rfl) q[KRHO] = rfl;
    if (q[KUU] < ufl) q[KUU] = ufl;
    St<double> s;
    get_state(q, geo, s);
    q[KRHO] = fmax(q[KRHO], s.bsq / g.sigma_max);
    q[KUU] = fmax(q[KUU], s.bsq / g.bu_max);
    gamma_cap(g, geo, q);
}

} // namespace grmhd
