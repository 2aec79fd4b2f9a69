// geometry.cu -- metric tables of the grid (Section 4.1, Eqs. 35-36).
//
// One thread per ghosted (I, J): g_{mu nu} at the zone centre and at the
// centres of the X1 and X2 faces, g^{mu nu} by the adjugate (Laplace
// expansion in complementary 2x2 minors), sqrt(-g), alpha = (-g^{tt})^-1/2,
// 1 - alpha, FP32 copies for the mixed path, and the connection
//   Gamma^l_{mn} = 1/2 g^{ls} (d_m g_{sn} + d_n g_{sm} - d_s g_{mn})
// at centres, with d_1, d_2 of the metric from forward-mode dual numbers
// (exact to rounding).  X2 faces on the poles (theta = 0, pi) are singular;
// they are marked and left zero (every flux through them vanishes).
#include "kernels.h"

namespace grmhd {

__device__ bool inv4(const double a[4][4], double b[4][4], double &det)
{
    double s0 = a[0][0] * a[1][1] - a[1][0] * a[0][1];
    double s1 = a[0][0] * a[1][2] - a[1][0] * a[0][2];
    double s2 = a[0][0] * a[1][3] - a[1][0] * a[0][3];
    double s3 = a[0][1] * a[1][2] - a[1][1] * a[0][2];
    double s4 = a[0][1] * a[1][3] - a[1][1] * a[0][3];
    double s5 = a[0][2] * a[1][3] - a[1][2] * a[0][3];
    double c5 = a[2][2] * a[3][3] - a[3][2] * a[2][3];
    double c4 = a[2][1] * a[3][3] - a[3][1] * a[2][3];
    double c3 = a[2][1] * a[3][2] - a[3][1] * a[2][2];
    double c2 = a[2][0] * a[3][3] - a[3][0] * a[2][3];
    double c1 = a[2][0] * a[3][2] - a[3][0] * a[2][2];
    double c0 = a[2][0] * a[3][1] - a[3][0] * a[2][1];
    det = s0 * c5 - s1 * c4 + s2 * c3 + s3 * c2 - s4 * c1 + s5 * c0;
    if (det == 0.0 || !isfinite(det)) return false;
    double id = 1.0 / det;
    b[0][0] = (a[1][1] * c5 - a[1][2] * c4 + a[1][3] * c3) * id;
    b[0][1] = (-a[0][1] * c5 + a[0][2] * c4 - a[0][3] * c3) * id;
    b[0][2] = (a[3][1] * s5 - a[3][2] * s4 + a[3][3] * s3) * id;
    b[0][3] = (-a[2][1] * s5 + a[2][2] * s4 - a[2][3] * s3) * id;
    b[1][0] = (-a[1][0] * c5 + a[1][2] * c2 - a[1][3] * c1) * id;
    b[1][1] = (a[0][0] * c5 - a[0][2] * c2 + a[0][3] * c1) * id;
    b[1][2] = (-a[3][0] * s5 + a[3][2] * s2 - a[3][3] * s1) * id;
    b[1][3] = (a[2][0] * s5 - a[2][2] * s2 + a[2][3] * s1) * id;
    b[2][0] = (a[1][0] * c4 - a[1][1] * c2 + a[1][3] * c0) * id;
    b[2][1] = (-a[0][0] * c4 + a[0][1] * c2 - a[0][3] * c0) * id;
    b[2][2] = (a[3][0] * s4 - a[3][1] * s2 + a[3][3] * s0) * id;
    b[2][3] = (-a[2][0] * s4 + a[2][1] * s2 - a[2][3] * s0) * id;
    b[3][0] = (-a[1][0] * c3 + a[1][1] * c1 - a[1][2] * c0) * id;
    b[3][1] = (a[0][0] * c3 - a[0][1] * c1 + a[0][2] * c0) * id;
    b[3][2] = (-a[3][0] * s3 + a[3][1] * s1 - a[3][2] * s0) * id;
    b[3][3] = (a[2][0] * s3 - a[2][1] * s1 + a[2][2] * s0) * id;
    return true;
}

__device__ void make_geo(const CoordParams &cp, double X1, double X2, Geo<double> &g, Geo<float> &gf,
                         double gcon_full[4][4])
{
    double gc[4][4], gi[4][4], det;
    code_gcov<double>(cp, X1, X2, gc);
    bool ok = inv4(gc, gi, det) && det < 0.0;
    for (int m = 0; m < 4; m++)
        for (int n = m; n < 4; n++) {
            g.gcov[sym(m, n)] = ok ? gc[m][n] : 0.0;
            g.gcon[sym(m, n)] = ok ? 0.5 * (gi[m][n] + gi[n][m]) : 0.0;
        }
    for (int m = 0; m < 4; m++)
        for (int n = 0; n < 4; n++) gcon_full[m][n] = ok ? gi[m][n] : 0.0;
    g.gdet = ok ? sqrt(-det) : 0.0;
    g.alpha = ok ? 1.0 / sqrt(-gi[0][0]) : 0.0;
    g.oma = ok ? 1.0 - g.alpha : 0.0;
    g.igdet = ok ? 1.0 / g.gdet : 0.0;
    g.ialpha = ok ? sqrt(-gi[0][0]) : 0.0;
    g.aig = ok ? g.alpha / g.gdet : 0.0;
    // floors of Eq. 34 at this radius (flat space: the absolute floors only)
    double r, dr;
    mks_radius<double>(cp, X1, r, dr);
    g.rfl = 1e-20;
    g.ufl = 1e-20;
    if (cp.metric == KERR_MKS) {
        g.rfl = fmax(g.rfl, 1e-5 * pow(r, -0.5));
        g.ufl = fmax(g.ufl, (1e-5 / 3.0) * pow(r, -2.5));
    }
    for (int a = 0; a < 10; a++) {
        gf.gcov[a] = (float)g.gcov[a];
        gf.gcon[a] = (float)g.gcon[a];
    }
    gf.gdet = (float)g.gdet;
    gf.alpha = (float)g.alpha;
    gf.oma = (float)g.oma;
    gf.igdet = (float)g.igdet;
    gf.ialpha = (float)g.ialpha;
    gf.aig = (float)g.aig;
    gf.rfl = (float)g.rfl;
    gf.ufl = (float)g.ufl;
}

__global__ void k_geometry(Grid g, GeomBuild b)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.N1 * g.N2) return;
    int i = t / g.N2 - NG, j = t % g.N2 - NG;
    double X1c = g.x1in + (i + 0.5) * g.dx[0], X1f = g.x1in + i * g.dx[0];
    const int jg = g.j0 + j; // the row in the whole grid (a theta slab's rows sit at their global X2)
    double X2c = g.x2in + (jg + 0.5) * g.dx[1], X2f = g.x2in + jg * g.dx[1];
    double gi[4][4];
    make_geo(b.cp, X1c, X2c, b.gc[t], b.gcF[t], gi);
    {
        // spatial part of the projector j^{mu nu} = g^{mu nu} + n^mu n^nu:
        // gamma^{ij} = g^{ij} - g^{ti} g^{tj} / g^{tt}
        const double *gu = b.gc[t].gcon;
        int q = 0;
        for (int a = 1; a < 4; a++)
            for (int c = a; c < 4; c++)
                b.gsp[(long long)t * 6 + q++] = gu[0] != 0.0 ? gu[sym(a, c)] - gu[sym(0, a)] * gu[sym(0, c)] / gu[0] : 0.0;
    }
    // connection at the centre
    Dual dg[2][4][4];
    {
        Dual X1d = mkd(X1c, 1.0), X2d = mkd(X2c, 0.0);
        code_gcov<Dual>(b.cp, X1d, X2d, dg[0]);
        X1d = mkd(X1c, 0.0);
        X2d = mkd(X2c, 1.0);
        code_gcov<Dual>(b.cp, X1d, X2d, dg[1]);
    }
    auto d = [&](int c, int m, int n) -> double { return (c == 1 || c == 2) ? dg[c - 1][m][n].d : 0.0; };
    for (int l = 0; l < 4; l++)
        for (int m = 0; m < 4; m++)
            for (int n = m; n < 4; n++) {
                double s = 0.0;
                for (int sg = 0; sg < 4; sg++) s += gi[l][sg] * (d(m, sg, n) + d(n, sg, m) - d(sg, m, n));
                b.conn[(long long)t * 40 + l * 10 + sym(m, n)] = 0.5 * s;
                b.connF[(long long)t * 40 + l * 10 + sym(m, n)] = (float)(0.5 * s);
            }
    make_geo(b.cp, X1f, X2c, b.gf1[t], b.gf1F[t], gi);
    bool polar = b.cp.metric == KERR_MKS && (jg == 0 || jg == g.n2t);
    b.polar2[t] = polar;
    if (polar) {
        Geo<double> z{};
        Geo<float> zf{};
        b.gf2[t] = z;
        b.gf2F[t] = zf;
    } else {
        make_geo(b.cp, X1c, X2f, b.gf2[t], b.gf2F[t], gi);
    }
    double r, dr;
    mks_radius<double>(b.cp, X1c, r, dr);
    b.rc[t] = b.cp.metric == KERR_MKS ? r : 1.0;
}

void launch_geometry(const Grid &g, const GeomBuild &b, cudaStream_t s)
{
    int n = g.N1 * g.N2;
    k_geometry<<<(n + 63) / 64, 64, 0, s>>>(g, b);
}

} // namespace grmhd
