// common.cuh -- device-side types of the GR-MHD step library.
//
// Layout in HBM (one context = one grid):
//   * primitives P[2][8][N1][N2][N3] (P^n and the half-step P-hat), FP64 in
//     FP64 mode, FP32 in mixed mode; conserved U[9][N1][N2][N3] always FP64;
//     face fluxes F[3][9][N1][N2][N3] and edge EMFs E[3][N1][N2][N3] in the
//     flux precision; N = n + 2*NG per direction, phi (k) fastest so that a
//     warp along phi shares one (r, theta) metric row (the metric does not
//     depend on phi, Section 3 of the paper).
//   * metric tables per (I, J) (ghosted): centre, X1-face and X2-face records
//     of g_{mu nu}, g^{mu nu}, sqrt(-g), alpha, 1 - alpha, and the 40
//     independent connection coefficients at centres.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace grmhd {

constexpr int NG = 3; // ghost layers per side: the PPM face stencil reaches three zones (Sec. 2.2)
constexpr int NP = 8;
constexpr int NU = 9;
enum { KRHO = 0, KUU, KU1, KU2, KU3, KB1, KB2, KB3, KENT };
enum { KERR_MKS = 0, MINK_CART = 1 };
enum { BC_INFLOW = 0, BC_POLAR = 1, BC_PERIODIC = 2, BC_OUTFLOW = 3, BC_EXTERNAL = 4 };

// packed index of a symmetric 4x4 tensor: 00 01 02 03 11 12 13 22 23 33
__host__ __device__ constexpr int sym(int m, int n)
{
    return m <= n ? (m == 0 ? n : (m == 1 ? 3 + n : (m == 2 ? 5 + n : 9)))
                  : (n == 0 ? m : (n == 1 ? 3 + m : (n == 2 ? 5 + m : 9)));
}

// splitmix64 (Steele, Lea & Flood 2014): one output of the generator whose
// state before the call is x
__host__ __device__ inline unsigned long long splitmix64(unsigned long long x)
{
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// counter-based uniform in [0, 1): the top 53 bits of splitmix64(seed ^ idx)
__host__ __device__ inline double counter_uniform(unsigned long long seed, unsigned long long idx)
{
    return (double)(splitmix64(seed ^ idx) >> 11) * (1.0 / 9007199254740992.0);
}

template <typename R>
struct Geo {
    R gcov[10];
    R gcon[10];
    R gdet;
    R alpha;
    R oma;    // 1 - alpha, evaluated in FP64 before rounding
    R igdet;  // 1 / sqrt(-g)
    R ialpha; // 1 / alpha
    R aig;    // alpha / sqrt(-g)
    R rfl;    // density floor of Eq. 34 at this radius (centre records)
    R ufl;    // internal-energy floor of Eq. 34
};

// counters accumulated on the device (indices into Grid::cnt)
enum {
    C_NR_ITERS = 0, C_NR, C_BRENT, C_ENT, C_ENT_BETA, C_FAIL, C_FLOOR, C_CEIL, C_GCAP,
    C_FIXED, C_SWEEPS, C_STEPS, C_LEARN, C_NCOUNT
};

// device status word bits
enum { ST_FIXUP = 1, ST_NONFINITE = 2, ST_FAILLIST = 4 };

struct Grid {
    int n1, n2, n3, N1, N2, N3;
    long long nz;
    int metric, bc1, bc2, bc3, riemann, mixed, i_h, nfix_cap;
    int x3warp;                 // X3 fluxes by row warps (rows of >= 32 faces)
    int flat3;                  // one phi zone with copied X3 ghosts: the face fluxes do not vary
    int recon;                  // 0 PLM (Eqs. 16-17), 1 PPM (faces read three zones on each side)
    int j0, n2t;                // a theta slab's first row and the whole grid's rows (0, n2: whole grid)
                                // along X3, so only k = 0 faces are computed and every k reads them
    double dx[3], idx[3], x1in, x2in, x3in;
    double gam, cfl, nr_tol, sigma_max, bu_max, gamma_max, beta_ent;
    double g1, igm1, isig, ibu; // (gam-1)/gam, 1/(gam-1), 1/sigma_max, 1/bu_max
    double ig;                  // 1/gam
    float isig_f, ibu_f;        // 1/sigma_max, 1/bu_max for the mixed path's FP32 ceiling test
    // FP32 copies of per-grid constants: the FP32 arithmetic of the mixed path
    // reads them instead of converting the FP64 values in every zone
    float gam_f, g1_f, beta_ent_f, gamma_max_f, tol_mixed_f, idx_f[3];
    float hidx_hi[3], hidx_lo[3]; // 1/(2 dX^d) as an FP32 pair (hi + lo, ~2^-48 relative)
    double nr_tol_mixed;        // sqrt(nr_tol): Newton acceptance of the mixed path
    int nr_maxit, brent_maxit, fix_maxsweep;
    int fcol;                   // faces per thread of the X1 / X2 flux sweeps (columns)
    // metric tables
    const Geo<double> *gc, *gf1, *gf2;
    const Geo<float> *gcF, *gf1F, *gf2F;
    const double *conn; // [N1*N2][40]: conn[l*10 + sym(m,n)]
    const float *connF;
    const double *rc;   // r of zone centres (1 for flat space)
    const double *gsp;  // [N1*N2][6] spatial inverse metric at centres, g^{ij} - g^{ti} g^{tj} / g^{tt}
                        // (packed 11 12 13 22 23 33)
    const unsigned char *polar2; // X2 face on a pole
    // state
    void *P[2];
    double *U;
    void *F[3];
    void *E[3];
    unsigned char *flag;
    double *scal;               // [0] dt, [1] t
    unsigned long long *dtmin;  // [3] per-direction CFL minima (bits of positive doubles)
    unsigned long long *cnt;    // [C_NCOUNT]
    int *status;
    int *faillist;              // compacted failed zones of a stage
    int *nfail;
    double *fixbuf;             // [5][nfix_cap] new primitives of a fixup sweep
    const float *mlp;           // learned Newton start of the inversion (null: start from the stage's primitives)
};

__host__ __device__ __forceinline__ long long zidx(const Grid &g, int i, int j, int k)
{
    return ((long long)(i + NG) * g.N2 + (j + NG)) * g.N3 + (k + NG);
}

__host__ __device__ __forceinline__ int midx(const Grid &g, int i, int j)
{
    return (i + NG) * g.N2 + (j + NG);
}

// ------------------------------------------------------------ dual numbers
// Forward-mode automatic differentiation: value and one directional derivative.
struct Dual {
    double v, d;
};
__host__ __device__ __forceinline__ Dual mkd(double v, double d = 0.0) { return Dual{v, d}; }
__host__ __device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__host__ __device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__host__ __device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__host__ __device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__host__ __device__ __forceinline__ Dual operator/(Dual a, Dual b)
{
    double q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
__host__ __device__ __forceinline__ Dual operator+(Dual a, double b) { return {a.v + b, a.d}; }
__host__ __device__ __forceinline__ Dual operator+(double a, Dual b) { return {a + b.v, b.d}; }
__host__ __device__ __forceinline__ Dual operator-(Dual a, double b) { return {a.v - b, a.d}; }
__host__ __device__ __forceinline__ Dual operator-(double a, Dual b) { return {a - b.v, -b.d}; }
__host__ __device__ __forceinline__ Dual operator*(Dual a, double b) { return {a.v * b, a.d * b}; }
__host__ __device__ __forceinline__ Dual operator*(double a, Dual b) { return {a * b.v, a * b.d}; }
__host__ __device__ __forceinline__ Dual operator/(Dual a, double b) { return {a.v / b, a.d / b}; }
__host__ __device__ __forceinline__ Dual operator/(double a, Dual b)
{
    double q = a / b.v;
    return {q, -q * b.d / b.v};
}
__host__ __device__ __forceinline__ Dual dsin(Dual a) { return {sin(a.v), cos(a.v) * a.d}; }
__host__ __device__ __forceinline__ Dual dcos(Dual a) { return {cos(a.v), -sin(a.v) * a.d}; }
__host__ __device__ __forceinline__ Dual dexp(Dual a)
{
    double e = exp(a.v);
    return {e, e * a.d};
}
__host__ __device__ __forceinline__ Dual dlog(Dual a) { return {log(a.v), a.d / a.v}; }
__host__ __device__ __forceinline__ Dual dsqrt(Dual a)
{
    double s = sqrt(a.v);
    return {s, 0.5 * a.d / s};
}
__host__ __device__ __forceinline__ double val(double a) { return a; }
__host__ __device__ __forceinline__ double val(Dual a) { return a.v; }
__host__ __device__ __forceinline__ double dsin(double a) { return sin(a); }
__host__ __device__ __forceinline__ double dcos(double a) { return cos(a); }
__host__ __device__ __forceinline__ double dexp(double a) { return exp(a); }
__host__ __device__ __forceinline__ double dlog(double a) { return log(a); }
__host__ __device__ __forceinline__ double dsqrt(double a) { return sqrt(a); }

// ------------------------------------------------ coordinates and metric
struct CoordParams {
    int metric;
    double a, hslope, xb, n_x, R0;
    double cyl_r, cyl_dx2; // polar cylindrification: radius r_c and band width in X2 (cyl_r <= 0: off)
};

// r(X1) of Eq. 36 and its Jacobian, for double or Dual arguments
template <typename T>
__host__ __device__ inline void mks_radius(const CoordParams &cp, T X1, T &r, T &drdx)
{
    if (val(X1) < cp.xb) {
        T e = dexp(X1);
        r = e + cp.R0;
        drdx = e;
    } else {
        T d = X1 - cp.xb;
        int n = (int)cp.n_x;
        T dn1 = d * 0.0 + 1.0;
        for (int m = 0; m < n - 1; m++) dn1 = dn1 * d;
        T e = dexp(X1 + dn1 * d);
        r = e + cp.R0;
        drdx = e * (1.0 + cp.n_x * dn1);
    }
}

// theta(X2) = pi/2 (1+X2) + (1-h)/2 sin(pi (1+X2))  (equator-refining form of Eq. 36)
template <typename T>
__host__ __device__ inline void mks_theta_raw(const CoordParams &cp, T X2, T &th, T &dthdx)
{
    const double pi = 3.141592653589793238462643;
    T y = (X2 + 1.0) * pi;
    th = (X2 + 1.0) * (0.5 * pi) + dsin(y) * (0.5 * (1.0 - cp.hslope));
    dthdx = dcos(y) * (0.5 * (1.0 - cp.hslope) * pi) + 0.5 * pi;
}

// theta(X1, X2) and its partial derivatives.  Without cylindrification the
// map of Eq. 36.  With it (Section 4.1 "cylindrifies" the cells next to the
// poles; the formula is not printed), inside a band of X2 width y_b next to
// each pole Eq. 36 is evaluated at a moved coordinate
//   X2' = pole -/+ y_b phi(s),  s = |X2 - pole| / y_b (negative past the pole),
//   phi(s) = s + (lambda - 1) s (1 - s^2)^3,  lambda(r) = (1 + (r_c / r)^4)^(1/4):
// the rows next to the pole are widened by lambda (r_c / r for r << r_c, so
// they keep a cylindrical radius of about r_c theta instead of shrinking
// with r), the rest of the band is narrowed, and phi(1) = phi'(1) = 1,
// phi''(1) = 0 join it smoothly to the MKS rows.  phi is odd, so the mirror
// across the pole is kept; lambda <= 5/2 (checked at grid creation) keeps
// phi' > 0.
template <typename T>
__host__ __device__ inline void mks_theta(const CoordParams &cp, T X1, T X2, T &th, T &dth1, T &dth2)
{
    if (!(cp.cyl_r > 0.0)) {
        mks_theta_raw(cp, X2, th, dth2);
        dth1 = X1 * 0.0;
        return;
    }
    const double yb = cp.cyl_dx2;
    const double sg = val(X2) < 0.0 ? 1.0 : -1.0; // +1 near the lower pole
    const T s = (X2 * sg + 1.0) * (1.0 / yb);
    if (!(fabs(val(s)) < 1.0)) {
        mks_theta_raw(cp, X2, th, dth2);
        dth1 = X1 * 0.0;
        return;
    }
    T r, drdx;
    mks_radius(cp, X1, r, drdx);
    T q = cp.cyl_r / r;
    q = q * q;
    q = q * q;
    const T lam = dsqrt(dsqrt(q + 1.0));
    const T dlam = -(lam * q) / (r * (q + 1.0)); // d lambda / dr
    const T c = 1.0 - s * s;
    const T c3 = c * c * c;
    const T lm1 = lam - 1.0;
    const T phi = s + lm1 * s * c3;
    const T dphi = 1.0 + lm1 * (c * c) * (1.0 - 7.0 * s * s); // d phi / ds
    T dthM;
    mks_theta_raw(cp, (phi * yb - 1.0) * sg, th, dthM);
    dth2 = dthM * dphi;                                  // dX2'/dX2 = phi'(s) on both sides
    dth1 = dthM * ((s * c3) * (dlam * drdx) * (yb * sg)); // via d lambda / dX1
}

// metric g_{mu nu} in code coordinates (Kerr-Schild, Eq. 35, pulled back by Eq. 36)
template <typename T>
__host__ __device__ inline void code_gcov(const CoordParams &cp, T X1, T X2, T g[4][4])
{
    for (int m = 0; m < 4; m++)
        for (int n = 0; n < 4; n++) g[m][n] = X1 * 0.0;
    if (cp.metric == MINK_CART) {
        g[0][0] = g[0][0] - 1.0;
        g[1][1] = g[1][1] + 1.0;
        g[2][2] = g[2][2] + 1.0;
        g[3][3] = g[3][3] + 1.0;
        return;
    }
    T r, dr, th, dth1, dth;
    mks_radius(cp, X1, r, dr);
    mks_theta(cp, X1, X2, th, dth1, dth);
    const double a = cp.a;
    T s = dsin(th), c = dcos(th);
    T s2 = s * s;
    T sig = r * r + (c * c) * (a * a);
    T z = (r * 2.0) / sig;
    T onez = z + 1.0;
    T gk[4][4];
    gk[0][0] = z - 1.0;
    gk[0][1] = z;
    gk[0][2] = z * 0.0;
    gk[0][3] = -(z * s2) * a;
    gk[1][1] = onez;
    gk[1][2] = z * 0.0;
    gk[1][3] = -(onez * s2) * a;
    gk[2][2] = sig;
    gk[2][3] = z * 0.0;
    gk[3][3] = s2 * (sig + onez * s2 * (a * a));
    if (!(cp.cyl_r > 0.0)) {
        T J[4] = {X1 * 0.0 + 1.0, dr, dth, X1 * 0.0 + 1.0};
        for (int m = 0; m < 4; m++)
            for (int n = m; n < 4; n++) {
                g[m][n] = gk[m][n] * J[m] * J[n];
                g[n][m] = g[m][n];
            }
        return;
    }
    // cylindrified: theta depends on X1 too, g_{mu nu} = J^a_mu J^b_nu g^KS_{ab}
    // with J^r_1 = dr/dX1, J^theta_1 = dtheta/dX1, J^theta_2 = dtheta/dX2
    for (int m = 0; m < 4; m++)
        for (int n = m; n < 4; n++) g[m][n] = gk[m][n];
    g[1][1] = gk[1][1] * dr * dr + gk[2][2] * dth1 * dth1;
    g[1][2] = gk[2][2] * dth1 * dth;
    g[2][2] = gk[2][2] * dth * dth;
    g[0][1] = gk[0][1] * dr;
    g[1][3] = gk[1][3] * dr;
    for (int m = 0; m < 4; m++)
        for (int n = 0; n < m; n++) g[m][n] = g[n][m];
}

} // namespace grmhd
