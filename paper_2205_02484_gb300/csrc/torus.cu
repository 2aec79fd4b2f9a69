// torus.cu -- initial state: Fishbone-Moncrief torus (Section 5), single
// poloidal loop A_phi = max(rho/rho_max - 0.2, 0) (Eq. 45) normalised to
// beta_0 = max p_g / max p_B, and a random internal-energy perturbation.
//
// Torus in Boyer-Lindquist coordinates (M = 1) with the FM invariant
// l = u^t u_phi, e^{2(nu - psi)} = Sigma^2 Delta / (A^2 sin^2):
//   ln h = 1/2 ln[(1 + R)/(Sigma Delta / A)] - R/2 - 2 a l r / A,
//   R = sqrt(1 + 4 l^2 e^{2(nu-psi)}),  minus its value at (r_in, pi/2);
// X^2 = (R - 1)/2 (ZAMO-frame u_(phi)^2), u^t = sqrt((1 + X^2) A/(Sigma Delta)),
// u^phi = 2 a r sqrt(1 + X^2)/sqrt(A Sigma Delta) + X sqrt(Sigma/A)/sin;
// l solves d ln h / dr = 0 at (r_max, pi/2).  With u^r = 0 the contravariant
// components are the same in Kerr-Schild coordinates.
#include "physics.cuh"
#include "kernels.h"

namespace grmhd {

template <typename T>
__host__ __device__ inline T fm_lnh_t(double a, double l, T r, double th)
{
    double s = sin(th), c = cos(th);
    T sig = r * r + a * a * c * c;
    T del = r * r - r * 2.0 + a * a;
    T rr = r * r + a * a;
    T A = rr * rr - del * (a * a * s * s);
    T R = dsqrt((sig * sig * del) * (4.0 * l * l) / (A * A * (s * s)) + 1.0);
    return dlog((R + 1.0) / (sig * del / A)) * 0.5 - R * 0.5 - r * (2.0 * a * l) / A;
}

double fm_lnh_host(double a, double ell, double r, double th) { return fm_lnh_t<double>(a, ell, r, th); }

double fm_ell_host(double a, double r_max)
{
    auto dlnh = [&](double l) { return fm_lnh_t<Dual>(a, l, mkd(r_max, 1.0), 1.5707963267948966).d; };
    double lo = 0.5, hi = 50.0, flo = dlnh(lo);
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi), fm = dlnh(mid);
        if ((fm > 0) == (flo > 0)) { lo = mid; flo = fm; }
        else hi = mid;
        if (hi - lo < 1e-15 * mid) break;
    }
    return 0.5 * (lo + hi);
}

__device__ inline double fm_rho(const TorusArgs &ta, double gam, double r, double th, bool &in)
{
    in = false;
    if (r < ta.r_in || fabs(sin(th)) < 1e-10) return 0.0;
    double lnh = fm_lnh_t<double>(ta.a, ta.ell, r, th) - ta.lnh_in;
    if (!(lnh > 0.0)) return 0.0;
    in = true;
    double hm1 = expm1(lnh);
    return pow(hm1 * (gam - 1.0) / (ta.kappa * gam), 1.0 / (gam - 1.0));
}

__device__ inline double atomic_max_pos(double *addr, double v)
{
    return __longlong_as_double(
        (long long)atomicMax((unsigned long long *)addr, (unsigned long long)__double_as_longlong(v)));
}

// Pd: active-zone FP64 primitives [8][nact]; red[0] = rho_max
__global__ void k_torus_prims(Grid g, TorusArgs ta, double *Pd, unsigned char *intorus, double *red)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.n1 * g.n2) return;
    int i = t / g.n2, j = t % g.n2;
    long long nact = (long long)g.n1 * g.n2 * g.n3;
    double X1 = g.x1in + (i + 0.5) * g.dx[0], X2 = g.x2in + (j + 0.5) * g.dx[1];
    double r, dr, th, dth1, dth;
    mks_radius<double>(ta.cp, X1, r, dr);
    mks_theta<double>(ta.cp, X1, X2, th, dth1, dth);
    bool in;
    double rho = fm_rho(ta, g.gam, r, th, in);
    double q[NP] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (in) {
        q[KRHO] = rho;
        q[KUU] = ta.kappa * pow(rho, g.gam) / (g.gam - 1.0);
        double s = sin(th), c = cos(th), a = ta.a;
        double sig = r * r + a * a * c * c, del = r * r - 2.0 * r + a * a;
        double A = (r * r + a * a) * (r * r + a * a) - del * a * a * s * s;
        double X2s = 0.5 * (sqrt(1.0 + 4.0 * ta.ell * ta.ell * sig * sig * del / (A * A * s * s)) - 1.0);
        double X = sqrt(X2s);
        double ut = sqrt((1.0 + X2s) * A / (sig * del));
        double uph = 2.0 * a * r * sqrt(1.0 + X2s) / sqrt(A * sig * del) + X * sqrt(sig / A) / s;
        const Geo<double> geo = g.gc[midx(g, i, j)];
        double lor = geo.alpha * ut;
        double ucon[4] = {ut, 0.0, 0.0, uph};
        for (int dd = 1; dd <= 3; dd++) q[KU1 + dd - 1] = ucon[dd] + lor * geo.alpha * geo.gcon[sym(0, dd)];
        atomic_max_pos(&red[0], rho);
    }
    intorus[t] = in;
    for (int k = 0; k < g.n3; k++) {
        long long a = ((long long)i * g.n2 + j) * g.n3 + k;
        for (int cc = 0; cc < NP; cc++) Pd[cc * nact + a] = q[cc];
    }
}

__global__ void k_torus_norm(Grid g, double *Pd, const double *red)
{
    long long nact = (long long)g.n1 * g.n2 * g.n3;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nact) return;
    double rm = red[0];
    Pd[t] /= rm;
    Pd[nact + t] /= rm;
}

// A_phi at corners (i-1/2, j-1/2), i in [0, n1], j in [0, n2]
__global__ void k_aphi(Grid g, TorusArgs ta, const double *red, double *Aph)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (g.n1 + 1) * (g.n2 + 1)) return;
    int i = t / (g.n2 + 1), j = t % (g.n2 + 1);
    double r, dr, th, dth1, dth;
    const double X1 = g.x1in + i * g.dx[0];
    mks_radius<double>(ta.cp, X1, r, dr);
    mks_theta<double>(ta.cp, X1, g.x2in + j * g.dx[1], th, dth1, dth);
    bool in;
    double rho = fm_rho(ta, g.gam, r, th, in);
    double v = rho / red[0] - 0.2;
    Aph[t] = v > 0.0 ? v : 0.0;
}

// B from the discrete curl so that the corner divergence of Eq. 24 vanishes;
// red[1] = max p_g, red[2] = max b^2
__global__ void k_bfield(Grid g, double *Pd, const double *Aph, double *red)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.n1 * g.n2) return;
    int i = t / g.n2, j = t % g.n2;
    long long nact = (long long)g.n1 * g.n2 * g.n3;
    int w = g.n2 + 1;
    double A00 = Aph[i * w + j], A01 = Aph[i * w + j + 1], A10 = Aph[(i + 1) * w + j], A11 = Aph[(i + 1) * w + j + 1];
    const Geo<double> geo = g.gc[midx(g, i, j)];
    double b1 = (A01 + A11 - A00 - A10) / (2.0 * g.dx[1]);
    double b2 = -(A10 + A11 - A00 - A01) / (2.0 * g.dx[0]);
    double pmax = 0.0, bmax = 0.0;
    for (int k = 0; k < g.n3; k++) {
        long long a = ((long long)i * g.n2 + j) * g.n3 + k;
        Pd[KB1 * nact + a] = b1 / geo.gdet;
        Pd[KB2 * nact + a] = b2 / geo.gdet;
        Pd[KB3 * nact + a] = 0.0;
        double q[NP];
        for (int c = 0; c < NP; c++) q[c] = Pd[c * nact + a];
        St<double> s;
        get_state(q, geo, s);
        pmax = fmax(pmax, (g.gam - 1.0) * q[KUU]);
        bmax = fmax(bmax, s.bsq);
    }
    atomic_max_pos(&red[1], pmax);
    atomic_max_pos(&red[2], bmax);
}

__global__ void k_bscale(Grid g, double *Pd, const double *red, double beta0)
{
    long long nact = (long long)g.n1 * g.n2 * g.n3;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nact || !(red[2] > 0.0)) return;
    double f = sqrt(red[1] / (0.5 * red[2]) / beta0);
    for (int c = KB1; c <= KB3; c++) Pd[c * nact + t] *= f;
}

// disk integrals (before the perturbation): per-block partial sums
__global__ void k_disk_partial(Grid g, const double *Pd, const unsigned char *intorus, double *part)
{
    long long nact = (long long)g.n1 * g.n2 * g.n3;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double m = 0.0, e = 0.0;
    if (t < nact) {
        int k = (int)(t % g.n3);
        long long r = t / g.n3;
        int j = (int)(r % g.n2), i = (int)(r / g.n2);
        (void)k;
        if (intorus[i * g.n2 + j]) {
            const Geo<double> geo = g.gc[midx(g, i, j)];
            double q[NP];
            for (int c = 0; c < NP; c++) q[c] = Pd[c * nact + t];
            St<double> s;
            get_state(q, geo, s);
            double dV = g.dx[0] * g.dx[1] * g.dx[2];
            m = geo.gdet * q[KRHO] * dV;
            e = geo.gdet * s.bsq * dV;
        }
    }
    __shared__ double sm[2][256];
    sm[0][threadIdx.x] = m;
    sm[1][threadIdx.x] = e;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sm[0][threadIdx.x] += sm[0][threadIdx.x + o];
            sm[1][threadIdx.x] += sm[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sm[0][0];
        part[2 * blockIdx.x + 1] = sm[1][0];
    }
}

__global__ void k_sum_pairs(const double *part, int n, double *out)
{
    if (threadIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int i = 0; i < n; i++) {
        a += part[2 * i];
        b += part[2 * i + 1];
    }
    out[0] = a;
    out[1] = b;
}

// perturbation, floors, conserved variables, write into the ghosted state
template <typename RS>
__global__ void k_torus_finish(Grid g, TorusArgs ta, const double *Pd, const unsigned char *intorus)
{
    long long nact = (long long)g.n1 * g.n2 * g.n3;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nact) return;
    int k = (int)(t % g.n3);
    long long r = t / g.n3;
    int j = (int)(r % g.n2), i = (int)(r / g.n2);
    double q[NP];
    for (int c = 0; c < NP; c++) q[c] = Pd[c * nact + t];
    if (intorus[i * g.n2 + j] && ta.pert_amp != 0.0) {
        double xi = counter_uniform(ta.seed, (unsigned long long)t);
        q[KUU] *= 1.0 + ta.pert_amp * (2.0 * xi - 1.0);
    }
    int m = midx(g, i, j);
    double rfl = 1e-20, ufl = 1e-20;
    if (g.metric == KERR_MKS) {
        rfl = fmax(rfl, 1e-5 * pow(g.rc[m], -0.5));
        ufl = fmax(ufl, (1e-5 / 3.0) * pow(g.rc[m], -2.5));
    }
    if (q[KRHO] < rfl) q[KRHO] = rfl;
    if (q[KUU] < ufl) q[KUU] = ufl;
    const Geo<double> geo = g.gc[m];
    St<double> s;
    get_state(q, geo, s);
    double U[NU];
    prim_to_UF<double, false>(q, geo, s, g.gam, 0, U);
    long long z = zidx(g, i, j, k);
    RS *P = (RS *)g.P[0];
    for (int c = 0; c < NP; c++) P[c * g.nz + z] = (RS)q[c];
    for (int c = 0; c < NU; c++) g.U[c * g.nz + z] = U[c];
}

void launch_torus(const Grid &g, const TorusArgs &ta, double *scratch, unsigned char *intorus,
                  double *out_host6, cudaStream_t s)
{
    long long nact = (long long)g.n1 * g.n2 * g.n3;
    double *Pd = scratch;
    double *red = scratch + 8 * nact;      // 8 slots
    double *Aph = red + 8;                 // (n1+1)(n2+1)
    double *part = Aph + (long long)(g.n1 + 1) * (g.n2 + 1);
    cudaMemsetAsync(red, 0, 8 * sizeof(double), s);
    int nij = g.n1 * g.n2;
    k_torus_prims<<<(nij + 127) / 128, 128, 0, s>>>(g, ta, Pd, intorus, red);
    unsigned nb = (unsigned)((nact + 255) / 256);
    k_torus_norm<<<nb, 256, 0, s>>>(g, Pd, red);
    if (ta.beta0 > 0.0) {
        int nc = (g.n1 + 1) * (g.n2 + 1);
        k_aphi<<<(nc + 127) / 128, 128, 0, s>>>(g, ta, red, Aph);
        k_bfield<<<(nij + 127) / 128, 128, 0, s>>>(g, Pd, Aph, red);
        k_bscale<<<nb, 256, 0, s>>>(g, Pd, red, ta.beta0);
    }
    k_disk_partial<<<nb, 256, 0, s>>>(g, Pd, intorus, part);
    k_sum_pairs<<<1, 32, 0, s>>>(part, (int)nb, red + 4);
    if (g.mixed) k_torus_finish<float><<<nb, 256, 0, s>>>(g, ta, Pd, intorus);
    else k_torus_finish<double><<<nb, 256, 0, s>>>(g, ta, Pd, intorus);
    cudaMemcpyAsync(out_host6, red, 6 * sizeof(double), cudaMemcpyDeviceToHost, s);
}

} // namespace grmhd
