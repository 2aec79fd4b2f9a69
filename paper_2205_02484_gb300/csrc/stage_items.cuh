// stage_items.cuh -- the per-element bodies of one RK2 stage, shared by the
// single-grid kernels (step.cu) and the persistent ensemble kernels
// (ensemble.cu).  Each item function processes one element (a face, an edge,
// a zone or a ghost zone) of one grid and returns what the caller reduces.
//
//   boundary fill (Section 4.1)  -> polar_item, bc1_item, bc2_item, bc3_item
//   face fluxes (Eqs. 16-21)     -> flux_item<D>: PLM-MC face states, U and F of
//                                   both states, LLF/HLL, c_w, CFL candidate (Eq. 27)
//   flux-CT EMFs (Eq. 22)        -> emf_item
//   update + inversion           -> update_item: flux divergence with the flux-CT
//                                   B-fluxes of Eq. 23 formed from the EMFs,
//                                   connection source (Eq. 15), RK2 stage update
//                                   (Eqs. 25-26) with FP64 accumulation, FP64
//                                   inversion (Section 2.3), floors/ceilings/cap
//                                   (Section 2.4); failed zones are compacted
//   fixups (Eq. 33)              -> fixup_block / fixup_sweep: Jacobi sweeps over the list (one block)
//   dt                           -> finalize_one
//
// R is the flux arithmetic type (double, or float in the mixed path), which is
// also the primitive storage type.
#pragma once
#include "fixes.cuh"
#include "mlp.cuh"

namespace grmhd {

struct Box {
    int lo[3], n[3];
    __host__ __device__ long long count() const { return (long long)n[0] * n[1] * n[2]; }
};

// element boxes of one grid: faces along X1..X3 (with the ring flux-CT
// needs), edges, active zones
__host__ __device__ inline Box flux_box(const Grid &g, int d)
{
    if (g.flat3) { // the k = 0 faces stand for every k
        if (d == 1) return Box{{0, -1, 0}, {g.n1 + 1, g.n2 + 2, 1}};
        if (d == 2) return Box{{-1, 0, 0}, {g.n1 + 2, g.n2 + 1, 1}};
        return Box{{-1, -1, 0}, {g.n1 + 2, g.n2 + 2, 1}};
    }
    if (d == 1) return Box{{0, -1, -1}, {g.n1 + 1, g.n2 + 2, g.n3 + 2}};
    if (d == 2) return Box{{-1, 0, -1}, {g.n1 + 2, g.n2 + 1, g.n3 + 2}};
    return Box{{-1, -1, 0}, {g.n1 + 2, g.n2 + 2, g.n3 + 1}};
}
__host__ __device__ inline Box edge_box(const Grid &g) { return Box{{0, 0, 0}, {g.n1 + 1, g.n2 + 1, g.n3 + 1}}; }
__host__ __device__ inline long long nact_of(const Grid &g) { return (long long)g.n1 * g.n2 * g.n3; }
// a theta slab holds the whole grid's low / high pole rows
__host__ __device__ inline bool has_pole_lo(const Grid &g) { return g.j0 == 0; }
__host__ __device__ inline bool has_pole_hi(const Grid &g) { return g.j0 + g.n2 == g.n2t; }
// the X2 ghost rows of a side come from the caller: a theta slab's side
// inside the grid, or a periodic side of the whole grid
__host__ __device__ inline bool x2_external(const Grid &g, int side)
{
    if (g.n2t == g.n2) return false;
    if (!(side == 0 ? has_pole_lo(g) : has_pole_hi(g))) return true;
    return g.metric != KERR_MKS && g.bc2 == BC_PERIODIC;
}
__host__ __device__ inline long long polar_count(const Grid &g)
{
    return (g.metric == KERR_MKS && g.n2t >= 6 && (has_pole_lo(g) || has_pole_hi(g))) ? (long long)g.n1 * g.n3
                                                                                       : 0;
}
__host__ __device__ inline long long bc1_count(const Grid &g) { return (long long)g.n2 * g.n3 * NG * 2; }
__host__ __device__ inline long long bc2_count(const Grid &g) { return (long long)(g.n1 + 2 * NG) * g.n3 * NG * 2; }
__host__ __device__ inline long long bc3_count(const Grid &g)
{
    return (long long)(g.n1 + 2 * NG) * (g.n2 + 2 * NG) * NG * 2;
}

__device__ __forceinline__ void box_decode(const Box &b, long long t, int &i, int &j, int &k)
{
    k = (int)(t % b.n[2]);
    long long r = t / b.n[2];
    j = (int)(r % b.n[1]);
    i = (int)(r / b.n[1]);
    i += b.lo[0];
    j += b.lo[1];
    k += b.lo[2];
}

template <typename T>
__device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// CFL step of a block's faces: min over faces of num / c_w = num / (max c_w)
// exactly (IEEE division is monotonic in the divisor), so the block reduces
// max c_w in the flux precision and divides once (num = cfl dX^D); every
// thread of the block must call it; *dst holds the bits of a positive double
template <typename R>
__device__ __forceinline__ void block_cfl_into(unsigned long long *dst, R cw, double num)
{
    __shared__ R sm[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cw = max(cw, __shfl_xor_sync(0xffffffffu, cw, o));
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[w] = cw;
    __syncthreads();
    if (w == 0) {
        R x = lane < (int)(blockDim.x >> 5) ? sm[lane] : R(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(0xffffffffu, x, o));
        if (lane == 0 && x > R(0)) atomicMin(dst, dbits(num / (double)x));
    }
}

__device__ __forceinline__ void block_count(unsigned long long *dst, unsigned v)
{
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, (unsigned long long)v);
}

// ------------------------------------------------------------ boundary fill

__device__ __forceinline__ int wrapi(int k, int n) { return ((k % n) + n) % n; }

template <typename RS>
__device__ __forceinline__ void polar_item(const Grid &g, RS *P, long long t)
{
    if (t >= polar_count(g)) return;
    int i = (int)(t / g.n3), k = (int)(t % g.n3);
    const long long f = (long long)KU2 * g.nz;
    if (has_pole_lo(g)) {
        RS a = P[f + zidx(g, i, 2, k)];
        P[f + zidx(g, i, 0, k)] = a * RS(0.5 / 2.5);
        P[f + zidx(g, i, 1, k)] = a * RS(1.5 / 2.5);
    }
    if (has_pole_hi(g)) {
        RS b = P[f + zidx(g, i, g.n2 - 3, k)];
        P[f + zidx(g, i, g.n2 - 1, k)] = b * RS(0.5 / 2.5);
        P[f + zidx(g, i, g.n2 - 2, k)] = b * RS(1.5 / 2.5);
    }
}

// u^1 = 0 at fixed ut^2, ut^3: ut^1 = Gamma alpha g^{t1}, Gamma from its quadratic
__device__ inline void zero_radial_velocity(const Geo<double> &geo, double q[NP])
{
    double c = geo.alpha * geo.gcon[1];
    double a2 = 1.0 - geo.gcov[4] * c * c;
    if (!(a2 > 0.0)) return;
    double b = -2.0 * c * (geo.gcov[5] * q[KU2] + geo.gcov[6] * q[KU3]);
    double rest = geo.gcov[7] * q[KU2] * q[KU2] + 2.0 * geo.gcov[8] * q[KU2] * q[KU3] +
                  geo.gcov[9] * q[KU3] * q[KU3];
    double cc = -(1.0 + rest);
    double disc = b * b - 4.0 * a2 * cc;
    double gm = (-b + sqrt(disc)) / (2.0 * a2);
    q[KU1] = gm * c;
}

// Mixed path: whether the radial ghost (id, j) of side `side` flows into the
// grid, from the FP32 state of the stored primitives of its source zone zs
// on the FP32 record (out of line, so that the single-grid and ensemble
// kernels take the same decision).
static __device__ __noinline__ bool ghost_inflow_f(const Grid &g, const float *P, long long zs, int id, int j,
                                                   int side)
{
    float qf[NP];
#pragma unroll
    for (int c = 0; c < NP; c++) qf[c] = P[c * g.nz + zs];
    const Geo<float> gf = g.gcF[midx(g, id, j)];
    St<float> sf;
    get_state(qf, gf, sf);
    return (side == 0 && sf.ucon[1] > 0.0f) || (side == 1 && sf.ucon[1] < 0.0f);
}

template <typename RS>
__device__ inline void bc1_item(const Grid &g, RS *P, long long t)
{
    if (t >= bc1_count(g)) return;
    int side = (int)(t % 2);
    long long r = t / 2;
    int gh = 1 + (int)(r % NG);
    r /= NG;
    int k = (int)(r % g.n3), j = (int)(r / g.n3);
    int bc = g.metric == KERR_MKS ? BC_INFLOW : g.bc1;
    int id = side == 0 ? -gh : g.n1 - 1 + gh;
    int is;
    if (bc == BC_PERIODIC) is = wrapi(id, g.n1);
    else is = side == 0 ? 0 : g.n1 - 1;
    long long zs = zidx(g, is, j, k), zd = zidx(g, id, j, k);
    bool copy = bc != BC_INFLOW;
    if constexpr (sizeof(RS) == 4) {
        // mixed path: the sign of u^r from the FP32 state of the stored
        // primitives on the FP32 record (the FP64 correction only where the
        // ghost flows into the grid; a sign within FP32 rounding of zero
        // moves u^r by that rounding either way)
        if (!copy) copy = !ghost_inflow_f(g, (const float *)P, zs, id, j, side);
    }
    if (copy) {
#pragma unroll
        for (int c = 0; c < NP; c++) P[c * g.nz + zd] = P[c * g.nz + zs];
        return;
    }
    double q[NP];
#pragma unroll
    for (int c = 0; c < NP; c++) q[c] = (double)P[c * g.nz + zs];
    Geo<double> geo = g.gc[midx(g, id, j)];
    if constexpr (sizeof(RS) == 4) {
        zero_radial_velocity(geo, q);
    } else {
        St<double> s;
        get_state(q, geo, s);
        if ((side == 0 && s.ucon[1] > 0.0) || (side == 1 && s.ucon[1] < 0.0)) zero_radial_velocity(geo, q);
    }
#pragma unroll
    for (int c = 0; c < NP; c++) P[c * g.nz + zd] = (RS)q[c];
}

template <typename RS>
__device__ __forceinline__ void bc2_item(const Grid &g, RS *P, long long t)
{
    if (t >= bc2_count(g)) return;
    int side = (int)(t % 2);
    long long r = t / 2;
    int gh = 1 + (int)(r % NG);
    r /= NG;
    int k = (int)(r % g.n3), i = (int)(r / g.n3) - NG;
    if (x2_external(g, side)) return; // a theta slab's inner side: the neighbour's rows
    int bc = g.metric == KERR_MKS ? BC_POLAR : g.bc2;
    int jd = side == 0 ? -gh : g.n2 - 1 + gh;
    int js;
    bool flip = false;
    if (bc == BC_POLAR) {
        js = side == 0 ? gh - 1 : g.n2 - gh;
        flip = true;
    } else if (bc == BC_PERIODIC) {
        js = wrapi(jd, g.n2);
    } else {
        js = side == 0 ? 0 : g.n2 - 1;
    }
    long long zs = zidx(g, i, js, k), zd = zidx(g, i, jd, k);
#pragma unroll
    for (int c = 0; c < NP; c++) {
        RS v = P[c * g.nz + zs];
        if (flip && (c == KU2 || c == KB2)) v = -v;
        P[c * g.nz + zd] = v;
    }
}

template <typename RS>
__device__ __forceinline__ void bc3_item(const Grid &g, RS *P, long long t)
{
    if (t >= bc3_count(g)) return;
    int side = (int)(t % 2);
    long long r = t / 2;
    int gh = 1 + (int)(r % NG);
    r /= NG;
    int j = (int)(r % (g.n2 + 2 * NG)) - NG, i = (int)(r / (g.n2 + 2 * NG)) - NG;
    int bc = (g.metric == KERR_MKS && g.bc3 != BC_EXTERNAL) ? BC_PERIODIC : g.bc3;
    if (bc == BC_EXTERNAL) return; // a slab's X3 ghosts come from its neighbours
    int kd = side == 0 ? -gh : g.n3 - 1 + gh;
    int ks = bc == BC_PERIODIC ? wrapi(kd, g.n3) : (side == 0 ? 0 : g.n3 - 1);
    long long zs = zidx(g, i, j, ks), zd = zidx(g, i, j, kd);
#pragma unroll
    for (int c = 0; c < NP; c++) P[c * g.nz + zd] = P[c * g.nz + zs];
}

// ------------------------------------------------------------- face fluxes

template <typename R>
__device__ __forceinline__ const Geo<R> *face_table(const Grid &g, int d);
template <>
__device__ __forceinline__ const Geo<double> *face_table<double>(const Grid &g, int d)
{
    return d == 1 ? g.gf1 : (d == 2 ? g.gf2 : g.gc);
}
template <>
__device__ __forceinline__ const Geo<float> *face_table<float>(const Grid &g, int d)
{
    return d == 1 ? g.gf1F : (d == 2 ? g.gf2F : g.gcF);
}

// Riemann flux of one face from its two reconstructed states (Eqs. 18-21);
// cw receives the face's c_w.
template <typename R, int D>
__device__ __forceinline__ void face_flux(const Grid &g, const Geo<R> &geo, const R ql[NP], const R qr[NP],
                                          R out[NU], R &cw)
{
    St<R> sl, sr;
    get_state(ql, geo, sl);
    get_state(qr, geo, sr);
    R gam = sizeof(R) == 4 ? (R)g.gam_f : (R)g.gam;
    R c1l, c2l, c1r, c2r;
    wave_speeds(ql, geo, sl, gam, D, c1l, c2l);
    wave_speeds(qr, geo, sr, gam, D, c1r, c2r);
    R cmax = fabs(fmax(R(0), fmax(c1r, c1l)));
    R cmin = fabs(fmax(R(0), fmax(-c2r, -c2l)));
    cw = fmax(cmax, cmin);
    R wlF, wlU, wrF, wrU;
    if (g.riemann == 1 && cmax + cmin > R(0)) {
        R inv = divr(R(1), cmax + cmin);
        wlF = cmax * inv;
        wrF = cmin * inv;
        wlU = cmax * cmin * inv;
        wrU = -wlU;
    } else if (g.riemann == 1) {
        wlF = wrF = R(0.5);
        wlU = wrU = R(0);
    } else {
        wlF = wrF = R(0.5);
        wlU = R(0.5) * cw;
        wrU = -wlU;
    }
    constexpr bool RMS = sizeof(R) == 4;
    R Ux[NU], Fx[NU];
    prim_to_UF2<R, RMS>(ql, geo, sl, gam, D, Ux, Fx);
#pragma unroll
    for (int c = 0; c < NU; c++) out[c] = wlF * Fx[c] + wlU * Ux[c];
    prim_to_UF2<R, RMS>(qr, geo, sr, gam, D, Ux, Fx);
#pragma unroll
    for (int c = 0; c < NU; c++) out[c] += wrF * Fx[c] + wrU * Ux[c];
}

// c_w of face (i, j, k) if it is an active face (it enters the CFL step of
// Eq. 27), else 0
template <typename R, int D>
__device__ __forceinline__ R face_cw(const Grid &g, int i, int j, int k, R cw)
{
    int ix[3] = {i, j, k}, nn[3] = {g.n1, g.n2, g.n3};
    bool act = true;
#pragma unroll
    for (int e = 0; e < 3; e++) act = act && ix[e] >= 0 && ix[e] < nn[e] + (e == D - 1 ? 1 : 0);
    return act ? cw : R(0);
}

// Face (i,j,k) of direction D lies between zone index-1 and index along D.
// Returns the face's c_w if it is active (else 0).
template <typename R, int D>
__device__ __forceinline__ R flux_item(const Grid &g, const R *__restrict__ P, R *__restrict__ F,
                                       const Box &box, int want_dt, long long t)
{
    if (t >= box.count()) return R(0);
    int i, j, k;
    box_decode(box, t, i, j, k);
    long long z = zidx(g, i, j, k);
    R out[NU];
    R cw = R(0);
    bool polar = (D == 2) && g.polar2[midx(g, i, j)];
    if (polar) {
#pragma unroll
        for (int c = 0; c < NU; c++) out[c] = R(0);
    } else {
        const long long st = D == 1 ? (long long)g.N2 * g.N3 : (D == 2 ? g.N3 : 1);
        R ql[NP], qr[NP];
#pragma unroll
        for (int c = 0; c < NP; c++) {
            const R *pc = P + c * g.nz + z;
            R qm2 = ldg(pc - 2 * st), qm1 = ldg(pc - st), q0 = ldg(pc), qp1 = ldg(pc + st);
            ql[c] = qm1 + R(0.5) * mc_slope(qm2, qm1, q0);
            qr[c] = q0 - R(0.5) * mc_slope(qm1, q0, qp1);
        }
        face_flux<R, D>(g, face_table<R>(g, D)[midx(g, i, j)], ql, qr, out, cw);
    }
#pragma unroll
    for (int c = 0; c < NU; c++) F[c * g.nz + z] = out[c];
    return want_dt ? face_cw<R, D>(g, i, j, k, cw) : R(0);
}

// One face of direction D with the PPM face states (six zones along D, idx-3
// .. idx+2); the same Riemann flux and c_w as flux_item.  Box: flux_box.
template <typename R, int D>
__device__ __forceinline__ R flux_item_ppm(const Grid &g, const R *__restrict__ P, R *__restrict__ F,
                                           const Box &box, int want_dt, long long t)
{
    if (t >= box.count()) return R(0);
    int i, j, k;
    box_decode(box, t, i, j, k);
    long long z = zidx(g, i, j, k);
    R out[NU];
    R cw = R(0);
    if ((D == 2) && g.polar2[midx(g, i, j)]) {
#pragma unroll
        for (int c = 0; c < NU; c++) out[c] = R(0);
    } else {
        const long long st = D == 1 ? (long long)g.N2 * g.N3 : (D == 2 ? g.N3 : 1);
        R ql[NP], qr[NP];
#pragma unroll
        for (int c = 0; c < NP; c++) {
            const R *pc = P + c * g.nz + z;
            R q6[6];
#pragma unroll
            for (int m = 0; m < 6; m++) q6[m] = ldg(pc + (m - 3) * st);
            ppm_face(q6, ql[c], qr[c]);
        }
        face_flux<R, D>(g, face_table<R>(g, D)[midx(g, i, j)], ql, qr, out, cw);
    }
#pragma unroll
    for (int c = 0; c < NU; c++) F[c * g.nz + z] = out[c];
    return want_dt ? face_cw<R, D>(g, i, j, k, cw) : R(0);
}

// Columns of g.fcol consecutive faces along X1 or X2: one thread walks its
// column with a three-zone window in registers, so each zone is loaded and
// its MC slope formed once instead of once per face (the face values are the
// same numbers flux_item forms, whatever the column length).  col_box counts
// columns: the face box with its extent along D divided into chunks of
// g.fcol (faces along D start at 0).  The host picks g.fcol per grid: long
// columns for large grids, single faces where columns would leave the GPU
// with too few threads.
__host__ __device__ inline Box col_box(const Grid &g, int d)
{
    Box b = flux_box(g, d);
    b.n[d - 1] = (b.n[d - 1] + g.fcol - 1) / g.fcol;
    return b;
}

template <typename R, int D>
__device__ __forceinline__ R flux_column(const Grid &g, const R *__restrict__ P, R *__restrict__ F,
                                         const Box &cb, int want_dt, long long t)
{
    static_assert(D == 1 || D == 2, "columns run along X1 or X2");
    R cwm = R(0); // largest c_w of the column's active faces
    if (t >= cb.count()) return cwm;
    int i, j, k;
    box_decode(cb, t, i, j, k);
    const int nf = (D == 1 ? g.n1 : g.n2) + 1;
    const int f0 = (D == 1 ? i : j) * g.fcol, f1 = min(f0 + g.fcol, nf);
    if (D == 1) i = f0;
    else j = f0;
    const long long st = D == 1 ? (long long)g.N2 * g.N3 : g.N3;
    const long long z0 = zidx(g, i, j, k); // zone f0; face f lies between zones f-1 and f
    // zones f-1, f, f+1 of the current face f and the slope of zone f-1
    R qa[NP], qb[NP], qc[NP], sa[NP];
#pragma unroll
    for (int c = 0; c < NP; c++) {
        const R *pc = P + c * g.nz + z0;
        R qm2 = ldg(pc - 2 * st);
        qa[c] = ldg(pc - st);
        qb[c] = ldg(pc);
        qc[c] = ldg(pc + st);
        sa[c] = mc_slope(qm2, qa[c], qb[c]);
    }
    for (int f = f0; f < f1; f++) {
        const int fi = D == 1 ? f : i, fj = D == 2 ? f : j;
        R ql[NP], qr[NP], sb[NP];
#pragma unroll
        for (int c = 0; c < NP; c++) {
            sb[c] = mc_slope(qa[c], qb[c], qc[c]);
            ql[c] = qa[c] + R(0.5) * sa[c];
            qr[c] = qb[c] - R(0.5) * sb[c];
        }
        // L1 prefetch of the next face's metric record and of the zone it adds
        // to the window, so that their latency overlaps this face's physics
        if (f + 1 < f1) {
            const int ni = D == 1 ? f + 1 : i, nj = D == 2 ? f + 1 : j;
            const char *gp = (const char *)&face_table<R>(g, D)[midx(g, ni, nj)];
#pragma unroll
            for (int o = 0; o < (int)sizeof(Geo<R>); o += 32) asm volatile("prefetch.global.L1 [%0];" ::"l"(gp + o));
#pragma unroll
            for (int c = 0; c < NP; c++)
                asm volatile("prefetch.global.L1 [%0];" ::"l"(P + c * g.nz + z0 + (long long)(f + 2 - f0) * st));
        }
        R out[NU];
        R cw = R(0);
        if (D == 2 && g.polar2[midx(g, fi, fj)]) {
#pragma unroll
            for (int c = 0; c < NU; c++) out[c] = R(0);
        } else {
            face_flux<R, D>(g, face_table<R>(g, D)[midx(g, fi, fj)], ql, qr, out, cw);
        }
        const long long zf = z0 + (long long)(f - f0) * st;
#pragma unroll
        for (int c = 0; c < NU; c++) F[c * g.nz + zf] = out[c];
        if (want_dt) cwm = max(cwm, face_cw<R, D>(g, fi, fj, k, cw));
        if (f + 1 < f1) {
#pragma unroll
            for (int c = 0; c < NP; c++) {
                qa[c] = qb[c];
                qb[c] = qc[c];
                sa[c] = sb[c];
                qc[c] = ldg(P + c * g.nz + zf + 2 * st);
            }
        }
    }
    return cwm;
}

// PPM faces of a column along X1 / X2: the column walk with a window of the
// zones f, f+1, f+2, the MC slope of zone f, the interface value a_{f-1/2}
// and the constrained upper value of zone f-1.  Each zone's slope, each
// interface value and each zone's constrained pair are formed once per column
// instead of once per face (flux_item_ppm forms them for every face), by the
// same operations as ppm_face.  Box: col_box.
template <typename R, int D>
__device__ __forceinline__ R flux_column_ppm(const Grid &g, const R *__restrict__ P, R *__restrict__ F,
                                             const Box &cb, int want_dt, long long t)
{
    static_assert(D == 1 || D == 2, "columns run along X1 or X2");
    R cwm = R(0);
    if (t >= cb.count()) return cwm;
    int i, j, k;
    box_decode(cb, t, i, j, k);
    const int nf = (D == 1 ? g.n1 : g.n2) + 1;
    const int f0 = (D == 1 ? i : j) * g.fcol, f1 = min(f0 + g.fcol, nf);
    if (D == 1) i = f0;
    else j = f0;
    const long long st = D == 1 ? (long long)g.N2 * g.N3 : g.N3;
    const long long z0 = zidx(g, i, j, k); // zone f0; face f lies between zones f-1 and f
    R q0[NP], q1[NP], q2[NP], s0[NP], am[NP], rp[NP];
#pragma unroll
    for (int c = 0; c < NP; c++) {
        const R *pc = P + c * g.nz + z0;
        const R qm3 = ldg(pc - 3 * st), qm2 = ldg(pc - 2 * st), qm1 = ldg(pc - st);
        q0[c] = ldg(pc);
        q1[c] = ldg(pc + st);
        q2[c] = ldg(pc + 2 * st);
        const R sm2 = mc_slope(qm3, qm2, qm1), sm1 = mc_slope(qm2, qm1, q0[c]);
        s0[c] = mc_slope(qm1, q0[c], q1[c]);
        // zone f0 - 1 between its interfaces f0 - 3/2 and f0 - 1/2
        R L = ppm_interface_s(qm2, qm1, sm2, sm1);
        R Rt = ppm_interface_s(qm1, q0[c], sm1, s0[c]);
        am[c] = Rt;
        ppm_monotone(qm1, L, Rt);
        rp[c] = Rt;
    }
    for (int f = f0; f < f1; f++) {
        const int fi = D == 1 ? f : i, fj = D == 2 ? f : j;
        R ql[NP], qr[NP];
#pragma unroll
        for (int c = 0; c < NP; c++) {
            const R s1 = mc_slope(q0[c], q1[c], q2[c]);
            const R ap = ppm_interface_s(q0[c], q1[c], s0[c], s1); // a_{f+1/2}
            R L = am[c], Rt = ap;
            ppm_monotone(q0[c], L, Rt);
            ql[c] = rp[c];
            qr[c] = L;
            rp[c] = Rt;
            am[c] = ap;
            s0[c] = s1;
        }
        if (f + 1 < f1) {
            const int ni = D == 1 ? f + 1 : i, nj = D == 2 ? f + 1 : j;
            const char *gp = (const char *)&face_table<R>(g, D)[midx(g, ni, nj)];
#pragma unroll
            for (int o = 0; o < (int)sizeof(Geo<R>); o += 32) asm volatile("prefetch.global.L1 [%0];" ::"l"(gp + o));
#pragma unroll
            for (int c = 0; c < NP; c++)
                asm volatile("prefetch.global.L1 [%0];" ::"l"(P + c * g.nz + z0 + (long long)(f + 3 - f0) * st));
        }
        R out[NU];
        R cw = R(0);
        if (D == 2 && g.polar2[midx(g, fi, fj)]) {
#pragma unroll
            for (int c = 0; c < NU; c++) out[c] = R(0);
        } else {
            face_flux<R, D>(g, face_table<R>(g, D)[midx(g, fi, fj)], ql, qr, out, cw);
        }
        const long long zf = z0 + (long long)(f - f0) * st;
#pragma unroll
        for (int c = 0; c < NU; c++) F[c * g.nz + zf] = out[c];
        if (want_dt) cwm = max(cwm, face_cw<R, D>(g, fi, fj, k, cw));
        if (f + 1 < f1) {
#pragma unroll
            for (int c = 0; c < NP; c++) {
                q0[c] = q1[c];
                q1[c] = q2[c];
                q2[c] = ldg(P + c * g.nz + zf + 3 * st);
            }
        }
    }
    return cwm;
}

// PPM faces of one (i, j) row by one warp: lane l holds zone k0 - 3 + l of a
// segment, forms its slope from the neighbours' values by shuffles, its upper
// interface value from its own and the upper neighbour's values and slopes,
// takes its lower one from the lane below, and constrains its parabola; lanes
// 3..29 evaluate the 27 faces k0 .. k0 + 26 between the zones of lanes l-1
// and l.  The next segment's zones are loaded before the faces are
// evaluated.  Box: x3_warp_box.
constexpr int X3W_PPM_FACES = 27;

template <typename R>
__device__ __forceinline__ R flux_x3_warp_ppm(const Grid &g, const R *__restrict__ P, R *__restrict__ F,
                                              const Box &wb, int want_dt, long long t)
{
    R cwm = R(0);
    if (t >= wb.count()) return cwm;
    int i, j, lane;
    box_decode(wb, t, i, j, lane);
    const long long zrow = zidx(g, i, j, 0);
    const Geo<R> &geo = face_table<R>(g, 3)[midx(g, i, j)];
    const int nseg = (g.n3 + 1 + X3W_PPM_FACES - 1) / X3W_PPM_FACES;
    // this lane's zone of a segment, clamped past the last ghost on lanes no face uses
    auto zone_of = [&](int seg) { return min(seg * X3W_PPM_FACES - 3 + lane, g.n3 + 2); };
    R qn[NP];
    {
        const long long z = zrow + zone_of(0);
#pragma unroll
        for (int c = 0; c < NP; c++) qn[c] = ldg(P + c * g.nz + z);
    }
    for (int seg = 0; seg < nseg; seg++) {
        const int k = zone_of(seg);
        R ql[NP], qr[NP];
#pragma unroll
        for (int c = 0; c < NP; c++) {
            const R q = qn[c];
            const R qm = __shfl_up_sync(0xffffffffu, q, 1), qp = __shfl_down_sync(0xffffffffu, q, 1);
            const R s = mc_slope(qm, q, qp);                              // lanes 1..30
            const R sp = __shfl_down_sync(0xffffffffu, s, 1);
            const R ap = ppm_interface_s(q, qp, s, sp);                   // a_{k+1/2}, lanes 1..29
            R L = __shfl_up_sync(0xffffffffu, ap, 1), Rt = ap;            // a_{k-1/2}, lanes 2..29
            ppm_monotone(q, L, Rt);
            ql[c] = __shfl_up_sync(0xffffffffu, Rt, 1);                   // lanes 3..29
            qr[c] = L;
        }
        if (seg + 1 < nseg) {
            const long long z = zrow + zone_of(seg + 1);
#pragma unroll
            for (int c = 0; c < NP; c++) qn[c] = ldg(P + c * g.nz + z);
        }
        if (lane >= 3 && lane <= 29 && k <= g.n3) {
            R out[NU];
            R cw = R(0);
            face_flux<R, 3>(g, geo, ql, qr, out, cw);
#pragma unroll
            for (int c = 0; c < NU; c++) F[c * g.nz + zrow + k] = out[c];
            if (want_dt) cwm = max(cwm, face_cw<R, 3>(g, i, j, k, cw));
        }
    }
    return cwm;
}

// X3 faces of one (i, j) row by one warp (the PLM stencil shared through
// warp-level primitives, Sec. 3).  The warp walks the row in segments of 29
// faces: lane l holds zone k0 - 2 + l of the segment, forms that zone's MC
// slope from its neighbours' values by shuffles, and lanes 2..30 evaluate
// the faces k0 .. k0 + 28 between them, so each zone is loaded and its slope
// formed once per segment instead of once per face; the next segment's
// zones are loaded before the current faces are evaluated, so their latency
// hides behind the face physics.  The face values are the numbers flux_item
// forms.  x3_warp_box counts lanes: rows (i, j) x 32.
constexpr int X3W_FACES = 29;

__host__ __device__ inline Box x3_warp_box(const Grid &g) { return Box{{-1, -1, 0}, {g.n1 + 2, g.n2 + 2, 32}}; }

template <typename R>
__device__ __forceinline__ R flux_x3_warp(const Grid &g, const R *__restrict__ P, R *__restrict__ F,
                                          const Box &wb, int want_dt, long long t)
{
    // the box count is a multiple of 32, so whole warps are in or out
    R cwm = R(0);
    if (t >= wb.count()) return cwm;
    int i, j, lane;
    box_decode(wb, t, i, j, lane);
    const long long zrow = zidx(g, i, j, 0);
    const Geo<R> &geo = face_table<R>(g, 3)[midx(g, i, j)];
    const int nseg = (g.n3 + 1 + X3W_FACES - 1) / X3W_FACES;
    // this lane's zone of a segment, clamped past the last ghost on lanes no face uses
    auto zone_of = [&](int seg) { return min(seg * X3W_FACES - 2 + lane, g.n3 + 1); };
    R qn[NP];
    {
        const long long z = zrow + zone_of(0);
#pragma unroll
        for (int c = 0; c < NP; c++) qn[c] = ldg(P + c * g.nz + z);
    }
    for (int seg = 0; seg < nseg; seg++) {
        const int k = zone_of(seg); // face k lies between the zones of lanes l-1 and l
        R ql[NP], qr[NP];
#pragma unroll
        for (int c = 0; c < NP; c++) {
            const R q = qn[c];
            const R qm = __shfl_up_sync(0xffffffffu, q, 1), qp = __shfl_down_sync(0xffffffffu, q, 1);
            const R sl = mc_slope(qm, q, qp); // valid on lanes 1..30
            const R up = q + R(0.5) * sl;     // the zone's value at its upper X3 face
            ql[c] = __shfl_up_sync(0xffffffffu, up, 1);
            qr[c] = q - R(0.5) * sl;
        }
        if (seg + 1 < nseg) {
            const long long z = zrow + zone_of(seg + 1);
#pragma unroll
            for (int c = 0; c < NP; c++) qn[c] = ldg(P + c * g.nz + z);
        }
        if (lane >= 2 && lane <= 30 && k <= g.n3) {
            R out[NU];
            R cw = R(0);
            face_flux<R, 3>(g, geo, ql, qr, out, cw);
#pragma unroll
            for (int c = 0; c < NU; c++) F[c * g.nz + zrow + k] = out[c];
            if (want_dt) cwm = max(cwm, face_cw<R, 3>(g, i, j, k, cw));
        }
    }
    return cwm;
}

// -------------------------------------------------------------------- EMFs

// E3 at (i-1/2, j-1/2, k), E1 at (i, j-1/2, k-1/2), E2 at (i-1/2, j, k-1/2) (Eq. 22)
template <typename R>
__device__ __forceinline__ void emf_item(const Grid &g, const R *__restrict__ F1, const R *__restrict__ F2,
                                         const R *__restrict__ F3, R *E1, R *E2, R *E3, const Box &box,
                                         long long t)
{
    if (t >= box.count()) return;
    int i, j, k;
    box_decode(box, t, i, j, k);
    const long long nz = g.nz;
    long long z = zidx(g, i, j, k);
    long long si = (long long)g.N2 * g.N3, sj = g.N3;
    // face fluxes of plane k (and k - 1); an axisymmetric grid keeps them at k = 0
    const long long zf = g.flat3 ? zidx(g, i, j, 0) : z, sk = g.flat3 ? 0 : 1;
    if (k < g.n3)
        E3[z] = R(0.25) * (F1[KB2 * nz + zf] + F1[KB2 * nz + zf - sj] - F2[KB1 * nz + zf] - F2[KB1 * nz + zf - si]);
    if (i < g.n1)
        E1[z] = R(0.25) * (F2[KB3 * nz + zf] + F2[KB3 * nz + zf - sk] - F3[KB2 * nz + zf] - F3[KB2 * nz + zf - sj]);
    if (j < g.n2)
        E2[z] = R(0.25) * (F3[KB1 * nz + zf] + F3[KB1 * nz + zf - si] - F1[KB3 * nz + zf] - F1[KB3 * nz + zf - sk]);
}

// ------------------------------------------------- FP32 pair arithmetic
// Values carried as an unevaluated sum hi + lo of two floats (Knuth's
// TwoSum; the product error by one FMA), for the mixed path's flux-CT
// increments: the corner divergence of Eq. 24 cancels only if the pair sums of
// the edge EMFs, paired along one direction for one B component and along the
// other for the next, are exact -- an FP32 rounding of each pair sum leaves
// div B at ~eps_32 of the step's change.
struct FPair {
    float hi, lo;
};

// hi + lo == a + b exactly
__device__ __forceinline__ FPair two_sum(float a, float b)
{
    float s = a + b;
    float bb = s - a;
    return FPair{s, (a - (s - bb)) + (b - bb)};
}

// (a.hi + a.lo) - (b.hi + b.lo), to ~2^-46 relative
__device__ __forceinline__ FPair ff_sub(FPair a, FPair b)
{
    FPair d = two_sum(a.hi, -b.hi);
    return two_sum(d.hi, d.lo + (a.lo - b.lo));
}

// (a.hi + a.lo) * (h + l) for a pair constant h + l
__device__ __forceinline__ FPair ff_mul(FPair a, float h, float l)
{
    float p = a.hi * h;
    float e = fmaf(a.hi, h, -p) + (a.hi * l + a.lo * h);
    return two_sum(p, e);
}

__device__ __forceinline__ FPair ff_add(FPair a, FPair b)
{
    FPair s = two_sum(a.hi, b.hi);
    return two_sum(s.hi, s.lo + (a.lo + b.lo));
}

// --------------------------------------------------------- update + invert

constexpr int NHZ = 4; // zones next to the horizon that keep the FP64 source in the mixed path

// per-thread counters of update_item: Newton iterations, methods, failures,
// floor/ceiling/cap hits
struct UpdCount {
    unsigned it, nr, br, en, eb, fail, fl, ce, gc, lr;
};

// Where Newton from the stage's starts does not converge and the grid has a
// network (g.mlp, set by grmhd_set_learned_guess), Newton from the learned W
// is tried before Brent; the choice is made at run time, so the plain and the
// learned order run the same machine code
template <typename R>
__device__ inline void update_item(const Grid &g, const R *__restrict__ Pin, R *__restrict__ Pout,
                                   const R *__restrict__ F1, const R *__restrict__ F2,
                                   const R *__restrict__ F3, const R *__restrict__ E1,
                                   const R *__restrict__ E2, const R *__restrict__ E3, double dtfac, int corr,
                                   long long t, UpdCount &cn)
{
    long long nact = nact_of(g);
    if (t >= nact) return;
    int k = (int)(t % g.n3);
    long long r = t / g.n3;
    int j = (int)(r % g.n2), i = (int)(r / g.n2);
    const long long nz = g.nz;
    long long z = zidx(g, i, j, k);
    int m = midx(g, i, j);
    const long long si = (long long)g.N2 * g.N3, sj = g.N3, sk = 1;
    const double dts = dtfac * g.scal[0];
    constexpr bool MX = sizeof(R) == 4;
    // the stage primitives: FP64 (FP64 path), or as stored in FP32 (mixed
    // path; widened only where the FP64 source needs them)
    double q[NP];
    float qin[NP];
    if constexpr (MX) {
#pragma unroll
        for (int c = 0; c < NP; c++) qin[c] = (float)Pin[c * nz + z];
    } else {
#pragma unroll
        for (int c = 0; c < NP; c++) q[c] = (double)Pin[c * nz + z];
    }
    const Geo<double> geo = g.gc[m];
    // source (Eq. 15): FP64, or FP32 in the mixed path away from the horizon
    double src[4];
    float sf[4];
    const bool src32 = MX && i >= g.i_h + NHZ;
    if (!src32) {
        if constexpr (MX) {
#pragma unroll
            for (int c = 0; c < NP; c++) q[c] = (double)qin[c];
        }
        St<double> s;
        get_state(q, geo, s);
        source_terms(q, geo, g.conn + (long long)m * 40, s, g.gam, src);
    } else {
        const Geo<float> gf = g.gcF[m];
        St<float> s;
        get_state(qin, gf, s);
        source_terms(qin, gf, g.connF + (long long)m * 40, s, g.gam_f, sf);
    }
    // flux divergence; B components from the flux-CT edge averages (Eq. 23),
    // formed exactly as the replaced face values.  The mixed path takes the
    // divergence in FP32 (the fluxes' own precision) and converts each
    // component once before the FP64 accumulation; the mass divergence is
    // added back to the rest-mass-subtracted energy in FP64 so that U_E and
    // U_rho see the same rounded mass flux.
    double Un[NU];
    {
        typedef R T;
        T ix1, ix2, ix3;
        if constexpr (MX) {
            ix1 = g.idx_f[0];
            ix2 = g.idx_f[1];
            ix3 = g.idx_f[2];
        } else {
            ix1 = g.idx[0];
            ix2 = g.idx[1];
            ix3 = g.idx[2];
        }
        T dv[NU];
#pragma unroll
        for (int c = 0; c < NU; c++) {
            if (c >= KB1 && c <= KB3) continue;
            const long long o = c * nz + z;
            T d1 = (F1[o + si] - F1[o]) * ix1;
            T d2 = (F2[o + sj] - F2[o]) * ix2;
            T d3 = (F3[o + (g.flat3 ? 0 : sk)] - F3[o]) * ix3; // axisymmetric: the k = 0 face twice
            dv[c] = d1 + d2 + d3;
        }
        T f2b1_j = T(-0.5) * (E3[z + si] + E3[z]);
        T f2b1_jp = T(-0.5) * (E3[z + si + sj] + E3[z + sj]);
        T f3b1_k = T(0.5) * (E2[z + si] + E2[z]);
        T f3b1_kp = T(0.5) * (E2[z + si + sk] + E2[z + sk]);
        T f1b2_i = T(0.5) * (E3[z + sj] + E3[z]);
        T f1b2_ip = T(0.5) * (E3[z + si + sj] + E3[z + si]);
        T f3b2_k = T(-0.5) * (E1[z + sj] + E1[z]);
        T f3b2_kp = T(-0.5) * (E1[z + sj + sk] + E1[z + sk]);
        T f1b3_i = T(-0.5) * (E2[z + sk] + E2[z]);
        T f1b3_ip = T(-0.5) * (E2[z + si + sk] + E2[z + si]);
        T f2b3_j = T(0.5) * (E1[z + sk] + E1[z]);
        T f2b3_jp = T(0.5) * (E1[z + sj + sk] + E1[z + sj]);
        double dB[3]; // the U_B increments' divergence terms (Eq. 23 fluxes, Eq. 26)
        if constexpr (MX) {
            // exact EMF pair sums (FP32 pairs), 1/(2 dX) as a pair: the
            // increments keep the corner divergence at FP64-like round-off
            const FPair e3a = two_sum(E3[z + si + sj], E3[z + sj]), e3b = two_sum(E3[z + si], E3[z]);
            const FPair e3c = two_sum(E3[z + si + sj], E3[z + si]), e3d = two_sum(E3[z + sj], E3[z]);
            const FPair e2a = two_sum(E2[z + si + sk], E2[z + sk]), e2b = two_sum(E2[z + si], E2[z]);
            const FPair e2c = two_sum(E2[z + si + sk], E2[z + si]), e2d = two_sum(E2[z + sk], E2[z]);
            const FPair e1a = two_sum(E1[z + sj + sk], E1[z + sk]), e1b = two_sum(E1[z + sj], E1[z]);
            const FPair e1c = two_sum(E1[z + sj + sk], E1[z + sj]), e1d = two_sum(E1[z + sk], E1[z]);
            const float *hh = g.hidx_hi, *hl = g.hidx_lo;
            // B1: -(E3 pairs along i) differenced along j, +(E2 pairs along i) along k
            const FPair b1 = ff_sub(ff_mul(ff_sub(e2a, e2b), hh[2], hl[2]), ff_mul(ff_sub(e3a, e3b), hh[1], hl[1]));
            // B2: +(E3 pairs along j) differenced along i, -(E1 pairs along j) along k
            const FPair b2 = ff_sub(ff_mul(ff_sub(e3c, e3d), hh[0], hl[0]), ff_mul(ff_sub(e1a, e1b), hh[2], hl[2]));
            // B3: -(E2 pairs along k) differenced along i, +(E1 pairs along k) along j
            const FPair b3 = ff_sub(ff_mul(ff_sub(e1c, e1d), hh[1], hl[1]), ff_mul(ff_sub(e2c, e2d), hh[0], hl[0]));
            dB[0] = (double)b1.hi + (double)b1.lo;
            dB[1] = (double)b2.hi + (double)b2.lo;
            dB[2] = (double)b3.hi + (double)b3.lo;
        } else {
            dB[0] = (f2b1_jp - f2b1_j) * ix2 + (f3b1_kp - f3b1_k) * ix3;
            dB[1] = (f1b2_ip - f1b2_i) * ix1 + (f3b2_kp - f3b2_k) * ix3;
            dB[2] = (f1b3_ip - f1b3_i) * ix1 + (f2b3_jp - f2b3_j) * ix2;
        }
        double dD = (double)dv[KRHO];
#pragma unroll
        for (int c = 0; c < NU; c++) {
            double rhs;
            if (c >= KB1 && c <= KB3) {
                rhs = -dB[c - KB1];
            } else if (c >= 1 && c <= 4 && src32) {
                // an FP32 source meets the FP32 divergence before the one conversion
                rhs = (double)(sf[c - 1] - (float)dv[c]);
            } else {
                rhs = -(double)dv[c];
                if (c >= 1 && c <= 4) rhs += src[c - 1];
            }
            if (c == 1 && MX) rhs += dD; // rest-mass-subtracted energy flux
            Un[c] = g.U[c * nz + z] + dts * rhs;
        }
    }
    double qn[NP];
    float qnf[NP];
    int it;
    const Geo<float> *gfr = MX ? &g.gcF[m] : nullptr;
    const double *gsp = g.gsp + 6LL * m;
    // mixed path: Newton starts from the stage input extrapolated by its change
    // over the previous half step, 2 P_in - P_out(old) (P_out still holds the
    // previous stage's result for this zone: P-hat before the corrector, the
    // previous step's P-hat before the predictor), an O(dt^2) start in place of
    // O(dt); used where rho and u move by less than 10%
    float qx[5];
    bool have_x = false;
    if constexpr (MX) {
#pragma unroll
        for (int c = 0; c < 5; c++) qx[c] = 2.0f * qin[c] - (float)Pout[c * nz + z];
        have_x = qx[KRHO] > 0.9f * qin[KRHO] && qx[KRHO] < 1.1f * qin[KRHO] && qx[KUU] > 0.9f * qin[KUU] &&
                 qx[KUU] < 1.1f * qin[KUU];
    }
    int fl = con2prim<MX>(Un, geo, gsp, q, qin, c2p_par(g), 15, qn, it, nullptr, gfr, qx, have_x,
                          g.mlp);
    bool ok = !(fl & C2P_FAIL);
    cn.it += it;
    int meth = fl & 7;
    if (fl & C2P_FAIL) {
        cn.fail += 1;
        // a non-finite conserved component cannot be repaired by the fixups
        // (they average the primitives, never B): report it
        bool fin = true;
#pragma unroll
        for (int c = 0; c < NU; c++) fin = fin && finite64(Un[c]);
        if (!fin) atomicOr(g.status, ST_NONFINITE);
        g.flag[z] = 1;
        int slot = atomicAdd(g.nfail, 1);
        if (slot < g.nfix_cap) g.faillist[slot] = (int)t;
    } else {
        g.flag[z] = 0;
        cn.nr += meth == C2P_NR;
        cn.br += meth == C2P_BRENT_W;
        cn.en += meth == C2P_ENTROPY;
        cn.eb += meth == C2P_ENTROPY_BETA;
        cn.lr += (fl & C2P_LEARNED) != 0;
        int res = post_inversion<MX>(g, geo, gsp, qn, Un, gfr, qnf);
        if (res & 1) {
            cn.fl += 1;
            cons_of<MX>(qn, geo, g.gam, Un, gfr, MX ? qnf : nullptr, g.gam_f, (res & 14) == 0);
        }
        cn.ce += (res & 2) != 0;
        cn.gc += (res & 4) != 0;
    }
    if (MX && ok) {
#pragma unroll
        for (int c = 0; c < NP; c++) Pout[c * nz + z] = (R)qnf[c];
    } else {
#pragma unroll
        for (int c = 0; c < NP; c++) Pout[c * nz + z] = (R)qn[c];
    }
    if (corr) {
#pragma unroll
        for (int c = 0; c < NU; c++) g.U[c * nz + z] = Un[c];
    }
}

__device__ __forceinline__ void flush_counts(const Grid &g, const UpdCount &cn)
{
    block_count(&g.cnt[C_NR_ITERS], cn.it);
    block_count(&g.cnt[C_NR], cn.nr);
    block_count(&g.cnt[C_BRENT], cn.br);
    block_count(&g.cnt[C_ENT], cn.en);
    block_count(&g.cnt[C_ENT_BETA], cn.eb);
    block_count(&g.cnt[C_FAIL], cn.fail);
    block_count(&g.cnt[C_FLOOR], cn.fl);
    block_count(&g.cnt[C_CEIL], cn.ce);
    block_count(&g.cnt[C_GCAP], cn.gc);
    block_count(&g.cnt[C_LEARN], cn.lr);
}

// ------------------------------------------------------------------ fixups

// a fixup neighbour (ii, jj) must be an active zone of the whole grid; a
// theta slab reads the rows jj = -1 and n2 from its ghost rows, which hold the
// neighbour slab's current edge rows (primitives and flags) during its fixups
__device__ __forceinline__ bool fix_inside(const Grid &g, int ii, int jj)
{
    const int jg = g.j0 + jj;
    return ii >= 0 && ii < g.n1 && jg >= 0 && jg < g.n2t;
}

// One Jacobi sweep of the fixups by one block over the compacted list of
// failed zones (nlist entries) of one grid: every repairable zone's average
// is formed from neighbours that were good at the start of the sweep, then
// all are written, so the result does not depend on the list order.  Every
// thread of the block calls it and gets the number of zones still failed.
// Out of line, so that the single-grid, ensemble and theta-slab kernels run
// the same machine code (inlined, the compiler may contract or schedule the
// FP64 arithmetic differently in each).
template <typename R>
__device__ __noinline__ int fixup_sweep(const Grid &g, R *P, int corr, int nlist)
{
    __shared__ int s_left;
    const long long nz = g.nz;
    const int cap = g.nfix_cap;
    double *nb = g.fixbuf;            // [5][cap]
    double *found = g.fixbuf + 5LL * cap;
    for (int a = threadIdx.x; a < nlist; a += blockDim.x) {
        int t = g.faillist[a];
        int k = t % g.n3, r = t / g.n3, j = r % g.n2, i = r / g.n2;
        found[a] = 0.0;
        if (!g.flag[zidx(g, i, j, k)]) continue;
        const int fo[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
        const int dg[4][2] = {{1, 1}, {1, -1}, {-1, 1}, {-1, -1}};
        bool done = false;
        for (int s = 0; s < 2 && !done; s++) {
            const int(*set)[2] = s == 0 ? fo : dg;
            bool all = true;
            for (int mm = 0; mm < 4; mm++) {
                int ii = i + set[mm][0], jj = j + set[mm][1];
                if (!fix_inside(g, ii, jj) || g.flag[zidx(g, ii, jj, k)]) all = false;
            }
            if (all) {
                for (int c = 0; c < 5; c++) {
                    double acc = 0.0;
                    for (int mm = 0; mm < 4; mm++)
                        acc += (double)P[c * nz + zidx(g, i + set[mm][0], j + set[mm][1], k)];
                    nb[(long long)c * cap + a] = 0.25 * acc;
                }
                done = true;
            }
        }
        if (!done) {
            int cnt = 0;
            double acc[5] = {0, 0, 0, 0, 0};
            for (int s = 0; s < 2; s++)
                for (int mm = 0; mm < 4; mm++) {
                    int ii = i + (s ? dg : fo)[mm][0], jj = j + (s ? dg : fo)[mm][1];
                    if (!fix_inside(g, ii, jj)) continue;
                    long long zz = zidx(g, ii, jj, k);
                    if (g.flag[zz]) continue;
                    for (int c = 0; c < 5; c++) acc[c] += (double)P[c * nz + zz];
                    cnt++;
                }
            if (cnt > 0) {
                for (int c = 0; c < 5; c++) nb[(long long)c * cap + a] = acc[c] / cnt;
                done = true;
            }
        }
        if (done) found[a] = 1.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_left = 0;
    __syncthreads();
    int left = 0;
    for (int a = threadIdx.x; a < nlist; a += blockDim.x) {
        int t = g.faillist[a];
        int k = t % g.n3, r = t / g.n3, j = r % g.n2, i = r / g.n2;
        long long z = zidx(g, i, j, k);
        if (found[a] != 0.0) {
            int m = midx(g, i, j);
            const Geo<double> geo = g.gc[m];
            double q[NP];
            for (int c = 0; c < NP; c++) q[c] = c < 5 ? nb[(long long)c * cap + a] : (double)P[c * nz + z];
            post_fixup(g, geo, q);
            for (int c = 0; c < NP; c++) P[c * nz + z] = (R)q[c];
            if (corr) {
                St<double> s;
                get_state(q, geo, s);
                double Uz[NU];
                prim_to_UF<double, false>(q, geo, s, g.gam, 0, Uz);
                for (int c = 0; c < NU; c++) g.U[c * nz + z] = Uz[c];
            }
            g.flag[z] = 0;
            atomicAdd(&g.cnt[C_FIXED], 1ULL);
        } else if (g.flag[z]) {
            left++;
        }
    }
    __syncthreads(); // all flag writes of this sweep done before the next reads
    if (left) atomicAdd(&s_left, left);
    __syncthreads();
    const int total = s_left;
    __syncthreads(); // every thread has read s_left before a next sweep resets it
    return total;
}

// The fixups of a stage on one grid: sweeps until no listed zone is left
// failed, at most fix_maxsweep of them; then the sweep count, the status and
// the list reset.  Every thread of the block calls it.
template <typename R>
__device__ inline void fixup_block(const Grid &g, R *P, int corr)
{
    const int nlist = min(*g.nfail, g.nfix_cap);
    if (nlist == 0) return;
    int sweep = 0, left = 1;
    while (sweep < g.fix_maxsweep) {
        left = fixup_sweep<R>(g, P, corr, nlist);
        sweep++;
        if (left == 0) break;
    }
    if (threadIdx.x == 0) {
        atomicAdd(&g.cnt[C_SWEEPS], (unsigned long long)sweep);
        if (left > 0 || *g.nfail > g.nfix_cap) atomicOr(g.status, ST_FIXUP);
        *g.nfail = 0;
    }
}

// ----------------------------------------------------- FP64 out-of-line calls
// The FP64 items are compiled out of line and called from both the
// single-grid and the ensemble kernels, so both run the same machine code:
// inlined into different kernels the compiler may contract or schedule the
// FP64 arithmetic differently and the two paths would differ in the last
// bit.  The FP32-flux path is inlined (its two instantiations already agree).

static __device__ __noinline__ double flux_column_d1(const Grid &g, const double *P, double *F, const Box &box,
                                                     int w, long long t)
{
    return flux_column<double, 1>(g, P, F, box, w, t);
}
static __device__ __noinline__ double flux_column_d2(const Grid &g, const double *P, double *F, const Box &box,
                                                     int w, long long t)
{
    return flux_column<double, 2>(g, P, F, box, w, t);
}
static __device__ __noinline__ double flux_item_d3(const Grid &g, const double *P, double *F, const Box &box, int w,
                                            long long t)
{
    return flux_item<double, 3>(g, P, F, box, w, t);
}
// the X3 row-warp sweep in FP64, out of line like the other FP64 items (all
// lanes of the warp call it together)
static __device__ __noinline__ double flux_x3_warp_d(const Grid &g, const double *P, double *F, const Box &box,
                                                     int w, long long t)
{
    return flux_x3_warp<double>(g, P, F, box, w, t);
}

// X3 faces of a row by one warp (x3_warp_box), either precision
template <typename R>
__device__ __forceinline__ R flux_x3_warp_call(const Grid &g, const R *P, R *F, const Box &box, int w, long long t)
{
    if constexpr (sizeof(R) == 8) return flux_x3_warp_d(g, P, F, box, w, t);
    else return flux_x3_warp<R>(g, P, F, box, w, t);
}
static __device__ __noinline__ void update_item_d(const Grid &g, const double *Pin, double *Pout, const double *F1,
                                           const double *F2, const double *F3, const double *E1,
                                           const double *E2, const double *E3, double dtfac, int corr,
                                           long long t, UpdCount &cn)
{
    update_item<double>(g, Pin, Pout, F1, F2, F3, E1, E2, E3, dtfac, corr, t, cn);
}
static __device__ __noinline__ void bc1_item_d(const Grid &g, double *P, long long t) { bc1_item<double>(g, P, t); }

// the flux element of direction D: a column of faces along X1 / X2, one face
// along X3; box = flux_elem_box(g, D)
template <typename R, int D>
__device__ __forceinline__ R flux_call(const Grid &g, const R *P, R *F, const Box &box, int w, long long t)
{
    if constexpr (sizeof(R) == 8) {
        if constexpr (D == 1) return flux_column_d1(g, P, F, box, w, t);
        else if constexpr (D == 2) return flux_column_d2(g, P, F, box, w, t);
        else return flux_item_d3(g, P, F, box, w, t);
    } else {
        if constexpr (D == 3) return flux_item<R, D>(g, P, F, box, w, t);
        else return flux_column<R, D>(g, P, F, box, w, t);
    }
}

__host__ __device__ inline Box flux_elem_box(const Grid &g, int d) { return d == 3 ? flux_box(g, 3) : col_box(g, d); }

template <typename R>
__device__ __forceinline__ void update_call(const Grid &g, const R *Pin, R *Pout, const R *F1, const R *F2,
                                            const R *F3, const R *E1, const R *E2, const R *E3, double dtfac,
                                            int corr, long long t, UpdCount &cn)
{
    if constexpr (sizeof(R) == 8) update_item_d(g, Pin, Pout, F1, F2, F3, E1, E2, E3, dtfac, corr, t, cn);
    else update_item<R>(g, Pin, Pout, F1, F2, F3, E1, E2, E3, dtfac, corr, t, cn);
}

template <typename R>
__device__ __forceinline__ void bc1_call(const Grid &g, R *P, long long t)
{
    if constexpr (sizeof(R) == 8) bc1_item_d(g, P, t);
    else bc1_item<R>(g, P, t);
}

template <typename R>
__device__ __forceinline__ void fixup_call(const Grid &g, R *P, int corr)
{
    fixup_block<R>(g, P, corr);
}

// --------------------------------------------------------------------- dt

// 1/dt = sum_l 1/dt^l (Eq. 27); t += dt for a finished step; minima reset.
// next dt from per-direction minima (Eq. 27: 1/dt = sum_l 1/dt^l)
__device__ __forceinline__ double combine_dt(const double dtd[3])
{
    double inv = 0.0;
#pragma unroll
    for (int d = 0; d < 3; d++)
        if (dtd[d] < INFINITY) inv += 1.0 / dtd[d];
    return inv > 0.0 ? 1.0 / inv : INFINITY;
}

__device__ inline void finalize_one(const Grid &g, int advance)
{
    double dtd[3];
    for (int d = 0; d < 3; d++) {
        dtd[d] = __longlong_as_double((long long)g.dtmin[d]);
        g.dtmin[d] = dbits(INFINITY);
    }
    if (advance) {
        g.scal[1] += g.scal[0];
        g.cnt[C_STEPS] += 1;
    }
    g.scal[0] = combine_dt(dtd);
}

} // namespace grmhd
