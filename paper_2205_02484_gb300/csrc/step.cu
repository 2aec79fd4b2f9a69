// step.cu -- single-grid kernels of the RK2 step and their launch sequence.
//
// Each kernel maps one thread to one element of one grid and runs the item
// function of stage_items.cuh; the fluxes reduce the CFL candidates of a
// block with warp shuffles and one atomic, the update reduces its counters
// the same way.  A step is 21 launches: per stage three face sweeps, EMFs,
// update + inversion, fixups, four boundary kernels; then the dt kernel.
#include "kernels.h"
#include "stage_items.cuh"

namespace grmhd {

template <typename RS>
__global__ void k_polar(Grid g, RS *P)
{
    polar_item(g, P, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

template <typename RS>
__global__ void k_bc1(Grid g, RS *P)
{
    bc1_call(g, P, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

template <typename RS>
__global__ void k_bc2(Grid g, RS *P)
{
    bc2_item(g, P, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

template <typename RS>
__global__ void k_bc3(Grid g, RS *P)
{
    bc3_item(g, P, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// mixed path: X1 / X2 column sweeps held to 4 resident blocks per SM, the X3
// row-warp sweep to 5
template <typename R, int D>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? (D < 3 ? 4 : 5) : 1) k_flux(Grid g, const R *__restrict__ P, R *__restrict__ F,
                                              Box box, int want_dt)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    R cw;
    if constexpr (D == 3) {
        if (g.x3warp) cw = flux_x3_warp_call<R>(g, P, F, box, want_dt, t);
        else cw = flux_call<R, D>(g, P, F, box, want_dt, t);
    } else {
        cw = flux_call<R, D>(g, P, F, box, want_dt, t);
    }
    if (want_dt) block_cfl_into(&g.dtmin[D - 1], cw, g.cfl * g.dx[D - 1]);
}

// PPM faces: X1 / X2 as columns (col_box), X3 as row warps where rows are
// long (x3_warp_box), else one face per thread (flux_box)
template <typename R, int D>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 4 : 1) k_flux_ppm(Grid g, const R *__restrict__ P,
                                                                          R *__restrict__ F, Box box, int want_dt)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    R cw;
    if constexpr (D < 3) {
        cw = flux_column_ppm<R, D>(g, P, F, box, want_dt, t);
    } else {
        if (g.x3warp) cw = flux_x3_warp_ppm<R>(g, P, F, box, want_dt, t);
        else cw = flux_item_ppm<R, D>(g, P, F, box, want_dt, t);
    }
    if (want_dt) block_cfl_into(&g.dtmin[D - 1], cw, g.cfl * g.dx[D - 1]);
}

template <typename R>
__global__ void k_emf(Grid g, const R *__restrict__ F1, const R *__restrict__ F2,
                      const R *__restrict__ F3, R *E1, R *E2, R *E3, Box box)
{
    emf_item(g, F1, F2, F3, E1, E2, E3, box, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

template <typename R>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 3 : 1) k_update(Grid g, const R *__restrict__ Pin, R *__restrict__ Pout,
                                                const R *__restrict__ F1, const R *__restrict__ F2,
                                                const R *__restrict__ F3, const R *__restrict__ E1,
                                                const R *__restrict__ E2, const R *__restrict__ E3,
                                                double dtfac, int corr)
{
    UpdCount cn{};
    update_call<R>(g, Pin, Pout, F1, F2, F3, E1, E2, E3, dtfac, corr,
                          blockIdx.x * (long long)blockDim.x + threadIdx.x, cn);
    flush_counts(g, cn);
}

template <typename R>
__global__ void __launch_bounds__(1024) k_fixup(Grid g, R *P, int corr)
{
    fixup_call(g, P, corr);
}

__global__ void k_finalize(Grid g, int advance)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    finalize_one(g, advance);
}

// ------------------------------------------------------------------ launch

static inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename R>
static void fill_bc(const Grid &g, R *P, cudaStream_t s)
{
    const int T = 128;
    if (polar_count(g) > 0) k_polar<R><<<nblk(polar_count(g), T), T, 0, s>>>(g, P);
    k_bc1<R><<<nblk(bc1_count(g), T), T, 0, s>>>(g, P);
    k_bc2<R><<<nblk(bc2_count(g), T), T, 0, s>>>(g, P);
    k_bc3<R><<<nblk(bc3_count(g), T), T, 0, s>>>(g, P);
}

// One part of a stage: 0-2 fluxes along X1..X3, 3 EMFs, 4 update + inversion,
// 5 fixups, 6 boundary fill.
template <typename R>
static void stage_part(const Grid &g, int part, int src, int dst, double dtfac, int corr, int want_dt,
                       cudaStream_t s)
{
    const int T = 128;
    const R *Pin = (const R *)g.P[src];
    R *Pout = (R *)g.P[dst];
    // the mixed path sweeps X3 by warps (x3_warp_box) where rows are long; else by faces
    Box b1 = flux_elem_box(g, 1), b2 = flux_elem_box(g, 2), be = edge_box(g);
    Box b3 = g.x3warp ? x3_warp_box(g) : flux_elem_box(g, 3);
    if (g.recon && part < 3) { // PPM faces: columns, row warps or single faces as for PLM
        const Box bp = part < 2 ? col_box(g, part + 1) : (g.x3warp ? x3_warp_box(g) : flux_box(g, 3));
        const unsigned nb = nblk(bp.count(), T);
        if (part == 0) k_flux_ppm<R, 1><<<nb, T, 0, s>>>(g, Pin, (R *)g.F[0], bp, want_dt);
        else if (part == 1) k_flux_ppm<R, 2><<<nb, T, 0, s>>>(g, Pin, (R *)g.F[1], bp, want_dt);
        else k_flux_ppm<R, 3><<<nb, T, 0, s>>>(g, Pin, (R *)g.F[2], bp, want_dt);
        return;
    }
    switch (part) {
    case 0: k_flux<R, 1><<<nblk(b1.count(), T), T, 0, s>>>(g, Pin, (R *)g.F[0], b1, want_dt); break;
    case 1: k_flux<R, 2><<<nblk(b2.count(), T), T, 0, s>>>(g, Pin, (R *)g.F[1], b2, want_dt); break;
    case 2: k_flux<R, 3><<<nblk(b3.count(), T), T, 0, s>>>(g, Pin, (R *)g.F[2], b3, want_dt); break;
    case 3:
        k_emf<R><<<nblk(be.count(), T), T, 0, s>>>(g, (const R *)g.F[0], (const R *)g.F[1], (const R *)g.F[2],
                                                    (R *)g.E[0], (R *)g.E[1], (R *)g.E[2], be);
        break;
    case 4:
        k_update<R><<<nblk(nact_of(g), T), T, 0, s>>>(g, Pin, Pout, (const R *)g.F[0], (const R *)g.F[1],
                                                      (const R *)g.F[2], (const R *)g.E[0], (const R *)g.E[1],
                                                      (const R *)g.E[2], dtfac, corr);
        break;
    case 5: k_fixup<R><<<1, 1024, 0, s>>>(g, Pout, corr); break;
    default: fill_bc<R>(g, Pout, s); break;
    }
}

template <typename R>
static void stage(const Grid &g, int src, int dst, double dtfac, int corr, int want_dt, cudaStream_t s)
{
    for (int part = 0; part < 7; part++) stage_part<R>(g, part, src, dst, dtfac, corr, want_dt, s);
}

// The same step as launch_step, with an event recorded before each part;
// ev holds 2 * 7 + 2 events.
void launch_step_profiled(const Grid &g, cudaStream_t s, cudaEvent_t *ev)
{
    int e = 0;
    for (int st = 0; st < 2; st++) {
        int src = st == 0 ? 0 : 1, dst = st == 0 ? 1 : 0;
        double fac = st == 0 ? 0.5 : 1.0;
        for (int part = 0; part < 7; part++) {
            cudaEventRecord(ev[e++], s);
            if (g.mixed) stage_part<float>(g, part, src, dst, fac, st, st == 0, s);
            else stage_part<double>(g, part, src, dst, fac, st, st == 0, s);
        }
    }
    cudaEventRecord(ev[e++], s);
    k_finalize<<<1, 32, 0, s>>>(g, 1);
    cudaEventRecord(ev[e++], s);
}

void launch_step(const Grid &g, cudaStream_t s)
{
    if (g.mixed) {
        stage<float>(g, 0, 1, 0.5, 0, 1, s);
        stage<float>(g, 1, 0, 1.0, 1, 0, s);
    } else {
        stage<double>(g, 0, 1, 0.5, 0, 1, s);
        stage<double>(g, 1, 0, 1.0, 1, 0, s);
    }
    k_finalize<<<1, 32, 0, s>>>(g, 1);
}

// one stage of the step (st 0: predictor, st 1: corrector) for a slab
void launch_stage(const Grid &g, int st, cudaStream_t s)
{
    int src = st == 0 ? 0 : 1, dst = st == 0 ? 1 : 0;
    double fac = st == 0 ? 0.5 : 1.0;
    if (g.mixed) stage<float>(g, src, dst, fac, st, st == 0, s);
    else stage<double>(g, src, dst, fac, st, st == 0, s);
}

__global__ void k_step_dtd(Grid g, double *dtd, int acc)
{
    if (threadIdx.x < 3) {
        double v = __longlong_as_double((long long)g.dtmin[threadIdx.x]);
        dtd[threadIdx.x] = acc ? fmin(dtd[threadIdx.x], v) : v;
        g.dtmin[threadIdx.x] = dbits(INFINITY);
    }
}

__global__ void k_finish_step(Grid g, const double *dtd)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double d[3] = {dtd[0], dtd[1], dtd[2]};
    g.scal[1] += g.scal[0];
    g.cnt[C_STEPS] += 1;
    g.scal[0] = combine_dt(d);
}

void launch_step_dtd(const Grid &g, double *dtd, int acc, cudaStream_t s) { k_step_dtd<<<1, 32, 0, s>>>(g, dtd, acc); }
void launch_finish_step(const Grid &g, const double *dtd, cudaStream_t s) { k_finish_step<<<1, 32, 0, s>>>(g, dtd); }

// X3 planes [NG][8][N1][N2]: pack k = base .. base+NG-1 into buf, or unpack buf there
template <typename R>
__global__ void k_x3_planes(Grid g, R *P, R *buf, int base, int unpack)
{
    long long plane = (long long)g.N1 * g.N2;
    long long n = (long long)NG * NP * plane;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    long long e = t % plane;
    int c = (int)((t / plane) % NP), gl = (int)(t / (plane * NP));
    int i = (int)(e / g.N2) - NG, j = (int)(e % g.N2) - NG;
    long long z = c * g.nz + zidx(g, i, j, base + gl);
    if (unpack) P[z] = buf[t];
    else buf[t] = P[z];
}

long long x3_plane_elems(const Grid &g) { return (long long)NG * NP * g.N1 * g.N2; }

// ------------------------------------------------------------ theta slabs

// stage st of a theta slab up to its fixups (parts 0-4 of stage_part)
void launch_stage_update(const Grid &g, int st, cudaStream_t s)
{
    int src = st == 0 ? 0 : 1, dst = st == 0 ? 1 : 0;
    double fac = st == 0 ? 0.5 : 1.0;
    for (int part = 0; part < 5; part++) {
        if (g.mixed) stage_part<float>(g, part, src, dst, fac, st, st == 0, s);
        else stage_part<double>(g, part, src, dst, fac, st, st == 0, s);
    }
}

__global__ void k_fail_count(Grid g, long long *acc)
{
    if (threadIdx.x == 0 && blockIdx.x == 0 && *g.nfail > 0)
        atomicAdd((unsigned long long *)acc, (unsigned long long)*g.nfail);
}

void launch_fail_count(const Grid &g, long long *acc, cudaStream_t s) { k_fail_count<<<1, 32, 0, s>>>(g, acc); }

template <typename R>
__global__ void __launch_bounds__(1024) k_fix_sweep(Grid g, R *P, int corr, long long *acc)
{
    const int nlist = min(*g.nfail, g.nfix_cap);
    if (nlist == 0) return;
    const int left = fixup_sweep<R>(g, P, corr, nlist);
    if (threadIdx.x == 0 && left > 0) atomicAdd((unsigned long long *)acc, (unsigned long long)left);
}

void launch_fix_sweep(const Grid &g, int st, long long *acc, cudaStream_t s)
{
    int dst = st == 0 ? 1 : 0;
    if (g.mixed) k_fix_sweep<float><<<1, 1024, 0, s>>>(g, (float *)g.P[dst], st, acc);
    else k_fix_sweep<double><<<1, 1024, 0, s>>>(g, (double *)g.P[dst], st, acc);
}

// close a theta slab's fixups: the sweeps its decomposed loop ran, the status
// if a listed zone is still failed (or the list overflowed), the list reset
__global__ void __launch_bounds__(256) k_fix_end(Grid g, int nsweeps)
{
    __shared__ int s_left;
    if (threadIdx.x == 0) s_left = 0;
    __syncthreads();
    const int nlist = min(*g.nfail, g.nfix_cap);
    int left = 0;
    for (int a = threadIdx.x; a < nlist; a += blockDim.x) {
        int t = g.faillist[a];
        int k = t % g.n3, r = t / g.n3, j = r % g.n2, i = r / g.n2;
        left += g.flag[zidx(g, i, j, k)] != 0;
    }
    if (left) atomicAdd(&s_left, left);
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&g.cnt[C_SWEEPS], (unsigned long long)nsweeps); // every slab counts the common rounds
        if (s_left > 0 || *g.nfail > g.nfix_cap) atomicOr(g.status, ST_FIXUP);
        *g.nfail = 0;
    }
}

void launch_fix_end(const Grid &g, int nsweeps, cudaStream_t s) { k_fix_end<<<1, 256, 0, s>>>(g, nsweeps); }

// The fixups of stage st of all theta slabs of one grid held on one device,
// in one block: the loop of fail counts, kind-1 row exchanges, Jacobi sweeps
// and closes that a host runs over the per-slab calls, with nothing read on
// the host.  A round copies every slab's neighbours' edge rows (the five
// averaged primitives and the flags) into its ghost rows before any slab
// sweeps, and a sweep reads across a slab face only those ghost rows, so
// the slabs' sweeps of a round see the same start state as the host loop's.
struct RingGrids {
    Grid g[RING_MAX];
};
static_assert(sizeof(RingGrids) < 32000, "kernel parameter block");

template <typename R>
__device__ void ring_edge_copy(const Grid &g, const Grid &gs, int jd, int js, int dst)
{
    R *P = (R *)g.P[dst];
    const R *Ps = (const R *)gs.P[dst];
    const long long plane = (long long)g.n1 * g.n3;
    for (long long t = threadIdx.x; t < 6 * plane; t += blockDim.x) {
        const int c = (int)(t / plane);
        const long long e = t % plane;
        const int i = (int)(e / g.n3), k = (int)(e % g.n3);
        const long long zd = zidx(g, i, jd, k), zs = zidx(gs, i, js, k);
        if (c < 5) P[c * g.nz + zd] = Ps[c * gs.nz + zs];
        else g.flag[zd] = gs.flag[zs] ? 1 : 0;
    }
}

template <typename R>
__global__ void __launch_bounds__(1024) k_fix_ring(RingGrids rg, int nslab, int st, int *nsweeps)
{
    __shared__ int s_left;
    const int dst = st == 0 ? 1 : 0;
    long long left = 0;
    for (int r = 0; r < nslab; r++) left += *rg.g[r].nfail;
    int n = 0;
    while (left > 0 && n < rg.g[0].fix_maxsweep) {
        for (int r = 0; r < nslab; r++) {
            const Grid &g = rg.g[r];
            if (x2_external(g, 0)) {
                const Grid &gs = rg.g[(r + nslab - 1) % nslab];
                ring_edge_copy<R>(g, gs, -1, gs.n2 - 1, dst);
            }
            if (x2_external(g, 1)) ring_edge_copy<R>(g, rg.g[(r + 1) % nslab], g.n2, 0, dst);
        }
        __syncthreads();
        left = 0;
        for (int r = 0; r < nslab; r++) {
            const Grid &g = rg.g[r];
            const int nlist = min(*g.nfail, g.nfix_cap);
            if (nlist > 0) left += fixup_sweep<R>(g, (R *)g.P[dst], st, nlist);
        }
        n++;
    }
    // close every slab as grmhd_fix_end does, with the common round count
    for (int r = 0; r < nslab; r++) {
        const Grid &g = rg.g[r];
        if (threadIdx.x == 0) s_left = 0;
        __syncthreads();
        const int nlist = min(*g.nfail, g.nfix_cap);
        int still = 0;
        for (int a = threadIdx.x; a < nlist; a += blockDim.x) {
            int t = g.faillist[a];
            int k = t % g.n3, q = t / g.n3, j = q % g.n2, i = q / g.n2;
            still += g.flag[zidx(g, i, j, k)] != 0;
        }
        if (still) atomicAdd(&s_left, still);
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicAdd(&g.cnt[C_SWEEPS], (unsigned long long)n);
            if (s_left > 0 || *g.nfail > g.nfix_cap) atomicOr(g.status, ST_FIXUP);
            *g.nfail = 0;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && nsweeps) *nsweeps = n;
}

void launch_fix_ring(const Grid *gs, int nslab, int st, int *nsweeps, cudaStream_t s)
{
    RingGrids rg;
    for (int r = 0; r < nslab; r++) rg.g[r] = gs[r];
    if (gs[0].mixed) k_fix_ring<float><<<1, 1024, 0, s>>>(rg, nslab, st, nsweeps);
    else k_fix_ring<double><<<1, 1024, 0, s>>>(rg, nslab, st, nsweeps);
}

__host__ __device__ inline long long x2_row_count(const Grid &g, int kind)
{
    return kind == 0 ? (long long)NG * NP * g.N1 * g.N3 : 6LL * g.n1 * g.n3;
}

long long x2_row_elems(const Grid &g, int kind) { return x2_row_count(g, kind); }

// X2 rows: kind 0 packs / unpacks rows base .. base+NG-1 as [NG][8][N1][N3];
// kind 1 row base as [6][n1][n3], the five averaged primitives and the flag
template <typename R>
__global__ void k_x2_rows(Grid g, R *P, R *buf, int kind, int base, int unpack)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= x2_row_count(g, kind)) return;
    if (kind == 0) {
        long long plane = (long long)g.N1 * g.N3;
        long long e = t % plane;
        int c = (int)((t / plane) % NP), gl = (int)(t / (plane * NP));
        int i = (int)(e / g.N3) - NG, k = (int)(e % g.N3) - NG;
        long long z = c * g.nz + zidx(g, i, base + gl, k);
        if (unpack) P[z] = buf[t];
        else buf[t] = P[z];
        return;
    }
    long long plane = (long long)g.n1 * g.n3;
    long long e = t % plane;
    int c = (int)(t / plane);
    int i = (int)(e / g.n3), k = (int)(e % g.n3);
    long long z = zidx(g, i, base, k);
    if (c < 5) {
        if (unpack) P[c * g.nz + z] = buf[t];
        else buf[t] = P[c * g.nz + z];
    } else {
        if (unpack) g.flag[z] = buf[t] != R(0) ? 1 : 0;
        else buf[t] = g.flag[z] ? R(1) : R(0);
    }
}

void launch_x2_rows(const Grid &g, int kind, int which, int side, void *buf, int unpack, cudaStream_t s)
{
    const int n = kind == 0 ? NG : 1;
    int base = unpack ? (side == 0 ? -n : g.n2) : (side == 0 ? 0 : g.n2 - n);
    long long ne = x2_row_elems(g, kind);
    unsigned nb = (unsigned)((ne + 255) / 256);
    if (g.mixed) k_x2_rows<float><<<nb, 256, 0, s>>>(g, (float *)g.P[which], (float *)buf, kind, base, unpack);
    else k_x2_rows<double><<<nb, 256, 0, s>>>(g, (double *)g.P[which], (double *)buf, kind, base, unpack);
}

void launch_x3_planes(const Grid &g, int which, int side, void *buf, int unpack, cudaStream_t s)
{
    int base = unpack ? (side == 0 ? -NG : g.n3) : (side == 0 ? 0 : g.n3 - NG);
    long long n = x3_plane_elems(g);
    unsigned nb = (unsigned)((n + 255) / 256);
    if (g.mixed) k_x3_planes<float><<<nb, 256, 0, s>>>(g, (float *)g.P[which], (float *)buf, base, unpack);
    else k_x3_planes<double><<<nb, 256, 0, s>>>(g, (double *)g.P[which], (double *)buf, base, unpack);
}

// Primitives re-derived from the conserved state alone: one stage's update
// with every face flux and edge EMF zero and a zero time-step factor, so U
// passes through unchanged (U + 0 x finite terms) and the step's own
// inversion, floors, ceilings, cap and fixups (Sections 2.3-2.4, Eq. 33)
// produce P from it, Newton starting from the primitives the context holds.
// Buffer 0 holds the result, ghosts filled.
void launch_reinvert(const Grid &g, cudaStream_t s)
{
    const size_t rs = g.mixed ? sizeof(float) : sizeof(double);
    for (int d = 0; d < 3; d++) {
        cudaMemsetAsync(g.F[d], 0, 9 * g.nz * rs, s);
        cudaMemsetAsync(g.E[d], 0, g.nz * rs, s);
    }
    const size_t bytes = (size_t)NP * g.nz * rs;
    cudaMemcpyAsync(g.P[1], g.P[0], bytes, cudaMemcpyDeviceToDevice, s); // no history: plain Newton start
    for (int part = 4; part < 7; part++) {
        if (g.mixed) stage_part<float>(g, part, 0, 1, 0.0, 1, 0, s);
        else stage_part<double>(g, part, 0, 1, 0.0, 1, 0, s);
    }
    cudaMemcpyAsync(g.P[0], g.P[1], bytes, cudaMemcpyDeviceToDevice, s);
}

void launch_bc(const Grid &g, int buf, cudaStream_t s)
{
    if (g.mixed) fill_bc<float>(g, (float *)g.P[buf], s);
    else fill_bc<double>(g, (double *)g.P[buf], s);
}

// flux sweep of buffer 0 only (CFL step of Eq. 27 at init, and the flux test entry)
void launch_fluxes_dt(const Grid &g, int set_dt, cudaStream_t s)
{
    for (int part = 0; part < 4; part++) {
        if (g.mixed) stage_part<float>(g, part, 0, 1, 0.0, 0, 1, s);
        else stage_part<double>(g, part, 0, 1, 0.0, 0, 1, s);
    }
    if (set_dt) k_finalize<<<1, 32, 0, s>>>(g, 0);
}

// flux-CT replaced fluxes of the current sweep, gathered to out[d][c][n1+1][n2+1][n3+1]
template <typename R>
__global__ void k_gather_fluxes(Grid g, double *out)
{
    long long m1 = g.n1 + 1, m2 = g.n2 + 1, m3 = g.n3 + 1;
    long long nf = m1 * m2 * m3;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= 3 * nf) return;
    int d = (int)(t / nf);
    long long o = t % nf;
    int k = (int)(o % m3), j = (int)((o / m3) % m2), i = (int)(o / (m2 * m3));
    int lim[3] = {g.n1 + (d == 0), g.n2 + (d == 1), g.n3 + (d == 2)};
    bool ok = i < lim[0] && j < lim[1] && k < lim[2];
    const R *F = (const R *)g.F[d];
    const R *E1 = (const R *)g.E[0], *E2 = (const R *)g.E[1], *E3 = (const R *)g.E[2];
    long long z = zidx(g, i, j, k);
    const long long zf = g.flat3 ? zidx(g, i, j, 0) : z; // axisymmetric grids keep the k = 0 faces
    const long long si = (long long)g.N2 * g.N3, sj = g.N3, sk = 1;
    for (int c = 0; c < NU; c++) {
        double v = 0.0;
        if (ok) {
            v = (double)F[c * g.nz + zf];
            if (d == 0) {
                if (c == KB1) v = 0.0;
                if (c == KB2) v = 0.5 * ((double)E3[z + sj] + (double)E3[z]);
                if (c == KB3) v = -0.5 * ((double)E2[z + sk] + (double)E2[z]);
            } else if (d == 1) {
                if (c == KB2) v = 0.0;
                if (c == KB1) v = -0.5 * ((double)E3[z + si] + (double)E3[z]);
                if (c == KB3) v = 0.5 * ((double)E1[z + sk] + (double)E1[z]);
            } else {
                if (c == KB3) v = 0.0;
                if (c == KB1) v = 0.5 * ((double)E2[z + si] + (double)E2[z]);
                if (c == KB2) v = -0.5 * ((double)E1[z + sj] + (double)E1[z]);
            }
        }
        out[((long long)d * NU + c) * nf + o] = v;
    }
}

void launch_gather_fluxes(const Grid &g, double *out, cudaStream_t s)
{
    long long nf = (long long)(g.n1 + 1) * (g.n2 + 1) * (g.n3 + 1);
    if (g.mixed) k_gather_fluxes<float><<<nblk(3 * nf, 128), 128, 0, s>>>(g, out);
    else k_gather_fluxes<double><<<nblk(3 * nf, 128), 128, 0, s>>>(g, out);
}

// FMA-chain throughput probe: 8 independent chains per thread.
template <typename T>
__global__ void k_fma_probe(T *out, int iters, T a, T b)
{
    T x[8];
#pragma unroll
    for (int c = 0; c < 8; c++) x[c] = T(threadIdx.x + c);
    for (int it = 0; it < iters; it++)
#pragma unroll
        for (int c = 0; c < 8; c++) x[c] = x[c] * a + b;
    T s = 0;
#pragma unroll
    for (int c = 0; c < 8; c++) s += x[c];
    if (s == T(-1.2345)) out[threadIdx.x] = s;
}

double launch_fma_probe(int fp64, int sms, cudaStream_t s)
{
    const int T = 256, iters = fp64 ? 4096 : 65536;
    int blocks = sms * 8;
    void *out;
    cudaMalloc(&out, 1024 * sizeof(double));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 0.0;
    for (int rep = 0; rep < 4; rep++) {
        cudaEventRecord(e0, s);
        if (fp64) k_fma_probe<double><<<blocks, T, 0, s>>>((double *)out, iters, 0.999999, 1e-7);
        else k_fma_probe<float><<<blocks, T, 0, s>>>((float *)out, iters, 0.9999f, 1e-7f);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms;
        cudaEventElapsedTime(&ms, e0, e1);
        double fl = 2.0 * 8.0 * iters * (double)blocks * T;
        if (rep > 0) best = fmax(best, fl / (ms * 1e-3) / 1e12);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return best;
}

} // namespace grmhd
