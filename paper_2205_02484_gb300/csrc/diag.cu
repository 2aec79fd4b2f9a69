// diag.cu -- horizon diagnostics (Section 4.2, Eqs. 38-42), the corner
// divergence of Eq. 24 (on the conserved sqrt(-g) B^i), batched stand-alone prim2cons / con2prim, and the
// active-zone state copies.
//
// Horizon sums are deterministic: fixed-size blocks write partial sums to
// scratch and one thread adds them in block order.  The divergence maximum
// uses an atomic max on the bit pattern of a non-negative double, which is
// order independent.
#include "fixes.cuh"
#include "kernels.h"
#include "mlp.cuh"

namespace grmhd {

template <typename RS>
__global__ void k_horizon_partial(Grid g, const RS *P, double *part)
{
    int n = g.n2 * g.n3;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    double v[4] = {0, 0, 0, 0};
    if (t < n && g.metric == KERR_MKS && g.i_h < g.n1) {
        int j = t / g.n3, k = t % g.n3, i = g.i_h;
        long long z = zidx(g, i, j, k);
        double q[NP];
        for (int c = 0; c < NP; c++) q[c] = (double)P[c * g.nz + z];
        const Geo<double> geo = g.gc[midx(g, i, j)];
        St<double> s;
        get_state(q, geo, s);
        double T[4];
        tmunu_row(q, s, g.gam, 1, T);
        double dA = g.dx[1] * g.dx[2];
        v[0] = geo.gdet * q[KRHO] * s.ucon[1] * dA;
        v[1] = 0.5 * geo.gdet * fabs(q[KB1]) * dA;
        v[2] = -geo.gdet * T[0] * dA;
        v[3] = geo.gdet * T[3] * dA;
    }
    __shared__ double sm[4][256];
    for (int c = 0; c < 4; c++) sm[c][threadIdx.x] = v[c];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int c = 0; c < 4; c++) sm[c][threadIdx.x] += sm[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 4; c++) part[4 * blockIdx.x + c] = sm[c][0];
}

// one warp: lanes take blocks lane, lane + 32, ...; the lane sums are then
// combined by a fixed shuffle tree (deterministic)
__global__ void k_horizon_sum(const double *part, int nb, double *out)
{
    double a[4] = {0, 0, 0, 0};
    for (int b = threadIdx.x; b < nb; b += 32)
        for (int c = 0; c < 4; c++) a[c] += part[4 * b + c];
    for (int o = 16; o > 0; o >>= 1)
        for (int c = 0; c < 4; c++) a[c] += __shfl_down_sync(0xffffffffu, a[c], o);
    if (threadIdx.x == 0)
        for (int c = 0; c < 4; c++) out[c] = a[c];
}

// Corner divergence of Eq. 24 on U_B = sqrt(-g) B^i: for each direction the
// four corner-adjacent values on the upper side minus the four on the lower
// side, times 1/(4 dX^d) (the grid's tabulated 1/dX^d).
__global__ void k_divb(Grid g, double *out)
{
    // a phi slab (external X3 ghosts) checks the corners inside it only: those
    // on its low phi face need the neighbour's conserved B
    bool per3 = g.bc3 != BC_EXTERNAL && (g.metric == KERR_MKS || g.bc3 == BC_PERIODIC);
    int k0 = (per3 || g.n3 == 1) ? 0 : 1;
    long long n = (long long)(g.n1 - 1) * (g.n2 - 1) * (g.n3 - k0);
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double dv = 0.0;
    if (t < n && n > 0) {
        int k = (int)(t % (g.n3 - k0)) + k0;
        long long r = t / (g.n3 - k0);
        int j = (int)(r % (g.n2 - 1)) + 1, i = (int)(r / (g.n2 - 1)) + 1;
        const int kl = k - 1 < 0 ? k - 1 + g.n3 : k - 1; // periodic in X3 (k >= 1 otherwise)
        double s1 = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll
        for (int l1 = 0; l1 < 2; l1++)
#pragma unroll
            for (int l2 = 0; l2 < 2; l2++)
#pragma unroll
                for (int l3 = 0; l3 < 2; l3++) {
                    long long z = zidx(g, i - 1 + l1, j - 1 + l2, l3 ? k : kl);
                    double b1 = g.U[KB1 * g.nz + z], b2 = g.U[KB2 * g.nz + z], b3 = g.U[KB3 * g.nz + z];
                    s1 += l1 ? b1 : -b1;
                    s2 += l2 ? b2 : -b2;
                    s3 += l3 ? b3 : -b3;
                }
        dv = 0.25 * (s1 * g.idx[0] + s2 * g.idx[1] + s3 * g.idx[2]);
    }
    dv = fabs(dv);
    for (int o = 16; o > 0; o >>= 1) dv = fmax(dv, __shfl_xor_sync(0xffffffffu, dv, o));
    if ((threadIdx.x & 31) == 0 && dv > 0.0)
        atomicMax((unsigned long long *)out, (unsigned long long)__double_as_longlong(dv));
}

// out_dev[0..3] = mdot, phib, edot, ldot; out_dev[4] = max corner divergence
void launch_diagnostics(const Grid &g, double *scratch, long scratch_len, double *out_dev, cudaStream_t s)
{
    int n = g.n2 * g.n3;
    int nb = (n + 255) / 256;
    (void)scratch_len;
    cudaMemsetAsync(out_dev, 0, 8 * sizeof(double), s);
    long long nc = (long long)(g.n1 - 1) * (g.n2 - 1) * g.n3;
    unsigned nbc = (unsigned)((nc + 255) / 256);
    if (g.mixed) {
        k_horizon_partial<float><<<nb, 256, 0, s>>>(g, (const float *)g.P[0], scratch);
        if (nc > 0) k_divb<<<nbc, 256, 0, s>>>(g, out_dev + 4);
    } else {
        k_horizon_partial<double><<<nb, 256, 0, s>>>(g, (const double *)g.P[0], scratch);
        if (nc > 0) k_divb<<<nbc, 256, 0, s>>>(g, out_dev + 4);
    }
    k_horizon_sum<<<1, 32, 0, s>>>(scratch, nb, out_dev);
}

// ----------------------------------------------- barycentric radius (Eq. 43)

// One block per radial row: the row's centre radius decides whether it is in
// [r_H, r_bar_max]; threads stride over its (j, k) zones (k fastest, so the
// density loads coalesce) and a fixed tree adds the block's terms.
template <typename RS>
__global__ void __launch_bounds__(256) k_bary_partial(Grid g, CoordParams cp, const RS *P, double rbar, double *part)
{
    const int i = blockIdx.x;
    double r, drdx;
    mks_radius<double>(cp, g.x1in + (i + 0.5) * g.dx[0], r, drdx);
    double num = 0.0, den = 0.0;
    if (i >= g.i_h && r <= rbar) {
        const int n = g.n2 * g.n3;
        const double dV = g.dx[0] * g.dx[1] * g.dx[2];
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            int j = t / g.n3, k = t - j * g.n3;
            double gdet = g.gc[midx(g, i, j)].gdet;
            double rho = (double)P[KRHO * g.nz + zidx(g, i, j, k)];
            num += r * rho * gdet * dV;
            den += rho * gdet * dV;
        }
    }
    __shared__ double sm[2][256];
    sm[0][threadIdx.x] = num;
    sm[1][threadIdx.x] = den;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sm[0][threadIdx.x] += sm[0][threadIdx.x + o];
            sm[1][threadIdx.x] += sm[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * i] = sm[0][0];
        part[2 * i + 1] = sm[1][0];
    }
}

// one warp adds the rows in a fixed order
__global__ void k_bary_sum(const double *part, int n1, double *out)
{
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n1; i += 32) {
        a += part[2 * i];
        b += part[2 * i + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (threadIdx.x == 0) {
        out[0] = a;
        out[1] = b;
    }
}

void launch_barycentric(const Grid &g, const CoordParams &cp, double r_bar_max, double *part, double *out,
                        cudaStream_t s)
{
    if (g.mixed) k_bary_partial<float><<<g.n1, 256, 0, s>>>(g, cp, (const float *)g.P[0], r_bar_max, part);
    else k_bary_partial<double><<<g.n1, 256, 0, s>>>(g, cp, (const double *)g.P[0], r_bar_max, part);
    k_bary_sum<<<1, 32, 0, s>>>(part, g.n1, out);
}

// ------------------------------------------- partial sums of a slab, combined
//
// The diagnostics of one context as a vector of DIAG_NPART doubles (its shell
// integrals, its corner div B maximum, its Eq. 43 sums, t, dt and counters),
// so that the slabs of a decomposed grid can gather the vectors on the device
// and the library can combine them.  Layout: [0..3] Mdot, phi_B, Edot, Ldot
// (Eqs. 38-41), [4] corner div B maximum (Eq. 24), [5] Eq. 43 numerator,
// [6] its mass sum, [7] t, [8] dt, [9 .. 9+C_NCOUNT) the counters; the
// combined vector adds [22] Phi_BH (Eq. 42), [23] (Edot - Mdot)/|Mdot|,
// [24] the barycentric radius.
__global__ void k_diag_pack(Grid g, const double *horizon, const double *bary, double *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int c = 0; c < 5; c++) out[c] = horizon[c];
    out[5] = bary ? bary[0] : 0.0;
    out[6] = bary ? bary[1] : 0.0;
    out[7] = g.scal[1];
    out[8] = g.scal[0];
    for (int c = 0; c < C_NCOUNT; c++) out[9 + c] = (double)g.cnt[c];
    for (int c = 9 + C_NCOUNT; c < DIAG_NPART; c++) out[c] = 0.0;
}

// Sum of nparts partial vectors in their order (one thread: the order of the
// additions is fixed, so every rank forms the same bits): integrals and
// counters add up, div B and the fixup sweep count take the largest, t, dt
// and the step count are the slabs' common values; then Eq. 42, the
// efficiency and the Eq. 43 quotient of the sums.
__global__ void k_diag_combine(const double *parts, int nparts, double *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double v[DIAG_NPART];
    for (int c = 0; c < DIAG_NPART; c++) v[c] = parts[c];
    for (int r = 1; r < nparts; r++) {
        const double *p = parts + (long long)r * DIAG_NPART;
        for (int c = 0; c < 4; c++) v[c] += p[c];
        v[4] = fmax(v[4], p[4]);
        v[5] += p[5];
        v[6] += p[6];
        for (int c = 0; c < C_NCOUNT; c++) {
            if (c == C_SWEEPS) v[9 + c] = fmax(v[9 + c], p[9 + c]);
            else if (c != C_STEPS) v[9 + c] += p[9 + c];
        }
    }
    const double mdot = v[0];
    v[22] = mdot != 0.0 ? v[1] / sqrt(fabs(mdot)) : 0.0;
    v[23] = mdot != 0.0 ? (v[2] - mdot) / fabs(mdot) : 0.0;
    v[24] = v[6] > 0.0 ? v[5] / v[6] : 0.0;
    v[25] = 0.0;
    for (int c = 0; c < DIAG_NPART; c++) out[c] = v[c];
}

void launch_diag_pack(const Grid &g, const double *horizon, const double *bary, double *out, cudaStream_t s)
{
    k_diag_pack<<<1, 32, 0, s>>>(g, horizon, bary, out);
}

void launch_diag_combine(const double *parts, int nparts, double *out, cudaStream_t s)
{
    k_diag_combine<<<1, 32, 0, s>>>(parts, nparts, out);
}

// ------------------------------------------------------------ point batches

__global__ void k_prim2cons(Grid g, const double *P, const int *loc, double *U, long n)
{
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    int l = loc[t];
    if (l < 0 || l >= g.n1 * g.n2) {
        for (int c = 0; c < NU; c++) U[c * n + t] = NAN;
        return;
    }
    const Geo<double> geo = g.gc[midx(g, l / g.n2, l % g.n2)];
    double q[NP], Uz[NU];
    for (int c = 0; c < NP; c++) q[c] = P[c * n + t];
    St<double> s;
    get_state(q, geo, s);
    prim_to_UF<double, false>(q, geo, s, g.gam, 0, Uz);
    for (int c = 0; c < NU; c++) U[c * n + t] = Uz[c];
}

// The stand-alone inversion runs in two passes so that the zones leaving
// Newton (the low-beta entropy inversions, Brent in W, the entropy inversion
// after an unphysical Newton root: loops of their own length) do not hold
// the lanes of Newton zones: the first pass (pass 1 of con2prim) finishes
// every zone Newton settles and appends the others to a compacted list; the
// second resumes each listed zone at its deferred step, 32 such zones to a
// warp.  The results are those of the whole chain in one pass.
//
// list: [0] the count, then the deferred indices.  On deferral the flag
// holds the step to resume at, P the input primitives (after an unphysical
// Newton root, that root's primitives, where the whole chain leaves them).
__device__ __forceinline__ void c2p_defer(int *list, long t, bool defer)
{
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, defer);
    if (!defer) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(list, __popc(m));
    base = __shfl_sync(m, base, leader);
    list[1 + base + __popc(m & ((1u << lane) - 1))] = (int)t;
}

__device__ __forceinline__ void c2p_store(const int fl, const double q[NP], double *P, int *flags, long n, long t,
                                          int *list)
{
    flags[t] = fl;
    const bool defer = (fl & C2P_DEFER) != 0;
    if (!defer || (fl & C2P_DEFER_ENT)) {
        for (int c = 0; c < (defer ? 5 : NP); c++) P[c * n + t] = q[c];
    }
    c2p_defer(list, t, defer);
}

// the first pass; mode 0: plain start from P; 1: the network's W first, then
// P; 2: P, then the network's W as a rescue before Brent (the step's use)
__global__ void __launch_bounds__(128) k_con2prim(Grid g, const double *U, const int *loc, double *P, int *flags,
                                                  int *iters, long n, const float *mlp, int mode, int *list)
{
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    int l = loc[t];
    if (l < 0 || l >= g.n1 * g.n2) {
        flags[t] = C2P_FAIL | C2P_FAIL_D;
        if (iters) iters[t] = 0;
        c2p_defer(list, t, false);
        return;
    }
    const Geo<double> geo = g.gc[midx(g, l / g.n2, l % g.n2)];
    double Uz[NU], q0[NP], q[NP];
    for (int c = 0; c < NU; c++) Uz[c] = U[c * n + t];
    for (int c = 0; c < NP; c++) q0[c] = P[c * n + t];
    int it;
    const int fl = con2prim(Uz, geo, g.gsp + 6LL * midx(g, l / g.n2, l % g.n2), q0, nullptr, c2p_par(g), 15, q,
                            it, mode == 1 ? mlp : nullptr, nullptr, nullptr, false, mode == 2 ? mlp : nullptr, 0.0,
                            1);
    if (iters) iters[t] = it;
    c2p_store(fl, q, P, flags, n, t, list);
}

// the second pass: the listed zones resumed at their deferred steps
__global__ void __launch_bounds__(128) k_con2prim_rest(Grid g, const double *U, const int *loc, double *P,
                                                       int *flags, long n, const int *list)
{
    const long a = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (a >= list[0]) return;
    const long t = list[1 + a];
    const int l = loc[t];
    const int m = midx(g, l / g.n2, l % g.n2);
    const Geo<double> geo = g.gc[m];
    double Uz[NU], q0[NP], q[NP];
    for (int c = 0; c < NU; c++) Uz[c] = U[c * n + t];
    for (int c = 0; c < NP; c++) q0[c] = P[c * n + t];
    int it;
    flags[t] = con2prim(Uz, geo, g.gsp + 6LL * m, q0, nullptr, c2p_par(g), 15, q, it, nullptr, nullptr, nullptr,
                        false, nullptr, 0.0, 2, flags[t]);
    for (int c = 0; c < NP; c++) P[c * n + t] = q[c];
}

// The inversion with the learned start first, the network evaluated per warp
// on the tensor cores (mlp_log_w_mma) from the invariants of each lane's
// state; lanes without a state (past n, bad loc, D not positive) take part
// in the warp's inference with the feature means and invert nothing.
__global__ void __launch_bounds__(128) k_con2prim_learned(Grid g, const double *U, const int *loc, double *P,
                                                          int *flags, int *iters, long n, const float *mlp,
                                                          int *list)
{
    __shared__ MlpSmem s;
    mlp_stage(mlp, s);
    __syncthreads();
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const int l = t < n ? loc[t] : -1;
    const bool ok = l >= 0 && l < g.n1 * g.n2;
    const int m = ok ? midx(g, l / g.n2, l % g.n2) : 0;
    const Geo<double> geo = g.gc[m];
    const double *gsp = g.gsp + 6LL * m;
    double Uz[NU];
    for (int c = 0; c < NU; c++) Uz[c] = ok ? U[c * n + t] : 0.0;
    C2PIn c;
    const bool have = ok && c2p_feature_invariants(Uz, geo, gsp, c);
    float f[MLP_IN];
    if (have) {
        c2p_learned_features(c, f);
    } else {
#pragma unroll
        for (int k = 0; k < MLP_IN; k++) f[k] = s.norm[k];
    }
    const float y = mlp_log_w_mma(s, f);
    if (t >= n) return;
    if (!ok) {
        flags[t] = C2P_FAIL | C2P_FAIL_D;
        if (iters) iters[t] = 0;
        c2p_defer(list, t, false);
        return;
    }
    double q0[NP], q[NP];
    for (int k = 0; k < NP; k++) q0[k] = P[k * n + t];
    int it;
    const int fl = con2prim(Uz, geo, gsp, q0, nullptr, c2p_par(g), 15, q, it, nullptr, nullptr, nullptr, false,
                            nullptr, have ? c2p_w_of(c.D, y) : 0.0, 1);
    if (iters) iters[t] = it;
    c2p_store(fl, q, P, flags, n, t, list);
}

void launch_prim2cons(const Grid &g, const double *P, const int *loc, double *U, long n, cudaStream_t s)
{
    if (n > 0) k_prim2cons<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(g, P, loc, U, n);
}

void launch_con2prim(const Grid &g, const double *U, const int *loc, double *P, int *flags, int *iters,
                     long n, const float *mlp, int mode, int *list, cudaStream_t s)
{
    if (n <= 0) return;
    const unsigned nb = (unsigned)((n + 127) / 128);
    cudaMemsetAsync(list, 0, sizeof(int), s);
    if (mode == 1) k_con2prim_learned<<<nb, 128, 0, s>>>(g, U, loc, P, flags, iters, n, mlp, list);
    else k_con2prim<<<nb, 128, 0, s>>>(g, U, loc, P, flags, iters, n, mlp, mode, list);
    k_con2prim_rest<<<nb, 128, 0, s>>>(g, U, loc, P, flags, n, list);
}

// ------------------------------------------------------------ state copies

template <typename RS>
__global__ void k_state_in(Grid g, const double *Pa, const double *Ua)
{
    long long nact = (long long)g.n1 * g.n2 * g.n3;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nact) return;
    int k = (int)(t % g.n3);
    long long r = t / g.n3;
    int j = (int)(r % g.n2), i = (int)(r / g.n2);
    long long z = zidx(g, i, j, k);
    RS *P = (RS *)g.P[0];
    // a value is finite unless its exponent bits are all set (integer test on the high word)
    unsigned bad = 0;
    if (Pa) // null: U alone (the primitives are re-derived afterwards)
        for (int c = 0; c < NP; c++) {
            const double v = Pa[c * nact + t];
            bad |= (__double2hiint(v) & 0x7ff00000) == 0x7ff00000;
            P[c * g.nz + z] = (RS)v;
        }
    for (int c = 0; c < NU; c++) {
        const double v = Ua[c * nact + t];
        bad |= (__double2hiint(v) & 0x7ff00000) == 0x7ff00000;
        g.U[c * g.nz + z] = v;
    }
    if (bad) atomicOr(g.status, ST_NONFINITE);
}

template <typename RS>
__global__ void k_state_out(Grid g, double *Pa, double *Ua)
{
    long long nact = (long long)g.n1 * g.n2 * g.n3;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nact) return;
    int k = (int)(t % g.n3);
    long long r = t / g.n3;
    int j = (int)(r % g.n2), i = (int)(r / g.n2);
    long long z = zidx(g, i, j, k);
    const RS *P = (const RS *)g.P[0];
    if (Pa)
        for (int c = 0; c < NP; c++) Pa[c * nact + t] = (double)P[c * g.nz + z];
    if (Ua)
        for (int c = 0; c < NU; c++) Ua[c * nact + t] = g.U[c * g.nz + z];
}

void launch_copy_state_in(const Grid &g, const double *P, const double *U, cudaStream_t s)
{
    long long nact = (long long)g.n1 * g.n2 * g.n3;
    unsigned nb = (unsigned)((nact + 255) / 256);
    if (g.mixed) k_state_in<float><<<nb, 256, 0, s>>>(g, P, U);
    else k_state_in<double><<<nb, 256, 0, s>>>(g, P, U);
}

void launch_copy_state_out(const Grid &g, double *P, double *U, cudaStream_t s)
{
    long long nact = (long long)g.n1 * g.n2 * g.n3;
    unsigned nb = (unsigned)((nact + 255) / 256);
    if (g.mixed) k_state_out<float><<<nb, 256, 0, s>>>(g, P, U);
    else k_state_out<double><<<nb, 256, 0, s>>>(g, P, U);
}

} // namespace grmhd
