// abi.cu -- the extern "C" entry points declared in include/grmhd.h.
//
// A context owns one grid: its device state, metric tables, scratch, stream
// and the CUDA graph of one full RK2 step.  The step graph is captured on the
// first grmhd_step call and replayed afterwards; the time step lives on the
// device, so replays need no host round trip.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/grmhd.h"
#include "kernels.h"
#include "mlp.cuh"

using namespace grmhd;

struct grmhd_ctx {
    grmhd_grid_params gp;
    grmhd_phys_params pp;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Grid g{};
    GeomBuild gb{};
    std::vector<void *> allocs;
    bool metric_set = false, state_set = false;
    double a = 0.0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    double *scratch = nullptr;
    long long scratch_len = 0;
    double *staging = nullptr;
    long long staging_len = 0;
    int *c2p_list = nullptr; // the stand-alone inversion's deferred zones (count, then indices)
    long long c2p_list_len = 0;
    unsigned char *intorus = nullptr;
    double *hpin = nullptr; // pinned host scratch (64 doubles)
    double disk_mass = 0.0, disk_eb = 0.0;
    CoordParams cp{}; // coordinate map of the metric (Kerr grids)
    // host <-> device state copies split over several streams (copy engines)
    static constexpr int NCOPY = 4;
    cudaStream_t cstream[NCOPY] = {};
    cudaEvent_t cfork = nullptr, cjoin[NCOPY] = {};
    float *mlp = nullptr;       // packed forward buffer of the learned Newton start
    float *mlp_theta = nullptr; // its FP32 parameters
    bool mlp_loaded = false;
    std::string err;
};

static thread_local std::string g_create_err;

static int fail(grmhd_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    else g_create_err = msg;
    return code;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(ctx, GRMHD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
    } while (0)

template <typename T>
static int dalloc(grmhd_ctx *ctx, T **p, size_t count)
{
    void *q = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return fail(ctx, GRMHD_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    cudaMemsetAsync(q, 0, bytes, ctx->stream);
    ctx->allocs.push_back(q);
    *p = (T *)q;
    return 0;
}

static long long nact_of(const grmhd_ctx *c) { return (long long)c->g.n1 * c->g.n2 * c->g.n3; }

const Grid *ctx_grid(const grmhd_ctx *ctx) { return ctx ? &ctx->g : nullptr; }
bool ctx_ready(const grmhd_ctx *ctx) { return ctx && ctx->metric_set && ctx->state_set; }
int ctx_device(const grmhd_ctx *ctx) { return ctx->gp.device; }
cudaStream_t ctx_stream(const grmhd_ctx *ctx) { return ctx->stream; }

extern "C" const char *grmhd_version(void) { return "grmhd-gb300 0.1 (sm_103a)"; }

extern "C" const char *grmhd_last_error(const grmhd_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

extern "C" void grmhd_destroy(grmhd_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    for (void *p : ctx->allocs) cudaFree(p);
    if (ctx->hpin) cudaFreeHost(ctx->hpin);
    for (int k = 0; k < grmhd_ctx::NCOPY; k++) {
        if (ctx->cstream[k]) cudaStreamDestroy(ctx->cstream[k]);
        if (ctx->cjoin[k]) cudaEventDestroy(ctx->cjoin[k]);
    }
    if (ctx->cfork) cudaEventDestroy(ctx->cfork);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

// A new state is copied into the second primitive buffer too: the mixed
// update reads that buffer's previous contents for its Newton start, which
// after a new state must be the state itself (no history).
static int copy_stage_buffer(grmhd_ctx *ctx)
{
    const Grid &g = ctx->g;
    size_t bytes = (size_t)NP * g.nz * (g.mixed ? sizeof(float) : sizeof(double));
    CK(cudaMemcpyAsync(g.P[1], g.P[0], bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    return 0;
}

extern "C" int grmhd_init_grid(const grmhd_grid_params *grid, const grmhd_phys_params *phys, grmhd_ctx **out)
{
    grmhd_ctx *ctx = nullptr;
    if (!grid || !phys || !out) return fail(nullptr, GRMHD_EINVAL, "null argument");
    if (grid->n1 < 1 || grid->n2 < 1 || grid->n3 < 1) return fail(nullptr, GRMHD_EINVAL, "grid sizes must be >= 1");
    if (grid->metric == GRMHD_KERR_MKS && grid->n1 < 2)
        return fail(nullptr, GRMHD_EINVAL, "Kerr grid needs n1 >= 2");
    if (grid->precision != GRMHD_FP64 && grid->precision != GRMHD_MIXED)
        return fail(nullptr, GRMHD_EINVAL, "precision must be GRMHD_FP64 or GRMHD_MIXED");
    if (grid->bc1 < 0 || grid->bc1 > GRMHD_BC_OUTFLOW || grid->bc2 < 0 || grid->bc2 > GRMHD_BC_OUTFLOW ||
        grid->bc3 < 0 || grid->bc3 > GRMHD_BC_EXTERNAL)
        return fail(nullptr, GRMHD_EINVAL, "bad boundary kind (external is for bc3 only)");
    if (grid->bc3 == GRMHD_BC_EXTERNAL && grid->n3 < 2)
        return fail(nullptr, GRMHD_EINVAL, "a phi slab needs n3 >= 2");
    if (grid->n2_total != 0) {
        if (grid->n2 < 4 || grid->j0 < 0 || (long long)grid->j0 + grid->n2 > grid->n2_total)
            return fail(nullptr, GRMHD_EINVAL, "a theta slab needs n2 >= 4 rows inside [0, n2_total)");
        if (grid->bc3 == GRMHD_BC_EXTERNAL)
            return fail(nullptr, GRMHD_EINVAL, "a grid is a theta slab or a phi slab, not both");
    } else if (grid->j0 != 0) {
        return fail(nullptr, GRMHD_EINVAL, "j0 needs n2_total (a theta slab)");
    }
    if (grid->riemann != GRMHD_LLF && grid->riemann != GRMHD_HLL)
        return fail(nullptr, GRMHD_EINVAL, "riemann must be GRMHD_LLF or GRMHD_HLL");
    if (grid->recon != GRMHD_PLM && grid->recon != GRMHD_PPM)
        return fail(nullptr, GRMHD_EINVAL, "recon must be GRMHD_PLM or GRMHD_PPM");
    if (!(phys->gam > 1.0) || !(phys->cfl > 0.0) || phys->nr_maxit < 1 || phys->brent_maxit < 1 ||
        phys->fix_maxsweep < 1 || !(phys->sigma_max > 0.0) || !(phys->bu_max > 0.0) || !(phys->gamma_max >= 1.0))
        return fail(nullptr, GRMHD_EINVAL, "bad physics parameters");
    long long N1 = grid->n1 + 2 * NG, N2 = grid->n2 + 2 * NG, N3 = grid->n3 + 2 * NG;
    long long nz = N1 * N2 * N3;
    if (nz > (1LL << 31) - 1) return fail(nullptr, GRMHD_EINVAL, "grid too large for 32-bit zone lists");
    if (cudaSetDevice(grid->device) != cudaSuccess) return fail(nullptr, GRMHD_ECUDA, "cudaSetDevice failed");
    ctx = new grmhd_ctx();
    ctx->gp = *grid;
    ctx->pp = *phys;
    if (grid->stream) {
        ctx->stream = (cudaStream_t)grid->stream;
    } else {
        CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamDefault));
        ctx->own_stream = true;
    }
    Grid &g = ctx->g;
    g.n1 = grid->n1; g.n2 = grid->n2; g.n3 = grid->n3;
    g.j0 = grid->j0;
    g.n2t = grid->n2_total > 0 ? grid->n2_total : grid->n2;
    g.N1 = (int)N1; g.N2 = (int)N2; g.N3 = (int)N3;
    g.nz = nz;
    g.metric = grid->metric;
    g.bc1 = grid->bc1; g.bc2 = grid->bc2; g.bc3 = grid->bc3;
    g.riemann = grid->riemann;
    g.recon = grid->recon;
    g.mixed = grid->precision == GRMHD_MIXED;
    // a row warp evaluates 29 faces per 32 lanes: worth it only for rows of >= 32 faces
    g.x3warp = g.n3 + 1 >= 32;
    // an axisymmetric grid (n3 = 1, X3 ghosts copies of the one plane) computes
    // the k = 0 faces only: the k = -1 and k = 1 planes hold the same states
    g.flat3 = g.n3 == 1 && (grid->metric == GRMHD_KERR_MKS || grid->bc3 == GRMHD_BC_PERIODIC ||
                            grid->bc3 == GRMHD_BC_OUTFLOW);
    g.gam = phys->gam; g.cfl = phys->cfl; g.nr_tol = phys->nr_tol; g.sigma_max = phys->sigma_max;
    g.bu_max = phys->bu_max; g.gamma_max = phys->gamma_max; g.beta_ent = phys->beta_entropy;
    g.g1 = (g.gam - 1.0) / g.gam;
    g.igm1 = 1.0 / (g.gam - 1.0);
    g.ig = 1.0 / g.gam;
    g.isig = 1.0 / g.sigma_max;
    g.ibu = 1.0 / g.bu_max;
    g.isig_f = (float)g.isig;
    g.ibu_f = (float)g.ibu;
    g.gam_f = (float)g.gam;
    g.g1_f = (float)g.g1;
    g.beta_ent_f = (float)g.beta_ent;
    g.gamma_max_f = (float)g.gamma_max;
    g.nr_tol_mixed = std::sqrt(g.nr_tol);
    g.tol_mixed_f = (float)g.nr_tol_mixed;
    {
        // column length of the X1 / X2 flux sweeps: at least ~2^17 threads per sweep
        long long faces = (long long)(g.n1 + 1) * (g.n2 + 2) * (g.n3 + 2);
        int fc = 1;
        while (fc < 16 && faces / (2LL * fc) >= (1LL << 17)) fc *= 2;
        g.fcol = fc;
    }
    g.nr_maxit = phys->nr_maxit; g.brent_maxit = phys->brent_maxit; g.fix_maxsweep = phys->fix_maxsweep;
    long long nact = (long long)g.n1 * g.n2 * g.n3;
    g.nfix_cap = (int)std::min<long long>(nact, 1LL << 20);
    size_t rs = g.mixed ? sizeof(float) : sizeof(double);
    int rc = 0;
    long long nm = N1 * N2;
    GeomBuild &b = ctx->gb;
    for (int s = 0; s < 2 && !rc; s++) rc = dalloc(ctx, (char **)&g.P[s], 8 * nz * rs);
    if (!rc) rc = dalloc(ctx, &g.U, 9 * nz);
    for (int d = 0; d < 3 && !rc; d++) rc = dalloc(ctx, (char **)&g.F[d], 9 * nz * rs);
    for (int d = 0; d < 3 && !rc; d++) rc = dalloc(ctx, (char **)&g.E[d], nz * rs);
    if (!rc) rc = dalloc(ctx, &g.flag, nz);
    if (!rc) rc = dalloc(ctx, &b.gc, nm);
    if (!rc) rc = dalloc(ctx, &b.gf1, nm);
    if (!rc) rc = dalloc(ctx, &b.gf2, nm);
    if (!rc) rc = dalloc(ctx, &b.gcF, nm);
    if (!rc) rc = dalloc(ctx, &b.gf1F, nm);
    if (!rc) rc = dalloc(ctx, &b.gf2F, nm);
    if (!rc) rc = dalloc(ctx, &b.conn, nm * 40);
    if (!rc) rc = dalloc(ctx, &b.connF, nm * 40);
    if (!rc) rc = dalloc(ctx, &b.rc, nm);
    if (!rc) rc = dalloc(ctx, &b.gsp, nm * 6);
    if (!rc) rc = dalloc(ctx, &b.polar2, nm);
    if (!rc) rc = dalloc(ctx, &g.scal, 8);
    if (!rc) rc = dalloc(ctx, &g.dtmin, 4);
    if (!rc) rc = dalloc(ctx, &g.cnt, C_NCOUNT);
    if (!rc) rc = dalloc(ctx, &g.status, 4);
    if (!rc) rc = dalloc(ctx, &g.nfail, 4);
    if (!rc) rc = dalloc(ctx, &g.faillist, g.nfix_cap);
    if (!rc) rc = dalloc(ctx, &g.fixbuf, 6LL * g.nfix_cap);
    if (!rc) rc = dalloc(ctx, &ctx->intorus, (long long)g.n1 * g.n2);
    long long nbz = (nact + 255) / 256;
    ctx->scratch_len = 8 * nact + 8 + (long long)(g.n1 + 1) * (g.n2 + 1) + 4 * nbz + 64;
    if (!rc) rc = dalloc(ctx, &ctx->scratch, ctx->scratch_len);
    if (!rc && cudaMallocHost(&ctx->hpin, 64 * sizeof(double)) != cudaSuccess) rc = GRMHD_ENOMEM;
    if (rc) {
        g_create_err = ctx->err.empty() ? "allocation failed" : ctx->err;
        grmhd_destroy(ctx);
        return rc;
    }
    g.gc = b.gc; g.gf1 = b.gf1; g.gf2 = b.gf2;
    g.gcF = b.gcF; g.gf1F = b.gf1F; g.gf2F = b.gf2F;
    g.conn = b.conn; g.connF = b.connF; g.rc = b.rc; g.polar2 = b.polar2; g.gsp = b.gsp;
    unsigned long long inf = 0x7FF0000000000000ULL;
    unsigned long long h[4] = {inf, inf, inf, inf};
    cudaMemcpyAsync(g.dtmin, h, sizeof(h), cudaMemcpyHostToDevice, ctx->stream);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        g_create_err = cudaGetErrorString(e);
        grmhd_destroy(ctx);
        return GRMHD_ECUDA;
    }
    *out = ctx;
    return 0;
}

static double x1_of_r(const CoordParams &cp, double r)
{
    double lo = -50.0, hi = 50.0;
    for (int it = 0; it < 300; it++) {
        double mid = 0.5 * (lo + hi), rr, dr;
        mks_radius<double>(cp, mid, rr, dr);
        if (rr < r) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

extern "C" int grmhd_set_metric(grmhd_ctx *ctx, double a, int kind)
{
    if (!ctx) return fail(nullptr, GRMHD_EINVAL, "null context");
    if (kind != GRMHD_KERR_MKS && kind != GRMHD_MINK_CART) return fail(ctx, GRMHD_EINVAL, "unknown metric kind");
    if (kind == GRMHD_KERR_MKS && !(std::fabs(a) < 1.0)) return fail(ctx, GRMHD_EINVAL, "spin must satisfy |a| < 1");
    Grid &g = ctx->g;
    const grmhd_grid_params &p = ctx->gp;
    g.metric = kind;
    CoordParams cp{};
    cp.metric = kind;
    cp.a = a;
    cp.hslope = p.hslope;
    cp.n_x = p.n_x;
    cp.R0 = p.R0;
    cp.cyl_r = p.cyl_r;
    cp.cyl_dx2 = p.cyl_dx2;
    if (p.cyl_r > 0.0 && kind != GRMHD_KERR_MKS)
        return fail(ctx, GRMHD_EINVAL, "cylindrification needs the Kerr grid");
    if (kind == GRMHD_KERR_MKS) {
        double rh =1.0 + std::sqrt(1.0 - a * a);
        if (!(p.r_in > p.R0) || !(p.r_out > p.r_in) || !(p.r_br > p.R0))
            return fail(ctx, GRMHD_EINVAL, "need R0 < r_in < r_out and r_br > R0");
        if (g.n2 < 2) return fail(ctx, GRMHD_EINVAL, "Kerr grid needs n2 >= 2");
        cp.xb = std::log(p.r_br - p.R0);
        g.x1in = std::log(p.r_in - p.R0);
        double x1out = p.r_out <= p.r_br ? std::log(p.r_out - p.R0) : x1_of_r(cp, p.r_out);
        g.x2in = -1.0;
        g.dx[0] = (x1out - g.x1in) / g.n1;
        g.dx[1] = 2.0 / g.n2t;
        if (g.bc3 == BC_EXTERNAL) { // a phi slab [x3min, x3max) of the full circle
            g.x3in = p.x3min;
            g.dx[2] = (p.x3max - p.x3min) / g.n3;
            if (!(g.dx[2] > 0.0)) return fail(ctx, GRMHD_EINVAL, "phi slab needs x3max > x3min");
        } else {
            g.x3in = 0.0;
            g.dx[2] = 2.0 * M_PI / g.n3;
        }
        if (p.cyl_r > 0.0) {
            // lambda(r) falls with r: its largest value is at the innermost ghost face
            double rmin, dr;
            mks_radius<double>(cp, g.x1in - NG * g.dx[0], rmin, dr);
            double x = p.cyl_r / rmin;
            if (!(p.cyl_dx2 > 0.0 && p.cyl_dx2 <= 1.0) || !std::isfinite(p.cyl_r) ||
                !(std::pow(1.0 + x * x * x * x, 0.25) <= 2.5))
                return fail(ctx, GRMHD_EINVAL, "cylindrification needs 0 < cyl_dx2 <= 1 and lambda <= 5/2");
        }
        g.i_h = g.n1;
        for (int i = 0; i < g.n1; i++) {
            double r, dr;
            mks_radius<double>(cp, g.x1in + (i + 0.5) * g.dx[0], r, dr);
            if (r >= rh) { g.i_h = i; break; }
        }
        ctx->cp = cp;
    } else {
        cp.xb = 1e300;
        g.x1in = p.x1min; g.x2in = p.x2min; g.x3in = p.x3min;
        g.dx[0] = (p.x1max - p.x1min) / g.n1;
        g.dx[1] = (p.x2max - p.x2min) / g.n2t;
        g.dx[2] = (p.x3max - p.x3min) / g.n3;
        g.i_h = 0;
        if (!(g.dx[0] > 0) || !(g.dx[1] > 0) || !(g.dx[2] > 0)) return fail(ctx, GRMHD_EINVAL, "empty box");
    }
    for (int d = 0; d < 3; d++) {
        g.idx[d] = 1.0 / g.dx[d];
        g.idx_f[d] = (float)g.idx[d];
        g.hidx_hi[d] = (float)(0.5 * g.idx[d]);
        g.hidx_lo[d] = (float)(0.5 * g.idx[d] - (double)g.hidx_hi[d]);
    }
    ctx->gb.cp = cp;
    ctx->a = a;
    (void)cudaGetLastError(); // a stale error of an unrelated earlier call is not ours
    launch_geometry(g, ctx->gb, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->metric_set = true;
    if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; }
    if (ctx->graph) { cudaGraphDestroy(ctx->graph); ctx->graph = nullptr; }
    return 0;
}

static int reset_counters(grmhd_ctx *ctx)
{
    Grid &g = ctx->g;
    CK(cudaMemsetAsync(g.cnt, 0, C_NCOUNT * sizeof(unsigned long long), ctx->stream));
    CK(cudaMemsetAsync(g.status, 0, 4 * sizeof(int), ctx->stream));
    CK(cudaMemsetAsync(g.nfail, 0, 4 * sizeof(int), ctx->stream));
    return 0;
}

static int set_scalars(grmhd_ctx *ctx, double t, double dt)
{
    ctx->hpin[0] = dt;
    ctx->hpin[1] = t;
    CK(cudaMemcpyAsync(ctx->g.scal, ctx->hpin, 2 * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return 0;
}

extern "C" int grmhd_init_torus(grmhd_ctx *ctx, const grmhd_torus_params *tp)
{
    if (!ctx || !tp) return fail(ctx, GRMHD_EINVAL, "null argument");
    if (!ctx->metric_set || ctx->g.metric != GRMHD_KERR_MKS)
        return fail(ctx, GRMHD_ESTATE, "init_torus needs grmhd_set_metric(GRMHD_KERR_MKS) first");
    if (!(tp->r_max > tp->r_in) || !(tp->r_in > 0.0)) return fail(ctx, GRMHD_EINVAL, "need 0 < r_in < r_max");
    if (ctx->g.n2t != ctx->g.n2)
        return fail(ctx, GRMHD_EINVAL, "a theta slab takes its state from set_state (the torus is normalised over the whole grid)");
    Grid &g = ctx->g;
    TorusArgs ta{};
    ta.a = ctx->a;
    ta.ell = fm_ell_host(ctx->a, tp->r_max);
    ta.lnh_in = fm_lnh_host(ctx->a, ta.ell, tp->r_in, 0.5 * M_PI);
    ta.r_in = tp->r_in;
    ta.kappa = tp->kappa > 0.0 ? tp->kappa : 1e-3;
    ta.beta0 = tp->beta0;
    ta.pert_amp = tp->pert_amp;
    ta.seed = tp->seed;
    ta.cp = ctx->gb.cp;
    if (reset_counters(ctx)) return GRMHD_ECUDA;
    (void)cudaGetLastError();
    launch_torus(g, ta, ctx->scratch, ctx->intorus, ctx->hpin, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    if (!(ctx->hpin[0] > 0.0)) return fail(ctx, GRMHD_EINVAL, "torus does not intersect the grid");
    ctx->disk_mass = ctx->hpin[4];
    ctx->disk_eb = ctx->hpin[5];
    launch_bc(g, 0, ctx->stream);
    if (copy_stage_buffer(ctx)) return GRMHD_ECUDA;
    if (set_scalars(ctx, 0.0, 0.0)) return GRMHD_ECUDA;
    launch_fluxes_dt(g, 1, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->state_set = true;
    return 0;
}

static int ensure_staging(grmhd_ctx *ctx, long long n)
{
    if (ctx->staging_len >= n) return 0;
    double *p;
    int rc = dalloc(ctx, &p, n);
    if (rc) return rc;
    ctx->staging = p;
    ctx->staging_len = n;
    return 0;
}

// A host <-> device copy of the state's parts (P, U) split into NCOPY nearly
// equal byte ranges on as many streams, so that several copy engines share
// it; forked from the context stream after the work already there and joined
// back before the work that follows.
struct CopyPart {
    char *dst;
    const char *src;
    size_t bytes;
};

static int copy_split(grmhd_ctx *ctx, const CopyPart *parts, int np, cudaMemcpyKind kind)
{
    const int NC = grmhd_ctx::NCOPY;
    if (!ctx->cfork) { // created once, all or nothing
        int dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaSetDevice(ctx->gp.device));
        cudaEvent_t fork = nullptr;
        bool ok = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
        for (int k = 0; k < NC && ok; k++)
            ok = cudaStreamCreateWithFlags(&ctx->cstream[k], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&ctx->cjoin[k], cudaEventDisableTiming) == cudaSuccess;
        cudaSetDevice(dev);
        if (!ok) {
            if (fork) cudaEventDestroy(fork);
            for (int k = 0; k < NC; k++) {
                if (ctx->cstream[k]) cudaStreamDestroy(ctx->cstream[k]);
                if (ctx->cjoin[k]) cudaEventDestroy(ctx->cjoin[k]);
                ctx->cstream[k] = nullptr;
                ctx->cjoin[k] = nullptr;
            }
            return fail(ctx, GRMHD_ECUDA, "copy streams could not be created");
        }
        ctx->cfork = fork;
    }
    size_t total = 0;
    for (int q = 0; q < np; q++) total += parts[q].bytes;
    const size_t align = 1 << 20;
    size_t per = ((total + NC - 1) / NC + align - 1) / align * align;
    CK(cudaEventRecord(ctx->cfork, ctx->stream));
    for (int k = 0; k < NC; k++) CK(cudaStreamWaitEvent(ctx->cstream[k], ctx->cfork, 0));
    int k = 0;
    size_t filled = 0;
    for (int q = 0; q < np; q++) {
        size_t off = 0;
        while (off < parts[q].bytes) {
            size_t take = std::min(parts[q].bytes - off, per - filled);
            CK(cudaMemcpyAsync(parts[q].dst + off, parts[q].src + off, take, kind, ctx->cstream[k]));
            off += take;
            filled += take;
            if (filled == per && k < NC - 1) {
                k++;
                filled = 0;
            }
        }
    }
    for (int j = 0; j < NC; j++) {
        CK(cudaEventRecord(ctx->cjoin[j], ctx->cstream[j]));
        CK(cudaStreamWaitEvent(ctx->stream, ctx->cjoin[j], 0));
    }
    return 0;
}

extern "C" int grmhd_set_state(grmhd_ctx *ctx, const double *P, const double *U, double t, double dt, int on_device)
{
    if (!ctx || !P || !U) return fail(ctx, GRMHD_EINVAL, "null argument");
    if (!ctx->metric_set) return fail(ctx, GRMHD_ESTATE, "set_state needs grmhd_set_metric first");
    long long na = nact_of(ctx);
    const double *Pd = P, *Ud = U;
    if (!on_device) {
        if (ensure_staging(ctx, 17 * na)) return GRMHD_ENOMEM;
        const CopyPart parts[2] = {{(char *)ctx->staging, (const char *)P, 8 * na * sizeof(double)},
                                   {(char *)(ctx->staging + 8 * na), (const char *)U, 9 * na * sizeof(double)}};
        if (int rc = copy_split(ctx, parts, 2, cudaMemcpyHostToDevice)) return rc;
        Pd = ctx->staging;
        Ud = ctx->staging + 8 * na;
    }
    (void)cudaGetLastError();
    ctx->state_set = false;
    // a new state starts with a clear status word (the counters keep running)
    CK(cudaMemsetAsync(ctx->g.status, 0, sizeof(int), ctx->stream));
    launch_copy_state_in(ctx->g, Pd, Ud, ctx->stream);
    launch_bc(ctx->g, 0, ctx->stream);
    CK(cudaGetLastError());
    if (copy_stage_buffer(ctx)) return GRMHD_ECUDA;
    CK(cudaMemcpyAsync(&ctx->hpin[8], ctx->g.status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    if (set_scalars(ctx, t, dt)) return GRMHD_ECUDA; // synchronises the stream
    int st = 0;
    std::memcpy(&st, &ctx->hpin[8], sizeof(int));
    if (st & ST_NONFINITE) {
        CK(cudaMemsetAsync(ctx->g.status, 0, sizeof(int), ctx->stream));
        return fail(ctx, GRMHD_ENONFINITE, "set_state: P or U holds a non-finite value; the context has no state");
    }
    ctx->state_set = true;
    return 0;
}

extern "C" int grmhd_set_state_u(grmhd_ctx *ctx, const double *U, double t, double dt, int on_device)
{
    if (!ctx || !U) return fail(ctx, GRMHD_EINVAL, "null argument");
    if (!ctx->metric_set) return fail(ctx, GRMHD_ESTATE, "set_state_u needs grmhd_set_metric first");
    if (!ctx->state_set)
        return fail(ctx, GRMHD_ESTATE, "set_state_u needs primitives to start from (grmhd_set_state or grmhd_init_torus)");
    if (ctx->gp.n2_total != 0 || ctx->g.bc3 == BC_EXTERNAL)
        return fail(ctx, GRMHD_EINVAL, "set_state_u: whole grids only (a slab's ghosts come from its neighbours)");
    if (!std::isfinite(t) || !std::isfinite(dt) || dt < 0.0)
        return fail(ctx, GRMHD_EINVAL, "set_state_u: t and dt must be finite, dt >= 0");
    long long na = nact_of(ctx);
    const double *Ud = U;
    if (!on_device) {
        if (ensure_staging(ctx, 9 * na)) return GRMHD_ENOMEM;
        const CopyPart part = {(char *)ctx->staging, (const char *)U, 9 * na * sizeof(double)};
        if (int rc = copy_split(ctx, &part, 1, cudaMemcpyHostToDevice)) return rc;
        Ud = ctx->staging;
    }
    (void)cudaGetLastError();
    ctx->state_set = false;
    CK(cudaMemsetAsync(ctx->g.status, 0, sizeof(int), ctx->stream));
    launch_copy_state_in(ctx->g, nullptr, Ud, ctx->stream);
    CK(cudaGetLastError());
    if (set_scalars(ctx, t, dt)) return GRMHD_ECUDA; // synchronises the stream
    CK(cudaMemcpyAsync(&ctx->hpin[8], ctx->g.status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    int st = 0;
    std::memcpy(&st, &ctx->hpin[8], sizeof(int));
    if (st & ST_NONFINITE) {
        CK(cudaMemsetAsync(ctx->g.status, 0, sizeof(int), ctx->stream));
        return fail(ctx, GRMHD_ENONFINITE, "set_state_u: U holds a non-finite value; the context has no state");
    }
    launch_reinvert(ctx->g, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->state_set = true;
    return 0;
}

extern "C" int grmhd_get_state(grmhd_ctx *ctx, double *P, double *U, double *t, double *dt, int on_device)
{
    if (!ctx) return fail(nullptr, GRMHD_EINVAL, "null context");
    if (!ctx->state_set) return fail(ctx, GRMHD_ESTATE, "no state yet");
    long long na = nact_of(ctx);
    (void)cudaGetLastError();
    if (P || U) {
        if (on_device) {
            launch_copy_state_out(ctx->g, P, U, ctx->stream);
        } else {
            if (ensure_staging(ctx, 17 * na)) return GRMHD_ENOMEM;
            launch_copy_state_out(ctx->g, P ? ctx->staging : nullptr, U ? ctx->staging + 8 * na : nullptr, ctx->stream);
            CopyPart parts[2];
            int np = 0;
            if (P) parts[np++] = CopyPart{(char *)P, (const char *)ctx->staging, 8 * na * sizeof(double)};
            if (U) parts[np++] = CopyPart{(char *)U, (const char *)(ctx->staging + 8 * na), 9 * na * sizeof(double)};
            if (int rc = copy_split(ctx, parts, np, cudaMemcpyDeviceToHost)) return rc;
        }
        CK(cudaGetLastError());
    }
    CK(cudaMemcpyAsync(ctx->hpin, ctx->g.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (dt) *dt = ctx->hpin[0];
    if (t) *t = ctx->hpin[1];
    return 0;
}

extern "C" int grmhd_step(grmhd_ctx *ctx, int nsteps)
{
    if (!ctx) return fail(nullptr, GRMHD_EINVAL, "null context");
    if (!ctx->state_set) return fail(ctx, GRMHD_ESTATE, "step needs a state (init_torus or set_state)");
    if (nsteps < 0) return fail(ctx, GRMHD_EINVAL, "nsteps < 0");
    if (ctx->g.bc3 == BC_EXTERNAL)
        return fail(ctx, GRMHD_EINVAL, "a phi slab steps by grmhd_stage with its ghost planes exchanged between stages");
    if (ctx->g.n2t != ctx->g.n2)
        return fail(ctx, GRMHD_EINVAL, "a theta slab steps by the stage parts with its rows exchanged");
    (void)cudaGetLastError();
    if (!ctx->gexec) {
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        launch_step(ctx->g, ctx->stream);
        cudaError_t le = cudaGetLastError();
        cudaGraph_t graph = nullptr;
        cudaError_t ee = cudaStreamEndCapture(ctx->stream, &graph);
        if (le != cudaSuccess || ee != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(ctx, GRMHD_ECUDA, std::string("step capture failed: ") +
                                              cudaGetErrorString(le != cudaSuccess ? le : ee));
        }
        ctx->graph = graph;
        CK(cudaGraphInstantiate(&ctx->gexec, ctx->graph, 0));
    }
    for (int s = 0; s < nsteps; s++) CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
    return 0;
}

extern "C" int grmhd_sync(grmhd_ctx *ctx)
{
    if (!ctx) return fail(nullptr, GRMHD_EINVAL, "null context");
    int st = 0;
    CK(cudaMemcpyAsync(&ctx->hpin[8], ctx->g.status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    std::memcpy(&st, &ctx->hpin[8], sizeof(int));
    if (st & ST_FIXUP) return fail(ctx, GRMHD_EFIXUP, "some failed zones could not be fixed");
    if (st & ST_NONFINITE) return fail(ctx, GRMHD_ENONFINITE, "non-finite state");
    return 0;
}

extern "C" int grmhd_diagnostics(grmhd_ctx *ctx, grmhd_diag *out)
{
    if (!ctx || !out) return fail(ctx, GRMHD_EINVAL, "null argument");
    if (!ctx->state_set) return fail(ctx, GRMHD_ESTATE, "no state yet");
    Grid &g = ctx->g;
    double *dout = ctx->scratch + ctx->scratch_len - 16;
    (void)cudaGetLastError();
    launch_diagnostics(g, ctx->scratch, ctx->scratch_len - 16, dout, ctx->stream);
    CK(cudaGetLastError());
    unsigned long long cnt[C_NCOUNT];
    CK(cudaMemcpyAsync(ctx->hpin, dout, 8 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->hpin + 8, g.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(cnt, g.cnt, sizeof(cnt), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    std::memset(out, 0, sizeof(*out));
    out->mdot = ctx->hpin[0];
    out->phib = ctx->hpin[1];
    out->edot = ctx->hpin[2];
    out->ldot = ctx->hpin[3];
    out->divb_max = ctx->hpin[4];
    out->PhiB = out->mdot != 0.0 ? out->phib / std::sqrt(std::fabs(out->mdot)) : 0.0;
    out->eta = out->mdot != 0.0 ? (out->edot - out->mdot) / std::fabs(out->mdot) : 0.0;
    out->dt = ctx->hpin[8];
    out->t = ctx->hpin[9];
    out->disk_mass = ctx->disk_mass;
    out->disk_eb = ctx->disk_eb;
    out->nr_iters = (long long)cnt[C_NR_ITERS];
    out->n_nr = (long long)cnt[C_NR];
    out->n_brent = (long long)cnt[C_BRENT];
    out->n_entropy = (long long)cnt[C_ENT];
    out->n_entropy_beta = (long long)cnt[C_ENT_BETA];
    out->n_fail = (long long)cnt[C_FAIL];
    out->n_floor = (long long)cnt[C_FLOOR];
    out->n_ceil = (long long)cnt[C_CEIL];
    out->n_gcap = (long long)cnt[C_GCAP];
    out->n_fixed = (long long)cnt[C_FIXED];
    out->fix_sweeps = (long long)cnt[C_SWEEPS];
    out->n_steps = (long long)cnt[C_STEPS];
    out->n_learned = (long long)cnt[C_LEARN];
    return grmhd_sync(ctx);
}

static_assert(GRMHD_DIAG_NPART == DIAG_NPART, "partial-vector length of the header and the kernels differ");

static void diag_from_vector(const grmhd_ctx *ctx, const double *v, grmhd_diag *out)
{
    std::memset(out, 0, sizeof(*out));
    out->mdot = v[0];
    out->phib = v[1];
    out->edot = v[2];
    out->ldot = v[3];
    out->divb_max = v[4];
    out->t = v[7];
    out->dt = v[8];
    out->PhiB = v[22];
    out->eta = v[23];
    out->disk_mass = ctx->disk_mass;
    out->disk_eb = ctx->disk_eb;
    long long *cnt[C_NCOUNT] = {&out->nr_iters, &out->n_nr,    &out->n_brent, &out->n_entropy, &out->n_entropy_beta,
                                &out->n_fail,   &out->n_floor, &out->n_ceil,  &out->n_gcap,    &out->n_fixed,
                                &out->fix_sweeps, &out->n_steps, &out->n_learned};
    for (int c = 0; c < C_NCOUNT; c++) *cnt[c] = (long long)v[9 + c];
}

extern "C" int grmhd_diag_partials(grmhd_ctx *ctx, double r_bar_max, double *out_dev)
{
    if (!ctx || !out_dev) return fail(ctx, GRMHD_EINVAL, "null argument");
    if (!ctx->state_set) return fail(ctx, GRMHD_ESTATE, "no state yet");
    const Grid &g = ctx->g;
    const bool bary = r_bar_max > 0.0 && g.metric == KERR_MKS;
    double *dout = ctx->scratch + ctx->scratch_len - 16;
    double *bpart = ctx->scratch + ctx->scratch_len - 16 - 2LL * g.n1 - 8;
    (void)cudaGetLastError();
    launch_diagnostics(g, ctx->scratch, ctx->scratch_len - 16 - 2LL * g.n1 - 8, dout, ctx->stream);
    if (bary) launch_barycentric(g, ctx->cp, r_bar_max, bpart, dout + 8, ctx->stream);
    launch_diag_pack(g, dout, bary ? dout + 8 : nullptr, out_dev, ctx->stream);
    CK(cudaGetLastError());
    return 0;
}

extern "C" int grmhd_diag_combine(grmhd_ctx *ctx, const double *parts_dev, int nparts, grmhd_diag *out, double *bary3)
{
    if (!ctx || !parts_dev || !out) return fail(ctx, GRMHD_EINVAL, "null argument");
    if (nparts < 1) return fail(ctx, GRMHD_EINVAL, "nparts < 1");
    double *dv = ctx->scratch + ctx->scratch_len - 16 - 2LL * ctx->g.n1 - 8 - DIAG_NPART;
    (void)cudaGetLastError();
    launch_diag_combine(parts_dev, nparts, dv, ctx->stream);
    CK(cudaGetLastError());
    double v[DIAG_NPART];
    CK(cudaMemcpyAsync(ctx->hpin, dv, DIAG_NPART * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    std::memcpy(v, ctx->hpin, sizeof(v));
    diag_from_vector(ctx, v, out);
    if (bary3) {
        bary3[0] = v[24];
        bary3[1] = v[6];
        bary3[2] = v[5];
    }
    return grmhd_sync(ctx);
}

extern "C" int grmhd_prim2cons(grmhd_ctx *ctx, const double *P, const int *loc, double *U, long n, int on_device)
{
    if (!ctx || (n > 0 && (!P || !loc || !U))) return fail(ctx, GRMHD_EINVAL, "null argument");
    if (!ctx->metric_set) return fail(ctx, GRMHD_ESTATE, "needs grmhd_set_metric first");
    if (n < 0) return fail(ctx, GRMHD_EINVAL, "n < 0");
    if (n == 0) return 0;
    const double *Pd = P;
    const int *ld = loc;
    double *Ud = U;
    if (!on_device) {
        long long need = 17LL * n + (n + 1) / 2 + 1;
        if (ensure_staging(ctx, need)) return GRMHD_ENOMEM;
        double *sp = ctx->staging, *su = sp + 8LL * n;
        int *sl = (int *)(su + 9LL * n);
        CK(cudaMemcpyAsync(sp, P, 8LL * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(sl, loc, n * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
        Pd = sp; ld = sl; Ud = su;
    }
    (void)cudaGetLastError();
    launch_prim2cons(ctx->g, Pd, ld, Ud, n, ctx->stream);
    CK(cudaGetLastError());
    if (!on_device) CK(cudaMemcpyAsync(U, Ud, 9LL * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return 0;
}

extern "C" int grmhd_con2prim(grmhd_ctx *ctx, const double *U, const int *loc, double *P, int *flags, int *iters,
                              long n, int use_learned_guess, int on_device)
{
    if (!ctx || (n > 0 && (!P || !loc || !U || !flags))) return fail(ctx, GRMHD_EINVAL, "null argument");
    if (!ctx->metric_set) return fail(ctx, GRMHD_ESTATE, "needs grmhd_set_metric first");
    if (n < 0) return fail(ctx, GRMHD_EINVAL, "n < 0");
    if (n >= INT_MAX) return fail(ctx, GRMHD_EINVAL, "n must be below 2^31 - 1");
    if (use_learned_guess < 0 || use_learned_guess > 2) return fail(ctx, GRMHD_EINVAL, "use_learned_guess must be 0, 1 or 2");
    if (use_learned_guess && !ctx->mlp_loaded) return fail(ctx, GRMHD_ESTATE, "no MLP loaded");
    if (n == 0) return 0;
    const double *Ud = U;
    const int *ld = loc;
    double *Pd = P;
    int *fd = flags, *id = iters;
    if (!on_device) {
        long long need = 17LL * n + 3 * ((n + 1) / 2) + 3;
        if (ensure_staging(ctx, need)) return GRMHD_ENOMEM;
        double *su = ctx->staging, *sp = su + 9LL * n;
        int *sl = (int *)(sp + 8LL * n);
        int *sf = sl + n, *si = sf + n;
        CK(cudaMemcpyAsync(su, U, 9LL * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(sp, P, 8LL * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(sl, loc, n * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
        Ud = su; Pd = sp; ld = sl; fd = sf; id = iters ? si : nullptr;
    }
    if (ctx->c2p_list_len < n + 1) {
        int *p;
        if (int rc = dalloc(ctx, &p, (size_t)n + 1)) return rc;
        ctx->c2p_list = p;
        ctx->c2p_list_len = n + 1;
    }
    (void)cudaGetLastError();
    launch_con2prim(ctx->g, Ud, ld, Pd, fd, id, n, use_learned_guess ? ctx->mlp : nullptr, use_learned_guess,
                    ctx->c2p_list, ctx->stream);
    CK(cudaGetLastError());
    if (!on_device) {
        CK(cudaMemcpyAsync(P, Pd, 8LL * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(flags, fd, n * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        if (iters) CK(cudaMemcpyAsync(iters, id, n * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return 0;
}

extern "C" int grmhd_fluxes(grmhd_ctx *ctx, double *out, double *dt_out, int on_device)
{
    if (!ctx || !out) return fail(ctx, GRMHD_EINVAL, "null argument");
    if (!ctx->state_set) return fail(ctx, GRMHD_ESTATE, "no state yet");
    Grid &g = ctx->g;
    long long nf = 3LL * NU * (g.n1 + 1) * (g.n2 + 1) * (g.n3 + 1);
    double *o = out;
    if (!on_device) {
        if (ensure_staging(ctx, nf)) return GRMHD_ENOMEM;
        o = ctx->staging;
    }
    // keep the state's dt: save it, sweep, read the sweep's dt, restore
    CK(cudaMemcpyAsync(ctx->hpin + 16, g.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    (void)cudaGetLastError();
    launch_fluxes_dt(g, 1, ctx->stream);
    launch_gather_fluxes(g, o, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ctx->hpin + 20, g.scal, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (dt_out) *dt_out = ctx->hpin[20];
    CK(cudaMemcpyAsync(g.scal, ctx->hpin + 16, 2 * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    if (!on_device) CK(cudaMemcpyAsync(out, o, nf * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return 0;
}

extern "C" int grmhd_step_profiled(grmhd_ctx *ctx, int nsteps, double *ms_out)
{
    if (!ctx || !ms_out) return fail(ctx, GRMHD_EINVAL, "null argument");
    if (!ctx->state_set) return fail(ctx, GRMHD_ESTATE, "step needs a state (init_torus or set_state)");
    const int NE = 16;
    cudaEvent_t ev[NE];
    for (int e = 0; e < NE; e++) CK(cudaEventCreate(&ev[e]));
    for (int p = 0; p < GRMHD_PROF_SLOTS; p++) ms_out[p] = 0.0;
    (void)cudaGetLastError();
    for (int s = 0; s < nsteps; s++) {
        launch_step_profiled(ctx->g, ctx->stream, ev);
        CK(cudaGetLastError());
        CK(cudaEventSynchronize(ev[NE - 1]));
        for (int st = 0; st < 2; st++)
            for (int part = 0; part < 7; part++) {
                float ms;
                int e = st * 7 + part;
                CK(cudaEventElapsedTime(&ms, ev[e], ev[e + 1]));
                ms_out[st * 7 + part] += ms;
            }
        float ms;
        CK(cudaEventElapsedTime(&ms, ev[14], ev[15]));
        ms_out[14] += ms;
        CK(cudaEventElapsedTime(&ms, ev[0], ev[15]));
        ms_out[15] += ms;
    }
    for (int e = 0; e < NE; e++) cudaEventDestroy(ev[e]);
    return 0;
}

extern "C" int grmhd_peak_probe(int device, int fp64, double *tflops)
{
    grmhd_ctx *ctx = nullptr;
    if (!tflops) return fail(nullptr, GRMHD_EINVAL, "null argument");
    CK(cudaSetDevice(device));
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    cudaStream_t s;
    CK(cudaStreamCreate(&s));
    *tflops = launch_fma_probe(fp64, sms, s);
    cudaError_t e = cudaGetLastError();
    cudaStreamDestroy(s);
    if (e != cudaSuccess) return fail(nullptr, GRMHD_ECUDA, cudaGetErrorString(e));
    return 0;
}

// ---------------------------------------------------------------------------
// Horizon diagnostics with no device allocation at all.
//
// grmhd_diagnostics reduces the horizon sums through per-block partial sums
// kept in the context's scratch buffer.  This variant runs the same kernels
// but keeps those partial sums in the file-scope array below, which the CUDA
// runtime reserves on every device that loads the library, once, for the
// life of the process.  Nothing in it needs to start at zero: every call
// writes all the partial sums it later reads.  Every call on a device shares
// the array, so two calls whose kernels overlap on the GPU (for instance two
// contexts on different streams) race on it.
static constexpr int NOALLOC_MAX_BLOCKS = 8192; // horizon shells up to 8192 * 256 (theta, phi) zones
static constexpr long long NOALLOC_DOUBLES = 4LL * NOALLOC_MAX_BLOCKS; // 256 KiB
static __device__ __align__(256) double g_noalloc_partials[NOALLOC_DOUBLES];

static constexpr int NOALLOC_MAX_DEVICES = 64;
static double *g_noalloc_addr[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mu;

// Device address of g_noalloc_partials on device dev, looked up once per
// device with that device current (host code may not use the symbol itself).
static int noalloc_partials(grmhd_ctx *ctx, int dev, double **out)
{
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        int prev = 0;
        CK(cudaGetDevice(&prev));
        CK(cudaSetDevice(dev));
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        cudaError_t e2 = cudaSetDevice(prev);
        if (e != cudaSuccess)
            return fail(ctx, GRMHD_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        CK(e2);
        g_noalloc_addr[dev] = (double *)p;
    }
    *out = g_noalloc_addr[dev];
    return 0;
}

extern "C" int grmhd_diagnostics_noalloc(grmhd_ctx *ctx, double *out_dev)
{
    if (!ctx || !out_dev) return fail(ctx, GRMHD_EINVAL, "null argument");
    if (!ctx->state_set) return fail(ctx, GRMHD_ESTATE, "no state yet");
    const Grid &g = ctx->g;
    long long shell = (long long)g.n2 * g.n3;
    long long blocks = (shell + 255) / 256;
    if (blocks > NOALLOC_MAX_BLOCKS)
        return fail(ctx, GRMHD_EINVAL,
                    "grmhd_diagnostics_noalloc: horizon shell of n2*n3 = " + std::to_string(shell) +
                        " zones exceeds its maximum of " + std::to_string(256LL * NOALLOC_MAX_BLOCKS) +
                        " zones; use grmhd_diagnostics");
    int dev = ctx->gp.device;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(ctx, GRMHD_EINVAL, "device ordinal out of range");
    double *partials = nullptr;
    int rc = noalloc_partials(ctx, dev, &partials);
    if (rc) return rc;
    (void)cudaGetLastError(); // an earlier asynchronous error is not this call's failure
    launch_diagnostics(g, partials, NOALLOC_DOUBLES, out_dev, ctx->stream);
    CK(cudaGetLastError());
    return 0;
}

// ---------------------------------------------------------------- learned start

static_assert(GRMHD_MLP_NPARAM == MLP_NPARAM, "parameter count of the header and the kernels differ");

namespace {

// device buffers of one call, freed when the call returns
struct DevTmp {
    std::vector<void *> p;
    bool bad = false;
    ~DevTmp()
    {
        for (void *q : p) cudaFree(q);
    }
    template <typename T>
    T *get(size_t count)
    {
        void *q = nullptr;
        if (cudaMalloc(&q, count * sizeof(T) > 16 ? count * sizeof(T) : 16) != cudaSuccess) {
            bad = true;
            return nullptr;
        }
        p.push_back(q);
        return (T *)q;
    }
};

int make_trainer(grmhd_ctx *ctx, DevTmp &tmp, int batch, long long hist, MlpTrainer &T)
{
    int nb = mlp_grad_blocks(batch);
    T.theta = tmp.get<float>(MLP_NPARAM);
    T.m = tmp.get<float>(MLP_NPARAM);
    T.v = tmp.get<float>(MLP_NPARAM);
    T.fwd = tmp.get<float>(MLP_FLOATS);
    T.part = tmp.get<float>((size_t)nb * MLP_NPARAM);
    T.lpart = tmp.get<double>(nb);
    T.step = tmp.get<long long>(1);
    T.ticket = tmp.get<unsigned int>(1);
    T.loss_hist = tmp.get<double>(hist);
    T.hist_len = hist;
    if (tmp.bad) return fail(ctx, GRMHD_ENOMEM, "cudaMalloc of the training buffers failed");
    CK(cudaMemsetAsync(T.m, 0, MLP_NPARAM * sizeof(float), ctx->stream));
    CK(cudaMemsetAsync(T.v, 0, MLP_NPARAM * sizeof(float), ctx->stream));
    CK(cudaMemsetAsync(T.fwd, 0, MLP_FLOATS * sizeof(float), ctx->stream));
    CK(cudaMemsetAsync(T.step, 0, sizeof(long long), ctx->stream));
    CK(cudaMemsetAsync(T.ticket, 0, sizeof(unsigned int), ctx->stream));
    CK(cudaMemsetAsync(T.loss_hist, 0, hist * sizeof(double), ctx->stream));
    CK(mlp_grad_setup());
    return 0;
}

int check_norm(grmhd_ctx *ctx, const float *norm)
{
    for (int k = 0; k < GRMHD_MLP_NNORM; k++)
        if (!std::isfinite(norm[k])) return fail(ctx, GRMHD_EINVAL, "norm has a non-finite entry");
    for (int k = 5; k < 10; k++)
        if (!(norm[k] > 0.0f)) return fail(ctx, GRMHD_EINVAL, "feature std must be positive");
    if (!(norm[11] > 0.0f)) return fail(ctx, GRMHD_EINVAL, "output std must be positive");
    return 0;
}

// the trainer's forward view of host parameters theta and norm
int trainer_load(grmhd_ctx *ctx, const MlpTrainer &T, const float *theta, const float *norm)
{
    CK(cudaMemcpyAsync(T.theta, theta, MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(T.fwd, norm, GRMHD_MLP_NNORM * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    (void)cudaGetLastError();
    launch_mlp_pack(T.theta, T.fwd, ctx->stream);
    CK(cudaGetLastError());
    return 0;
}

int ensure_mlp_bufs(grmhd_ctx *ctx)
{
    if (!ctx->mlp) {
        int rc = dalloc(ctx, &ctx->mlp, MLP_FLOATS);
        if (rc) return rc;
    }
    if (!ctx->mlp_theta) {
        int rc = dalloc(ctx, &ctx->mlp_theta, MLP_NPARAM);
        if (rc) return rc;
    }
    return 0;
}

// device copies of host inputs (or the caller's device pointers)
template <typename T>
const T *dev_in(grmhd_ctx *ctx, DevTmp &tmp, const T *p, size_t count, int on_device)
{
    if (on_device || !p) return p;
    T *d = tmp.get<T>(count);
    if (!d) return nullptr;
    if (cudaMemcpyAsync(d, p, count * sizeof(T), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) {
        tmp.bad = true;
        return nullptr;
    }
    return d;
}

} // namespace

extern "C" int grmhd_mlp_load(grmhd_ctx *ctx, const float *theta, const float *norm)
{
    if (!ctx || !theta || !norm) return fail(ctx, GRMHD_EINVAL, "null argument");
    for (int k = 0; k < MLP_NPARAM; k++)
        if (!std::isfinite(theta[k])) return fail(ctx, GRMHD_EINVAL, "theta has a non-finite entry");
    if (int rc = check_norm(ctx, norm)) return rc;
    if (int rc = ensure_mlp_bufs(ctx)) return rc;
    CK(cudaMemcpyAsync(ctx->mlp_theta, theta, MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->mlp, norm, GRMHD_MLP_NNORM * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    (void)cudaGetLastError();
    launch_mlp_pack(ctx->mlp_theta, ctx->mlp, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->mlp_loaded = true;
    return 0;
}

extern "C" int grmhd_mlp_get(grmhd_ctx *ctx, float *theta, float *norm)
{
    if (!ctx || (!theta && !norm)) return fail(ctx, GRMHD_EINVAL, "null argument");
    if (!ctx->mlp_loaded) return fail(ctx, GRMHD_ESTATE, "no MLP loaded");
    if (theta)
        CK(cudaMemcpyAsync(theta, ctx->mlp_theta, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    if (norm)
        CK(cudaMemcpyAsync(norm, ctx->mlp, GRMHD_MLP_NNORM * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return 0;
}

extern "C" int grmhd_mlp_samples(grmhd_ctx *ctx, unsigned long long seed, long first, long n, double *P, int *loc,
                                 double *U, float *feat, float *label, int on_device)
{
    if (!ctx) return fail(ctx, GRMHD_EINVAL, "null argument");
    if (!ctx->metric_set) return fail(ctx, GRMHD_ESTATE, "needs grmhd_set_metric first");
    if (n < 0 || first < 0) return fail(ctx, GRMHD_EINVAL, "first and n must be >= 0");
    if (n == 0) return 0;
    DevTmp tmp;
    double *Pd = P, *Ud = U;
    int *ld = loc;
    float *fd = feat, *yd = label;
    if (!on_device) {
        if (P) Pd = tmp.get<double>((size_t)NP * n);
        if (U) Ud = tmp.get<double>((size_t)NU * n);
        if (loc) ld = tmp.get<int>(n);
        if (feat) fd = tmp.get<float>((size_t)MLP_IN * n);
        if (label) yd = tmp.get<float>(n);
        if (tmp.bad) return fail(ctx, GRMHD_ENOMEM, "cudaMalloc of the sample buffers failed");
    }
    (void)cudaGetLastError();
    launch_mlp_samples(ctx->g, seed, first, n, Pd, ld, Ud, fd, yd, ctx->stream);
    CK(cudaGetLastError());
    if (!on_device) {
        if (P) CK(cudaMemcpyAsync(P, Pd, (size_t)NP * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        if (U) CK(cudaMemcpyAsync(U, Ud, (size_t)NU * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        if (loc) CK(cudaMemcpyAsync(loc, ld, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        if (feat)
            CK(cudaMemcpyAsync(feat, fd, (size_t)MLP_IN * n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        if (label) CK(cudaMemcpyAsync(label, yd, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return 0;
}

extern "C" int grmhd_mlp_forward(grmhd_ctx *ctx, const float *feat, long n, float *y, int on_device)
{
    if (!ctx || (n > 0 && (!feat || !y))) return fail(ctx, GRMHD_EINVAL, "null argument");
    if (!ctx->mlp_loaded) return fail(ctx, GRMHD_ESTATE, "no MLP loaded");
    if (n < 0) return fail(ctx, GRMHD_EINVAL, "n < 0");
    if (n == 0) return 0;
    DevTmp tmp;
    const float *fd = dev_in(ctx, tmp, feat, (size_t)MLP_IN * n, on_device);
    float *yd = on_device ? y : tmp.get<float>(n);
    if (tmp.bad) return fail(ctx, GRMHD_ENOMEM, "cudaMalloc or copy of the forward buffers failed");
    (void)cudaGetLastError();
    launch_mlp_forward(ctx->mlp, fd, n, yd, ctx->stream);
    CK(cudaGetLastError());
    if (!on_device) CK(cudaMemcpyAsync(y, yd, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return 0;
}

static const long MLP_MAX_BATCH = 1L << 18;

extern "C" int grmhd_mlp_loss_grad(grmhd_ctx *ctx, const float *theta, const float *norm, const float *feat,
                                   const float *label, long n, float *grad, double *loss, int on_device)
{
    if (!ctx || !theta || !norm || !feat || !label || !grad) return fail(ctx, GRMHD_EINVAL, "null argument");
    if (n < 1 || n > MLP_MAX_BATCH) return fail(ctx, GRMHD_EINVAL, "n must be in [1, 262144]");
    if (int rc = check_norm(ctx, norm)) return rc;
    DevTmp tmp;
    MlpTrainer T{};
    if (int rc = make_trainer(ctx, tmp, (int)n, 1, T)) return rc;
    if (int rc = trainer_load(ctx, T, theta, norm)) return rc;
    const float *fd = dev_in(ctx, tmp, feat, (size_t)MLP_IN * n, on_device);
    const float *ld = dev_in(ctx, tmp, label, (size_t)n, on_device);
    float *gd = on_device ? grad : tmp.get<float>(MLP_NPARAM);
    if (tmp.bad) return fail(ctx, GRMHD_ENOMEM, "cudaMalloc or copy of the gradient buffers failed");
    (void)cudaGetLastError();
    launch_mlp_grad(T, fd, ld, n, (int)n, 1ull, ctx->stream);
    launch_mlp_reduce_grad(T, (int)n, gd, ctx->stream);
    CK(cudaGetLastError());
    if (!on_device) CK(cudaMemcpyAsync(grad, gd, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    int nb = mlp_grad_blocks((int)n);
    std::vector<double> lp(nb);
    CK(cudaMemcpyAsync(lp.data(), T.lpart, nb * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (loss) {
        double l = 0.0;
        for (double v : lp) l += v;
        *loss = l / (double)n;
    }
    return 0;
}

extern "C" int grmhd_mlp_train_steps(grmhd_ctx *ctx, float *theta, const float *norm, const float *feat,
                                     const float *label, long n, long batch, long nsteps, double lr, double beta1,
                                     double beta2, double eps, double wd, double *loss_last, int on_device)
{
    if (!ctx || !theta || !norm || !feat || !label) return fail(ctx, GRMHD_EINVAL, "null argument");
    if (n < 1 || batch < 1 || batch > MLP_MAX_BATCH || nsteps < 1)
        return fail(ctx, GRMHD_EINVAL, "need n >= 1, 1 <= batch <= 262144, nsteps >= 1");
    if (!(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
        return fail(ctx, GRMHD_EINVAL, "bad optimiser parameters");
    if (int rc = check_norm(ctx, norm)) return rc;
    DevTmp tmp;
    MlpTrainer T{};
    if (int rc = make_trainer(ctx, tmp, (int)batch, nsteps, T)) return rc;
    if (int rc = trainer_load(ctx, T, theta, norm)) return rc;
    const float *fd = dev_in(ctx, tmp, feat, (size_t)MLP_IN * n, on_device);
    const float *ld = dev_in(ctx, tmp, label, (size_t)n, on_device);
    if (tmp.bad) return fail(ctx, GRMHD_ENOMEM, "cudaMalloc or copy of the training data failed");
    MlpHyper h{lr, lr, beta1, beta2, eps, wd, 0};
    (void)cudaGetLastError();
    for (long s = 0; s < nsteps; s++) {
        launch_mlp_grad(T, fd, ld, n, (int)batch, 1ull, ctx->stream);
        launch_mlp_adam(T, (int)batch, h, ctx->stream);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(theta, T.theta, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    double ll = 0.0;
    CK(cudaMemcpyAsync(&ll, T.loss_hist + (nsteps - 1), sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (loss_last) *loss_last = ll;
    return 0;
}

static unsigned long long coprime_multiplier(long long n)
{
    unsigned long long c = ((unsigned long long)(0.6180339887498949 * (double)n)) | 1ull;
    while (std::gcd(c, (unsigned long long)n) != 1ull) c += 2;
    return c;
}

extern "C" int grmhd_mlp_train(grmhd_ctx *ctx, const grmhd_mlp_train_params *tp, grmhd_mlp_train_report *rep)
{
    if (!ctx || !tp) return fail(ctx, GRMHD_EINVAL, "null argument");
    if (!ctx->metric_set) return fail(ctx, GRMHD_ESTATE, "needs grmhd_set_metric first");
    const long long N = tp->n_samples, V = tp->n_val;
    if (N < 1 || N > (1LL << 31) - 1 || V < 0 || tp->epochs < 1 || tp->batch < 1 || tp->batch > MLP_MAX_BATCH)
        return fail(ctx, GRMHD_EINVAL, "need 1 <= n_samples < 2^31, n_val >= 0, epochs >= 1, 1 <= batch <= 262144");
    if (!(tp->lr >= 0.0) || !(tp->lr_min >= 0.0) || !(tp->beta1 >= 0.0 && tp->beta1 < 1.0) ||
        !(tp->beta2 >= 0.0 && tp->beta2 < 1.0) || !(tp->eps > 0.0))
        return fail(ctx, GRMHD_EINVAL, "bad optimiser parameters");
    const long long steps = ((long long)tp->epochs * N + tp->batch - 1) / tp->batch;
    DevTmp tmp;
    float *feat = tmp.get<float>((size_t)MLP_IN * N), *lab = tmp.get<float>((size_t)N);
    float *vfeat = tmp.get<float>((size_t)MLP_IN * (V > 0 ? V : 1)), *vlab = tmp.get<float>((size_t)(V > 0 ? V : 1));
    const int mblk = 1024;
    double *mpart = tmp.get<double>((size_t)12 * mblk);
    const int nbv = V > 0 ? mlp_eval_blocks(V) : 1;
    double *vpart = tmp.get<double>((size_t)2 * nbv);
    if (tmp.bad) return fail(ctx, GRMHD_ENOMEM, "cudaMalloc of the training set failed");
    (void)cudaGetLastError();
    launch_mlp_samples(ctx->g, tp->seed, 0, N, nullptr, nullptr, nullptr, feat, lab, ctx->stream);
    if (V > 0) launch_mlp_samples(ctx->g, tp->seed, N, V, nullptr, nullptr, nullptr, vfeat, vlab, ctx->stream);
    launch_mlp_moments(feat, lab, N, mpart, mblk, ctx->stream);
    CK(cudaGetLastError());
    std::vector<double> mp((size_t)12 * mblk);
    CK(cudaMemcpyAsync(mp.data(), mpart, mp.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    float norm[GRMHD_MLP_NNORM];
    for (int c = 0; c < 6; c++) {
        double s1 = 0.0, s2 = 0.0;
        for (int b = 0; b < mblk; b++) {
            s1 += mp[(size_t)b * 12 + 2 * c];
            s2 += mp[(size_t)b * 12 + 2 * c + 1];
        }
        double mean = s1 / (double)N, var = s2 / (double)N - mean * mean;
        double sd = var > 1e-24 ? std::sqrt(var) : 1.0;
        if (c < 5) {
            norm[c] = (float)mean;
            norm[5 + c] = (float)sd;
        } else {
            norm[10] = (float)mean;
            norm[11] = (float)sd;
        }
    }
    MlpTrainer T{};
    if (int rc = make_trainer(ctx, tmp, tp->batch, steps, T)) return rc;
    (void)cudaGetLastError();
    launch_mlp_init(T.theta, tp->init_seed, ctx->stream);
    CK(cudaMemcpyAsync(T.fwd, norm, sizeof(norm), cudaMemcpyHostToDevice, ctx->stream));
    launch_mlp_pack(T.theta, T.fwd, ctx->stream);
    CK(cudaGetLastError());
    const unsigned long long mul = coprime_multiplier(N);
    MlpHyper h{tp->lr, tp->lr_min, tp->beta1, tp->beta2, tp->eps, tp->weight_decay, steps};

    // the steps as CUDA graphs of up to 32 steps each
    const long long chunk = steps < 32 ? steps : 32;
    cudaGraph_t gr[2] = {nullptr, nullptr};
    cudaGraphExec_t ge[2] = {nullptr, nullptr};
    long long lens[2] = {chunk, steps % chunk};
    int err = 0;
    for (int q = 0; q < 2 && !err; q++) {
        if (lens[q] == 0) continue;
        if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            err = 1;
            break;
        }
        for (long long s = 0; s < lens[q]; s++) {
            launch_mlp_grad(T, feat, lab, N, tp->batch, mul, ctx->stream);
            launch_mlp_adam(T, tp->batch, h, ctx->stream);
        }
        if (cudaStreamEndCapture(ctx->stream, &gr[q]) != cudaSuccess ||
            cudaGraphInstantiate(&ge[q], gr[q], 0) != cudaSuccess)
            err = 1;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.0f;
    if (!err && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        cudaEventRecord(e0, ctx->stream);
        for (long long r = 0; r < steps / chunk; r++) cudaGraphLaunch(ge[0], ctx->stream);
        if (ge[1]) cudaGraphLaunch(ge[1], ctx->stream);
        cudaEventRecord(e1, ctx->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) err = 1;
    } else {
        err = 1;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (int q = 0; q < 2; q++) {
        if (ge[q]) cudaGraphExecDestroy(ge[q]);
        if (gr[q]) cudaGraphDestroy(gr[q]);
    }
    if (err) {
        cudaError_t e = cudaGetLastError();
        return fail(ctx, GRMHD_ECUDA, std::string("training graph failed: ") + cudaGetErrorString(e));
    }

    double vr = 0.0, vm = 0.0;
    if (V > 0) {
        launch_mlp_eval(T.fwd, vfeat, vlab, V, vpart, ctx->stream);
        CK(cudaGetLastError());
        std::vector<double> ev((size_t)2 * nbv);
        CK(cudaMemcpyAsync(ev.data(), vpart, ev.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        double se = 0.0;
        for (int b = 0; b < nbv; b++) {
            se += ev[2 * b];
            vm = std::max(vm, ev[2 * b + 1]);
        }
        vr = std::sqrt(se / (double)V);
    }
    double lf = 0.0, ll = 0.0;
    CK(cudaMemcpyAsync(&lf, T.loss_hist, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(&ll, T.loss_hist + (steps - 1), sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (int rc = ensure_mlp_bufs(ctx)) return rc;
    CK(cudaMemcpyAsync(ctx->mlp, T.fwd, MLP_FLOATS * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->mlp_theta, T.theta, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->mlp_loaded = true;
    if (rep) {
        rep->loss_first = lf;
        rep->loss_last = ll;
        rep->val_rmse = vr;
        rep->val_maxerr = vm;
        rep->train_ms = ms;
        rep->samples_per_s = ms > 0.0f ? (double)steps * tp->batch / (ms * 1e-3) : 0.0;
        rep->steps = (long)steps;
    }
    return 0;
}

extern "C" int grmhd_set_learned_guess(grmhd_ctx *ctx, int on)
{
    if (!ctx) return fail(nullptr, GRMHD_EINVAL, "null context");
    if (on && !ctx->mlp_loaded) return fail(ctx, GRMHD_ESTATE, "no MLP loaded");
    const float *want = on ? ctx->mlp : nullptr;
    if (ctx->g.mlp == want) return 0;
    // the captured step holds the grid record by value: capture again
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    ctx->gexec = nullptr;
    ctx->graph = nullptr;
    ctx->g.mlp = want;
    return 0;
}

// ------------------------------------------------------------- phi slabs

extern "C" int grmhd_stage(grmhd_ctx *ctx, int st)
{
    if (!ctx) return fail(nullptr, GRMHD_EINVAL, "null context");
    if (!ctx->state_set) return fail(ctx, GRMHD_ESTATE, "stage needs a state (init_torus or set_state)");
    if (st != 0 && st != 1) return fail(ctx, GRMHD_EINVAL, "st must be 0 or 1");
    if (ctx->g.n2t != ctx->g.n2)
        return fail(ctx, GRMHD_EINVAL, "a theta slab steps by the stage parts (its fixups exchange rows)");
    (void)cudaGetLastError();
    launch_stage(ctx->g, st, ctx->stream);
    CK(cudaGetLastError());
    return 0;
}

extern "C" int grmhd_step_dtd(grmhd_ctx *ctx, double *dtd_dev, int accumulate)
{
    if (!ctx || !dtd_dev) return fail(ctx, GRMHD_EINVAL, "null argument");
    (void)cudaGetLastError();
    launch_step_dtd(ctx->g, dtd_dev, accumulate != 0, ctx->stream);
    CK(cudaGetLastError());
    return 0;
}

extern "C" int grmhd_finish_step(grmhd_ctx *ctx, const double *dtd_dev)
{
    if (!ctx || !dtd_dev) return fail(ctx, GRMHD_EINVAL, "null argument");
    (void)cudaGetLastError();
    launch_finish_step(ctx->g, dtd_dev, ctx->stream);
    CK(cudaGetLastError());
    return 0;
}

extern "C" int grmhd_x3_plane_bytes(grmhd_ctx *ctx, unsigned long long *bytes)
{
    if (!ctx || !bytes) return fail(ctx, GRMHD_EINVAL, "null argument");
    *bytes = (unsigned long long)x3_plane_elems(ctx->g) * (ctx->g.mixed ? sizeof(float) : sizeof(double));
    return 0;
}

static int x3_planes(grmhd_ctx *ctx, int which, int side, void *buf, int unpack)
{
    if (!ctx || !buf) return fail(ctx, GRMHD_EINVAL, "null argument");
    if ((which != 0 && which != 1) || (side != 0 && side != 1))
        return fail(ctx, GRMHD_EINVAL, "which and side must be 0 or 1");
    if (ctx->g.n3 < NG) return fail(ctx, GRMHD_EINVAL, "a slab needs n3 >= 2");
    (void)cudaGetLastError();
    launch_x3_planes(ctx->g, which, side, buf, unpack, ctx->stream);
    CK(cudaGetLastError());
    return 0;
}

extern "C" int grmhd_x3_pack(grmhd_ctx *ctx, int which, int side, void *buf_dev)
{
    return x3_planes(ctx, which, side, buf_dev, 0);
}

extern "C" int grmhd_x3_unpack(grmhd_ctx *ctx, int which, int side, const void *buf_dev)
{
    return x3_planes(ctx, which, side, const_cast<void *>(buf_dev), 1);
}

// ----------------------------------------------------------- theta slabs

static int theta_check(grmhd_ctx *ctx, int st)
{
    if (!ctx) return fail(nullptr, GRMHD_EINVAL, "null context");
    if (!ctx->state_set) return fail(ctx, GRMHD_ESTATE, "a stage needs a state (set_state)");
    if (st != 0 && st != 1) return fail(ctx, GRMHD_EINVAL, "st must be 0 or 1");
    if (ctx->g.n2t == ctx->g.n2) return fail(ctx, GRMHD_EINVAL, "not a theta slab (n2_total)");
    (void)cudaGetLastError();
    return 0;
}

extern "C" int grmhd_stage_update(grmhd_ctx *ctx, int st)
{
    if (int rc = theta_check(ctx, st)) return rc;
    launch_stage_update(ctx->g, st, ctx->stream);
    CK(cudaGetLastError());
    return 0;
}

extern "C" int grmhd_fail_count(grmhd_ctx *ctx, long long *acc_dev)
{
    if (int rc = theta_check(ctx, 0)) return rc;
    if (!acc_dev) return fail(ctx, GRMHD_EINVAL, "null argument");
    launch_fail_count(ctx->g, acc_dev, ctx->stream);
    CK(cudaGetLastError());
    return 0;
}

extern "C" int grmhd_fix_sweep(grmhd_ctx *ctx, int st, long long *acc_dev)
{
    if (int rc = theta_check(ctx, st)) return rc;
    if (!acc_dev) return fail(ctx, GRMHD_EINVAL, "null argument");
    launch_fix_sweep(ctx->g, st, acc_dev, ctx->stream);
    CK(cudaGetLastError());
    return 0;
}

extern "C" int grmhd_fix_end(grmhd_ctx *ctx, int st, int nsweeps)
{
    if (int rc = theta_check(ctx, st)) return rc;
    if (nsweeps < 0) return fail(ctx, GRMHD_EINVAL, "nsweeps < 0");
    launch_fix_end(ctx->g, nsweeps, ctx->stream);
    CK(cudaGetLastError());
    return 0;
}

extern "C" int grmhd_theta_ring_fix(grmhd_ctx *const *ctxs, int nslab, int st, int *nsweeps_dev)
{
    if (!ctxs || !ctxs[0]) return fail(nullptr, GRMHD_EINVAL, "null argument");
    grmhd_ctx *c0 = ctxs[0];
    if (nslab < 1 || nslab > RING_MAX) return fail(c0, GRMHD_EINVAL, "a ring holds 1 to 16 theta slabs");
    Grid gs[RING_MAX];
    for (int r = 0; r < nslab; r++) {
        grmhd_ctx *c = ctxs[r];
        if (!c) return fail(c0, GRMHD_EINVAL, "null slab " + std::to_string(r));
        if (int rc = theta_check(c, st)) return fail(c0, rc, "slab " + std::to_string(r) + ": " + c->err);
        const int j0 = r == 0 ? 0 : ctxs[r - 1]->g.j0 + ctxs[r - 1]->g.n2;
        if (c->g.j0 != j0 || c->g.n2t != c0->g.n2t || c->g.n1 != c0->g.n1 || c->g.n3 != c0->g.n3 ||
            c->g.mixed != c0->g.mixed || c->g.metric != c0->g.metric || c->g.bc2 != c0->g.bc2 ||
            c->g.fix_maxsweep != c0->g.fix_maxsweep || c->gp.device != c0->gp.device ||
            c->stream != c0->stream)
            return fail(c0, GRMHD_EINVAL, "slab " + std::to_string(r) +
                                              ": the slabs of a ring split one grid in theta order, on one device "
                                              "and one stream");
        gs[r] = c->g;
    }
    if (ctxs[nslab - 1]->g.j0 + ctxs[nslab - 1]->g.n2 != c0->g.n2t)
        return fail(c0, GRMHD_EINVAL, "the slabs of a ring cover every row of the grid");
    grmhd_ctx *ctx = c0;
    launch_fix_ring(gs, nslab, st, nsweeps_dev, ctx->stream);
    CK(cudaGetLastError());
    return 0;
}

extern "C" int grmhd_stage_bc(grmhd_ctx *ctx, int st)
{
    if (int rc = theta_check(ctx, st)) return rc;
    launch_bc(ctx->g, st == 0 ? 1 : 0, ctx->stream);
    CK(cudaGetLastError());
    return 0;
}

extern "C" int grmhd_x2_row_bytes(grmhd_ctx *ctx, int kind, unsigned long long *bytes)
{
    if (!ctx || !bytes) return fail(ctx, GRMHD_EINVAL, "null argument");
    if (kind != 0 && kind != 1) return fail(ctx, GRMHD_EINVAL, "kind must be 0 or 1");
    *bytes = (unsigned long long)x2_row_elems(ctx->g, kind) * (ctx->g.mixed ? sizeof(float) : sizeof(double));
    return 0;
}

static int x2_rows(grmhd_ctx *ctx, int kind, int which, int side, void *buf, int unpack)
{
    if (!ctx || !buf) return fail(ctx, GRMHD_EINVAL, "null argument");
    if ((kind != 0 && kind != 1) || (which != 0 && which != 1) || (side != 0 && side != 1))
        return fail(ctx, GRMHD_EINVAL, "kind, which and side must be 0 or 1");
    if (ctx->g.n2t == ctx->g.n2) return fail(ctx, GRMHD_EINVAL, "not a theta slab (n2_total)");
    (void)cudaGetLastError();
    launch_x2_rows(ctx->g, kind, which, side, buf, unpack, ctx->stream);
    CK(cudaGetLastError());
    return 0;
}

extern "C" int grmhd_x2_pack(grmhd_ctx *ctx, int kind, int which, int side, void *buf_dev)
{
    return x2_rows(ctx, kind, which, side, buf_dev, 0);
}

extern "C" int grmhd_x2_unpack(grmhd_ctx *ctx, int kind, int which, int side, const void *buf_dev)
{
    return x2_rows(ctx, kind, which, side, const_cast<void *>(buf_dev), 1);
}

// ------------------------------------------------------ disk diagnostics

extern "C" int grmhd_barycentric_radius(grmhd_ctx *ctx, double r_bar_max, double *out)
{
    if (!ctx || !out) return fail(ctx, GRMHD_EINVAL, "null argument");
    if (!ctx->state_set) return fail(ctx, GRMHD_ESTATE, "no state yet");
    if (ctx->g.metric != KERR_MKS) return fail(ctx, GRMHD_EINVAL, "the barycentric radius needs a Kerr grid");
    const Grid &g = ctx->g;
    double *part = ctx->scratch, *dout = ctx->scratch + 2LL * g.n1;
    (void)cudaGetLastError();
    launch_barycentric(g, ctx->cp, r_bar_max, part, dout, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ctx->hpin, dout, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    double num = ctx->hpin[0], den = ctx->hpin[1];
    out[0] = den > 0.0 ? num / den : 0.0;
    out[1] = den;
    out[2] = num;
    return 0;
}
