// ensemble.cu -- a batch of independent tori (different sizes, spins,
// adiabatic indices, field strengths) advanced together: every kernel class
// of the RK2 step is one persistent launch over a ragged work list that
// spans all members, and the whole ensemble step is one captured CUDA graph.
//
// Work list: for kernel class c and batched member m the elements (faces,
// edges, zones, ghost zones) are cut into tiles of blockDim * items elements;
// prefix[c][m] counts the tiles of members < m.  A persistent grid of
// (SM count x blocks per SM) blocks walks the tiles; a block finds its
// member by binary search on the prefix (staged in shared memory), copies
// that member's descriptor into shared memory and runs the same item
// functions as the single-grid kernels, so every member evolves bit-for-bit
// as it would alone.  Fixups run one block per member, the CFL step and
// counters stay per member.
//
// Members at or above a size threshold are not batched: they run their own
// single-grid step kernels inside the same captured graph.  One launch per
// kernel class over the batch keeps every member's face and EMF arrays of a
// stage alive until the update of the whole batch, which for large members
// overflows L2; a large member's own step keeps them in L2.
//
// Tunables (tile length in elements per thread, persistent blocks per SM,
// the solo threshold) are picked by grmhd_ensemble_autotune from timed trial
// steps.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/grmhd.h"
#include "kernels.h"
#include "stage_items.cuh"

namespace grmhd {

enum { W_F1 = 0, W_F2, W_F3, W_EMF, W_UPD, W_POL, W_BC1, W_BC2, W_BC3, W_NCLASS };
constexpr int ENS_THREADS = 128;

struct EnsDev {
    const Grid *grids;       // [n]
    const long long *prefix; // [W_NCLASS][n + 1]
    int n;
    int items[W_NCLASS];
};

__host__ __device__ inline long long class_count(const Grid &g, int cls)
{
    switch (cls) {
    case W_F1: return flux_elem_box(g, 1).count();
    case W_F2: return flux_elem_box(g, 2).count();
    case W_F3: return g.x3warp ? x3_warp_box(g).count() : flux_elem_box(g, 3).count(); // long rows: warps
    case W_EMF: return edge_box(g).count();
    case W_UPD: return nact_of(g);
    case W_POL: return polar_count(g);
    case W_BC1: return bc1_count(g);
    case W_BC2: return bc2_count(g);
    default: return bc3_count(g);
    }
}

__device__ __forceinline__ int find_member(const long long *pre, int n, long long w)
{
    int lo = 0, hi = n; // pre[lo] <= w < pre[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (pre[mid] <= w) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <typename R, int CLS>
__global__ void __launch_bounds__(ENS_THREADS) ek_sweep(EnsDev E, int src, int dst, double dtfac, int corr,
                                                       int want_dt)
{
    __shared__ Grid sg;
    extern __shared__ long long s_pre[]; // this class's tile prefix, [n + 1]
    const long long *gpre = E.prefix + (long long)CLS * (E.n + 1);
    for (int q = threadIdx.x; q <= E.n; q += blockDim.x) s_pre[q] = gpre[q];
    __syncthreads();
    const long long *pre = s_pre;
    const long long total = pre[E.n];
    const int items = E.items[CLS];
    const long long tile = (long long)blockDim.x * items;
    int cur = -1;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        int m = find_member(pre, E.n, w);
        if (m != cur) {
            // the member's descriptor, copied by the whole block word by word
            __syncthreads();
            const unsigned *gw = (const unsigned *)&E.grids[m];
            unsigned *sw = (unsigned *)&sg;
            for (int q = threadIdx.x; q < (int)(sizeof(Grid) / 4); q += blockDim.x) sw[q] = gw[q];
            __syncthreads();
            cur = m;
        }
        const long long base = (w - pre[m]) * tile;
        const R *Pin = (const R *)sg.P[src];
        R *Pout = (R *)sg.P[dst];
        R cwm = R(0);
        UpdCount cn{};
        for (int it = 0; it < items; it++) {
            long long t = base + (long long)it * blockDim.x + threadIdx.x;
            if (CLS == W_F1)
                cwm = max(cwm, flux_call<R, 1>(sg, Pin, (R *)sg.F[0], flux_elem_box(sg, 1), want_dt, t));
            if (CLS == W_F2)
                cwm = max(cwm, flux_call<R, 2>(sg, Pin, (R *)sg.F[1], flux_elem_box(sg, 2), want_dt, t));
            if (CLS == W_F3) {
                // tiles are whole warps (blockDim and items multiples of 32), as the
                // mixed path's row-warp X3 sweep needs
                if (sg.x3warp)
                    cwm = max(cwm, flux_x3_warp_call<R>(sg, Pin, (R *)sg.F[2], x3_warp_box(sg), want_dt, t));
                else
                    cwm = max(cwm, flux_call<R, 3>(sg, Pin, (R *)sg.F[2], flux_elem_box(sg, 3), want_dt, t));
            }
            if (CLS == W_EMF)
                emf_item(sg, (const R *)sg.F[0], (const R *)sg.F[1], (const R *)sg.F[2], (R *)sg.E[0], (R *)sg.E[1],
                         (R *)sg.E[2], edge_box(sg), t);
            if (CLS == W_UPD)
                update_call<R>(sg, Pin, Pout, (const R *)sg.F[0], (const R *)sg.F[1], (const R *)sg.F[2],
                            (const R *)sg.E[0], (const R *)sg.E[1], (const R *)sg.E[2], dtfac, corr, t, cn);
            if (CLS == W_POL) polar_item(sg, Pout, t);
            if (CLS == W_BC1) bc1_call(sg, Pout, t);
            if (CLS == W_BC2) bc2_item(sg, Pout, t);
            if (CLS == W_BC3) bc3_item(sg, Pout, t);
        }
        if ((CLS == W_F1 || CLS == W_F2 || CLS == W_F3) && want_dt)
            block_cfl_into(&sg.dtmin[CLS - W_F1], cwm, sg.cfl * sg.dx[CLS - W_F1]);
        if (CLS == W_UPD) flush_counts(sg, cn);
    }
}

// The update class as one block per tile (no persistent loop), so that its
// registers match the single-grid update kernel's (3 resident blocks of 128
// threads per SM in the mixed path)
template <typename R>
__global__ void __launch_bounds__(ENS_THREADS, sizeof(R) == 4 ? 3 : 1) ek_update(EnsDev E, int src, int dst,
                                                                                 double dtfac, int corr)
{
    __shared__ Grid sg;
    const long long *pre = E.prefix + (long long)W_UPD * (E.n + 1);
    const long long w = blockIdx.x;
    if (w >= pre[E.n]) return;
    const int m = find_member(pre, E.n, w);
    {
        const unsigned *gw = (const unsigned *)&E.grids[m];
        unsigned *sw = (unsigned *)&sg;
        for (int q = threadIdx.x; q < (int)(sizeof(Grid) / 4); q += blockDim.x) sw[q] = gw[q];
    }
    __syncthreads();
    const int items = E.items[W_UPD];
    const long long base = (w - pre[m]) * (long long)blockDim.x * items;
    UpdCount cn{};
    for (int it = 0; it < items; it++)
        update_call<R>(sg, (const R *)sg.P[src], (R *)sg.P[dst], (const R *)sg.F[0], (const R *)sg.F[1],
                       (const R *)sg.F[2], (const R *)sg.E[0], (const R *)sg.E[1], (const R *)sg.E[2], dtfac, corr,
                       base + (long long)it * blockDim.x + threadIdx.x, cn);
    flush_counts(sg, cn);
}

template <typename R>
__global__ void __launch_bounds__(1024) ek_fixup(EnsDev E, int dst, int corr)
{
    const Grid &g = E.grids[blockIdx.x];
    fixup_call(g, (R *)g.P[dst], corr);
}

__global__ void ek_finalize(EnsDev E)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < E.n) finalize_one(E.grids[m], 1);
}

} // namespace grmhd

using namespace grmhd;

// solo members step on up to this many branch streams, which a captured
// ensemble graph turns into parallel branches beside the batched kernels
static constexpr int ENS_BRANCHES = 16;

struct grmhd_ens {
    std::vector<grmhd_ctx *> members;
    std::vector<Grid> hgrids;
    std::vector<int> batched, solo; // member indices: batched kernels / own step kernels
    std::vector<int> branch_of;     // branch stream of each solo member (balanced by zones)
    cudaStream_t bstream[ENS_BRANCHES] = {};
    cudaEvent_t bjoin[ENS_BRANCHES] = {};
    cudaEvent_t bfork = nullptr;
    std::vector<Grid> bgrids;       // descriptors of the batched members
    Grid *dgrids = nullptr;
    long long *dprefix = nullptr;
    cudaStream_t stream = nullptr;
    int device = 0, mixed = 0, sms = 0;
    grmhd_ens_tiling tiling{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    long long tiles[W_NCLASS] = {0};
    std::string err;
};

static int efail(grmhd_ens *e, int code, const std::string &m)
{
    if (e) e->err = m;
    return code;
}

#define ECK(call)                                                                                     \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return efail(ens, GRMHD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static void drop_graph(grmhd_ens *ens)
{
    if (ens->gexec) cudaGraphExecDestroy(ens->gexec);
    if (ens->graph) cudaGraphDestroy(ens->graph);
    ens->gexec = nullptr;
    ens->graph = nullptr;
}

// the batched / solo split and the tile prefix tables for the current tiling
static int build_tables(grmhd_ens *ens)
{
    ens->batched.clear();
    ens->solo.clear();
    ens->bgrids.clear();
    const int sl = ens->tiling.solo_log2;
    for (int m = 0; m < (int)ens->members.size(); m++) {
        long long na = nact_of(ens->hgrids[m]);
        if (sl > 0 && na >= (1LL << sl)) {
            ens->solo.push_back(m);
        } else {
            ens->batched.push_back(m);
            ens->bgrids.push_back(ens->hgrids[m]);
        }
    }
    // solo members to branches: largest first, each to the least loaded branch
    {
        const int ns = (int)ens->solo.size(), K = std::min(ns, ENS_BRANCHES);
        std::vector<int> order(ns);
        for (int i = 0; i < ns; i++) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            return nact_of(ens->hgrids[ens->solo[x]]) > nact_of(ens->hgrids[ens->solo[y]]);
        });
        std::vector<long long> load(K > 0 ? K : 1, 0);
        ens->branch_of.assign(ns, 0);
        for (int i : order) {
            int b = (int)(std::min_element(load.begin(), load.begin() + K) - load.begin());
            ens->branch_of[i] = b;
            load[b] += nact_of(ens->hgrids[ens->solo[i]]);
        }
    }
    int n = (int)ens->batched.size();
    if (n > 0)
        ECK(cudaMemcpyAsync(ens->dgrids, ens->bgrids.data(), sizeof(Grid) * n, cudaMemcpyHostToDevice,
                            ens->stream));
    int items[W_NCLASS];
    for (int c = 0; c < W_NCLASS; c++) items[c] = 4;
    items[W_F1] = items[W_F2] = items[W_F3] = ens->tiling.items_flux;
    items[W_UPD] = ens->tiling.items_update;
    std::vector<long long> pre((size_t)W_NCLASS * (n + 1));
    for (int c = 0; c < W_NCLASS; c++) {
        long long acc = 0;
        long long tile = (long long)ENS_THREADS * items[c];
        for (int m = 0; m < n; m++) {
            pre[(size_t)c * (n + 1) + m] = acc;
            acc += (class_count(ens->bgrids[m], c) + tile - 1) / tile;
        }
        pre[(size_t)c * (n + 1) + n] = acc;
        ens->tiles[c] = acc;
    }
    if (n > 0)
        ECK(cudaMemcpyAsync(ens->dprefix, pre.data(), pre.size() * sizeof(long long), cudaMemcpyHostToDevice,
                            ens->stream));
    ECK(cudaStreamSynchronize(ens->stream));
    return 0;
}

static EnsDev ens_dev(const grmhd_ens *ens)
{
    EnsDev E{};
    E.grids = ens->dgrids;
    E.prefix = ens->dprefix;
    E.n = (int)ens->batched.size();
    for (int c = 0; c < W_NCLASS; c++) E.items[c] = 4;
    E.items[W_F1] = E.items[W_F2] = E.items[W_F3] = ens->tiling.items_flux;
    E.items[W_UPD] = ens->tiling.items_update;
    return E;
}

// Launch one ensemble step; with ev != nullptr an event is recorded before
// each batched launch (2 stages x 10 launches + finalize + end = 22 events);
// the solo members' own steps follow.
template <typename R>
static void launch_ens_step(const grmhd_ens *ens, cudaStream_t s, cudaEvent_t *ev)
{
    EnsDev E = ens_dev(ens);
    const int n = E.n;
    const size_t smem = sizeof(long long) * (n + 1);
    auto grid_of = [&](int cls) {
        int bps = (cls == W_UPD) ? ens->tiling.blocks_per_sm_update
                                 : (cls <= W_F3 ? ens->tiling.blocks_per_sm_flux : 8);
        long long b = std::min<long long>((long long)ens->sms * bps, ens->tiles[cls]);
        return (unsigned)std::max<long long>(b, 1);
    };
    // solo members: their own step graphs on the branch streams, forked from s
    // before the batched kernels and joined after them (in a capture: parallel
    // branches of the ensemble graph); under profiling events, after them on s
    const int nsolo = (int)ens->solo.size();
    const int K = std::min(nsolo, ENS_BRANCHES);
    const bool fork = ev == nullptr && nsolo > 0;
    if (fork) {
        cudaEventRecord(ens->bfork, s);
        for (int b = 0; b < K; b++) cudaStreamWaitEvent(ens->bstream[b], ens->bfork, 0);
        for (int i = 0; i < nsolo; i++) launch_step(ens->hgrids[ens->solo[i]], ens->bstream[ens->branch_of[i]]);
        for (int b = 0; b < K; b++) cudaEventRecord(ens->bjoin[b], ens->bstream[b]);
    }
    int e = 0;
    for (int st = 0; st < 2 && n > 0; st++) {
        int src = st == 0 ? 0 : 1, dst = st == 0 ? 1 : 0;
        double fac = st == 0 ? 0.5 : 1.0;
        int corr = st, wdt = st == 0;
#define REC() do { if (ev) cudaEventRecord(ev[e++], s); } while (0)
        REC(); ek_sweep<R, W_F1><<<grid_of(W_F1), ENS_THREADS, smem, s>>>(E, src, dst, fac, corr, wdt);
        REC(); ek_sweep<R, W_F2><<<grid_of(W_F2), ENS_THREADS, smem, s>>>(E, src, dst, fac, corr, wdt);
        REC(); ek_sweep<R, W_F3><<<grid_of(W_F3), ENS_THREADS, smem, s>>>(E, src, dst, fac, corr, wdt);
        REC(); ek_sweep<R, W_EMF><<<grid_of(W_EMF), ENS_THREADS, smem, s>>>(E, src, dst, fac, corr, wdt);
        REC(); ek_update<R><<<(unsigned)std::max<long long>(ens->tiles[W_UPD], 1), ENS_THREADS, 0, s>>>(E, src, dst, fac, corr);
        REC(); ek_fixup<R><<<n, 1024, 0, s>>>(E, dst, corr);
        REC(); ek_sweep<R, W_POL><<<grid_of(W_POL), ENS_THREADS, smem, s>>>(E, src, dst, fac, corr, wdt);
        REC(); ek_sweep<R, W_BC1><<<grid_of(W_BC1), ENS_THREADS, smem, s>>>(E, src, dst, fac, corr, wdt);
        REC(); ek_sweep<R, W_BC2><<<grid_of(W_BC2), ENS_THREADS, smem, s>>>(E, src, dst, fac, corr, wdt);
        REC(); ek_sweep<R, W_BC3><<<grid_of(W_BC3), ENS_THREADS, smem, s>>>(E, src, dst, fac, corr, wdt);
    }
    REC();
    if (n > 0) ek_finalize<<<(n + 127) / 128, 128, 0, s>>>(E);
    REC();
#undef REC
    if (fork) {
        for (int b = 0; b < K; b++) cudaStreamWaitEvent(s, ens->bjoin[b], 0);
    } else {
        for (int m : ens->solo) launch_step(ens->hgrids[m], s);
    }
}

static void ens_step_launch(const grmhd_ens *ens, cudaStream_t s, cudaEvent_t *ev)
{
    if (ens->mixed) launch_ens_step<float>(ens, s, ev);
    else launch_ens_step<double>(ens, s, ev);
}

extern "C" int grmhd_ensemble_create(grmhd_ctx *const *members, int n, grmhd_ens **out)
{
    grmhd_ens *ens = nullptr;
    if (!members || n < 1 || !out) return GRMHD_EINVAL;
    ens = new grmhd_ens();
    for (int m = 0; m < n; m++) {
        const Grid *g = ctx_grid(members[m]);
        if (!g || !ctx_ready(members[m])) {
            delete ens;
            return GRMHD_ESTATE;
        }
        // a slab of a decomposed grid steps with its neighbours, not as a member
        // the batched face sweeps walk PLM columns: a PPM member steps on its own
        if ((m > 0 && (g->mixed != ens->hgrids[0].mixed || ctx_device(members[m]) != ctx_device(members[0]))) ||
            g->bc3 == BC_EXTERNAL || g->n2t != g->n2 || g->recon != 0) {
            delete ens;
            return GRMHD_EINVAL;
        }
        ens->members.push_back(members[m]);
        ens->hgrids.push_back(*g);
        ens->hgrids.back().mlp = nullptr; // ensemble steps keep the plain method order
    }
    ens->mixed = ens->hgrids[0].mixed;
    ens->device = ctx_device(members[0]);
    ens->stream = ctx_stream(members[0]);
    cudaDeviceGetAttribute(&ens->sms, cudaDevAttrMultiProcessorCount, ens->device);
    ens->tiling = grmhd_ens_tiling{2, 2, 8, 4, 0};
    if (cudaMalloc(&ens->dgrids, sizeof(Grid) * n) != cudaSuccess ||
        cudaMalloc(&ens->dprefix, sizeof(long long) * W_NCLASS * (n + 1)) != cudaSuccess) {
        grmhd_ensemble_destroy(ens);
        return GRMHD_ENOMEM;
    }
    {
        // branch streams and their events on the members' device
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(ens->device);
        bool ok = cudaEventCreateWithFlags(&ens->bfork, cudaEventDisableTiming) == cudaSuccess;
        for (int b = 0; b < ENS_BRANCHES && ok; b++)
            ok = cudaStreamCreateWithFlags(&ens->bstream[b], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&ens->bjoin[b], cudaEventDisableTiming) == cudaSuccess;
        cudaSetDevice(prev);
        if (!ok) {
            grmhd_ensemble_destroy(ens);
            return GRMHD_ECUDA;
        }
    }
    cudaMemcpyAsync(ens->dgrids, ens->hgrids.data(), sizeof(Grid) * n, cudaMemcpyHostToDevice, ens->stream);
    if (build_tables(ens) != 0) {
        grmhd_ensemble_destroy(ens);
        return GRMHD_ECUDA;
    }
    *out = ens;
    return 0;
}

extern "C" void grmhd_ensemble_destroy(grmhd_ens *ens)
{
    if (!ens) return;
    // The stream belongs to the first member, which may already be gone;
    // cudaFree below waits for all device work anyway.
    drop_graph(ens);
    for (int b = 0; b < ENS_BRANCHES; b++) {
        if (ens->bstream[b]) cudaStreamDestroy(ens->bstream[b]);
        if (ens->bjoin[b]) cudaEventDestroy(ens->bjoin[b]);
    }
    if (ens->bfork) cudaEventDestroy(ens->bfork);
    if (ens->dgrids) cudaFree(ens->dgrids);
    if (ens->dprefix) cudaFree(ens->dprefix);
    delete ens;
}

extern "C" const char *grmhd_ensemble_last_error(const grmhd_ens *ens) { return ens ? ens->err.c_str() : ""; }

extern "C" int grmhd_ensemble_set_tiling(grmhd_ens *ens, const grmhd_ens_tiling *t)
{
    if (!ens || !t) return GRMHD_EINVAL;
    if (t->items_flux < 1 || t->items_flux > 16 || t->items_update < 1 || t->items_update > 16 ||
        t->blocks_per_sm_flux < 1 || t->blocks_per_sm_flux > 64 || t->blocks_per_sm_update < 1 ||
        t->blocks_per_sm_update > 64 || (t->solo_log2 != 0 && (t->solo_log2 < 10 || t->solo_log2 > 40)))
        return efail(ens, GRMHD_EINVAL, "tiling out of range (items 1-16, blocks per SM 1-64, solo 0 or 10-40)");
    ECK(cudaStreamSynchronize(ens->stream));
    ens->tiling = *t;
    drop_graph(ens);
    return build_tables(ens);
}

extern "C" int grmhd_ensemble_get_tiling(const grmhd_ens *ens, grmhd_ens_tiling *t)
{
    if (!ens || !t) return GRMHD_EINVAL;
    *t = ens->tiling;
    return 0;
}

extern "C" int grmhd_ensemble_step(grmhd_ens *ens, int nsteps)
{
    if (!ens) return GRMHD_EINVAL;
    if (nsteps < 0) return efail(ens, GRMHD_EINVAL, "nsteps < 0");
    (void)cudaGetLastError(); // a stale error of an unrelated earlier call is not ours
    if (!ens->gexec) {
        ECK(cudaStreamBeginCapture(ens->stream, cudaStreamCaptureModeThreadLocal));
        ens_step_launch(ens, ens->stream, nullptr);
        cudaError_t le = cudaGetLastError();
        cudaGraph_t graph = nullptr;
        cudaError_t ee = cudaStreamEndCapture(ens->stream, &graph);
        if (le != cudaSuccess || ee != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return efail(ens, GRMHD_ECUDA, std::string("ensemble capture failed: ") +
                                               cudaGetErrorString(le != cudaSuccess ? le : ee));
        }
        ens->graph = graph;
        ECK(cudaGraphInstantiate(&ens->gexec, ens->graph, 0));
    }
    for (int s = 0; s < nsteps; s++) ECK(cudaGraphLaunch(ens->gexec, ens->stream));
    return 0;
}

extern "C" int grmhd_ensemble_sync(grmhd_ens *ens)
{
    if (!ens) return GRMHD_EINVAL;
    ECK(cudaStreamSynchronize(ens->stream));
    for (grmhd_ctx *c : ens->members) {
        int rc = grmhd_sync(c);
        if (rc) return efail(ens, rc, grmhd_last_error(c));
    }
    return 0;
}

// Snapshot of one member's evolving state (P^n, U, dt/t, counters, CFL minima).
struct Snap {
    void *P = nullptr, *U = nullptr;
    size_t pbytes = 0, ubytes = 0;
    double scal[8];
    unsigned long long cnt[C_NCOUNT], dtmin[4];
};

extern "C" int grmhd_ensemble_autotune(grmhd_ens *ens, int trial_steps, grmhd_ens_tiling *best, double *best_ms)
{
    if (!ens) return GRMHD_EINVAL;
    if (trial_steps < 1) return efail(ens, GRMHD_EINVAL, "trial_steps < 1");
    cudaStream_t s = ens->stream;
    ECK(cudaStreamSynchronize(s));
    // save every member so that the trials leave the state unchanged
    std::vector<Snap> snaps(ens->members.size());
    size_t rs = ens->mixed ? sizeof(float) : sizeof(double);
    for (size_t m = 0; m < snaps.size(); m++) {
        const Grid &g = ens->hgrids[m];
        Snap &sn = snaps[m];
        sn.pbytes = 8 * (size_t)g.nz * rs;
        sn.ubytes = 9 * (size_t)g.nz * sizeof(double);
        ECK(cudaMalloc(&sn.P, 2 * sn.pbytes));
        ECK(cudaMalloc(&sn.U, sn.ubytes));
        ECK(cudaMemcpyAsync(sn.P, g.P[0], sn.pbytes, cudaMemcpyDeviceToDevice, s));
        // the second buffer too: the mixed update's Newton start reads it
        ECK(cudaMemcpyAsync((char *)sn.P + sn.pbytes, g.P[1], sn.pbytes, cudaMemcpyDeviceToDevice, s));
        ECK(cudaMemcpyAsync(sn.U, g.U, sn.ubytes, cudaMemcpyDeviceToDevice, s));
        ECK(cudaMemcpyAsync(sn.scal, g.scal, sizeof(sn.scal), cudaMemcpyDeviceToHost, s));
        ECK(cudaMemcpyAsync(sn.cnt, g.cnt, sizeof(sn.cnt), cudaMemcpyDeviceToHost, s));
        ECK(cudaMemcpyAsync(sn.dtmin, g.dtmin, sizeof(sn.dtmin), cudaMemcpyDeviceToHost, s));
    }
    ECK(cudaStreamSynchronize(s));
    const int NE = 22;
    cudaEvent_t ev[NE];
    for (int e = 0; e < NE; e++) ECK(cudaEventCreate(&ev[e]));
    // flux sweeps and the update are timed separately; each picks its own
    // (items per thread, blocks per SM) from a small grid of candidates
    const int items_c[3] = {1, 2, 4};
    const int bps_c[4] = {2, 4, 8, 16};
    grmhd_ens_tiling keep = ens->tiling, cur = keep;
    double best_flux = 1e300, best_upd = 1e300, best_step = 1e300;
    cur.solo_log2 = 0; // tiles are timed with every member batched
    grmhd_ens_tiling bt = cur;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 4; b++) {
            cur.items_flux = items_c[a];
            cur.blocks_per_sm_flux = bps_c[b];
            cur.items_update = items_c[a];
            cur.blocks_per_sm_update = std::min(bps_c[b], 4);
            ens->tiling = cur;
            if (build_tables(ens)) goto done;
            double tf = 0.0, tu = 0.0;
            for (int it = 0; it <= trial_steps; it++) {
                ens_step_launch(ens, s, ev);
                ECK(cudaEventSynchronize(ev[NE - 1]));
                if (it == 0) continue; // first run of a configuration warms up
                for (int st = 0; st < 2; st++) {
                    float ms;
                    for (int k = 0; k < 3; k++) {
                        ECK(cudaEventElapsedTime(&ms, ev[st * 10 + k], ev[st * 10 + k + 1]));
                        tf += ms;
                    }
                    ECK(cudaEventElapsedTime(&ms, ev[st * 10 + 4], ev[st * 10 + 5]));
                    tu += ms;
                }
            }
            if (tf < best_flux) {
                best_flux = tf;
                bt.items_flux = cur.items_flux;
                bt.blocks_per_sm_flux = cur.blocks_per_sm_flux;
            }
            if (tu < best_upd) {
                best_upd = tu;
                bt.items_update = cur.items_update;
                bt.blocks_per_sm_update = cur.blocks_per_sm_update;
            }
        }
    {
        // the solo threshold, on whole steps with the chosen tiles: members of at
        // least 2^k zones step on their own (k = 0: none); candidates that give
        // the same split as the previous one are skipped
        const int cands[10] = {0, 22, 21, 20, 19, 18, 16, 14, 12, 10};
        long long last_nsolo = -1;
        int best_sl = 0;
        for (int q = 0; q < 10; q++) {
            grmhd_ens_tiling t = bt;
            t.solo_log2 = cands[q];
            ens->tiling = t;
            if (build_tables(ens)) break;
            if ((long long)ens->solo.size() == last_nsolo) continue;
            last_nsolo = (long long)ens->solo.size();
            // timed as the step runs: a captured graph (the solo members'
            // launches are many; launched one by one the host would bound them)
            drop_graph(ens);
            if (grmhd_ensemble_step(ens, 1) != 0) break; // capture and warm-up
            cudaEventRecord(ev[0], s);
            if (grmhd_ensemble_step(ens, trial_steps) != 0) break;
            cudaEventRecord(ev[1], s);
            if (cudaEventSynchronize(ev[1]) != cudaSuccess) break;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, ev[0], ev[1]);
            if (ms < best_step) {
                best_step = ms;
                best_sl = cands[q];
            }
        }
        bt.solo_log2 = best_sl;
    }
done:
    for (int e = 0; e < NE; e++) cudaEventDestroy(ev[e]);
    cudaError_t err = cudaGetLastError();
    // restore the members
    for (size_t m = 0; m < snaps.size(); m++) {
        const Grid &g = ens->hgrids[m];
        Snap &sn = snaps[m];
        cudaMemcpyAsync(g.P[0], sn.P, sn.pbytes, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(g.P[1], (char *)sn.P + sn.pbytes, sn.pbytes, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(g.U, sn.U, sn.ubytes, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(g.scal, sn.scal, sizeof(sn.scal), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(g.cnt, sn.cnt, sizeof(sn.cnt), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(g.dtmin, sn.dtmin, sizeof(sn.dtmin), cudaMemcpyHostToDevice, s);
    }
    cudaStreamSynchronize(s);
    for (Snap &sn : snaps) {
        cudaFree(sn.P);
        cudaFree(sn.U);
    }
    for (size_t m = 0; m < snaps.size(); m++) launch_bc(ens->hgrids[m], 0, s);
    if (err != cudaSuccess) {
        ens->tiling = keep;
        build_tables(ens);
        return efail(ens, GRMHD_ECUDA, cudaGetErrorString(err));
    }
    ens->tiling = bt;
    drop_graph(ens);
    int rc = build_tables(ens);
    if (rc) return rc;
    if (best) *best = bt;
    if (best_ms) *best_ms = best_step < 1e300 ? best_step / trial_steps : (best_flux + best_upd) / trial_steps;
    return 0;
}
