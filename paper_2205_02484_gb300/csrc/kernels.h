// kernels.h -- host-side launchers of the device kernels (internal).
#pragma once
#include "common.cuh"

namespace grmhd {

// step.cu
void launch_step(const Grid &g, cudaStream_t s);
void launch_step_profiled(const Grid &g, cudaStream_t s, cudaEvent_t *ev);
double launch_fma_probe(int fp64, int sms, cudaStream_t s);
void launch_bc(const Grid &g, int buf, cudaStream_t s);
void launch_reinvert(const Grid &g, cudaStream_t s);
// Eq. 43 sums over rows i_h.. with centre radius <= r_bar_max: out[0] = numerator, out[1] = mass
void launch_barycentric(const Grid &g, const CoordParams &cp, double r_bar_max, double *part, double *out,
                        cudaStream_t s);
void launch_stage(const Grid &g, int st, cudaStream_t s);
void launch_step_dtd(const Grid &g, double *dtd, int acc, cudaStream_t s);
void launch_finish_step(const Grid &g, const double *dtd, cudaStream_t s);
long long x3_plane_elems(const Grid &g);
void launch_x3_planes(const Grid &g, int which, int side, void *buf, int unpack, cudaStream_t s);
void launch_stage_update(const Grid &g, int st, cudaStream_t s);
void launch_fail_count(const Grid &g, long long *acc, cudaStream_t s);
void launch_fix_sweep(const Grid &g, int st, long long *acc, cudaStream_t s);
void launch_fix_end(const Grid &g, int nsweeps, cudaStream_t s);
// the fixup loop of stage st over the theta slabs gs[0..nslab) of one grid on
// one device, in theta order; nsweeps (device, may be null) <- the sweeps run
constexpr int RING_MAX = 16;
void launch_fix_ring(const Grid *gs, int nslab, int st, int *nsweeps, cudaStream_t s);
long long x2_row_elems(const Grid &g, int kind);
void launch_x2_rows(const Grid &g, int kind, int which, int side, void *buf, int unpack, cudaStream_t s);
void launch_fluxes_dt(const Grid &g, int set_dt, cudaStream_t s);
void launch_gather_fluxes(const Grid &g, double *out, cudaStream_t s);

// geometry.cu
struct GeomBuild {
    CoordParams cp;
    Geo<double> *gc, *gf1, *gf2;
    Geo<float> *gcF, *gf1F, *gf2F;
    double *conn;
    float *connF;
    double *rc;
    double *gsp;
    unsigned char *polar2;
};
void launch_geometry(const Grid &g, const GeomBuild &b, cudaStream_t s);

// torus.cu
struct TorusArgs {
    double a, ell, lnh_in, r_in, kappa, beta0, pert_amp;
    unsigned long long seed;
    CoordParams cp;
};
double fm_ell_host(double a, double r_max);
double fm_lnh_host(double a, double ell, double r, double th);
// scratch: >= 2 * nact doubles + 8 (reductions); intorus: nact bytes
void launch_torus(const Grid &g, const TorusArgs &ta, double *scratch, unsigned char *intorus,
                  double *out_host6, cudaStream_t s);

// points.cu
void launch_prim2cons(const Grid &g, const double *P, const int *loc, double *U, long n, cudaStream_t s);
// list: n + 1 ints of device scratch (the deferred zones of the first pass)
void launch_con2prim(const Grid &g, const double *U, const int *loc, double *P, int *flags, int *iters,
                     long n, const float *mlp, int mode, int *list, cudaStream_t s);

// mlp.cu (learned Newton start)
struct MlpHyper {
    double lr0, lr_min, b1, b2, eps, wd;
    long long total_steps; // > 0: cosine from lr0 to lr_min over total_steps; else constant lr0
};
struct MlpTrainer {
    float *theta, *m, *v; // FP32 master parameters and AdamW moments [MLP_NPARAM]
    float *fwd;           // packed forward buffer (norm, biases, BF16 weights)
    float *part;          // per-block gradient rows [blocks][MLP_NPARAM]
    double *lpart;        // per-block loss sums [blocks]
    long long *step;      // steps taken (device)
    unsigned int *ticket; // last-block detection of the AdamW kernel
    double *loss_hist;    // mean loss of step s at [s % hist_len]
    long long hist_len;
};
void launch_mlp_samples(const Grid &g, unsigned long long seed, long long first, long long n, double *P, int *loc,
                        double *U, float *feat, float *label, cudaStream_t s);
void launch_mlp_forward(const float *fwd, const float *feat, long long n, float *y, cudaStream_t s);
void launch_mlp_moments(const float *feat, const float *label, long long n, double *part, int nblk, cudaStream_t s);
void launch_mlp_init(float *theta, unsigned long long seed, cudaStream_t s);
void launch_mlp_pack(const float *theta, float *fwd, cudaStream_t s);
size_t mlp_grad_smem();
int mlp_grad_blocks(int batch);
cudaError_t mlp_grad_setup();
void launch_mlp_grad(const MlpTrainer &T, const float *feat, const float *label, long long n, int batch,
                     unsigned long long mul, cudaStream_t s);
void launch_mlp_adam(const MlpTrainer &T, int batch, const MlpHyper &h, cudaStream_t s);
void launch_mlp_reduce_grad(const MlpTrainer &T, int batch, float *grad, cudaStream_t s);
int mlp_eval_blocks(long long n);
// part: 2 * mlp_eval_blocks(n) doubles
void launch_mlp_eval(const float *fwd, const float *feat, const float *label, long long n, double *part,
                     cudaStream_t s);

// diag.cu
void launch_diagnostics(const Grid &g, double *scratch, long scratch_len, double *out_dev, cudaStream_t s);
constexpr int DIAG_NPART = 26; // partial-sum vector of one context (see diag.cu)
void launch_diag_pack(const Grid &g, const double *horizon, const double *bary, double *out, cudaStream_t s);
void launch_diag_combine(const double *parts, int nparts, double *out, cudaStream_t s);
void launch_copy_state_in(const Grid &g, const double *P, const double *U, cudaStream_t s);
void launch_copy_state_out(const Grid &g, double *P, double *U, cudaStream_t s);

} // namespace grmhd

// context accessors for the ensemble (abi.cu)
struct grmhd_ctx;
const grmhd::Grid *ctx_grid(const grmhd_ctx *ctx);
bool ctx_ready(const grmhd_ctx *ctx);
int ctx_device(const grmhd_ctx *ctx);
cudaStream_t ctx_stream(const grmhd_ctx *ctx);
