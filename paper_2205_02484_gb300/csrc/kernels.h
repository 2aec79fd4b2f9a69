// kernels.h -- host-side launchers of the device kernels (internal).
#pragma once
#include "common.cuh"

namespace grmhd {

// step.cu
void launch_step(const Grid &g, cudaStream_t s);
void launch_step_profiled(const Grid &g, cudaStream_t s, cudaEvent_t *ev);
double launch_fma_probe(int fp64, int sms, cudaStream_t s);
void launch_bc(const Grid &g, int buf, cudaStream_t s);
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
void launch_con2prim(const Grid &g, const double *U, const int *loc, double *P, int *flags, int *iters,
                     long n, const float *mlp, cudaStream_t s);

// diag.cu
void launch_diagnostics(const Grid &g, double *scratch, long scratch_len, double *out_dev, cudaStream_t s);
void launch_copy_state_in(const Grid &g, const double *P, const double *U, cudaStream_t s);
void launch_copy_state_out(const Grid &g, double *P, double *U, cudaStream_t s);

} // namespace grmhd

// context accessors for the ensemble (abi.cu)
struct grmhd_ctx;
const grmhd::Grid *ctx_grid(const grmhd_ctx *ctx);
bool ctx_ready(const grmhd_ctx *ctx);
int ctx_device(const grmhd_ctx *ctx);
cudaStream_t ctx_stream(const grmhd_ctx *ctx);
