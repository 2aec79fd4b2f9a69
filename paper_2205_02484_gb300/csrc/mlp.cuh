// mlp.cuh -- learned Newton starting point for the inversion: a 5-64-64-1
// ReLU MLP with BF16 weights and FP32 accumulation that maps the normalised
// conserved-variable invariants of Section 2.3 to log(W/D).  Newton from the
// resulting (W, v^2(W) of Eq. 29) decides convergence exactly as from the
// previous-step primitives, so the guess changes the iteration count, never
// the root.
//
// Features (scale free: under D, Q -> lambda D, lambda Q and Bf -> sqrt(lambda) Bf
// the ratios below are invariant and W/D is unchanged):
//   x0 = log(tau / D), tau = -n.Q - D      (energy minus rest mass)
//   x1 = log(Qt^2 / D^2)                   (momentum squared)
//   x2 = log(Bf^2 / D)                     (field energy)
//   x3 = log((Q.Bf)^2 / D^3)
//   x4 = log(D)
// each argument clamped below at 1e-30, then standardised with the stored
// mean/std.  Inputs, biases and activations stay FP32; only the weight
// matrices are BF16.
//
// FP32 parameter vector (training master copy), MLP_NPARAM entries:
//   W1[64][5], b1[64], W2[64][64], b2[64], W3[64], b3   (row = output unit)
// Packed forward buffer (float words):
//   [0..4] feature mean, [5..9] feature std, [10] output mean, [11] output std,
//   [12..75] b1, [76..139] b2, [140] b3, [141..143] pad,
//   then BF16 words: W1[64][5], W2[64][64], W3[64].
#pragma once
#include <cuda_bf16.h>

#include "physics.cuh"

namespace grmhd {

constexpr int MLP_H = 64;
constexpr int MLP_IN = 5;
constexpr int MLP_OFF_B1 = 12, MLP_OFF_B2 = 76, MLP_OFF_B3 = 140, MLP_OFF_W = 144;
constexpr int MLP_NW1 = MLP_H * MLP_IN, MLP_NW2 = MLP_H * MLP_H, MLP_NW3 = MLP_H;
constexpr int MLP_FLOATS = MLP_OFF_W + (MLP_NW1 + MLP_NW2 + MLP_NW3 + 1) / 2;

// offsets in the FP32 parameter vector
constexpr int TH_W1 = 0, TH_B1 = TH_W1 + MLP_NW1, TH_W2 = TH_B1 + MLP_H, TH_B2 = TH_W2 + MLP_NW2,
              TH_W3 = TH_B2 + MLP_H, TH_B3 = TH_W3 + MLP_NW3, MLP_NPARAM = TH_B3 + 1;

__device__ __forceinline__ double mlp_clamp_log(double v) { return log(fmax(v, 1e-30)); }

// Section 2.3 variables of one conserved state (U includes sqrt(-g)) at the
// centre metric g; false (and zero features) when D is not positive.
__device__ inline bool mlp_features(const double U[NU], const Geo<double> &g, double feat[MLP_IN], double &D)
{
    double f = g.aig;
    D = f * U[KRHO];
    if (!(D > 0.0) || !isfinite(D)) {
#pragma unroll
        for (int k = 0; k < MLP_IN; k++) feat[k] = 0.0;
        return false;
    }
    double Q[4] = {f * U[1], f * U[2], f * U[3], f * U[4]};
    double nq = g.ialpha * Q[0] - g.alpha * (g.gcon[1] * Q[1] + g.gcon[2] * Q[2] + g.gcon[3] * Q[3]);
    double Qsq = 0.0;
#pragma unroll
    for (int m = 0; m < 4; m++)
        Qsq += (g.gcon[sym(m, 0)] * Q[0] + g.gcon[sym(m, 1)] * Q[1] + g.gcon[sym(m, 2)] * Q[2] +
                g.gcon[sym(m, 3)] * Q[3]) * Q[m];
    double Qt2 = Qsq + nq * nq;
    double Bf[3] = {g.alpha * U[KB1] * g.igdet, g.alpha * U[KB2] * g.igdet, g.alpha * U[KB3] * g.igdet};
    double B2 = spatial_sq(g, Bf[0], Bf[1], Bf[2]);
    double QB = Q[1] * Bf[0] + Q[2] * Bf[1] + Q[3] * Bf[2];
    double tau = -nq - D;
    feat[0] = mlp_clamp_log(tau / D);
    feat[1] = mlp_clamp_log(Qt2 / (D * D));
    feat[2] = mlp_clamp_log(B2 / D);
    feat[3] = mlp_clamp_log(QB * QB / (D * D * D));
    feat[4] = log(D);
    return true;
}

// log(W/D) predicted by the packed network for FP32 features f
__device__ inline float mlp_log_w_guess(const float *buf, const float f[MLP_IN])
{
    const __nv_bfloat16 *W1 = reinterpret_cast<const __nv_bfloat16 *>(buf + MLP_OFF_W);
    const __nv_bfloat16 *W2 = W1 + MLP_NW1;
    const __nv_bfloat16 *W3 = W2 + MLP_NW2;
    float x[MLP_IN];
#pragma unroll
    for (int i = 0; i < MLP_IN; i++) x[i] = (f[i] - buf[i]) / buf[5 + i];
    float h1[MLP_H];
#pragma unroll
    for (int o = 0; o < MLP_H; o++) {
        float a = buf[MLP_OFF_B1 + o];
#pragma unroll
        for (int i = 0; i < MLP_IN; i++) a = fmaf(__bfloat162float(W1[o * MLP_IN + i]), x[i], a);
        h1[o] = fmaxf(a, 0.0f);
    }
    float y = buf[MLP_OFF_B3];
#pragma unroll 1
    for (int o = 0; o < MLP_H; o++) {
        float a = buf[MLP_OFF_B2 + o];
        const __nv_bfloat162 *w = reinterpret_cast<const __nv_bfloat162 *>(W2 + o * MLP_H);
#pragma unroll
        for (int i = 0; i < MLP_H / 2; i++) {
            float2 wf = __bfloat1622float2(w[i]);
            a = fmaf(wf.x, h1[2 * i], a);
            a = fmaf(wf.y, h1[2 * i + 1], a);
        }
        y = fmaf(__bfloat162float(W3[o]), fmaxf(a, 0.0f), y);
    }
    return y * buf[11] + buf[10];
}

} // namespace grmhd
