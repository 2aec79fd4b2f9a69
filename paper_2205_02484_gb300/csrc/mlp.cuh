// mlp.cuh -- learned Newton starting point for the inversion: a 5-64-64-1
// MLP with BF16 weights and FP32 accumulation that maps the normalised
// conserved-variable invariants of Section 2.3 to log(W/D).  Newton from the
// previous-step primitives stays the fallback and decides convergence.
//
// Features (scale free: under D, Q -> lambda D, lambda Q and Bf -> sqrt(lambda) Bf
// the ratios below are invariant and W/D is unchanged):
//   x0 = log(tau / D), tau = -Q.n - D     (energy minus rest mass)
//   x1 = log(Qt^2 / D^2)                   (momentum squared)
//   x2 = log(Bf^2 / D)                     (field energy)
//   x3 = log((Q.Bf)^2 / D^3)
//   x4 = log(D)
// each clamped at log(1e-30), then standardised with the stored mean/std.
//
// Packed parameter buffer (float words):
//   [0..4] feature mean, [5..9] feature std, [10] output mean, [11] output std,
//   [12..75] b1, [76..139] b2, [140] b3, [141..143] pad,
//   then BF16 words: W1[64][5], W2[64][64], W3[64] (row = output unit).
#pragma once
#include <cuda_bf16.h>

namespace grmhd {

constexpr int MLP_H = 64;
constexpr int MLP_IN = 5;
constexpr int MLP_OFF_B1 = 12, MLP_OFF_B2 = 76, MLP_OFF_B3 = 140, MLP_OFF_W = 144;
constexpr int MLP_NW1 = MLP_H * MLP_IN, MLP_NW2 = MLP_H * MLP_H, MLP_NW3 = MLP_H;
constexpr int MLP_FLOATS = MLP_OFF_W + (MLP_NW1 + MLP_NW2 + MLP_NW3 + 1) / 2;

__device__ inline float mlp_log_w_guess(const float *buf, const double feat[5])
{
    const __nv_bfloat16 *W1 = reinterpret_cast<const __nv_bfloat16 *>(buf + MLP_OFF_W);
    const __nv_bfloat16 *W2 = W1 + MLP_NW1;
    const __nv_bfloat16 *W3 = W2 + MLP_NW2;
    float x[MLP_IN];
#pragma unroll
    for (int i = 0; i < MLP_IN; i++) x[i] = ((float)feat[i] - buf[i]) / buf[5 + i];
    float h1[MLP_H];
#pragma unroll 4
    for (int o = 0; o < MLP_H; o++) {
        float a = buf[MLP_OFF_B1 + o];
#pragma unroll
        for (int i = 0; i < MLP_IN; i++) a = fmaf(__bfloat162float(W1[o * MLP_IN + i]), x[i], a);
        h1[o] = fmaxf(a, 0.0f);
    }
    float y = buf[MLP_OFF_B3];
    for (int o = 0; o < MLP_H; o++) {
        float a = buf[MLP_OFF_B2 + o];
#pragma unroll 8
        for (int i = 0; i < MLP_H; i++) a = fmaf(__bfloat162float(W2[o * MLP_H + i]), h1[i], a);
        y = fmaf(__bfloat162float(W3[o]), fmaxf(a, 0.0f), y);
    }
    return y * buf[11] + buf[10];
}

} // namespace grmhd
