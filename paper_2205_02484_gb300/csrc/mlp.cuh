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

// ------------------------------------------ tensor-core inference (one warp)
//
// The same network on the tensor cores, for a warp of 32 inversions that all
// reach the network (the stand-alone inversion with the learned start first,
// the forward entry point).  mma.sync m16n8k16 with BF16 operands and FP32
// accumulation: the BF16 weights are the operands as stored; each FP32
// activation is split into three BF16 parts (hi + mid + lo, 24 bits), so the
// products are those of the FP32 activations and only the FP32 summation
// order differs from mlp_log_w_guess.  Hidden layer 1 comes out of the
// accumulators in the layout of layer 2's A operand (the fragments of two
// adjacent 8-column tiles are one 16-column k-step), so no shuffles are
// needed between the layers.

// weights staged in shared memory: W1 rows padded to 8 BF16 (k = 5..7 zero,
// 4 words per row), W2 rows padded to 72 BF16 (36 words: the eight rows a
// B fragment reads fall into distinct banks)
struct MlpSmem {
    float norm[12];
    float b1[MLP_H], b2[MLP_H], w3[MLP_H], b3;
    unsigned w1[MLP_H * 4];
    unsigned w2[MLP_H * 36];
};

// block-cooperative copy of the packed forward buffer into s (the caller
// synchronises the block afterwards)
__device__ inline void mlp_stage(const float *buf, MlpSmem &s)
{
    const unsigned short *W = reinterpret_cast<const unsigned short *>(buf + MLP_OFF_W);
    for (int a = threadIdx.x; a < MLP_H * 36; a += blockDim.x) {
        const int o = a / 36, w = a % 36;
        const unsigned lo = w < 32 ? W[MLP_NW1 + o * MLP_H + 2 * w] : 0u;
        const unsigned hi = w < 32 ? W[MLP_NW1 + o * MLP_H + 2 * w + 1] : 0u;
        s.w2[a] = lo | (hi << 16);
    }
    for (int a = threadIdx.x; a < MLP_H * 4; a += blockDim.x) {
        const int o = a / 4, k0 = 2 * (a % 4);
        const unsigned lo = k0 < MLP_IN ? W[o * MLP_IN + k0] : 0u;
        const unsigned hi = k0 + 1 < MLP_IN ? W[o * MLP_IN + k0 + 1] : 0u;
        s.w1[a] = lo | (hi << 16);
    }
    for (int a = threadIdx.x; a < MLP_H; a += blockDim.x) {
        s.b1[a] = buf[MLP_OFF_B1 + a];
        s.b2[a] = buf[MLP_OFF_B2 + a];
        s.w3[a] = __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(W)[MLP_NW1 + MLP_NW2 + a]);
    }
    for (int a = threadIdx.x; a < 12; a += blockDim.x) s.norm[a] = buf[a];
    if (threadIdx.x == 0) s.b3 = buf[MLP_OFF_B3];
}

// x = hi + mid + lo exactly to FP32 rounding, each part BF16; packed pairs
// (element of the lower index in the low half)
__device__ __forceinline__ void mlp_split3(float x0, float x1, unsigned p[3])
{
#pragma unroll
    for (int q = 0; q < 3; q++) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
        p[q] = (unsigned)__bfloat16_as_ushort(h0) | ((unsigned)__bfloat16_as_ushort(h1) << 16);
        x0 -= __bfloat162float(h0);
        x1 -= __bfloat162float(h1);
    }
}

__device__ __forceinline__ void mlp_mma(const unsigned a[4], unsigned b0, unsigned b1, float c[4])
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// log(W/D) for this lane's features f; all 32 lanes of the warp must call it
// together (a lane without an inversion passes any finite features)
__device__ inline float mlp_log_w_mma(const MlpSmem &s, const float f[MLP_IN])
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
    float x[MLP_IN];
#pragma unroll
    for (int i = 0; i < MLP_IN; i++) x[i] = (f[i] - s.norm[i]) / s.norm[5 + i];
    float y00 = 0.0f, y01 = 0.0f, y10 = 0.0f, y11 = 0.0f; // [tile][row g, g + 8]: this quad's sums
#pragma unroll 1
    for (int m = 0; m < 2; m++) {
        // layer 1 A operand: rows g and g + 8 of tile m are lanes 16 m + g (+ 8);
        // this lane's columns are the features 2 tq and 2 tq + 1 (zero from 5 on)
        unsigned a1[3][4];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int src = 16 * m + gq + 8 * h;
            float v[MLP_IN];
#pragma unroll
            for (int i = 0; i < MLP_IN; i++) v[i] = __shfl_sync(full, x[i], src);
            const float c0 = tq == 0 ? v[0] : (tq == 1 ? v[2] : (tq == 2 ? v[4] : 0.0f));
            const float c1 = tq == 0 ? v[1] : (tq == 1 ? v[3] : 0.0f);
            unsigned p[3];
            mlp_split3(c0, c1, p);
#pragma unroll
            for (int q = 0; q < 3; q++) a1[q][h] = p[q];
        }
#pragma unroll
        for (int q = 0; q < 3; q++) a1[q][2] = a1[q][3] = 0u;
        // layer 1 -> ReLU -> layer 2's A operand (three BF16 parts per k-step)
        unsigned a2[4][3][4];
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            const float bb0 = s.b1[nt * 8 + 2 * tq], bb1 = s.b1[nt * 8 + 2 * tq + 1];
            float c[4] = {bb0, bb1, bb0, bb1};
            const unsigned b0 = s.w1[(nt * 8 + gq) * 4 + tq];
#pragma unroll
            for (int q = 0; q < 3; q++) mlp_mma(a1[q], b0, 0u, c);
            unsigned pg[3], pg8[3];
            mlp_split3(fmaxf(c[0], 0.0f), fmaxf(c[1], 0.0f), pg);
            mlp_split3(fmaxf(c[2], 0.0f), fmaxf(c[3], 0.0f), pg8);
            const int kk = nt >> 1, hi = (nt & 1) * 2;
#pragma unroll
            for (int q = 0; q < 3; q++) {
                a2[kk][q][hi] = pg[q];
                a2[kk][q][hi + 1] = pg8[q];
            }
        }
        // layer 2 -> ReLU -> the output weights, summed over this lane's columns
        float yg = 0.0f, yg8 = 0.0f;
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            const float bb0 = s.b2[nt * 8 + 2 * tq], bb1 = s.b2[nt * 8 + 2 * tq + 1];
            float c[4] = {bb0, bb1, bb0, bb1};
#pragma unroll
            for (int kk = 0; kk < 4; kk++) {
                const unsigned *wr = s.w2 + (nt * 8 + gq) * 36 + kk * 8;
                const unsigned b0 = wr[tq], b1 = wr[4 + tq];
#pragma unroll
                for (int q = 0; q < 3; q++) mlp_mma(a2[kk][q], b0, b1, c);
            }
            const float w0 = s.w3[nt * 8 + 2 * tq], w1 = s.w3[nt * 8 + 2 * tq + 1];
            yg = fmaf(w1, fmaxf(c[1], 0.0f), fmaf(w0, fmaxf(c[0], 0.0f), yg));
            yg8 = fmaf(w1, fmaxf(c[3], 0.0f), fmaf(w0, fmaxf(c[2], 0.0f), yg8));
        }
        yg += __shfl_xor_sync(full, yg, 1);
        yg += __shfl_xor_sync(full, yg, 2);
        yg8 += __shfl_xor_sync(full, yg8, 1);
        yg8 += __shfl_xor_sync(full, yg8, 2);
        if (m == 0) {
            y00 = yg;
            y01 = yg8;
        } else {
            y10 = yg;
            y11 = yg8;
        }
    }
    // zone `lane` is row (lane & 15) of tile lane >> 4, held by quad (lane & 7)
    const int src = 4 * (lane & 7);
    const float t00 = __shfl_sync(full, y00, src), t01 = __shfl_sync(full, y01, src);
    const float t10 = __shfl_sync(full, y10, src), t11 = __shfl_sync(full, y11, src);
    const int m = lane >> 4, h = (lane >> 3) & 1;
    const float y = s.b3 + (m == 0 ? (h == 0 ? t00 : t01) : (h == 0 ? t10 : t11));
    return y * s.norm[11] + s.norm[10];
}

} // namespace grmhd
