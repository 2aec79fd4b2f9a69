// mlp.cu -- the learned Newton start on the GPU: seeded training samples of
// the inversion (labels exact: W = Gamma^2 (rho + u + p) of the sampled
// primitives, no Newton needed), the batched forward pass, and one minibatch
// training step (BF16-weight forward, FP32 backward, AdamW on an FP32
// master copy), all written so that a training run is a chain of graph-
// capturable launches with its step counter on the device.
//
// Samples: sample i draws xi_k = counter_uniform(seed, 16 i + k), k = 0..9:
//   zone (floor(xi_0 n1), floor(xi_1 n2)) of the grid, centre metric;
//   rho = 1e-6^(1 - xi_2), u/rho = 1e-4 1e5^xi_3, Gamma = 50^xi_4,
//   sigma = b^2/rho = 1e-3 1e5^xi_5; velocity and field directions from
//   (cos th, ph) = (2 xi - 1, 2 pi xi') with components e^i / sqrt(g_ii),
//   scaled to g_ij ut^i ut^j = Gamma^2 - 1 and b^2 = sigma rho.
#include "kernels.h"
#include "mlp.cuh"

namespace grmhd {

// ----------------------------------------------------------------- samples

__global__ void k_mlp_samples(Grid g, unsigned long long seed, long long first, long long n, double *P, int *loc,
                              double *U, float *feat, float *label)
{
    long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (a >= n) return;
    unsigned long long i = (unsigned long long)(first + a);
    double xi[10];
#pragma unroll
    for (int k = 0; k < 10; k++) xi[k] = counter_uniform(seed, 16ull * i + (unsigned long long)k);
    int i1 = min((int)(xi[0] * g.n1), g.n1 - 1), j1 = min((int)(xi[1] * g.n2), g.n2 - 1);
    const Geo<double> geo = g.gc[midx(g, i1, j1)];
    double rho = exp(log(1e-6) * (1.0 - xi[2]));
    double uu = rho * 1e-4 * exp(log(1e5) * xi[3]);
    double lor = exp(log(50.0) * xi[4]);
    double sigma = 1e-3 * exp(log(1e5) * xi[5]);
    const double gd[3] = {geo.gcov[sym(1, 1)], geo.gcov[sym(2, 2)], geo.gcov[sym(3, 3)]};

    double q[NP];
    q[KRHO] = rho;
    q[KUU] = uu;
    {
        double ct = 2.0 * xi[6] - 1.0, st = sqrt(fmax(0.0, 1.0 - ct * ct)), ph = 2.0 * M_PI * xi[7];
        double e[3] = {st * cos(ph) / sqrt(gd[0]), st * sin(ph) / sqrt(gd[1]), ct / sqrt(gd[2])};
        double n2u = spatial_sq(geo, e[0], e[1], e[2]);
        double us = sqrt(lor * lor - 1.0) / sqrt(n2u);
        for (int c = 0; c < 3; c++) q[KU1 + c] = us * e[c];
    }
    {
        double ct = 2.0 * xi[8] - 1.0, st = sqrt(fmax(0.0, 1.0 - ct * ct)), ph = 2.0 * M_PI * xi[9];
        q[KB1] = st * cos(ph) / sqrt(gd[0]);
        q[KB2] = st * sin(ph) / sqrt(gd[1]);
        q[KB3] = ct / sqrt(gd[2]);
    }
    St<double> s;
    get_state(q, geo, s);
    double lam = sqrt(sigma * rho / s.bsq);
    for (int c = 0; c < 3; c++) q[KB1 + c] *= lam;
    get_state(q, geo, s);
    double Uz[NU];
    prim_to_UF<double, false>(q, geo, s, g.gam, 0, Uz);
    double f[MLP_IN], D;
    mlp_features(Uz, geo, f, D);
    double W = s.gamma * s.gamma * (rho + uu + (g.gam - 1.0) * uu);
    if (P)
        for (int c = 0; c < NP; c++) P[c * n + a] = q[c];
    if (loc) loc[a] = i1 * g.n2 + j1;
    if (U)
        for (int c = 0; c < NU; c++) U[c * n + a] = Uz[c];
    if (feat)
        for (int k = 0; k < MLP_IN; k++) feat[k * n + a] = (float)f[k];
    if (label) label[a] = (float)log(W / D);
}

void launch_mlp_samples(const Grid &g, unsigned long long seed, long long first, long long n, double *P, int *loc,
                        double *U, float *feat, float *label, cudaStream_t s)
{
    if (n > 0)
        k_mlp_samples<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(g, seed, first, n, P, loc, U, feat, label);
}

// ----------------------------------------------------------------- forward

// tensor-core inference, one warp per 32 samples; lanes past n pass the
// feature means and write nothing
__global__ void __launch_bounds__(128) k_mlp_forward(const float *buf, const float *feat, long long n, float *y)
{
    __shared__ MlpSmem s;
    mlp_stage(buf, s);
    __syncthreads();
    const long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool in = a < n;
    float f[MLP_IN];
#pragma unroll
    for (int k = 0; k < MLP_IN; k++) f[k] = in ? feat[k * n + a] : s.norm[k];
    const float r = mlp_log_w_mma(s, f);
    if (in) y[a] = r;
}

void launch_mlp_forward(const float *buf, const float *feat, long long n, float *y, cudaStream_t s)
{
    if (n > 0) k_mlp_forward<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(buf, feat, n, y);
}

// ------------------------------------------------- standardisation moments

// per block: sum and sum of squares of the 5 features and the label
__global__ void k_mlp_moments(const float *feat, const float *label, long long n, double *part)
{
    __shared__ double red[12][4];
    double acc[12];
    for (int c = 0; c < 12; c++) acc[c] = 0.0;
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        for (int c = 0; c < 6; c++) {
            double v = c < 5 ? (double)feat[c * n + a] : (double)label[a];
            acc[2 * c] += v;
            acc[2 * c + 1] += v * v;
        }
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int c = 0; c < 12; c++) {
        double v = acc[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[c][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        double v = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) v += red[threadIdx.x][k];
        part[blockIdx.x * 12 + threadIdx.x] = v;
    }
}

void launch_mlp_moments(const float *feat, const float *label, long long n, double *part, int nblk, cudaStream_t s)
{
    k_mlp_moments<<<nblk, 128, 0, s>>>(feat, label, n, part);
}

// -------------------------------------------------------- parameter setup

// He-uniform weights (bound sqrt(6 / fan_in)), zero biases, linear output
// layer with bound 1 / sqrt(64)
__global__ void k_mlp_init(float *theta, unsigned long long seed)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= MLP_NPARAM) return;
    double u = 2.0 * counter_uniform(seed, (unsigned long long)k) - 1.0;
    float v = 0.0f;
    if (k < TH_B1) v = (float)(u * sqrt(6.0 / MLP_IN));
    else if (k >= TH_W2 && k < TH_B2) v = (float)(u * sqrt(6.0 / MLP_H));
    else if (k >= TH_W3 && k < TH_B3) v = (float)(u / sqrt((double)MLP_H));
    theta[k] = v;
}

__device__ __forceinline__ void pack_one(float *fwd, int k, float v)
{
    __nv_bfloat16 *wb = reinterpret_cast<__nv_bfloat16 *>(fwd + MLP_OFF_W);
    if (k < TH_B1) wb[k - TH_W1] = __float2bfloat16_rn(v);
    else if (k < TH_W2) fwd[MLP_OFF_B1 + (k - TH_B1)] = v;
    else if (k < TH_B2) wb[MLP_NW1 + (k - TH_W2)] = __float2bfloat16_rn(v);
    else if (k < TH_W3) fwd[MLP_OFF_B2 + (k - TH_B2)] = v;
    else if (k < TH_B3) wb[MLP_NW1 + MLP_NW2 + (k - TH_W3)] = __float2bfloat16_rn(v);
    else fwd[MLP_OFF_B3] = v;
}

// the forward buffer's view of theta (weights rounded to BF16, ties to even)
__global__ void k_mlp_pack(const float *theta, float *fwd)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < MLP_NPARAM) pack_one(fwd, k, theta[k]);
}

void launch_mlp_init(float *theta, unsigned long long seed, cudaStream_t s)
{
    k_mlp_init<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(theta, seed);
}

void launch_mlp_pack(const float *theta, float *fwd, cudaStream_t s)
{
    k_mlp_pack<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(theta, fwd);
}

// ------------------------------------------------------- training: gradient
//
// One block takes SB = 32 samples of the minibatch with 128 threads.  The
// three 64-wide products of the pass are register-tiled block GEMMs in shared
// memory (4 x 4 outputs per thread, W2 kept in both orientations so every
// read is a conflict-free row or a float4 broadcast):
//   forward   A2 = H1 W2^T (+ b2), h2 = relu(A2), s = h2 . W3 + b3;
//   backward  ds = 2 (s - t) / B; dh2 = ds W3 [h2 > 0]; dh1 = dh2 W2 [h1 > 0];
//   weights   dW2 = dh2^T H1, dW1 = dh1^T x, db1, db2, dW3 = ds^T h2, db3,
// summed over the block's samples into its own row of part[]; the AdamW
// kernel adds the rows in block order.  Inputs, activations and accumulation
// are FP32, the weights the BF16 values of the forward buffer.
//
// Sample of batch position b at step s: k = s B + b, epoch e = k / n,
// index ((k mod n) mul + e * 0x9E3779B1) mod n with mul coprime with n (one
// permutation of the set per epoch); mul = 1 takes the set in order,
// (k mod n), in every epoch.

constexpr int SB = 32;      // samples per block
constexpr int NT = 128;     // threads per block
constexpr int LDH = 68;     // padded activation row (16-byte aligned)

struct GradArgs {
    const float *fwd, *feat, *label;
    long long n;
    int batch;
    unsigned long long mul;
    const long long *step;
    float *part;
    double *lpart;
};

__global__ void __launch_bounds__(NT) k_mlp_grad(GradArgs A)
{
    extern __shared__ __align__(16) float sm[];
    float *W2R = sm;                   // [o][i]
    float *W2T = W2R + MLP_NW2;        // [i][o]
    float *H1 = W2T + MLP_NW2;         // [SB][LDH]  h1
    float *H2 = H1 + SB * LDH;         // [SB][LDH]  h2
    float *G1 = H2 + SB * LDH;         // [SB][LDH]  dL/da1
    float *W1s = G1 + SB * LDH;        // [64][5]
    float *b1s = W1s + MLP_NW1;        // [64]
    float *b2s = b1s + MLP_H;          // [64]
    float *W3s = b2s + MLP_H;          // [64]
    float *X = W3s + MLP_H;            // [SB][5]
    float *DS = X + SB * MLP_IN;       // [SB]
    __shared__ double lred[NT / 32];

    const float *buf = A.fwd;
    const __nv_bfloat16 *Wb = reinterpret_cast<const __nv_bfloat16 *>(buf + MLP_OFF_W);
    const int tid = threadIdx.x;
    for (int k = tid; k < MLP_NW2; k += NT) {
        float w = __bfloat162float(Wb[MLP_NW1 + k]);
        W2R[k] = w;
        W2T[(k & 63) * MLP_H + (k >> 6)] = w;
    }
    for (int k = tid; k < MLP_NW1; k += NT) W1s[k] = __bfloat162float(Wb[k]);
    if (tid < MLP_H) {
        b1s[tid] = buf[MLP_OFF_B1 + tid];
        b2s[tid] = buf[MLP_OFF_B2 + tid];
        W3s[tid] = __bfloat162float(Wb[MLP_NW1 + MLP_NW2 + tid]);
    }
    // standardised inputs of the block's samples (zero rows past the batch)
    const long long step = *A.step;
    if (tid < SB) {
        const int b = blockIdx.x * SB + tid;
        float x[MLP_IN] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (b < A.batch) {
            long long k = step * (long long)A.batch + b;
            long long e = k / A.n;
            unsigned long long kk = (unsigned long long)(k % A.n);
            unsigned long long off = A.mul == 1ull ? 0ull : (unsigned long long)e * 0x9E3779B1ull;
            long long idx = (long long)((kk * A.mul + off) % (unsigned long long)A.n);
#pragma unroll
            for (int i = 0; i < MLP_IN; i++) x[i] = (A.feat[i * A.n + idx] - buf[i]) / buf[5 + i];
            DS[tid] = (A.label[idx] - buf[10]) / buf[11]; // target, replaced by dL/ds below
        } else {
            DS[tid] = 0.0f;
        }
#pragma unroll
        for (int i = 0; i < MLP_IN; i++) X[tid * MLP_IN + i] = x[i];
    }
    __syncthreads();

    // h1 = relu(W1 x + b1): thread (sample tid/4, outputs 16 (tid%4) .. +16)
    {
        const int s = tid >> 2, o0 = (tid & 3) * 16;
        float x[MLP_IN];
#pragma unroll
        for (int i = 0; i < MLP_IN; i++) x[i] = X[s * MLP_IN + i];
#pragma unroll
        for (int oo = 0; oo < 16; oo++) {
            const int o = o0 + oo;
            float a = b1s[o];
#pragma unroll
            for (int i = 0; i < MLP_IN; i++) a = fmaf(W1s[o * MLP_IN + i], x[i], a);
            H1[s * LDH + o] = fmaxf(a, 0.0f);
        }
    }
    __syncthreads();

    // forward layer 2 and the output: thread (samples 4 (tid/16) .. +4, outputs 4 (tid%16) .. +4)
    const int sb = tid >> 4, ob = tid & 15;
    float r2 = 0.0f;
    {
        float acc[4][4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const float bb = b2s[4 * ob + c];
#pragma unroll
            for (int r = 0; r < 4; r++) acc[r][c] = bb;
        }
#pragma unroll 8
        for (int k = 0; k < MLP_H; k++) {
            const float4 w = *reinterpret_cast<const float4 *>(W2T + k * MLP_H + 4 * ob);
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const float h = H1[(4 * sb + r) * LDH + k];
                acc[r][0] = fmaf(h, w.x, acc[r][0]);
                acc[r][1] = fmaf(h, w.y, acc[r][1]);
                acc[r][2] = fmaf(h, w.z, acc[r][2]);
                acc[r][3] = fmaf(h, w.w, acc[r][3]);
            }
        }
        float y[4];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            y[r] = 0.0f;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const float h2 = fmaxf(acc[r][c], 0.0f);
                H2[(4 * sb + r) * LDH + 4 * ob + c] = h2;
                y[r] = fmaf(W3s[4 * ob + c], h2, y[r]);
            }
        }
        // sum over the 16 threads of the sample group (one half-warp)
#pragma unroll
        for (int off = 8; off > 0; off >>= 1)
#pragma unroll
            for (int r = 0; r < 4; r++) y[r] += __shfl_xor_sync(0xffffffffu, y[r], off);
        if (ob == 0) {
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const int s = 4 * sb + r;
                const bool act = blockIdx.x * SB + s < A.batch;
                const float res = (y[r] + buf[MLP_OFF_B3]) - DS[s];
                r2 += act ? res * res : 0.0f;
                DS[s] = act ? 2.0f * res / (float)A.batch : 0.0f;
            }
        }
    }
    __syncthreads();

    // dh1 = dh2 W2, masked by h1 > 0: thread (samples 4 sb .. +4, inputs 4 ob .. +4)
    {
        float acc[4][4] = {};
        float d[4];
#pragma unroll
        for (int r = 0; r < 4; r++) d[r] = DS[4 * sb + r];
#pragma unroll 4
        for (int o = 0; o < MLP_H; o++) {
            const float4 w = *reinterpret_cast<const float4 *>(W2R + o * MLP_H + 4 * ob);
            const float w3 = W3s[o];
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const float g = H2[(4 * sb + r) * LDH + o] > 0.0f ? d[r] * w3 : 0.0f;
                acc[r][0] = fmaf(g, w.x, acc[r][0]);
                acc[r][1] = fmaf(g, w.y, acc[r][1]);
                acc[r][2] = fmaf(g, w.z, acc[r][2]);
                acc[r][3] = fmaf(g, w.w, acc[r][3]);
            }
        }
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const int s = 4 * sb + r, i = 4 * ob + c;
                G1[s * LDH + i] = H1[s * LDH + i] > 0.0f ? acc[r][c] : 0.0f;
            }
    }
    // loss of the block
    float lv = r2;
    for (int off = 16; off > 0; off >>= 1) lv += __shfl_down_sync(0xffffffffu, lv, off);
    if ((tid & 31) == 0) lred[tid >> 5] = (double)lv;
    __syncthreads();

    float *gout = A.part + (size_t)blockIdx.x * MLP_NPARAM;
    // dW2[o][i] = sum_s dh2[s][o] h1[s][i]: thread (outputs 4 (tid/8) .. +4, inputs 8 (tid%8) .. +8)
    {
        const int o0 = 4 * (tid >> 3), i0 = 8 * (tid & 7);
        float acc[4][8] = {};
        float w3[4];
#pragma unroll
        for (int r = 0; r < 4; r++) w3[r] = W3s[o0 + r];
#pragma unroll 4
        for (int s = 0; s < SB; s++) {
            const float ds = DS[s];
            const float4 h0 = *reinterpret_cast<const float4 *>(H1 + s * LDH + i0);
            const float4 h1 = *reinterpret_cast<const float4 *>(H1 + s * LDH + i0 + 4);
            const float hv[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const float g = H2[s * LDH + o0 + r] > 0.0f ? ds * w3[r] : 0.0f;
#pragma unroll
                for (int c = 0; c < 8; c++) acc[r][c] = fmaf(g, hv[c], acc[r][c]);
            }
        }
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int c = 0; c < 8; c++) gout[TH_W2 + (o0 + r) * MLP_H + i0 + c] = acc[r][c];
    }
    if (tid < MLP_H) {
        // dW1[o][i] = sum_s dh1[s][o] x[s][i]; db1[o] = sum_s dh1[s][o]
        const int o = tid;
        float acc[MLP_IN] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, bsum = 0.0f;
        for (int s = 0; s < SB; s++) {
            const float d1 = G1[s * LDH + o];
            bsum += d1;
#pragma unroll
            for (int i = 0; i < MLP_IN; i++) acc[i] = fmaf(d1, X[s * MLP_IN + i], acc[i]);
        }
#pragma unroll
        for (int i = 0; i < MLP_IN; i++) gout[TH_W1 + o * MLP_IN + i] = acc[i];
        gout[TH_B1 + o] = bsum;
    } else {
        // db2[o] = sum_s dh2[s][o]; dW3[o] = sum_s ds[s] h2[s][o]; db3 = sum_s ds[s]
        const int o = tid - MLP_H;
        const float w3 = W3s[o];
        float b2sum = 0.0f, w3sum = 0.0f, b3sum = 0.0f;
        for (int s = 0; s < SB; s++) {
            const float h = H2[s * LDH + o], d = DS[s];
            b2sum += h > 0.0f ? d * w3 : 0.0f;
            w3sum = fmaf(d, h, w3sum);
            b3sum += d;
        }
        gout[TH_B2 + o] = b2sum;
        gout[TH_W3 + o] = w3sum;
        if (o == 0) gout[TH_B3] = b3sum;
    }
    if (tid == 0) {
        double l = 0.0;
        for (int w = 0; w < NT / 32; w++) l += lred[w];
        A.lpart[blockIdx.x] = l;
    }
}

size_t mlp_grad_smem()
{
    return sizeof(float) * (2 * MLP_NW2 + 3 * SB * LDH + MLP_NW1 + 3 * MLP_H + SB * MLP_IN + SB);
}

int mlp_grad_blocks(int batch) { return (batch + SB - 1) / SB; }

cudaError_t mlp_grad_setup()
{
    return cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_grad_smem());
}

void launch_mlp_grad(const MlpTrainer &T, const float *feat, const float *label, long long n, int batch,
                     unsigned long long mul, cudaStream_t s)
{
    GradArgs A{T.fwd, feat, label, n, batch, mul, T.step, T.part, T.lpart};
    k_mlp_grad<<<mlp_grad_blocks(batch), NT, mlp_grad_smem(), s>>>(A);
}

// ------------------------------------------------------------ training: AdamW
//
// g = sum of the block rows of part[] (FP64, fixed order); bias-corrected
// AdamW (Kingma & Ba 2015; decoupled decay of Loshchilov & Hutter 2019) in
// FP32 on the FP32 master, weight decay on W1, W2, W3 only; learning rate
// constant, or cosine from lr0 to lr_min over total_steps (rate and bias
// corrections formed once per block); then the BF16 forward view.
// The last block to finish advances the device step counter and records
// the mean loss of the step.

struct AdamArgs {
    float *theta, *m, *v, *fwd;
    const float *part;
    const double *lpart;
    int nblk, batch;
    long long *step;
    unsigned int *ticket;
    double *loss_hist;
    long long hist_len;
    MlpHyper h;
};

// sum of the block rows of one parameter: eight independent partial sums
// (so the loads overlap), combined in a fixed order.  T = double for the
// gradient entry point; the optimiser sums in FP32 (the FP64 pipe would put
// 128 dependent-rate adds per warp on every step's critical path).
template <typename T>
__device__ __forceinline__ T sum_rows(const float *part, int nblk, int k)
{
    T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int b = 0;
    for (; b + 8 <= nblk; b += 8)
#pragma unroll
        for (int u = 0; u < 8; u++) acc[u] += (T)part[(size_t)(b + u) * MLP_NPARAM + k];
    for (; b < nblk; b++) acc[0] += (T)part[(size_t)b * MLP_NPARAM + k];
    return ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
}

__global__ void k_mlp_adam(AdamArgs A)
{
    // the step's learning rate and bias corrections, once per block
    __shared__ float sc[3];
    const long long s = *A.step;
    if (threadIdx.x == 0) {
        // FP32 transcendentals: a single thread's FP64 pow/cos chain costs tens of
        // microseconds at the FP64 issue rate, and these scalars need no FP64
        float lr = (float)A.h.lr0;
        if (A.h.total_steps > 0) {
            float fr = fminf((float)s, (float)A.h.total_steps) / (float)A.h.total_steps;
            lr = (float)A.h.lr_min + 0.5f * (float)(A.h.lr0 - A.h.lr_min) * (1.0f + cosf(3.14159265358979f * fr));
        }
        const float t = (float)(s + 1);
        sc[0] = lr;
        sc[1] = 1.0f / (1.0f - powf((float)A.h.b1, t));
        sc[2] = 1.0f / (1.0f - powf((float)A.h.b2, t));
    }
    __syncthreads();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < MLP_NPARAM) {
        const float g = sum_rows<float>(A.part, A.nblk, k);
        const float b1 = (float)A.h.b1, b2 = (float)A.h.b2, lr = sc[0];
        const float m = b1 * A.m[k] + (1.0f - b1) * g;
        const float v = b2 * A.v[k] + (1.0f - b2) * g * g;
        float th = A.theta[k];
        const bool decay = k < TH_B1 || (k >= TH_W2 && k < TH_B2) || (k >= TH_W3 && k < TH_B3);
        if (decay) th -= lr * (float)A.h.wd * th;
        th -= lr * (m * sc[1]) / (sqrtf(v * sc[2]) + (float)A.h.eps);
        A.m[k] = m;
        A.v[k] = v;
        A.theta[k] = th;
        pack_one(A.fwd, k, th);
    }
    // the last block to finish records the step's mean loss and advances the step
    __shared__ unsigned int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(A.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        double l = 0.0;
        for (int b = threadIdx.x; b < A.nblk; b += blockDim.x) l += A.lpart[b];
        for (int off = 16; off > 0; off >>= 1) l += __shfl_down_sync(0xffffffffu, l, off);
        __shared__ double lw[2];
        if ((threadIdx.x & 31) == 0) lw[threadIdx.x >> 5] = l;
        __syncthreads();
        if (threadIdx.x == 0) {
            if (A.loss_hist && A.hist_len > 0) A.loss_hist[s % A.hist_len] = (lw[0] + lw[1]) / (double)A.batch;
            *A.ticket = 0u;
            *A.step = s + 1;
        }
    }
}

void launch_mlp_adam(const MlpTrainer &T, int batch, const MlpHyper &h, cudaStream_t s)
{
    AdamArgs A{T.theta, T.m, T.v, T.fwd, T.part, T.lpart, mlp_grad_blocks(batch), batch,
               T.step, T.ticket, T.loss_hist, T.hist_len, h};
    k_mlp_adam<<<(MLP_NPARAM + 63) / 64, 64, 0, s>>>(A);
}

// gradient of the whole batch without an update (gradient checks)
__global__ void k_mlp_reduce_grad(const float *part, int nblk, float *grad)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= MLP_NPARAM) return;
    grad[k] = (float)sum_rows<double>(part, nblk, k);
}

void launch_mlp_reduce_grad(const MlpTrainer &T, int batch, float *grad, cudaStream_t s)
{
    k_mlp_reduce_grad<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(T.part, mlp_grad_blocks(batch), grad);
}

// ------------------------------------------------------------- evaluation

// per block (one sample per thread): sum of squared and maximum absolute
// error of log(W/D)
__global__ void k_mlp_eval(const float *buf, const float *feat, const float *label, long long n, double *part)
{
    __shared__ double red[2][8];
    long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double se = 0.0, me = 0.0;
    if (a < n) {
        float f[MLP_IN];
#pragma unroll
        for (int k = 0; k < MLP_IN; k++) f[k] = feat[k * n + a];
        double e = (double)mlp_log_w_guess(buf, f) - (double)label[a];
        se = e * e;
        me = fabs(e);
    }
    for (int o = 16; o > 0; o >>= 1) {
        se += __shfl_down_sync(0xffffffffu, se, o);
        me = fmax(me, __shfl_down_sync(0xffffffffu, me, o));
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][w] = se;
        red[1][w] = me;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) {
            sa += red[0][k];
            sb = fmax(sb, red[1][k]);
        }
        part[2 * blockIdx.x] = sa;
        part[2 * blockIdx.x + 1] = sb;
    }
}

int mlp_eval_blocks(long long n) { return (int)((n + 255) / 256); }

void launch_mlp_eval(const float *buf, const float *feat, const float *label, long long n, double *part,
                     cudaStream_t s)
{
    if (n > 0) k_mlp_eval<<<mlp_eval_blocks(n), 256, 0, s>>>(buf, feat, label, n, part);
}
} // namespace grmhd
