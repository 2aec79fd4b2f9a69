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

constexpr int TB = 128; // samples (= threads) per block of the gradient kernel
constexpr int LD = 65;  // padded row of the per-sample activations in shared memory

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

__global__ void k_mlp_forward(const float *buf, const float *feat, long long n, float *y)
{
    long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (a >= n) return;
    float f[MLP_IN];
#pragma unroll
    for (int k = 0; k < MLP_IN; k++) f[k] = feat[k * n + a];
    y[a] = mlp_log_w_guess(buf, f);
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
// One block takes TB samples of the minibatch, one per thread.  Forward:
// h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), s = W3 h2 + b3 with the BF16
// weights expanded to FP32 in shared memory.  Backward of L = (1/B) sum
// (s - t)^2: ds = 2 (s - t) / B, dh2 = ds W3 [a2 > 0], dh1 = W2^T dh2 [a1 > 0].
// Weight gradients of the block are sums over its samples, written to its
// own row of part[]; the AdamW kernel adds the rows in block order.
//
// Sample of batch position b at step s: k = s B + b, epoch e = k / n,
// index ((k mod n) mul + e * 0x9E3779B1) mod n with mul coprime with n (one
// permutation of the set per epoch); mul = 1 takes the set in order,
// (k mod n), in every epoch.

struct GradArgs {
    const float *fwd, *feat, *label;
    long long n;
    int batch;
    unsigned long long mul;
    const long long *step;
    float *part;
    double *lpart;
};

__global__ void __launch_bounds__(TB) k_mlp_grad(GradArgs A)
{
    extern __shared__ float sm[];
    float *W2s = sm;                  // [64][64]
    float *W1s = W2s + MLP_NW2;       // [64][5]
    float *b1s = W1s + MLP_NW1;       // [64]
    float *b2s = b1s + MLP_H;         // [64]
    float *W3s = b2s + MLP_H;         // [64]
    float *H1 = W3s + MLP_H;          // [TB][LD]  h1
    float *H2 = H1 + TB * LD;         // [TB][LD]  h2
    float *G1 = H2 + TB * LD;         // [TB][LD]  dL/da1
    float *X = G1 + TB * LD;          // [TB][5]   standardised inputs
    float *DS = X + TB * MLP_IN;      // [TB]      dL/ds
    __shared__ double lred[TB / 32];

    const float *buf = A.fwd;
    const __nv_bfloat16 *Wb = reinterpret_cast<const __nv_bfloat16 *>(buf + MLP_OFF_W);
    const int tid = threadIdx.x;
    for (int k = tid; k < MLP_NW2; k += TB) W2s[k] = __bfloat162float(Wb[MLP_NW1 + k]);
    for (int k = tid; k < MLP_NW1; k += TB) W1s[k] = __bfloat162float(Wb[k]);
    if (tid < MLP_H) {
        b1s[tid] = buf[MLP_OFF_B1 + tid];
        b2s[tid] = buf[MLP_OFF_B2 + tid];
        W3s[tid] = __bfloat162float(Wb[MLP_NW1 + MLP_NW2 + tid]);
    }
    __syncthreads();

    const int b = blockIdx.x * TB + tid;
    const bool act = b < A.batch;
    float ds = 0.0f, r2 = 0.0f;
    float *h1r = H1 + tid * LD, *h2r = H2 + tid * LD, *g1r = G1 + tid * LD;
    if (act) {
        long long k = *A.step * (long long)A.batch + b;
        long long e = k / A.n;
        unsigned long long kk = (unsigned long long)(k % A.n);
        unsigned long long off = A.mul == 1ull ? 0ull : (unsigned long long)e * 0x9E3779B1ull;
        long long idx = (long long)((kk * A.mul + off) % (unsigned long long)A.n);
        float x[MLP_IN];
#pragma unroll
        for (int i = 0; i < MLP_IN; i++) {
            x[i] = (A.feat[i * A.n + idx] - buf[i]) / buf[5 + i];
            X[tid * MLP_IN + i] = x[i];
        }
        float h1[MLP_H];
#pragma unroll
        for (int o = 0; o < MLP_H; o++) {
            float a = b1s[o];
#pragma unroll
            for (int i = 0; i < MLP_IN; i++) a = fmaf(W1s[o * MLP_IN + i], x[i], a);
            h1[o] = fmaxf(a, 0.0f);
            h1r[o] = h1[o];
        }
        float s = buf[MLP_OFF_B3];
        for (int o = 0; o < MLP_H; o += 4) {
            float a0 = b2s[o], a1 = b2s[o + 1], a2 = b2s[o + 2], a3 = b2s[o + 3];
            const float4 *w0 = reinterpret_cast<const float4 *>(W2s + o * MLP_H);
#pragma unroll
            for (int i = 0; i < MLP_H / 4; i++) {
                float4 p0 = w0[i], p1 = w0[i + 16], p2 = w0[i + 32], p3 = w0[i + 48];
                a0 = fmaf(p0.x, h1[4 * i], fmaf(p0.y, h1[4 * i + 1], fmaf(p0.z, h1[4 * i + 2], fmaf(p0.w, h1[4 * i + 3], a0))));
                a1 = fmaf(p1.x, h1[4 * i], fmaf(p1.y, h1[4 * i + 1], fmaf(p1.z, h1[4 * i + 2], fmaf(p1.w, h1[4 * i + 3], a1))));
                a2 = fmaf(p2.x, h1[4 * i], fmaf(p2.y, h1[4 * i + 1], fmaf(p2.z, h1[4 * i + 2], fmaf(p2.w, h1[4 * i + 3], a2))));
                a3 = fmaf(p3.x, h1[4 * i], fmaf(p3.y, h1[4 * i + 1], fmaf(p3.z, h1[4 * i + 2], fmaf(p3.w, h1[4 * i + 3], a3))));
            }
            float v0 = fmaxf(a0, 0.0f), v1 = fmaxf(a1, 0.0f), v2 = fmaxf(a2, 0.0f), v3 = fmaxf(a3, 0.0f);
            h2r[o] = v0;
            h2r[o + 1] = v1;
            h2r[o + 2] = v2;
            h2r[o + 3] = v3;
            s = fmaf(W3s[o], v0, s);
            s = fmaf(W3s[o + 1], v1, s);
            s = fmaf(W3s[o + 2], v2, s);
            s = fmaf(W3s[o + 3], v3, s);
        }
        float t = (A.label[idx] - buf[10]) / buf[11];
        float r = s - t;
        r2 = r * r;
        ds = 2.0f * r / (float)A.batch;
    } else {
        for (int o = 0; o < MLP_H; o++) h1r[o] = h2r[o] = 0.0f;
        for (int i = 0; i < MLP_IN; i++) X[tid * MLP_IN + i] = 0.0f;
    }
    DS[tid] = ds;

    // dh1 = W2^T dh2, masked by a1 > 0
    if (act) {
        float acc[MLP_H];
#pragma unroll
        for (int i = 0; i < MLP_H; i++) acc[i] = 0.0f;
        for (int o = 0; o < MLP_H; o++) {
            float d2 = h2r[o] > 0.0f ? ds * W3s[o] : 0.0f;
            const float4 *w = reinterpret_cast<const float4 *>(W2s + o * MLP_H);
#pragma unroll
            for (int i = 0; i < MLP_H / 4; i++) {
                float4 p = w[i];
                acc[4 * i] = fmaf(p.x, d2, acc[4 * i]);
                acc[4 * i + 1] = fmaf(p.y, d2, acc[4 * i + 1]);
                acc[4 * i + 2] = fmaf(p.z, d2, acc[4 * i + 2]);
                acc[4 * i + 3] = fmaf(p.w, d2, acc[4 * i + 3]);
            }
        }
#pragma unroll
        for (int i = 0; i < MLP_H; i++) g1r[i] = h1r[i] > 0.0f ? acc[i] : 0.0f;
    } else {
        for (int i = 0; i < MLP_H; i++) g1r[i] = 0.0f;
    }

    // loss of the block
    float lv = r2;
    for (int o = 16; o > 0; o >>= 1) lv += __shfl_down_sync(0xffffffffu, lv, o);
    if ((tid & 31) == 0) lred[tid >> 5] = (double)lv;
    __syncthreads();

    float *gout = A.part + (size_t)blockIdx.x * MLP_NPARAM;
    // dW2[o][i] = sum_t dh2[t][o] h1[t][i]: thread owns row o = tid/2, columns i = tid%2 + 2c
    {
        const int o = tid >> 1, i0 = tid & 1;
        const float w3 = W3s[o];
        float acc[MLP_H / 2];
#pragma unroll
        for (int c = 0; c < MLP_H / 2; c++) acc[c] = 0.0f;
        for (int t = 0; t < TB; t++) {
            float d2 = H2[t * LD + o] > 0.0f ? DS[t] * w3 : 0.0f;
            const float *h = H1 + t * LD + i0;
#pragma unroll
            for (int c = 0; c < MLP_H / 2; c++) acc[c] = fmaf(d2, h[2 * c], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < MLP_H / 2; c++) gout[TH_W2 + o * MLP_H + i0 + 2 * c] = acc[c];
    }
    if (tid < MLP_H) {
        // dW1[o][i] = sum_t dh1[t][o] x[t][i]; db1[o] = sum_t dh1[t][o]
        const int o = tid;
        float acc[MLP_IN] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, bsum = 0.0f;
        for (int t = 0; t < TB; t++) {
            float d1 = G1[t * LD + o];
            bsum += d1;
#pragma unroll
            for (int i = 0; i < MLP_IN; i++) acc[i] = fmaf(d1, X[t * MLP_IN + i], acc[i]);
        }
#pragma unroll
        for (int i = 0; i < MLP_IN; i++) gout[TH_W1 + o * MLP_IN + i] = acc[i];
        gout[TH_B1 + o] = bsum;
    } else {
        // db2[o] = sum_t dh2[t][o]; dW3[o] = sum_t ds[t] h2[t][o]; db3 = sum_t ds[t]
        const int o = tid - MLP_H;
        const float w3 = W3s[o];
        float b2sum = 0.0f, w3sum = 0.0f, b3sum = 0.0f;
        for (int t = 0; t < TB; t++) {
            float h = H2[t * LD + o], d = DS[t];
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
        for (int w = 0; w < TB / 32; w++) l += lred[w];
        A.lpart[blockIdx.x] = l;
    }
}

size_t mlp_grad_smem()
{
    return sizeof(float) * (MLP_NW2 + MLP_NW1 + 3 * MLP_H + 3 * TB * LD + TB * MLP_IN + TB);
}

int mlp_grad_blocks(int batch) { return (batch + TB - 1) / TB; }

cudaError_t mlp_grad_setup()
{
    return cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_grad_smem());
}

void launch_mlp_grad(const MlpTrainer &T, const float *feat, const float *label, long long n, int batch,
                     unsigned long long mul, cudaStream_t s)
{
    GradArgs A{T.fwd, feat, label, n, batch, mul, T.step, T.part, T.lpart};
    k_mlp_grad<<<mlp_grad_blocks(batch), TB, mlp_grad_smem(), s>>>(A);
}

// ------------------------------------------------------------ training: AdamW
//
// g = sum of the block rows of part[] (FP64, block order); bias-corrected
// AdamW (Kingma & Ba 2015; decoupled decay of Loshchilov & Hutter 2019) on
// the FP32 master, weight decay on W1, W2, W3 only; learning rate constant,
// or cosine from lr0 to lr_min over total_steps; then the BF16 forward view.
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

__global__ void k_mlp_adam(AdamArgs A)
{
    const long long s = *A.step;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < MLP_NPARAM) {
        double g = 0.0;
        for (int b = 0; b < A.nblk; b++) g += (double)A.part[(size_t)b * MLP_NPARAM + k];
        double lr = A.h.lr0;
        if (A.h.total_steps > 0) {
            double fr = fmin((double)s, (double)A.h.total_steps) / (double)A.h.total_steps;
            lr = A.h.lr_min + 0.5 * (A.h.lr0 - A.h.lr_min) * (1.0 + cos(M_PI * fr));
        }
        double t = (double)(s + 1);
        double m = A.h.b1 * (double)A.m[k] + (1.0 - A.h.b1) * g;
        double v = A.h.b2 * (double)A.v[k] + (1.0 - A.h.b2) * g * g;
        double mh = m / (1.0 - pow(A.h.b1, t)), vh = v / (1.0 - pow(A.h.b2, t));
        double th = (double)A.theta[k];
        bool decay = k < TH_B1 || (k >= TH_W2 && k < TH_B2) || (k >= TH_W3 && k < TH_B3);
        if (decay) th -= lr * A.h.wd * th;
        th -= lr * mh / (sqrt(vh) + A.h.eps);
        A.m[k] = (float)m;
        A.v[k] = (float)v;
        A.theta[k] = (float)th;
        pack_one(A.fwd, k, (float)th);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int done = atomicAdd(A.ticket, 1u);
        if (done == gridDim.x - 1) {
            double l = 0.0;
            for (int b = 0; b < A.nblk; b++) l += A.lpart[b];
            if (A.loss_hist && A.hist_len > 0) A.loss_hist[s % A.hist_len] = l / (double)A.batch;
            *A.ticket = 0u;
            *A.step = s + 1;
        }
    }
}

void launch_mlp_adam(const MlpTrainer &T, int batch, const MlpHyper &h, cudaStream_t s)
{
    AdamArgs A{T.theta, T.m, T.v, T.fwd, T.part, T.lpart, mlp_grad_blocks(batch), batch,
               T.step, T.ticket, T.loss_hist, T.hist_len, h};
    k_mlp_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(A);
}

// gradient of the whole batch without an update (gradient checks)
__global__ void k_mlp_reduce_grad(const float *part, int nblk, float *grad)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= MLP_NPARAM) return;
    double g = 0.0;
    for (int b = 0; b < nblk; b++) g += (double)part[(size_t)b * MLP_NPARAM + k];
    grad[k] = (float)g;
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
