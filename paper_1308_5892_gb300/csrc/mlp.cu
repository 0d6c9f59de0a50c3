// mlp.cu -- learned inverse cumulative distribution of the drift component of
// a drifting Maxwell-Juttner distribution, used by the loader as method
// PIC_MJ_MLP in place of the table inversion of App. D.
//
// Network: 3 -> 64 -> 64 -> 64 -> 1, tanh on the hidden layers, linear output.
// Inputs  x0 = (log10 theta + 0.5) / 1.5,  x1 = 2 beta0 / 0.95 - 1,
//         x2 = probit(w) / 3   (w the uniform of the marginal, Eq. distr_y);
// output  o, and s = asinh(p_par) = psi + asinh(sqrt(theta)) o, psi = atanh(beta0).
// Parameters, flat FP32: W1[64][3] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[64] b4.
//
// Training, FP32 on the GPU: every step draws a fresh batch from the exact
// loader (table + Newton inversion on a 16 x 12 grid of (theta, beta0)),
// runs one fused forward + backward kernel (one thread per sample,
// activations and deltas in shared memory, per-CTA weight gradients reduced
// in shared memory and added once to global memory) and one Adam step.
// Inference: FP16 weights and activations, FP32 accumulation.
#include <algorithm>
#include <cmath>
#include <vector>

#include <cuda_fp16.h>

#include "mj_common.cuh"

namespace pic {

namespace {

constexpr int H = 64;
constexpr int OW1 = 0, OB1 = OW1 + H * 3, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + H * H,
              OW4 = OB3 + H, OB4 = OW4 + H;
constexpr int NP = OB4 + 1;
static_assert(NP == kMlpParams, "parameter count");
constexpr int kT = 128;          // training threads per CTA, one sample each
constexpr int kS = kT + 1;       // padded row of the feature-major activations

// smem: weights | a1 a2 a3 dA dB [H][kS] | d4 [kT]
__global__ void __launch_bounds__(kT) k_mlp_fwd_bwd(const float *__restrict__ W, const float *__restrict__ X,
                                                    const float *__restrict__ T, int n, float *grad, double *loss) {
    extern __shared__ float sm[];
    float *w = sm;
    float *a1 = w + NP + 3;
    float *a2 = a1 + H * kS;
    float *a3 = a2 + H * kS;
    float *dA = a3 + H * kS;
    float *dB = dA + H * kS;
    float *d4s = dB + H * kS;
    float *xs = d4s + kT;            // [3][kT]
    for (int q = threadIdx.x; q < NP; q += kT) w[q] = W[q];
    const int t = threadIdx.x;
    const int idx = blockIdx.x * kT + t;
    const bool valid = idx < n;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f, target = 0.f;
    if (valid) {
        x0 = X[idx]; x1 = X[n + idx]; x2 = X[2 * n + idx];
        target = T[idx];
    }
    xs[t] = x0; xs[kT + t] = x1; xs[2 * kT + t] = x2;
    __syncthreads();
    // forward: each thread owns column t of the activations
    for (int j = 0; j < H; ++j)
        a1[j * kS + t] = tanhf(w[OB1 + j] + w[OW1 + 3 * j] * x0 + w[OW1 + 3 * j + 1] * x1 + w[OW1 + 3 * j + 2] * x2);
    for (int j = 0; j < H; ++j) {
        float v = w[OB2 + j];
        for (int i = 0; i < H; ++i) v += w[OW2 + H * j + i] * a1[i * kS + t];
        a2[j * kS + t] = tanhf(v);
    }
    float o = w[OB4];
    for (int j = 0; j < H; ++j) {
        float v = w[OB3 + j];
        for (int i = 0; i < H; ++i) v += w[OW3 + H * j + i] * a2[i * kS + t];
        const float a = tanhf(v);
        a3[j * kS + t] = a;
        o += w[OW4 + j] * a;
    }
    // loss = mean over the batch of (o - target)^2; backward
    const float e = valid ? (o - target) : 0.f;
    const float d4 = valid ? 2.f * e / (float)n : 0.f;
    d4s[t] = d4;
    for (int j = 0; j < H; ++j) {
        const float a = a3[j * kS + t];
        dA[j * kS + t] = d4 * w[OW4 + j] * (1.f - a * a);     // layer-3 pre-activation deltas
    }
    for (int i = 0; i < H; ++i) {
        float v = 0.f;
        for (int j = 0; j < H; ++j) v += w[OW3 + H * j + i] * dA[j * kS + t];
        const float a = a2[i * kS + t];
        dB[i * kS + t] = v * (1.f - a * a);                   // layer-2 deltas
    }
    __syncthreads();
    // W3, W2 gradients: sums over the CTA's samples
    for (int q = t; q < H * H; q += kT) {
        const int j = q / H, i = q % H;
        float g3 = 0.f, g2 = 0.f;
        for (int s = 0; s < kT; ++s) {
            g3 += dA[j * kS + s] * a2[i * kS + s];
            g2 += dB[j * kS + s] * a1[i * kS + s];
        }
        atomicAdd(grad + OW3 + q, g3);
        atomicAdd(grad + OW2 + q, g2);
    }
    if (t < H) {
        float gb3 = 0.f, gb2 = 0.f, gw4 = 0.f;
        for (int s = 0; s < kT; ++s) {
            gb3 += dA[t * kS + s];
            gb2 += dB[t * kS + s];
            gw4 += d4s[s] * a3[t * kS + s];
        }
        atomicAdd(grad + OB3 + t, gb3);
        atomicAdd(grad + OB2 + t, gb2);
        atomicAdd(grad + OW4 + t, gw4);
    }
    if (t == 0) {
        float g = 0.f;
        for (int s = 0; s < kT; ++s) g += d4s[s];
        atomicAdd(grad + OB4, g);
    }
    __syncthreads();
    // layer-1 deltas (dA is free again)
    for (int i = 0; i < H; ++i) {
        float v = 0.f;
        for (int j = 0; j < H; ++j) v += w[OW2 + H * j + i] * dB[j * kS + t];
        const float a = a1[i * kS + t];
        dA[i * kS + t] = v * (1.f - a * a);
    }
    __syncthreads();
    if (t < H) {
        float gb1 = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
        for (int s = 0; s < kT; ++s) {
            const float dl = dA[t * kS + s];
            gb1 += dl;
            g0 += dl * xs[s];
            g1 += dl * xs[kT + s];
            g2 += dl * xs[2 * kT + s];
        }
        atomicAdd(grad + OB1 + t, gb1);
        atomicAdd(grad + OW1 + 3 * t, g0);
        atomicAdd(grad + OW1 + 3 * t + 1, g1);
        atomicAdd(grad + OW1 + 3 * t + 2, g2);
    }
    double l = (double)e * (double)e;
    for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
    if ((t & 31) == 0) atomicAdd(loss, l / (double)n);
}

// Adam (Kingma and Ba 2015) with bias correction; zeroes the gradient.
__global__ void k_adam(float *W, float *g, float *m, float *v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const float gq = g[q];
        const float mq = b1 * m[q] + (1.f - b1) * gq;
        const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
        m[q] = mq;
        v[q] = vq;
        W[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
        g[q] = 0.f;
    }
}

__global__ void k_to_half(const float *W, __half *Wh, int n) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) Wh[q] = __float2half_rn(W[q]);
}

// FP16 weights and activations, FP32 accumulation; fully unrolled so the
// activations stay in registers.
__device__ __forceinline__ float mlp_eval_half(const __half *__restrict__ w, float x0, float x1, float x2) {
    __half h1[H], h2[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
        const float v = __half2float(w[OB1 + j]) + __half2float(w[OW1 + 3 * j]) * x0 +
                        __half2float(w[OW1 + 3 * j + 1]) * x1 + __half2float(w[OW1 + 3 * j + 2]) * x2;
        h1[j] = __float2half_rn(tanhf(v));
    }
#pragma unroll
    for (int j = 0; j < H; ++j) {
        float v = __half2float(w[OB2 + j]);
#pragma unroll
        for (int i = 0; i < H; ++i) v += __half2float(w[OW2 + H * j + i]) * __half2float(h1[i]);
        h2[j] = __float2half_rn(tanhf(v));
    }
    float o = __half2float(w[OB4]);
#pragma unroll
    for (int j = 0; j < H; ++j) {
        float v = __half2float(w[OB3 + j]);
#pragma unroll
        for (int i = 0; i < H; ++i) v += __half2float(w[OW3 + H * j + i]) * __half2float(h2[i]);
        o += __half2float(w[OW4 + j]) * __half2float(__float2half_rn(tanhf(v)));
    }
    return o;
}

__device__ __forceinline__ void features(double theta, double beta0, double w, float &x0, float &x1, float &x2) {
    x0 = (float)((log10(theta) + 0.5) / 1.5);
    x1 = (float)(2.0 * beta0 / 0.95 - 1.0);
    x2 = (float)(normcdfinv(w) / 3.0);
}

__global__ void k_mlp_infer(const __half *Wg, const float *X, int n, float *out) {
    __shared__ __align__(16) __half w[NP + 7];
    for (int q = threadIdx.x; q < NP; q += blockDim.x) w[q] = Wg[q];
    __syncthreads();
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x)
        out[idx] = mlp_eval_half(w, X[idx], X[n + idx], X[2 * n + idx]);
}

// Training batch from the exact sampler: a random grid point (theta_k, beta_j)
// and a uniform w per sample, the exact drift component s, and the network
// target o = (s - psi) / asinh(sqrt(theta)).
struct TabSet {
    const double *F;         // ncombo x (kMjTable + 1)
    const double *par;       // ncombo x 8: mu, G0, psi, Z, s0, h, theta, beta0
    int ncombo;
};

__global__ void k_mlp_data(TabSet ts, unsigned long long seed, long long base, int n, float *X, float *T) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double u[6];
        mjk::uniforms6(seed, 7, base + i, u);
        const int k = min((int)(u[0] * ts.ncombo), ts.ncombo - 1);
        const double *p = ts.par + 8 * k;
        mjk::Table tb;
        tb.m = mjk::Marg{p[0], p[1], p[2], p[3]};
        tb.s0 = p[4];
        tb.h = p[5];
        tb.n = kMjTable;
        tb.F = ts.F + (size_t)k * (kMjTable + 1);
        const double w = fmin(fmax(u[1], 1e-7), 1.0 - 1e-7);
        const double y = mjk::inverse_marginal(tb, w);
        const double s = asinh(y);
        float x0, x1, x2;
        features(p[6], p[7], w, x0, x1, x2);
        X[i] = x0; X[n + i] = x1; X[2 * n + i] = x2;
        T[i] = (float)((s - p[2]) / asinh(sqrt(p[6])));
    }
}

// Drift component from the network, for the loader.
struct MlpPar {
    const __half *w;
    double psi, scale;
    __device__ double operator()(const mjk::LoadArgs &a, double wv) const {
        const double wc = fmin(fmax(wv, 1e-7), 1.0 - 1e-7);
        float x0, x1, x2;
        features(a.theta, a.beta0, wc, x0, x1, x2);
        const float o = mlp_eval_half(w, x0, x1, x2);
        return sinh(psi + scale * (double)o);
    }
};

// Drift component of given uniforms, exact or learned (tests and the gain measurement).
__global__ void k_sample_par(mjk::Table tb, MlpPar mp, int use_mlp, double theta, double beta0, const double *wv,
                             int n, double *y) {
    mjk::LoadArgs a{};
    a.theta = theta;
    a.beta0 = beta0;
    a.tab = tb;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] = use_mlp ? mp(a, wv[i]) : mjk::inverse_marginal(tb, wv[i]);
}

}  // namespace

size_t mlp_train_smem() { return sizeof(float) * (NP + 3 + 5 * H * kS + 4 * kT); }

void launch_mlp_fwd_bwd(const float *W, const float *X, const float *T, int n, float *grad, double *loss,
                        cudaStream_t s) {
    const size_t smem = mlp_train_smem();
    cudaFuncSetAttribute(k_mlp_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_mlp_fwd_bwd<<<(n + kT - 1) / kT, kT, smem, s>>>(W, X, T, n, grad, loss);
}

void launch_adam(float *W, float *g, float *m, float *v, int step, float lr, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<(NP + 255) / 256, 256, 0, s>>>(W, g, m, v, NP, lr, b1, b2, 1e-8f, c1, c2);
}

void launch_mlp_to_half(const float *W, void *Wh, cudaStream_t s) {
    k_to_half<<<(NP + 255) / 256, 256, 0, s>>>(W, (__half *)Wh, NP);
}

void launch_mlp_infer(const void *Wh, const float *X, int n, float *out, cudaStream_t s) {
    if (n <= 0) return;
    const int blocks = std::min((n + 255) / 256, 152 * 8);
    k_mlp_infer<<<blocks, 256, 0, s>>>((const __half *)Wh, X, n, out);
}

void launch_mlp_data(const double *F, const double *par, int ncombo, unsigned long long seed, long long base, int n,
                     float *X, float *T, cudaStream_t s) {
    TabSet ts{F, par, ncombo};
    const int blocks = std::min((n + 255) / 256, 152 * 8);
    k_mlp_data<<<blocks, 256, 0, s>>>(ts, seed, base, n, X, T);
}

void launch_sample_par(const double *F, double s0, double h, double psi, double Z, const void *Wh, int use_mlp,
                       double theta, double beta0, const double *w, int n, double *y, cudaStream_t s) {
    mjk::Table tb;
    const double mu = 1.0 / theta;
    const double G0 = 1.0 / std::sqrt(1.0 - beta0 * beta0);
    tb.m = mjk::Marg{mu, G0, psi, Z};
    tb.s0 = s0;
    tb.h = h;
    tb.n = kMjTable;
    tb.F = F;
    MlpPar mp{(const __half *)Wh, std::atanh(beta0), std::asinh(std::sqrt(theta))};
    const int blocks = std::max(1, std::min((n + 255) / 256, 152 * 16));
    k_sample_par<<<blocks, 256, 0, s>>>(tb, mp, use_mlp, theta, beta0, w, n, y);
}

void launch_load_mj_mlp(const Geom &g, int ndim, long long n, int species, unsigned long long seed, int profile,
                        double L, double x0, double theta, const double beta[3], const void *Wh, int colocate,
                        Species64 d64, Species64 c64, SpeciesMixed dmx, SpeciesMixed cmx, int mixed, int *err,
                        cudaStream_t s) {
    mjk::LoadArgs a = mjk::make_load_args(g, ndim, n, species, seed, profile, L, x0, theta, beta, 0, nullptr, 0.0, 0.0,
                                          0, 0.0, 1.0, colocate, d64, c64, dmx, cmx, mixed, err);
    MlpPar mp{(const __half *)Wh, std::atanh(a.beta0), std::asinh(std::sqrt(theta))};
    if (n <= 0) return;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    mjk::k_load_mj<MlpPar><<<blocks, 256, 0, s>>>(a, mp);
}

}  // namespace pic
