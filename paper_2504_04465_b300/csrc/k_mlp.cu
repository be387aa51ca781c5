// Batched training and inference kernels of the Newton-guess network (mlp.cuh): forward pass,
// gradient of the loss 1/(2n) sum ||y - t||^2, and an Adam update.  FP32 master parameters,
// bf16-rounded weight matrices in every pass, FP32 accumulation.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/lbmtree.h"
#include "mlp.cuh"

namespace lbm {
int set_error(int code, const std::string& msg);
}

namespace {
using namespace lbm;

constexpr int GS = 64;      // samples (threads) per block of the gradient kernel

// parameters with rounded weight matrices into shared memory
__device__ __forceinline__ void load_params(const float* __restrict__ P, float* sP) {
    for (int k = threadIdx.x; k < MLP_NP; k += blockDim.x) {
        const bool w = (k < MLP_B1) || (k >= MLP_W2 && k < MLP_B2) || (k >= MLP_W3 && k < MLP_B3);
        sP[k] = w ? bf16r(P[k]) : P[k];
    }
}

__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ P, const double* __restrict__ X,
                                                     long long n, float* __restrict__ Y) {
    __shared__ float sP[MLP_NP];
    load_params(P, sP);
    __syncthreads();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float h1[MLP_H], h2[MLP_H], y[MLP_OUT];
    mlp_eval(sP, (float)X[3 * i], (float)X[3 * i + 1], (float)X[3 * i + 2], h1, h2, y);
#pragma unroll
    for (int o = 0; o < MLP_OUT; ++o) Y[MLP_OUT * i + o] = y[o];
}

__global__ void __launch_bounds__(GS) k_mlp_grad(const float* __restrict__ P, const double* __restrict__ X,
                                                 const float* __restrict__ Tg, long long n, float* __restrict__ G,
                                                 float* __restrict__ loss) {
    extern __shared__ float sm[];
    float* sP = sm;                              // MLP_NP
    float* H1 = sP + MLP_NP;                     // GS x 64
    float* H2 = H1 + GS * MLP_H;                 // GS x 64
    float* D2 = H2 + GS * MLP_H;                 // GS x 64
    float* D1 = D2 + GS * MLP_H;                 // GS x 64
    float* D3 = D1 + GS * MLP_H;                 // GS x 8
    float* XS = D3 + GS * MLP_OUT;               // GS x 3
    float* LS = XS + GS * 3;                     // GS
    load_params(P, sP);
    __syncthreads();
    const int t = threadIdx.x;
    const long long i = (long long)blockIdx.x * GS + t;
    const bool live = i < n;
    const float inv_n = 1.0f / (float)n;
    float h1[MLP_H], h2[MLP_H], y[MLP_OUT];
    float x0 = 0, x1 = 0, x2 = 0;
    if (live) {
        x0 = (float)X[3 * i]; x1 = (float)X[3 * i + 1]; x2 = (float)X[3 * i + 2];
    }
    mlp_eval(sP, x0, x1, x2, h1, h2, y);
    float l = 0.0f;
#pragma unroll
    for (int o = 0; o < MLP_OUT; ++o) {
        const float e = live ? y[o] - Tg[MLP_OUT * i + o] : 0.0f;
        l = fmaf(e, e, l);
        D3[MLP_OUT * t + o] = e * inv_n;
    }
    LS[t] = 0.5f * l * inv_n;
    XS[3 * t] = live ? x0 : 0.0f; XS[3 * t + 1] = live ? x1 : 0.0f; XS[3 * t + 2] = live ? x2 : 0.0f;
    // back-propagation for this sample
#pragma unroll 4
    for (int j = 0; j < MLP_H; ++j) {
        float s = 0.0f;
#pragma unroll
        for (int o = 0; o < MLP_OUT; ++o) s = fmaf(D3[MLP_OUT * t + o], sP[MLP_W3 + MLP_H * o + j], s);
        const float d2 = live ? s * (1.0f - h2[j] * h2[j]) : 0.0f;
        D2[MLP_H * t + j] = d2;
        H2[MLP_H * t + j] = live ? h2[j] : 0.0f;
        H1[MLP_H * t + j] = live ? h1[j] : 0.0f;
    }
#pragma unroll 2
    for (int i1 = 0; i1 < MLP_H; ++i1) {
        float s = 0.0f;
#pragma unroll 16
        for (int j = 0; j < MLP_H; ++j) s = fmaf(D2[MLP_H * t + j], sP[MLP_W2 + MLP_H * j + i1], s);
        D1[MLP_H * t + i1] = live ? s * (1.0f - h1[i1] * h1[i1]) : 0.0f;
    }
    __syncthreads();
    // weight gradients summed over the block's samples; thread t owns row t of W1, W2 and
    // column t of W3
    {
        float g2[MLP_H];
#pragma unroll
        for (int k = 0; k < MLP_H; ++k) g2[k] = 0.0f;
        float g1[3] = {0, 0, 0}, gb1 = 0, gb2 = 0, g3[MLP_OUT];
#pragma unroll
        for (int o = 0; o < MLP_OUT; ++o) g3[o] = 0.0f;
        for (int s = 0; s < GS; ++s) {
            const float d2 = D2[MLP_H * s + t], d1 = D1[MLP_H * s + t], h2t = H2[MLP_H * s + t];
#pragma unroll
            for (int k = 0; k < MLP_H; ++k) g2[k] = fmaf(d2, H1[MLP_H * s + k], g2[k]);
            g1[0] = fmaf(d1, XS[3 * s], g1[0]);
            g1[1] = fmaf(d1, XS[3 * s + 1], g1[1]);
            g1[2] = fmaf(d1, XS[3 * s + 2], g1[2]);
            gb1 += d1;
            gb2 += d2;
#pragma unroll
            for (int o = 0; o < MLP_OUT; ++o) g3[o] = fmaf(D3[MLP_OUT * s + o], h2t, g3[o]);
        }
#pragma unroll
        for (int k = 0; k < MLP_H; ++k) atomicAdd(&G[MLP_W2 + MLP_H * t + k], g2[k]);
#pragma unroll
        for (int k = 0; k < 3; ++k) atomicAdd(&G[MLP_W1 + 3 * t + k], g1[k]);
        atomicAdd(&G[MLP_B1 + t], gb1);
        atomicAdd(&G[MLP_B2 + t], gb2);
#pragma unroll
        for (int o = 0; o < MLP_OUT; ++o) atomicAdd(&G[MLP_W3 + MLP_H * o + t], g3[o]);
        if (t < MLP_OUT) {
            float gb3 = 0.0f;
            for (int s = 0; s < GS; ++s) gb3 += D3[MLP_OUT * s + t];
            atomicAdd(&G[MLP_B3 + t], gb3);
        }
        if (t == 0) {
            float ls = 0.0f;
            for (int s = 0; s < GS; ++s) ls += LS[s];
            atomicAdd(loss, ls);
        }
    }
}

__global__ void k_mlp_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ Mo,
                           float* __restrict__ Vo, float lr, float c1, float c2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= MLP_NP) return;
    const float g = G[k];
    const float m = 0.9f * Mo[k] + 0.1f * g;
    const float v = 0.999f * Vo[k] + 0.001f * g * g;
    Mo[k] = m;
    Vo[k] = v;
    P[k] -= lr * (m / c1) / (sqrtf(v / c2) + 1e-8f);
}

// ---------------------------------------------------------------- training on solver equilibria
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// per-output mean and standard deviation of the targets (one block per output, FP64)
__global__ void __launch_bounds__(256) k_lambda_stats(const double* __restrict__ lam, long long n, double* __restrict__ ms) {
    __shared__ double s1[256], s2[256];
    const int a = blockIdx.x;
    double a1 = 0.0, a2 = 0.0;
    for (long long i = threadIdx.x; i < n; i += 256) {
        const double v = lam[MLP_OUT * i + a];
        a1 += v;
        a2 = fma(v, v, a2);
    }
    s1[threadIdx.x] = a1;
    s2[threadIdx.x] = a2;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) { s1[threadIdx.x] += s1[threadIdx.x + w]; s2[threadIdx.x] += s2[threadIdx.x + w]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mean = s1[0] / (double)n;
        const double var = fmax(s2[0] / (double)n - mean * mean, 0.0);
        ms[a] = mean;
        ms[MLP_OUT + a] = fmax(sqrt(var), 1e-12);
    }
}

// features x = (u_x, u_y, T/T0 - 1) and normalised targets (lambda - m) / s
__global__ void k_prepare(const double* __restrict__ uT, const double* __restrict__ lam, long long n, double T0,
                          const double* __restrict__ ms, double* __restrict__ X, float* __restrict__ Tg) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    X[3 * i] = uT[3 * i];
    X[3 * i + 1] = uT[3 * i + 1];
    X[3 * i + 2] = uT[3 * i + 2] / T0 - 1.0;
#pragma unroll
    for (int a = 0; a < MLP_OUT; ++a) Tg[MLP_OUT * i + a] = (float)((lam[MLP_OUT * i + a] - ms[a]) / ms[MLP_OUT + a]);
}

// Glorot-uniform weights from a counter-based hash of (seed, index), zero biases
__global__ void k_init_params(float* __restrict__ P, unsigned long long seed) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= MLP_NP) return;
    float b = 0.0f;
    if (k < MLP_B1) b = sqrtf(6.0f / (MLP_IN + MLP_H));
    else if (k >= MLP_W2 && k < MLP_B2) b = sqrtf(6.0f / (MLP_H + MLP_H));
    else if (k >= MLP_W3 && k < MLP_B3) b = sqrtf(6.0f / (MLP_H + MLP_OUT));
    const double r = (double)(mix64(seed * 0x100000001B3ull + (unsigned long long)k) >> 11) * 0x1.0p-53;
    P[k] = b * (float)(2.0 * r - 1.0);
}

// minibatch of samples drawn with replacement by a hash of (seed, step, slot)
__global__ void k_gather_batch(const double* __restrict__ X, const float* __restrict__ Tg, long long n, int batch,
                               unsigned long long seed, int step, double* __restrict__ Xb, float* __restrict__ Tb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= batch) return;
    const unsigned long long h = mix64(seed ^ mix64(((unsigned long long)step << 32) | (unsigned)i));
    const long long j = (long long)(h % (unsigned long long)n);
#pragma unroll
    for (int c = 0; c < 3; ++c) Xb[3 * i + c] = X[3 * j + c];
#pragma unroll
    for (int a = 0; a < MLP_OUT; ++a) Tb[MLP_OUT * i + a] = Tg[MLP_OUT * j + a];
}

__global__ void k_round_weights(const float* __restrict__ P, float* __restrict__ R) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= MLP_NP) return;
    const bool w = (k < MLP_B1) || (k >= MLP_W2 && k < MLP_B2) || (k >= MLP_W3 && k < MLP_B3);
    R[k] = w ? bf16r(P[k]) : P[k];
}

size_t grad_smem() { return sizeof(float) * (MLP_NP + 4 * GS * MLP_H + GS * MLP_OUT + 4 * GS); }

}  // namespace

namespace lbm {

int mlp_train_device(const double* d_uT, const double* d_lam, int64_t n, double T0, const lbm_mlp_train_params& p,
                     float* d_master, float* d_rounded, double* h_ms, float* h_loss, cudaStream_t s) {
    float *Tg = nullptr, *Tb = nullptr, *G = nullptr, *Mo = nullptr, *Vo = nullptr, *L = nullptr;
    double *X = nullptr, *Xb = nullptr, *ms = nullptr;
    const int B = p.batch;
    auto fail_cuda = [&](cudaError_t e) {
        cudaFree(Tg); cudaFree(Tb); cudaFree(G); cudaFree(Mo); cudaFree(Vo); cudaFree(L);
        cudaFree(X); cudaFree(Xb); cudaFree(ms);
        return set_error(e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, cudaGetErrorString(e));
    };
    cudaError_t e;
    if ((e = cudaMalloc(&X, sizeof(double) * 3 * n)) || (e = cudaMalloc(&Tg, sizeof(float) * MLP_OUT * n)) ||
        (e = cudaMalloc(&Xb, sizeof(double) * 3 * B)) || (e = cudaMalloc(&Tb, sizeof(float) * MLP_OUT * B)) ||
        (e = cudaMalloc(&G, sizeof(float) * MLP_NP)) || (e = cudaMalloc(&Mo, sizeof(float) * MLP_NP)) ||
        (e = cudaMalloc(&Vo, sizeof(float) * MLP_NP)) || (e = cudaMalloc(&L, sizeof(float))) ||
        (e = cudaMalloc(&ms, sizeof(double) * 2 * MLP_OUT)))
        return fail_cuda(e);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem());
        attr = true;
    }
    k_lambda_stats<<<MLP_OUT, 256, 0, s>>>(d_lam, n, ms);
    k_prepare<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d_uT, d_lam, n, T0, ms, X, Tg);
    k_init_params<<<(MLP_NP + 255) / 256, 256, 0, s>>>(d_master, p.seed);
    cudaMemsetAsync(Mo, 0, sizeof(float) * MLP_NP, s);
    cudaMemsetAsync(Vo, 0, sizeof(float) * MLP_NP, s);
    for (int step = 1; step <= p.steps; ++step) {
        // learning rate: linear decay from lr to lr_final over the run
        const double frac = p.steps > 1 ? (double)(step - 1) / (p.steps - 1) : 0.0;
        const float lr = (float)(p.lr + (p.lr_final - p.lr) * frac);
        k_gather_batch<<<(B + 255) / 256, 256, 0, s>>>(X, Tg, n, B, p.seed, step, Xb, Tb);
        cudaMemsetAsync(G, 0, sizeof(float) * MLP_NP, s);
        cudaMemsetAsync(L, 0, sizeof(float), s);
        k_mlp_grad<<<(B + GS - 1) / GS, GS, grad_smem(), s>>>(d_master, Xb, Tb, B, G, L);
        const double c1 = 1.0 - std::pow(0.9, step), c2 = 1.0 - std::pow(0.999, step);
        k_mlp_adam<<<(MLP_NP + 255) / 256, 256, 0, s>>>(d_master, G, Mo, Vo, lr, (float)c1, (float)c2);
    }
    k_round_weights<<<(MLP_NP + 255) / 256, 256, 0, s>>>(d_master, d_rounded);
    // loss of the final parameters over the whole sample set
    cudaMemsetAsync(G, 0, sizeof(float) * MLP_NP, s);
    cudaMemsetAsync(L, 0, sizeof(float), s);
    k_mlp_grad<<<(unsigned)((n + GS - 1) / GS), GS, grad_smem(), s>>>(d_master, X, Tg, n, G, L);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_ms, ms, sizeof(double) * 2 * MLP_OUT, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_loss, L, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(e);
    cudaFree(Tg); cudaFree(Tb); cudaFree(G); cudaFree(Mo); cudaFree(Vo); cudaFree(L);
    cudaFree(X); cudaFree(Xb); cudaFree(ms);
    return LBM_OK;
}

}  // namespace lbm

extern "C" {

int lbm_mlp_forward(const float* d_params, const double* d_x, int64_t n, float* d_y, void* stream) {
    if (!d_params || !d_x || !d_y || n < 0) return set_error(LBM_ERR_ARG, "bad arguments");
    if (n == 0) return LBM_OK;
    k_mlp_forward<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(d_params, d_x, n, d_y);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : set_error(LBM_ERR_CUDA, cudaGetErrorString(e));
}

int lbm_mlp_grad(const float* d_params, const double* d_x, const float* d_t, int64_t n, float* d_grad,
                 float* d_loss, void* stream) {
    if (!d_params || !d_x || !d_t || !d_grad || !d_loss || n <= 0) return set_error(LBM_ERR_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem());
        attr = true;
    }
    cudaMemsetAsync(d_grad, 0, sizeof(float) * MLP_NP, s);
    cudaMemsetAsync(d_loss, 0, sizeof(float), s);
    k_mlp_grad<<<(unsigned)((n + GS - 1) / GS), GS, grad_smem(), s>>>(d_params, d_x, d_t, n, d_grad, d_loss);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : set_error(LBM_ERR_CUDA, cudaGetErrorString(e));
}

int lbm_mlp_adam(float* d_params, const float* d_grad, float* d_m, float* d_v, int step, float lr, void* stream) {
    if (!d_params || !d_grad || !d_m || !d_v || step < 1) return set_error(LBM_ERR_ARG, "bad arguments");
    const double c1 = 1.0 - std::pow(0.9, step), c2 = 1.0 - std::pow(0.999, step);
    k_mlp_adam<<<(MLP_NP + 255) / 256, 256, 0, (cudaStream_t)stream>>>(d_params, d_grad, d_m, d_v, lr, (float)c1, (float)c2);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : set_error(LBM_ERR_CUDA, cudaGetErrorString(e));
}

int lbm_mlp_nparams(void) { return MLP_NP; }

}  // extern "C"
