// Small multilayer perceptron used as the initial guess of the Newton solve of the numerical
// equilibrium (an extension beyond the paper).  3 -> 64 -> 64 -> 8 with tanh hidden layers:
//   x = (u_x, u_y, T/T0 - 1),  h1 = tanh(W1 x + b1),  h2 = tanh(W2 h1 + b2),  y = W3 h2 + b3,
//   lambda = m + s * y.
// Parameters are one FP32 vector [W1 (64x3), b1, W2 (64x64), b2, W3 (8x64), b3] (row-major);
// weight matrices are used rounded to bfloat16 (round to nearest even), arithmetic is FP32.
#pragma once
#include <cuda_bf16.h>

namespace lbm {

constexpr int MLP_H = 64, MLP_IN = 3, MLP_OUT = 8;
constexpr int MLP_W1 = 0, MLP_B1 = MLP_W1 + MLP_H * MLP_IN, MLP_W2 = MLP_B1 + MLP_H, MLP_B2 = MLP_W2 + MLP_H * MLP_H,
              MLP_W3 = MLP_B2 + MLP_H, MLP_B3 = MLP_W3 + MLP_OUT * MLP_H, MLP_NP = MLP_B3 + MLP_OUT;

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// forward pass of one sample with parameters P whose weight matrices are already bf16-rounded
__device__ __forceinline__ void mlp_eval(const float* P, float x0, float x1, float x2, float* h1, float* h2, float* y) {
#pragma unroll 4
    for (int j = 0; j < MLP_H; ++j)
        h1[j] = tanhf(fmaf(P[MLP_W1 + 3 * j], x0, fmaf(P[MLP_W1 + 3 * j + 1], x1, fmaf(P[MLP_W1 + 3 * j + 2], x2, P[MLP_B1 + j]))));
#pragma unroll 2
    for (int j = 0; j < MLP_H; ++j) {
        float s = P[MLP_B2 + j];
#pragma unroll 16
        for (int i = 0; i < MLP_H; ++i) s = fmaf(P[MLP_W2 + MLP_H * j + i], h1[i], s);
        h2[j] = tanhf(s);
    }
#pragma unroll
    for (int o = 0; o < MLP_OUT; ++o) {
        float s = P[MLP_B3 + o];
#pragma unroll 16
        for (int i = 0; i < MLP_H; ++i) s = fmaf(P[MLP_W3 + MLP_H * o + i], h2[i], s);
        y[o] = s;
    }
}

// network guess lambda0 = m + s * y(u_x, u_y, T/T0 - 1) for the Newton solve, evaluated without
// per-thread arrays in memory: layer-1 units one at a time into 64 layer-2 accumulators (same
// summation order as mlp_eval).  P holds bf16-rounded weights; mm, ms the output scaling.
template <typename R>
__device__ __forceinline__ void mlp_guess(const float* P, double T0, const double* mm, const double* ms,
                                          R ux, R uy, R Tt, R* lam) {
    const float x0 = (float)ux, x1 = (float)uy, x2 = (float)((double)Tt / T0 - 1.0);
    float acc[MLP_H];
#pragma unroll
    for (int j = 0; j < MLP_H; ++j) acc[j] = __ldg(P + MLP_B2 + j);
#pragma unroll 1
    for (int i = 0; i < MLP_H; ++i) {
        const float h1 = tanhf(fmaf(__ldg(P + MLP_W1 + 3 * i), x0, fmaf(__ldg(P + MLP_W1 + 3 * i + 1), x1,
                               fmaf(__ldg(P + MLP_W1 + 3 * i + 2), x2, __ldg(P + MLP_B1 + i)))));
#pragma unroll
        for (int j = 0; j < MLP_H; ++j) acc[j] = fmaf(__ldg(P + MLP_W2 + MLP_H * j + i), h1, acc[j]);
    }
    float y[MLP_OUT];
#pragma unroll
    for (int o = 0; o < MLP_OUT; ++o) y[o] = __ldg(P + MLP_B3 + o);
#pragma unroll
    for (int j = 0; j < MLP_H; ++j) {
        const float h2 = tanhf(acc[j]);
#pragma unroll
        for (int o = 0; o < MLP_OUT; ++o) y[o] = fmaf(__ldg(P + MLP_W3 + MLP_H * o + j), h2, y[o]);
    }
#pragma unroll
    for (int a = 0; a < MLP_OUT; ++a) lam[a] = R(mm[a] + ms[a] * (double)y[a]);
}

}  // namespace lbm
