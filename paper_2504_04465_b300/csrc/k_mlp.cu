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

// ---------------------------------------------------------------- BF16 tensor-core form
// The 64-wide products (layers 2 and 3 and their gradients) on the tensor cores: warp-level
// mma.sync m16n8k16 with bfloat16 operands and FP32 accumulation.  A warp carries 16 samples
// (the M dimension); layer 1 (three inputs), tanh, the biases and dW1 stay on the FP32 cores.
// Fragments (g = lane / 4, t = lane % 4): A (16 x 16, row-major) holds (g, 2t..2t+1),
// (g+8, 2t..), (g, 2t+8..), (g+8, 2t+8..); B (16 x 8, k x n) holds (2t..2t+1, g) and
// (2t+8..2t+9, g); the FP32 accumulator (16 x 8) holds (g, 2t..2t+1) and (g+8, 2t..2t+1).
// Two adjacent accumulator tiles (columns 0-7 and 8-15) are therefore exactly one A fragment of
// k = 16, so a layer's output feeds the next product from registers.
constexpr int TCW = 4;                       // warps per block
constexpr int TCS = 16 * TCW;                // samples per block

__device__ __forceinline__ void mma_bf16(float* c, const unsigned* a, unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// two values as one register of bfloat16 (the first in the low half)
__device__ __forceinline__ unsigned pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<unsigned*>(&v);
}
__device__ __forceinline__ unsigned pack2h(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}
// A fragments of k-block kb from an accumulator-layout array v[8][4] (64 columns)
__device__ __forceinline__ void a_frag(const float (*v)[4], int kb, unsigned* a) {
    a[0] = pack2(v[2 * kb][0], v[2 * kb][1]);
    a[1] = pack2(v[2 * kb][2], v[2 * kb][3]);
    a[2] = pack2(v[2 * kb + 1][0], v[2 * kb + 1][1]);
    a[3] = pack2(v[2 * kb + 1][2], v[2 * kb + 1][3]);
}

struct TcSmem {
    __nv_bfloat16 w2[MLP_H * MLP_H];         // W2[j][i], rounded
    __nv_bfloat16 w3[MLP_OUT * MLP_H];       // W3[o][i], rounded
    float p1[MLP_W2];                        // W1 (rounded), b1
    float b2[MLP_H], b3[MLP_OUT];
};

__device__ __forceinline__ void tc_load(const float* __restrict__ P, TcSmem& S) {
    for (int k = threadIdx.x; k < MLP_H * MLP_H; k += blockDim.x) S.w2[k] = __float2bfloat16_rn(P[MLP_W2 + k]);
    for (int k = threadIdx.x; k < MLP_OUT * MLP_H; k += blockDim.x) S.w3[k] = __float2bfloat16_rn(P[MLP_W3 + k]);
    for (int k = threadIdx.x; k < MLP_W2; k += blockDim.x) S.p1[k] = k < MLP_B1 ? bf16r(P[k]) : P[k];
    for (int k = threadIdx.x; k < MLP_H; k += blockDim.x) S.b2[k] = P[MLP_B2 + k];
    if (threadIdx.x < MLP_OUT) S.b3[threadIdx.x] = P[MLP_B3 + threadIdx.x];
}

// forward pass of the warp's 16 samples (rows g and g+8 are samples s0 + g, s0 + g + 8):
// h1, h2 (FP32, accumulator layout) and y (accumulator layout, 8 outputs)
__device__ __forceinline__ void tc_forward(const TcSmem& S, const float* x /* [2][3] rows g, g+8 */,
                                           float (*h1)[4], float (*h2)[4], float* y) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int j = 8 * nt + 2 * t + (r & 1);
            const float* xs = x + 3 * (r >> 1);
            h1[nt][r] = tanhf(fmaf(S.p1[MLP_W1 + 3 * j], xs[0], fmaf(S.p1[MLP_W1 + 3 * j + 1], xs[1],
                              fmaf(S.p1[MLP_W1 + 3 * j + 2], xs[2], S.p1[MLP_B1 + j]))));
        }
    // layer 2: h2 = tanh(h1 W2^T + b2)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int j0 = 8 * nt + 2 * t;
        float c[4] = {S.b2[j0], S.b2[j0 + 1], S.b2[j0], S.b2[j0 + 1]};
        const int jn = 8 * nt + g;            // this lane's column of B
#pragma unroll
        for (int kb = 0; kb < 4; ++kb) {
            unsigned a[4];
            a_frag(h1, kb, a);
            const unsigned b0 = *reinterpret_cast<const unsigned*>(S.w2 + jn * MLP_H + 16 * kb + 2 * t);
            const unsigned b1 = *reinterpret_cast<const unsigned*>(S.w2 + jn * MLP_H + 16 * kb + 2 * t + 8);
            mma_bf16(c, a, b0, b1);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) h2[nt][r] = tanhf(c[r]);
    }
    // layer 3: y = h2 W3^T + b3
    y[0] = S.b3[2 * t]; y[1] = S.b3[2 * t + 1]; y[2] = y[0]; y[3] = y[1];
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) {
        unsigned a[4];
        a_frag(h2, kb, a);
        const unsigned b0 = *reinterpret_cast<const unsigned*>(S.w3 + g * MLP_H + 16 * kb + 2 * t);
        const unsigned b1 = *reinterpret_cast<const unsigned*>(S.w3 + g * MLP_H + 16 * kb + 2 * t + 8);
        mma_bf16(y, a, b0, b1);
    }
}

__device__ __forceinline__ void tc_inputs(const double* __restrict__ X, long long n, long long s0, float* x, bool* live) {
    const int g = (threadIdx.x & 31) >> 2;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const long long i = s0 + g + 8 * h;
        live[h] = i < n;
#pragma unroll
        for (int c = 0; c < 3; ++c) x[3 * h + c] = live[h] ? (float)X[3 * i + c] : 0.0f;
    }
}

__global__ void __launch_bounds__(32 * TCW) k_mlp_forward_tc(const float* __restrict__ P, const double* __restrict__ X,
                                                            long long n, float* __restrict__ Y) {
    __shared__ TcSmem S;
    tc_load(P, S);
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const long long s0 = (long long)blockIdx.x * TCS + 16 * w;
    float x[6];
    bool live[2];
    tc_inputs(X, n, s0, x, live);
    float h1[8][4], h2[8][4], y[4];
    tc_forward(S, x, h1, h2, y);
#pragma unroll
    for (int h = 0; h < 2; ++h)
        if (live[h]) {
            const long long i = s0 + g + 8 * h;
            Y[MLP_OUT * i + 2 * t] = y[2 * h];
            Y[MLP_OUT * i + 2 * t + 1] = y[2 * h + 1];
        }
}

// per-block staging of the backward pass, samples of the whole block
struct TcBack {
    __nv_bfloat16 d2[TCS * MLP_H];           // d2[s][j], rounded
    __nv_bfloat16 h1[TCS * MLP_H];           // h1[s][i], rounded
    __nv_bfloat16 h2[TCS * MLP_H];           // h2[s][i], rounded
    __nv_bfloat16 d3[TCS * MLP_OUT];         // d3[s][o], rounded
    float d2f[TCS * MLP_H], d1f[TCS * MLP_H], d3f[TCS * MLP_OUT], x[TCS * 3], loss[TCW];
};

__global__ void __launch_bounds__(32 * TCW) k_mlp_grad_tc(const float* __restrict__ P, const double* __restrict__ X,
                                                         const float* __restrict__ Tg, long long n,
                                                         float* __restrict__ G, float* __restrict__ loss) {
    extern __shared__ unsigned char tc_raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(tc_raw);
    TcBack& B = *reinterpret_cast<TcBack*>(tc_raw + ((sizeof(TcSmem) + 15) / 16) * 16);
    tc_load(P, S);
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const long long s0 = (long long)blockIdx.x * TCS + 16 * w;
    const int ls0 = 16 * w;                  // block-local sample of row 0
    float x[6];
    bool live[2];
    tc_inputs(X, n, s0, x, live);
    float h1[8][4], h2[8][4], y[4];
    tc_forward(S, x, h1, h2, y);
    const float inv_n = 1.0f / (float)n;
    // d3 = (y - t) / n, loss
    float d3[4], l = 0.0f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int h = r >> 1, o = 2 * t + (r & 1);
        const long long i = s0 + g + 8 * h;
        const float e = live[h] ? y[r] - Tg[MLP_OUT * i + o] : 0.0f;
        l = fmaf(e, e, l);
        d3[r] = e * inv_n;
        const int ls = ls0 + g + 8 * h;
        B.d3[MLP_OUT * ls + o] = __float2bfloat16_rn(d3[r]);
        B.d3f[MLP_OUT * ls + o] = d3[r];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if (lane == 0) B.loss[w] = 0.5f * l * inv_n;
    // d2 = (d3 W3) * (1 - h2^2): k = 8 outputs, padded to 16 with zeros
    float d2[8][4];
    {
        const unsigned a[4] = {pack2(d3[0], d3[1]), pack2(d3[2], d3[3]), 0u, 0u};
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int in = 8 * nt + g;
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            const unsigned b0 = pack2h(S.w3[(2 * t) * MLP_H + in], S.w3[(2 * t + 1) * MLP_H + in]);
            mma_bf16(c, a, b0, 0u);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                d2[nt][r] = c[r] * (1.0f - h2[nt][r] * h2[nt][r]);
                const int ls = ls0 + g + 8 * (r >> 1), j = 8 * nt + 2 * t + (r & 1);
                B.d2[MLP_H * ls + j] = __float2bfloat16_rn(d2[nt][r]);
                B.h2[MLP_H * ls + j] = __float2bfloat16_rn(h2[nt][r]);
                B.d2f[MLP_H * ls + j] = d2[nt][r];
            }
        }
    }
    // d1 = (d2 W2) * (1 - h1^2)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int in = 8 * nt + g;
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kb = 0; kb < 4; ++kb) {
            unsigned a[4];
            a_frag(d2, kb, a);
            const int j0 = 16 * kb + 2 * t;
            const unsigned b0 = pack2h(S.w2[j0 * MLP_H + in], S.w2[(j0 + 1) * MLP_H + in]);
            const unsigned b1 = pack2h(S.w2[(j0 + 8) * MLP_H + in], S.w2[(j0 + 9) * MLP_H + in]);
            mma_bf16(c, a, b0, b1);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float d1v = c[r] * (1.0f - h1[nt][r] * h1[nt][r]);
            const int ls = ls0 + g + 8 * (r >> 1), j = 8 * nt + 2 * t + (r & 1);
            B.h1[MLP_H * ls + j] = __float2bfloat16_rn(h1[nt][r]);
            B.d1f[MLP_H * ls + j] = d1v;
        }
    }
    // the block's samples are staged for the products over samples
    if (t == 0) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int c = 0; c < 3; ++c) B.x[3 * (ls0 + g + 8 * h) + c] = x[3 * h + c];
    }
    __syncthreads();
    // dW2[j][i] = sum_s d2[s][j] h1[s][i]: warp w takes rows j = 16w .. 16w + 15
    {
        float acc[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[nt][r] = 0.0f;
        const int jr = 16 * w + g;
#pragma unroll
        for (int ks = 0; ks < TCS / 16; ++ks) {
            const int sa = 16 * ks + 2 * t;
            const unsigned a[4] = {pack2h(B.d2[MLP_H * sa + jr], B.d2[MLP_H * (sa + 1) + jr]),
                                   pack2h(B.d2[MLP_H * sa + jr + 8], B.d2[MLP_H * (sa + 1) + jr + 8]),
                                   pack2h(B.d2[MLP_H * (sa + 8) + jr], B.d2[MLP_H * (sa + 9) + jr]),
                                   pack2h(B.d2[MLP_H * (sa + 8) + jr + 8], B.d2[MLP_H * (sa + 9) + jr + 8])};
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const int in = 8 * nt + g;
                const unsigned b0 = pack2h(B.h1[MLP_H * sa + in], B.h1[MLP_H * (sa + 1) + in]);
                const unsigned b1 = pack2h(B.h1[MLP_H * (sa + 8) + in], B.h1[MLP_H * (sa + 9) + in]);
                mma_bf16(acc[nt], a, b0, b1);
            }
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int j = 16 * w + g + 8 * (r >> 1), i = 8 * nt + 2 * t + (r & 1);
                atomicAdd(&G[MLP_W2 + MLP_H * j + i], acc[nt][r]);
            }
    }
    // dW3[o][i] = sum_s d3[s][o] h2[s][i]: rows o = 0..7 (padded to 16), warp w takes i = 16w .. 16w + 15
    {
        float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int ks = 0; ks < TCS / 16; ++ks) {
            const int sa = 16 * ks + 2 * t;
            const unsigned a[4] = {pack2h(B.d3[MLP_OUT * sa + g], B.d3[MLP_OUT * (sa + 1) + g]), 0u,
                                   pack2h(B.d3[MLP_OUT * (sa + 8) + g], B.d3[MLP_OUT * (sa + 9) + g]), 0u};
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int in = 16 * w + 8 * q + g;
                const unsigned b0 = pack2h(B.h2[MLP_H * sa + in], B.h2[MLP_H * (sa + 1) + in]);
                const unsigned b1 = pack2h(B.h2[MLP_H * (sa + 8) + in], B.h2[MLP_H * (sa + 9) + in]);
                mma_bf16(acc[q], a, b0, b1);
            }
        }
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int r = 0; r < 2; ++r)
                atomicAdd(&G[MLP_W3 + MLP_H * g + 16 * w + 8 * q + 2 * t + r], acc[q][r]);
    }
    // FP32 cores: dW1, b1, b2 (threads 0..63: unit j), b3 (threads 64..71), the loss
    const int tid = threadIdx.x;
    if (tid < MLP_H) {
        float g1[3] = {0.f, 0.f, 0.f}, gb1 = 0.f, gb2 = 0.f;
        for (int s2 = 0; s2 < TCS; ++s2) {
            const float dd1 = B.d1f[MLP_H * s2 + tid];
            g1[0] = fmaf(dd1, B.x[3 * s2], g1[0]);
            g1[1] = fmaf(dd1, B.x[3 * s2 + 1], g1[1]);
            g1[2] = fmaf(dd1, B.x[3 * s2 + 2], g1[2]);
            gb1 += dd1;
            gb2 += B.d2f[MLP_H * s2 + tid];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) atomicAdd(&G[MLP_W1 + 3 * tid + c], g1[c]);
        atomicAdd(&G[MLP_B1 + tid], gb1);
        atomicAdd(&G[MLP_B2 + tid], gb2);
    } else if (tid < MLP_H + MLP_OUT) {
        const int o = tid - MLP_H;
        float gb3 = 0.f;
        for (int s2 = 0; s2 < TCS; ++s2) gb3 += B.d3f[MLP_OUT * s2 + o];
        atomicAdd(&G[MLP_B3 + o], gb3);
    } else if (tid == MLP_H + MLP_OUT) {
        float ls = 0.f;
#pragma unroll
        for (int k = 0; k < TCW; ++k) ls += B.loss[k];
        atomicAdd(loss, ls);
    }
}

size_t grad_tc_smem() { return ((sizeof(TcSmem) + 15) / 16) * 16 + sizeof(TcBack); }

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
        cudaFuncSetAttribute(k_mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_tc_smem());
        attr = true;
    }
    // the gradient of a batch: FP32 cores, or the BF16 tensor-core form
    auto grad = [&](const double* Xg, const float* Tgg, long long m) {
        if (p.tensor_cores)
            k_mlp_grad_tc<<<(unsigned)((m + TCS - 1) / TCS), 32 * TCW, grad_tc_smem(), s>>>(d_master, Xg, Tgg, m, G, L);
        else
            k_mlp_grad<<<(unsigned)((m + GS - 1) / GS), GS, grad_smem(), s>>>(d_master, Xg, Tgg, m, G, L);
    };
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
        grad(Xb, Tb, B);
        const double c1 = 1.0 - std::pow(0.9, step), c2 = 1.0 - std::pow(0.999, step);
        k_mlp_adam<<<(MLP_NP + 255) / 256, 256, 0, s>>>(d_master, G, Mo, Vo, lr, (float)c1, (float)c2);
    }
    k_round_weights<<<(MLP_NP + 255) / 256, 256, 0, s>>>(d_master, d_rounded);
    // loss of the final parameters over the whole sample set
    cudaMemsetAsync(G, 0, sizeof(float) * MLP_NP, s);
    cudaMemsetAsync(L, 0, sizeof(float), s);
    grad(X, Tg, n);
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

int lbm_mlp_forward_tc(const float* d_params, const double* d_x, int64_t n, float* d_y, void* stream) {
    if (!d_params || !d_x || !d_y || n < 0) return set_error(LBM_ERR_ARG, "bad arguments");
    if (n == 0) return LBM_OK;
    k_mlp_forward_tc<<<(unsigned)((n + TCS - 1) / TCS), 32 * TCW, 0, (cudaStream_t)stream>>>(d_params, d_x, n, d_y);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : set_error(LBM_ERR_CUDA, cudaGetErrorString(e));
}

int lbm_mlp_grad_tc(const float* d_params, const double* d_x, const float* d_t, int64_t n, float* d_grad,
                    float* d_loss, void* stream) {
    if (!d_params || !d_x || !d_t || !d_grad || !d_loss || n <= 0) return set_error(LBM_ERR_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_tc_smem());
        attr = true;
    }
    cudaMemsetAsync(d_grad, 0, sizeof(float) * MLP_NP, s);
    cudaMemsetAsync(d_loss, 0, sizeof(float), s);
    k_mlp_grad_tc<<<(unsigned)((n + TCS - 1) / TCS), 32 * TCW, grad_tc_smem(), s>>>(d_params, d_x, d_t, n, d_grad, d_loss);
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
