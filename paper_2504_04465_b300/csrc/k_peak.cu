// Throughput of the FP32 and FP64 fused multiply-add pipes (and of the packed FP32-pair FMA), the compute denominators of the
// roofline of the compute-bound step kernels (the FP64-storage paths, the D2Q37 polynomial
// equilibrium and the Newton-solved equilibria).  Measurement support: the paper has no
// counterpart.
//
// Each thread runs 8 independent FMA chains (enough independent work to hide the pipe latency
// at full occupancy) for `iters` rounds; the grid is one wave of resident blocks on every SM.
// A round is 8 FMAs = 16 floating-point operations per thread.  The coefficients are run-time
// arguments (a < 1, so the chains converge to b / (1 - a) and stay finite) and every chain
// feeds the stored sum, so the compiler can neither fold nor drop the arithmetic.
#include <cuda_runtime.h>

#include <string>

#include "../../include/lbmtree.h"

namespace lbm {
int set_error(int code, const std::string& msg);
}

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* __restrict__ out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = T(threadIdx.x + 37 * j) * T(1e-3);
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// the same with packed FP32 pairs: one fma.rn.f32x2 does two FMAs (4 flops) per thread
__global__ void __launch_bounds__(256) k_fma2_peak(float* __restrict__ out, int iters, float a, float b) {
    float2 x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = make_float2(float(threadIdx.x + 37 * j) * 1e-3f, float(threadIdx.x + 41 * j) * 1e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = __ffma2_rn(x[j], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j].x + x[j].y;
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T, bool PACKED = false>
int measure(int device, int iters, int repeats, double* flop_per_s, float* best_ms) {
    using lbm::set_error;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if constexpr (PACKED) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma2_peak, 256, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak<T>, 256, 0);
    if (sms <= 0 || per_sm <= 0) return set_error(LBM_ERR_CUDA, "occupancy query failed");
    const int blocks = sms * per_sm;
    T* out = nullptr;
    if ((e = cudaMalloc(&out, sizeof(T) * (size_t)blocks * 256)) != cudaSuccess)
        return set_error(LBM_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    cudaStream_t s = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    float best = 0.f;
    for (int r = 0; r <= repeats; ++r) {          // r = 0 is the warm-up launch
        cudaEventRecord(t0, s);
        if constexpr (PACKED) k_fma2_peak<<<blocks, 256, 0, s>>>((float*)out, iters, 0.999f, 1e-4f);
        else k_fma_peak<T><<<blocks, 256, 0, s>>>(out, iters, T(0.999), T(1e-4));
        cudaEventRecord(t1, s);
        if ((e = cudaEventSynchronize(t1)) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0, t1);
        if (r > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaStreamDestroy(s);
    cudaFree(out);
    if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, std::string("peak kernel: ") + cudaGetErrorString(e));
    const double flops = (PACKED ? 32.0 : 16.0) * (double)iters * (double)blocks * 256.0;
    *flop_per_s = flops / (best * 1e-3);
    if (best_ms) *best_ms = best;
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_pipe_peak(int device, int kind, int iters, double* flop_per_s, float* ms) {
    if (!flop_per_s || iters <= 0 || device < 0 || kind < 0 || kind > 2) return lbm::set_error(LBM_ERR_ARG, "bad argument");
    if (kind == 1) return measure<double>(device, iters, 5, flop_per_s, ms);
    if (kind == 2) return measure<float, true>(device, iters, 5, flop_per_s, ms);
    return measure<float>(device, iters, 5, flop_per_s, ms);
}
