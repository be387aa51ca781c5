// D2Q21 compressible double-distribution model with the numerical (max-entropy) equilibrium
// of Eq. exponential solved by Newton-Raphson (FP64, or FP32 in a kernel set of its own), and the
// kinetic shock sensor
// (Appendix A of arXiv 2504.04465).  The multipliers are stored per cell (warm start) and carried
// through coalescence/explosion (Sec. 3.2).  The polynomial guess fits -1 - ln f_poly, f_poly the
// 3rd-order thermal Hermite equilibrium about theta = 2/3 (positive populations only), onto the
// eight basis functions by weighted least squares.
//
// Shared by the translation units that compile its kernel sets.  The constant tables are internal
// to each unit that includes this header; every such unit exports an upload function that fills
// its own copy (k_d2q21.cu calls them all).
#pragma once
#include <type_traits>

#include "kernels_impl.cuh"
#include "mlp.cuh"

namespace lbm {

static __constant__ double cw21[21];
static __constant__ float cw21f[21], cinvw21f[21];   // the weights in FP32 and their reciprocals
static __constant__ double cH21[21][10];
static __constant__ float cH21f[21][10];   // the same in FP32

template <typename R>
__device__ __forceinline__ void poly_guess21(R ux, R uy, R Tt, R* lam) {
    R a[15];
    thermal_moments<R>(R(1), ux, uy, Tt - R(2.0 / 3.0), 3, a);
    poly_guess_fit<21, R>(ux, uy, Tt, [&](int q, R& w) {
        R s = R(0);
#pragma unroll
        for (int k = 0; k < 10; ++k) s += (sizeof(R) == 4 ? R(cH21f[q][k]) : R(cH21[q][k])) * a[k];
        w = sizeof(R) == 4 ? R(cw21f[q]) : R(cw21[q]);
        return w * s;
    }, lam);
}

// N32: Newton in FP32 (the multipliers stay FP64 between steps), else FP64
template <bool N32>
struct D2Q21M {
    static constexpr int D = 2, Q = 21;
    // resident 128-thread blocks per SM the step kernels are compiled for (simple / other blocks)
    static constexpr int MINB_FAST = N32 ? 4 : 2, MINB_GEN = 2;
    // compile occupancy variants for the autotuner: a warm start (few iterations) runs fastest
    // at 32 resident warps, the polynomial and network guesses at 16 (their state spills below
    // 128 registers)
    static constexpr bool TUNE = N32;
    static constexpr int TUNE_V[3] = {62, 82, 84};   // their targets, 10 * interior + general
    static constexpr bool BATCH = false;  // compile the batched multi-case launch
    static constexpr bool DEV = false;
    static constexpr bool HAS_G = true, HAS_LAM = true, RR = false;
    __host__ __device__ static constexpr int cx(int q) { return Lat<21>::cx(q); }
    __host__ __device__ static constexpr int cy(int q) { return Lat<21>::cy(q); }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __device__ static double w(int q) { return cw21[q]; }
    __device__ static float wf(int q) { return cw21f[q]; }
    __device__ static float inv_wf(int q) { return cinvw21f[q]; }
    template <int ST>
    __device__ static void feq(const ModelDev& m, typename Store<ST>::T rho, typename Store<ST>::T ux,
                               typename Store<ST>::T uy, typename Store<ST>::T Tt, double* lam,
                               typename Store<ST>::T* f, int* iters, int* conv) {
        using T = typename Store<ST>::T;
        using R = typename std::conditional<N32, float, double>::type;
        R l[8];
        if (m.guess == 1) {
#pragma unroll
            for (int a = 0; a < 8; ++a) l[a] = R(0);
        } else if (m.guess == 2) {
            poly_guess21<R>(R(ux), R(uy), R(Tt), l);
        } else if (m.guess == 3) {
            mlp_guess<R>(m.mlp, m.T0, m.mlp_m, m.mlp_s, R(ux), R(uy), R(Tt), l);
        } else {
#pragma unroll
            for (int a = 0; a < 8; ++a) l[a] = R(lam[a]);
        }
        R e[21];
        if constexpr (N32) *iters = newton_solve_inl<21, float>(R(ux), R(uy), R(Tt), l, e, R(m.newton_tol), m.newton_max_iter, conv);
        else *iters = newton_solve<21>(R(ux), R(uy), R(Tt), l, e, R(m.newton_tol), m.newton_max_iter, conv);
#pragma unroll
        for (int a = 0; a < 8; ++a) lam[a] = double(l[a]);
#pragma unroll
        for (int q = 0; q < 21; ++q) f[q] = T(R(rho) * e[q]);
    }
    __device__ static void init_guess(double ux, double uy, double Tt, double* lam) { poly_guess21<double>(ux, uy, Tt, lam); }
};

static cudaError_t upload21_here(const double* w21, const double* H21) {
    cudaError_t e;
    if ((e = cudaMemcpyToSymbol(cw21, w21, sizeof(double) * 21)) != cudaSuccess) return e;
    float wf[21], iwf[21];
    for (int q = 0; q < 21; ++q) {
        wf[q] = (float)w21[q];
        iwf[q] = (float)(1.0 / w21[q]);
    }
    if ((e = cudaMemcpyToSymbol(cw21f, wf, sizeof(wf))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(cinvw21f, iwf, sizeof(iwf))) != cudaSuccess) return e;
    float hf[21 * 10];
    for (int i = 0; i < 21 * 10; ++i) hf[i] = (float)H21[i];
    if ((e = cudaMemcpyToSymbol(cH21f, hf, sizeof(hf))) != cudaSuccess) return e;
    return cudaMemcpyToSymbol(cH21, H21, sizeof(double) * 21 * 10);
}


}  // namespace lbm
