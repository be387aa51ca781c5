// D2Q37 compressible double-distribution models (Appendix A of arXiv 2504.04465), shared by the
// translation units that compile their kernel sets.
//
// D2Q37N: the max-entropy equilibrium of Eq. exponential, Newton-solved in FP64 or FP32; its
// polynomial guess uses the per-velocity thermal Hermite table H37[i][k] =
// h_a(xi_x) h_b(xi_y) / (a! b! theta^(a+b)) for component k = (a, b) (weights.cpp).  The
// polynomial-equilibrium model D2Q37M lives in k_d2q37.cu.
//
// The constant tables are internal to each translation unit that includes this header; every
// such unit exports an upload function that fills its own copy (k_d2q37.cu calls them all).
#pragma once
#include <type_traits>

#include "kernels_impl.cuh"
#include "mlp.cuh"

namespace lbm {

static __constant__ double cw37[37];
static __constant__ float cw37f[37], cinvw37f[37];   // the weights in FP32 and their reciprocals
static __constant__ double cH37[37][15];
static __constant__ float cH37f[37][15];   // the same in FP32 (no conversion in the FP32 kernels)
static __constant__ double ccs2_37;
static __constant__ float ccs2_37f;

// ---------------------------------------------------------------- numerical equilibrium
// The max-entropy equilibrium of Eq. exponential on D2Q37 (the paper's lattice for Mach 1.75 to
// 2.5): the same eight constraints and Newton solve as D2Q21, the polynomial guess fitted to the
// 4th-order thermal Hermite equilibrium about c_s^2 of D2Q37 (positive populations only, kept
// where it beats lambda = 0), the learned guess evaluated like D2Q21's.
template <typename R>
__device__ __forceinline__ void poly_guess37(R ux, R uy, R Tt, R* lam) {
    constexpr bool F = sizeof(R) == 4;
    R a[15];
    thermal_moments<R>(R(1), ux, uy, Tt - (F ? R(ccs2_37f) : R(ccs2_37)), 4, a);
    poly_guess_fit<37, R>(ux, uy, Tt, [&](int q, R& w) {
        R s = R(0);
#pragma unroll
        for (int k = 0; k < 15; ++k) s += (F ? R(cH37f[q][k]) : R(cH37[q][k])) * a[k];
        w = F ? R(cw37f[q]) : R(cw37[q]);
        return w * s;
    }, lam);
}

template <bool N32>
struct D2Q37N {
    static constexpr int D = 2, Q = 37;
    // resident 128-thread blocks per SM the step kernels are compiled for (simple / other blocks)
    static constexpr int MINB_FAST = N32 ? 4 : 2, MINB_GEN = 2;
    static constexpr bool TUNE = N32;        // compile occupancy variants for the autotuner
    static constexpr int TUNE_V[3] = {62, 82, 44};   // their targets, 10 * interior + general
    static constexpr bool BATCH = false;
    static constexpr bool DEV = false;
    static constexpr bool HAS_G = true, HAS_LAM = true, RR = false;
    __host__ __device__ static constexpr int cx(int q) { return Lat<37>::cx(q); }
    __host__ __device__ static constexpr int cy(int q) { return Lat<37>::cy(q); }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __device__ static double w(int q) { return cw37[q]; }
    __device__ static float wf(int q) { return cw37f[q]; }
    __device__ static float inv_wf(int q) { return cinvw37f[q]; }
    template <int ST>
    __device__ static void feq(const ModelDev& m, typename Store<ST>::T rho, typename Store<ST>::T ux,
                               typename Store<ST>::T uy, typename Store<ST>::T Tt, double* lam,
                               typename Store<ST>::T* f, int* iters, int* conv) {
        using T = typename Store<ST>::T;
        using R = typename std::conditional<N32, float, double>::type;
        R l[8];
        if (m.guess == 1) {
#pragma unroll
            for (int a2 = 0; a2 < 8; ++a2) l[a2] = R(0);
        } else if (m.guess == 2) {
            poly_guess37<R>(R(ux), R(uy), R(Tt), l);
        } else if (m.guess == 3) {
            mlp_guess<R>(m.mlp, m.T0, m.mlp_m, m.mlp_s, R(ux), R(uy), R(Tt), l);
        } else {
#pragma unroll
            for (int a2 = 0; a2 < 8; ++a2) l[a2] = R(lam[a2]);
        }
        R e[37];
        if constexpr (N32) *iters = newton_solve_inl<37, float>(R(ux), R(uy), R(Tt), l, e, R(m.newton_tol), m.newton_max_iter, conv);
        else *iters = newton_solve<37>(R(ux), R(uy), R(Tt), l, e, R(m.newton_tol), m.newton_max_iter, conv);
#pragma unroll
        for (int a2 = 0; a2 < 8; ++a2) lam[a2] = double(l[a2]);
#pragma unroll
        for (int q = 0; q < 37; ++q) f[q] = T(R(rho) * e[q]);
    }
    __device__ static void init_guess(double ux, double uy, double Tt, double* lam) { poly_guess37<double>(ux, uy, Tt, lam); }
};

static cudaError_t upload37_here(const double* w37, const double* H37, double cs2_37) {
    cudaError_t e;
    if ((e = cudaMemcpyToSymbol(cw37, w37, sizeof(double) * 37)) != cudaSuccess) return e;
    float wf[37], iwf[37];
    for (int q = 0; q < 37; ++q) {
        wf[q] = (float)w37[q];
        iwf[q] = (float)(1.0 / w37[q]);
    }
    if ((e = cudaMemcpyToSymbol(cw37f, wf, sizeof(wf))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(cinvw37f, iwf, sizeof(iwf))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(cH37, H37, sizeof(double) * 37 * 15)) != cudaSuccess) return e;
    float hf[37 * 15];
    for (int i = 0; i < 37 * 15; ++i) hf[i] = (float)H37[i];
    if ((e = cudaMemcpyToSymbol(cH37f, hf, sizeof(hf))) != cudaSuccess) return e;
    const float c2f = (float)cs2_37;
    if ((e = cudaMemcpyToSymbol(ccs2_37f, &c2f, sizeof(float))) != cudaSuccess) return e;
    return cudaMemcpyToSymbol(ccs2_37, &cs2_37, sizeof(double));
}


}  // namespace lbm
