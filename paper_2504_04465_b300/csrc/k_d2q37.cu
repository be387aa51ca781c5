// D2Q37 compressible double-distribution kernels with the thermal polynomial equilibrium and
// the kinetic shock sensor (Appendix A of arXiv 2504.04465).  The equilibrium is the Hermite
// expansion of Eq. GenEq to 4th order about theta = c_s^2 of the lattice with the thermal
// moments of models_comp.cuh: f_eq,i = w_i sum_k H37[i][k] a_k, where H37[i][k] holds
// h_a(xi_x) h_b(xi_y) / (a! b! theta^(a+b)) for component k = (a, b) (weights.cpp).
#include "kernels_impl.cuh"

namespace lbm {

static __constant__ double cw37[37];
static __constant__ float cw37f[37], cinvw37f[37];   // the weights in FP32 and their reciprocals
static __constant__ double cH37[37][15];
static __constant__ float cH37f[37][15];   // the same in FP32 (no conversion in the FP32 kernels)
static __constant__ double ccs2_37;
static __constant__ float ccs2_37f;

struct D2Q37M {
    static constexpr int D = 2, Q = 37;
    // resident 128-thread blocks per SM the step kernels are compiled for (simple / other blocks)
    static constexpr int MINB_FAST = 4, MINB_GEN = 2;
    static constexpr bool TUNE = false;      // compile occupancy variants for the autotuner
    static constexpr bool BATCH = true;   // compile the batched multi-case launch
    static constexpr bool DEV = false;
    static constexpr bool HAS_G = true, HAS_LAM = false, RR = false;
    __host__ __device__ static constexpr int cx(int q) { return Lat<37>::cx(q); }
    __host__ __device__ static constexpr int cy(int q) { return Lat<37>::cy(q); }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __device__ static double w(int q) { return cw37[q]; }
    __device__ static float wf(int q) { return cw37f[q]; }
    __device__ static float inv_wf(int q) { return cinvw37f[q]; }
    template <int ST>
    __device__ static void feq(const ModelDev&, typename Store<ST>::T rho, typename Store<ST>::T ux,
                               typename Store<ST>::T uy, typename Store<ST>::T Tt, double*,
                               typename Store<ST>::T* f, int* iters, int* conv) {
        using T = typename Store<ST>::T;
        constexpr bool F = sizeof(T) == 4;
        T a[15];
        thermal_moments<T>(rho, ux, uy, Tt - (F ? T(ccs2_37f) : T(ccs2_37)), 4, a);
#pragma unroll
        for (int i = 0; i < 37; ++i) {
            T s = 0;
#pragma unroll
            for (int k = 0; k < 15; ++k) s += (F ? T(cH37f[i][k]) : T(cH37[i][k])) * a[k];
            f[i] = (F ? T(cw37f[i]) : T(cw37[i])) * s;
        }
        *iters = 0;
        *conv = 1;
    }
    __device__ static void init_guess(double, double, double, double*) {}
};

bool find_kernels_d2q37(int model, int storage, const int* blk, KernelSet& out) {
    if (model == 3 && blk[0] == 16 && blk[1] == 16 && blk[2] == 1) return pick_storage<D2Q37M, 16, 16, 1>(storage, out);
    return false;
}

cudaError_t upload_tables_d2q37(const double* w37, const double* H37, double cs2_37) {
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
