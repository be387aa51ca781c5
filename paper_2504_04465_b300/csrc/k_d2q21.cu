// D2Q21 compressible double-distribution kernels with the numerical (max-entropy) equilibrium
// of Eq. exponential solved by Newton-Raphson in FP64, and the kinetic shock sensor
// (Appendix A of arXiv 2504.04465).  The multipliers are stored per cell (warm start) and carried
// through coalescence/explosion (Sec. 3.2).  The polynomial guess fits -1 - ln f_poly, f_poly the
// 3rd-order thermal Hermite equilibrium about theta = 2/3 (positive populations only), onto the
// eight basis functions by weighted least squares.
#include "kernels_impl.cuh"
#include "mlp.cuh"

namespace lbm {

static __constant__ double cw21[21];
static __constant__ float cw21f[21], cinvw21f[21];   // the weights in FP32 and their reciprocals
static __constant__ double cH21[21][10];

__device__ __forceinline__ void poly_guess21(double ux, double uy, double Tt, double* lam) {
    double a[15];
    thermal_moments<double>(1.0, ux, uy, Tt - 2.0 / 3.0, 3, a);
    double A[36], b[8];
#pragma unroll
    for (int k = 0; k < 36; ++k) A[k] = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) b[k] = 0.0;
#pragma unroll
    for (int q = 0; q < 21; ++q) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < 10; ++k) s += cH21[q][k] * a[k];
        const double fp = cw21[q] * s;
        if (fp > 0.0) {
            const double y = -1.0 - log(fp);
            const double w = cw21[q];
            int k = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                b[i] += w * MB<21>::m(q, i) * y;
#pragma unroll
                for (int j = 0; j <= i; ++j) A[k++] += w * (MB<21>::m(q, i) * MB<21>::m(q, j));
            }
        }
    }
    double fit[8];
    chol8_solve(A, b, fit);
    // keep the fit where it is finite and closer to the root than lambda = 0 (at large |u| or T
    // far from the lattice temperature the truncated polynomial is a poor start)
    const double u2 = ux * ux + uy * uy, t2 = u2 + 4.0 * Tt;
    const double tgt[8] = {1.0, ux, uy, ux * ux + Tt, ux * uy, uy * uy + Tt, ux * t2, uy * t2};
    bool fin = true;
#pragma unroll
    for (int a = 0; a < 8; ++a) fin = fin && isfinite(fit[a]);
    double e[21], G[8], gf = 0.0, g0 = 0.0;
    if (fin) {
        newton_eval<21>(fit, tgt, e, G);
#pragma unroll
        for (int a = 0; a < 8; ++a) gf += G[a] * G[a];
        const double zero[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        newton_eval<21>(zero, tgt, e, G);
#pragma unroll
        for (int a = 0; a < 8; ++a) g0 += G[a] * G[a];
    }
    const bool keep = fin && (gf < g0);
#pragma unroll
    for (int a = 0; a < 8; ++a) lam[a] = keep ? fit[a] : 0.0;
}

// network guess lambda0 = m + s * y(u_x, u_y, T/T0 - 1)
__device__ __forceinline__ void mlp_guess21(const ModelDev& m, double ux, double uy, double Tt, double* lam) {
    float h1[MLP_H], h2[MLP_H], y[MLP_OUT];
    mlp_eval(m.mlp, (float)ux, (float)uy, (float)(Tt / m.T0 - 1.0), h1, h2, y);
#pragma unroll
    for (int a = 0; a < 8; ++a) lam[a] = m.mlp_m[a] + m.mlp_s[a] * (double)y[a];
}

struct D2Q21M {
    static constexpr int D = 2, Q = 21;
    // resident 128-thread blocks per SM the step kernels are compiled for (simple / other blocks)
    static constexpr int MINB_FAST = 2, MINB_GEN = 2;
    static constexpr bool TUNE = false;      // compile occupancy variants for the autotuner
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
        if (m.guess == 1) {
#pragma unroll
            for (int a = 0; a < 8; ++a) lam[a] = 0.0;
        } else if (m.guess == 2) {
            poly_guess21((double)ux, (double)uy, (double)Tt, lam);
        } else if (m.guess == 3) {
            mlp_guess21(m, (double)ux, (double)uy, (double)Tt, lam);
        }
        if (m.newton_fp32) {
            // single-precision solve (FP32 pipe); the multipliers stay FP64 between steps
            float lf[8], ef[21];
#pragma unroll
            for (int a = 0; a < 8; ++a) lf[a] = (float)lam[a];
            *iters = newton_solve<21, float>((float)ux, (float)uy, (float)Tt, lf, ef, (float)m.newton_tol,
                                             m.newton_max_iter, conv);
#pragma unroll
            for (int a = 0; a < 8; ++a) lam[a] = (double)lf[a];
#pragma unroll
            for (int q = 0; q < 21; ++q) f[q] = T((float)rho * ef[q]);
            return;
        }
        double e[21];
        *iters = newton_solve<21>((double)ux, (double)uy, (double)Tt, lam, e, m.newton_tol, m.newton_max_iter, conv);
#pragma unroll
        for (int q = 0; q < 21; ++q) f[q] = T((double)rho * e[q]);
    }
    __device__ static void init_guess(double ux, double uy, double Tt, double* lam) { poly_guess21(ux, uy, Tt, lam); }
};

// batched equilibrium solve: samples (u_x, u_y, T), guess 1 zero, 2 polynomial, 3 network
__global__ void __launch_bounds__(128) k_newton_batch(const double* __restrict__ uT, long long n, ModelDev m,
                                                      double* __restrict__ lam_out, int* __restrict__ iters) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double ux = uT[3 * i], uy = uT[3 * i + 1], Tt = uT[3 * i + 2];
    double lam[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (m.guess == 2) poly_guess21(ux, uy, Tt, lam);
    else if (m.guess == 3) mlp_guess21(m, ux, uy, Tt, lam);
    double e[21];
    int conv = 0;
    const int it = newton_solve<21>(ux, uy, Tt, lam, e, m.newton_tol, m.newton_max_iter, &conv);
#pragma unroll
    for (int a = 0; a < 8; ++a) lam_out[8 * i + a] = lam[a];
    iters[i] = conv ? it : -1;
}

void launch_newton_batch_d2q21(const double* uT, long long n, const ModelDev& m, double* lam, int* iters, cudaStream_t s) {
    if (n) k_newton_batch<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(uT, n, m, lam, iters);
}

bool find_kernels_d2q21(int model, int storage, const int* blk, KernelSet& out) {
    if (model == 4 && blk[0] == 16 && blk[1] == 16 && blk[2] == 1) return pick_storage<D2Q21M, 16, 16, 1>(storage, out);
    return false;
}

cudaError_t upload_tables_d2q21(const double* w21, const double* H21) {
    cudaError_t e;
    if ((e = cudaMemcpyToSymbol(cw21, w21, sizeof(double) * 21)) != cudaSuccess) return e;
    float wf[21], iwf[21];
    for (int q = 0; q < 21; ++q) {
        wf[q] = (float)w21[q];
        iwf[q] = (float)(1.0 / w21[q]);
    }
    if ((e = cudaMemcpyToSymbol(cw21f, wf, sizeof(wf))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(cinvw21f, iwf, sizeof(iwf))) != cudaSuccess) return e;
    return cudaMemcpyToSymbol(cH21, H21, sizeof(double) * 21 * 10);
}

}  // namespace lbm
