// D2Q37 compressible double-distribution kernels (Appendix A of arXiv 2504.04465): the kernel
// sets of the thermal polynomial equilibrium, the batched equilibrium solve, and the lookup of
// every D2Q37 kernel set.  The Newton-solved sets are compiled in translation units of their
// own (k_d2q37_n64.cu: FP64 Newton; k_d2q37_n32_*.cu: FP32 Newton, one per storage format).
//
// D2Q37M, the thermal polynomial equilibrium with the kinetic shock sensor: the Hermite expansion
// of Eq. GenEq to 4th order about theta = c_s^2 of the lattice with the thermal moments a_k of
// models_comp.cuh, f_eq,i = sum_k w_i h_a(xi_x) h_b(xi_y) / (a! b! theta^(a+b)) a_k over the
// components k = (a, b).  The sum runs per velocity class (X, Y) = (|xi_x|, |xi_y|): h_a is even or
// odd with a, so with the coefficients C[c][k] of the class's positive velocity (weights.cpp) the
// partial sums over the four parity groups of k,
//     ee = sum_{a, b even} C a_k, oe = sum_{a odd, b even}, eo = sum_{a even, b odd}, oo = sum_{a, b odd},
// give all (up to four) velocities (sx X, sy Y) of the class as ee + sx oe + sy eo + sx sy oo:
// about 210 operations per cell instead of the 590 of the per-velocity sum.  The FP32 table is
// rounded so that the reconstruction conserves mass, momentum and energy exactly.
#include "d2q37.cuh"

namespace lbm {

static __constant__ double cC37[13][15];
static __constant__ float cC37f[13][15];
static __constant__ double cth37;
static __constant__ float cth37f;

// index of velocity (x, y) in the lattice order
__host__ __device__ constexpr int q37(int x, int y) {
    for (int q = 0; q < 37; ++q)
        if (Lat<37>::cx(q) == x && Lat<37>::cy(q) == y) return q;
    return -1;
}

// f_eq of the 37 velocities from the thermal moments a (class form above)
template <typename T>
__device__ __forceinline__ void feq37_classes(const T* a, T* f) {
    constexpr bool F = sizeof(T) == 4;
    static_for<13>([&](auto cc) {
        constexpr int c = decltype(cc)::value;
        constexpr int X = d2q37_class_x(c), Y = d2q37_class_y(c);
        auto C = [&](int k) -> T { return F ? T(cC37f[c][k]) : T(cC37[c][k]); };
        const T ee = C(0) * a[0] + C(3) * a[3] + C(5) * a[5] + C(10) * a[10] + C(12) * a[12] + C(14) * a[14];
        if constexpr (X == 0 && Y == 0) {
            f[q37(0, 0)] = ee;
        } else if constexpr (Y == 0) {
            const T oe = C(1) * a[1] + C(6) * a[6] + C(8) * a[8];
            constexpr int qp = q37(X, 0), qm = q37(-X, 0);
            f[qp] = ee + oe;
            f[qm] = ee - oe;
        } else if constexpr (X == 0) {
            const T eo = C(2) * a[2] + C(7) * a[7] + C(9) * a[9];
            constexpr int qp = q37(0, Y), qm = q37(0, -Y);
            f[qp] = ee + eo;
            f[qm] = ee - eo;
        } else {
            const T oe = C(1) * a[1] + C(6) * a[6] + C(8) * a[8];
            const T eo = C(2) * a[2] + C(7) * a[7] + C(9) * a[9];
            const T oo = C(4) * a[4] + C(11) * a[11] + C(13) * a[13];
            const T p = ee + oe, m = ee - oe, po = eo + oo, mo = eo - oo;
            constexpr int q1 = q37(X, Y), q2 = q37(X, -Y), q3 = q37(-X, Y), q4 = q37(-X, -Y);
            f[q1] = p + po;
            f[q2] = p - po;
            f[q3] = m + mo;
            f[q4] = m - mo;
        }
    });
}

struct D2Q37M {
    static constexpr int D = 2, Q = 37;
    // resident 128-thread blocks per SM the step kernels are compiled for (simple / other blocks)
    static constexpr int MINB_FAST = 4, MINB_GEN = 2;
    static constexpr bool TUNE = false;      // compile occupancy variants for the autotuner
    static constexpr bool BATCH = true;   // compile the batched multi-case launch
    static constexpr bool AA = true;      // compile the AA-pattern (in-place) kernels
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
        thermal_moments<T>(rho, ux, uy, Tt - (F ? T(cth37f) : T(cth37)), 4, a);
        feq37_classes<T>(a, f);
        *iters = 0;
        *conv = 1;
    }
    __device__ static void init_guess(double, double, double, double*) {}
};

extern template KernelSet make_set<D2Q37N<false>, ST_F64, 16, 16, 1>();
extern template KernelSet make_set<D2Q37N<false>, ST_F32, 16, 16, 1>();
extern template KernelSet make_set<D2Q37N<false>, ST_F16DEV, 16, 16, 1>();
extern template KernelSet make_set<D2Q37N<true>, ST_F64, 16, 16, 1>();
extern template KernelSet make_set<D2Q37N<true>, ST_F32, 16, 16, 1>();
extern template KernelSet make_set<D2Q37N<true>, ST_F16DEV, 16, 16, 1>();
cudaError_t upload_tables_d2q37_n64(const double*, const double*, double);
cudaError_t upload_tables_d2q37_n32_f64(const double*, const double*, double);
cudaError_t upload_tables_d2q37_n32_f32(const double*, const double*, double);
cudaError_t upload_tables_d2q37_n32_f16(const double*, const double*, double);

// batched equilibrium solve: samples (u_x, u_y, T), guess 1 zero, 2 polynomial, 3 network
__global__ void __launch_bounds__(128) k_newton_batch37(const double* __restrict__ uT, long long n, ModelDev m,
                                                        double* __restrict__ lam_out, int* __restrict__ iters) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double ux = uT[3 * i], uy = uT[3 * i + 1], Tt = uT[3 * i + 2];
    double lam[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (m.guess == 2) poly_guess37<double>(ux, uy, Tt, lam);
    else if (m.guess == 3) mlp_guess<double>(m.mlp, m.T0, m.mlp_m, m.mlp_s, ux, uy, Tt, lam);
    double e[37];
    int conv = 0;
    const int it = newton_solve<37>(ux, uy, Tt, lam, e, m.newton_tol, m.newton_max_iter, &conv);
#pragma unroll
    for (int a2 = 0; a2 < 8; ++a2) lam_out[8 * i + a2] = lam[a2];
    iters[i] = conv ? it : -1;
}

void launch_newton_batch_d2q37(const double* uT, long long n, const ModelDev& m, double* lam, int* iters, cudaStream_t s) {
    if (n) k_newton_batch37<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(uT, n, m, lam, iters);
}

template <bool N32>
static bool numerical_set(int storage, KernelSet& out) {
    switch (storage) {
        case ST_F64: out = make_set<D2Q37N<N32>, ST_F64, 16, 16, 1>(); return true;
        case ST_F32: out = make_set<D2Q37N<N32>, ST_F32, 16, 16, 1>(); return true;
        case ST_F16DEV: out = make_set<D2Q37N<N32>, ST_F16DEV, 16, 16, 1>(); return true;
    }
    return false;
}

bool find_kernels_d2q37(int model, int storage, const int* blk, bool newton_fp32, KernelSet& out) {
    if (blk[0] != 16 || blk[1] != 16 || blk[2] != 1) return false;
    if (model == 4) return newton_fp32 ? numerical_set<true>(storage, out) : numerical_set<false>(storage, out);
    if (model == 3) return pick_storage<D2Q37M, 16, 16, 1>(storage, out);
    return false;
}

cudaError_t upload_tables_d2q37(const double* w37, const double* H37, double cs2_37) {
    double C64[13 * 15], th64, resid;
    float C32[13 * 15], th32;
    d2q37_class_tables(C64, C32, &th64, &th32, &resid);
    cudaError_t e = cudaMemcpyToSymbol(cC37, C64, sizeof(C64));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(cC37f, C32, sizeof(C32));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(cth37, &th64, sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(cth37f, &th32, sizeof(float));
    if (e == cudaSuccess) e = upload37_here(w37, H37, cs2_37);
    if (e == cudaSuccess) e = upload_tables_d2q37_n64(w37, H37, cs2_37);
    if (e == cudaSuccess) e = upload_tables_d2q37_n32_f64(w37, H37, cs2_37);
    if (e == cudaSuccess) e = upload_tables_d2q37_n32_f32(w37, H37, cs2_37);
    if (e == cudaSuccess) e = upload_tables_d2q37_n32_f16(w37, H37, cs2_37);
    return e;
}

}  // namespace lbm
