// D2Q13 kernels (Appendix A of arXiv 2504.04465; the lattice the paper uses for Mach <= 0.98 and
// on which it chose the sensor constant A): the weakly compressible BGK and recursive-regularized
// models of weak_h3.cuh (every Hermite component to order 3, c_s^2 = 1/2), and the compressible
// double distribution with the numerical (max-entropy) equilibrium of Eq. exponential, the eight
// constraints solved by Newton-Raphson in FP64 or FP32 (the solver of models_comp.cuh), the
// polynomial guess fitted to the 3rd-order thermal Hermite equilibrium about c_s^2.
#include <type_traits>

#include "mlp.cuh"
#include "weak_h3.cuh"

namespace lbm {

// 288 w_i H[i][k] as an integer: 288 w_i is 108, 24, 18, 3 for the classes (0,0), (1,0), (1,1),
// (2,0) (w = 36/96, 8/96, 6/96, 1/96); per axis h_a(xi) / (a! c_s^2a) with c_s^2 = 1/2 is 1, 2 xi,
// 2 xi^2 - 1 and (4 xi^3 - 6 xi) / 3 for a = 0..3, and every product divides exactly.
struct P13 {
    static constexpr int Q = 13;
    static constexpr long DEN = 288;
    static constexpr double CS2 = 0.5;
    __host__ __device__ static constexpr int cx(int q) { return Lat<13>::cx(q); }
    __host__ __device__ static constexpr int cy(int q) { return Lat<13>::cy(q); }
    __host__ __device__ static constexpr int wint(int x, int y) {
        const int a = x < 0 ? -x : x, b = y < 0 ? -y : y;
        return a + b == 0 ? 108 : (a + b == 1 ? 24 : (a == 1 && b == 1 ? 18 : 3));
    }
    __host__ __device__ static constexpr int hnum(int a, int x) {
        return a == 0 ? 1 : a == 1 ? 2 * x : a == 2 ? 2 * x * x - 1 : 4 * x * x * x - 6 * x;
    }
    __host__ __device__ static constexpr int hden(int a) { return a == 3 ? 3 : 1; }
    __host__ __device__ static constexpr int G(int q, int k) {
        return wint(cx(q), cy(q)) * hnum(h3_a(k), cx(q)) * hnum(h3_b(k), cy(q)) / (hden(h3_a(k)) * hden(h3_b(k)));
    }
};
static_assert(h3_table_ok<P13>(), "D2Q13 integer reconstruction table");

// polynomial guess: weighted least squares of -1 - ln f_poly onto the eight monomials, f_poly the
// 3rd-order thermal Hermite equilibrium about theta = c_s^2 = 1/2 (positive populations only,
// kept where it beats lambda = 0)
template <typename R>
__device__ __forceinline__ void poly_guess13(R ux, R uy, R Tt, R* lam) {
    R a[15];
    thermal_moments<R>(R(1), ux, uy, Tt - R(0.5), 3, a);
    poly_guess_fit<13, R>(ux, uy, Tt, [&](int q, R& w) {
        R s = R(0);
#pragma unroll
        for (int k = 0; k < 10; ++k) s += R(P13::G(q, k)) * a[k];
        w = R(double(P13::G(q, 0)) / double(P13::DEN));
        return s / R(P13::DEN);
    }, lam);
}

// N32: Newton in FP32 (the multipliers stay FP64 between steps), else FP64
template <bool N32>
struct D2Q13N {
    static constexpr int D = 2, Q = 13;
    // occupancy targets of the step kernels (simple / other blocks) in units of 128 resident
    // threads per SM
    static constexpr int MINB_FAST = N32 ? 4 : 2, MINB_GEN = 2;
    static constexpr bool TUNE = false, BATCH = false, DEV = false;
    static constexpr bool HAS_G = true, HAS_LAM = true, RR = false;
    __host__ __device__ static constexpr int cx(int q) { return Lat<13>::cx(q); }
    __host__ __device__ static constexpr int cy(int q) { return Lat<13>::cy(q); }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr double w(int q) { return double(P13::G(q, 0)) / double(P13::DEN); }
    __host__ __device__ static constexpr float wf(int q) { return float(w(q)); }
    __host__ __device__ static constexpr float inv_wf(int q) { return float(1.0 / w(q)); }
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
            poly_guess13<R>(R(ux), R(uy), R(Tt), l);
        } else if (m.guess == 3) {
            mlp_guess<R>(m.mlp, m.T0, m.mlp_m, m.mlp_s, R(ux), R(uy), R(Tt), l);
        } else {
#pragma unroll
            for (int a = 0; a < 8; ++a) l[a] = R(lam[a]);
        }
        R e[13];
        if constexpr (N32) *iters = newton_solve_inl<13, float>(R(ux), R(uy), R(Tt), l, e, R(m.newton_tol), m.newton_max_iter, conv);
        else *iters = newton_solve<13>(R(ux), R(uy), R(Tt), l, e, R(m.newton_tol), m.newton_max_iter, conv);
#pragma unroll
        for (int a = 0; a < 8; ++a) lam[a] = double(l[a]);
#pragma unroll
        for (int q = 0; q < 13; ++q) f[q] = T(R(rho) * e[q]);
    }
    __device__ static void init_guess(double ux, double uy, double Tt, double* lam) { poly_guess13<double>(ux, uy, Tt, lam); }
};

// batched equilibrium solve: samples (u_x, u_y, T), guess 1 zero, 2 polynomial, 3 network
__global__ void __launch_bounds__(128) k_newton_batch13(const double* __restrict__ uT, long long n, ModelDev m,
                                                        double* __restrict__ lam_out, int* __restrict__ iters) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double ux = uT[3 * i], uy = uT[3 * i + 1], Tt = uT[3 * i + 2];
    double lam[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (m.guess == 2) poly_guess13<double>(ux, uy, Tt, lam);
    else if (m.guess == 3) mlp_guess<double>(m.mlp, m.T0, m.mlp_m, m.mlp_s, ux, uy, Tt, lam);
    double e[13];
    int conv = 0;
    const int it = newton_solve<13>(ux, uy, Tt, lam, e, m.newton_tol, m.newton_max_iter, &conv);
#pragma unroll
    for (int a = 0; a < 8; ++a) lam_out[8 * i + a] = lam[a];
    iters[i] = conv ? it : -1;
}

void launch_newton_batch_d2q13(const double* uT, long long n, const ModelDev& m, double* lam, int* iters, cudaStream_t s) {
    if (n) k_newton_batch13<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(uT, n, m, lam, iters);
}

// weakly compressible: FP64 and FP32 deviations; numerical: FP64 Newton with FP64 or FP32
// populations, FP32 Newton with FP32 populations
bool find_kernels_d2q13(int model, int storage, const int* blk, bool newton_fp32, KernelSet& out) {
    if (blk[0] != 16 || blk[1] != 16 || blk[2] != 1) return false;
    if (model == 1 || model == 2) {
        if (storage != ST_F64 && storage != ST_F32) return false;
        return model == 1 ? pick_storage<WeakH3<P13, false>, 16, 16, 1>(storage, out)
                          : pick_storage<WeakH3<P13, true>, 16, 16, 1>(storage, out);
    }
    if (model != 4) return false;
    if (newton_fp32) {
        if (storage != ST_F32) return false;
        out = make_set<D2Q13N<true>, ST_F32, 16, 16, 1>();
        return true;
    }
    if (storage == ST_F64) out = make_set<D2Q13N<false>, ST_F64, 16, 16, 1>();
    else if (storage == ST_F32) out = make_set<D2Q13N<false>, ST_F32, 16, 16, 1>();
    else return false;
    return true;
}

}  // namespace lbm
