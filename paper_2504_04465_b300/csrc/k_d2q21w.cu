// D2Q21 weakly compressible BGK and recursive-regularized kernels (Appendix A.2 of arXiv
// 2504.04465): the Hermite equilibrium of Eq. GenEq about T0 = c_s^2 = 2/3 on every tensor
// component up to order 3 (the D2Q21 basis of Tab. lattices_hermite), and the regularized
// collision of Eq. GenRegCollision with the pair-sum non-equilibrium moments of order 2 and 3.
// Populations are stored as deviations f_i - w_i rho_ref, like the D2Q9/D3Q27 sets.
//   f_i = w_i sum_k H[i][k] a_k,  H[i][k] = h_a(xi_x) h_b(xi_y) / (a! b! c_s^(2(a+b))) for
//   component k = (a, b) in the order (0,0) (1,0) (0,1) (2,0) (1,1) (0,2) (3,0) (2,1) (1,2) (0,3).
#include "kernels_impl.cuh"

namespace lbm {

static __constant__ double cw21w[21];
static __constant__ float cw21wf[21], cinvw21wf[21];
static __constant__ double cH21w[21][10];
static __constant__ float cH21wf[21][10];

template <bool RR_>
struct D2Q21W {
    static constexpr int D = 2, Q = 21;
    // occupancy targets of the step kernels (simple / other blocks) in units of 128 resident
    // threads per SM: 4 is two resident 16x16 blocks (512 threads, at most 128 registers each)
    static constexpr int MINB_FAST = 4, MINB_GEN = 2;
    static constexpr bool TUNE = false, BATCH = false, DEV = true;
    static constexpr bool HAS_G = false, HAS_LAM = false, RR = RR_;
    static constexpr bool HERMITE_WEAK = true;   // equilibrium and collision by the tables below
    __host__ __device__ static constexpr int cx(int q) { return Lat<21>::cx(q); }
    __host__ __device__ static constexpr int cy(int q) { return Lat<21>::cy(q); }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __device__ static double w(int q) { return cw21w[q]; }
    __device__ static float wf(int q) { return cw21wf[q]; }
    __device__ static float inv_wf(int q) { return cinvw21wf[q]; }
    template <typename T>
    __device__ static T Hk(int q, int k) { return sizeof(T) == 4 ? T(cH21wf[q][k]) : T(cH21w[q][k]); }
    template <typename T>
    __device__ static T wq(int q) { return sizeof(T) == 4 ? T(cw21wf[q]) : T(cw21w[q]); }

    // 25920 w_i H[i][k] as an integer (exact in FP32 and FP64): 25920 w_i is 7280, 2160, 1920, 504,
    // 60, 16 for the velocity classes (0,0), (1,0), (1,1), (2,0), (2,2), (3,0); per axis the
    // factor h_a(xi) / (a! c_s^2a) with c_s^2 = 2/3 is 1, 3 xi / 2, 3 (3 xi^2 - 2) / 8 and
    // 9 (xi^3 - 2 xi) / 16 for a = 0..3, and every product divides exactly.
    __host__ __device__ static constexpr int wint(int x, int y) {
        const int a = x < 0 ? -x : x, b = y < 0 ? -y : y;
        const int m = a > b ? a : b, n = a > b ? b : a;
        return m == 0 ? 7280 : m == 1 ? (n == 0 ? 2160 : 1920) : m == 2 ? (n == 0 ? 504 : 60) : 16;
    }
    __host__ __device__ static constexpr int hnum(int a, int x) {
        return a == 0 ? 1 : a == 1 ? 3 * x : a == 2 ? 3 * (3 * x * x - 2) : 9 * (x * x * x - 2 * x);
    }
    __host__ __device__ static constexpr int hden(int a) { return a == 0 ? 1 : a == 1 ? 2 : a == 2 ? 8 : 16; }
    __host__ __device__ static constexpr int ka(int k) { return k == 0 ? 0 : k <= 2 ? 2 - k : k <= 5 ? 5 - k : 9 - k; }
    __host__ __device__ static constexpr int kb(int k) { return k == 0 ? 0 : k <= 2 ? k - 1 : k <= 5 ? k - 3 : k - 6; }
    __host__ __device__ static constexpr int G(int q, int k) {
        return wint(cx(q), cy(q)) * hnum(ka(k), cx(q)) * hnum(kb(k), cy(q)) / (hden(ka(k)) * hden(kb(k)));
    }
    // deviations f_i - w_i rho_ref of the expansion with coefficients a (a[0] = rho - rho_ref):
    // f_i = (sum_k G(i, k) a_k) / 25920, one correctly rounded division per population, so the
    // reconstruction carries no rounded weight or Hermite constant (an FP32 table scaled the
    // momentum by 1 + O(1e-8) every step, a drift that grows linearly with the step count)
    template <typename T>
    __device__ static void expand(const T* a, T* f) {
        const T den = T(25920), rden = T(1) / den;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            T s = T(0);
#pragma unroll
            for (int k = 0; k < 10; ++k)
                if (G(q, k) != 0) s += T(G(q, k)) * a[k];
            f[q] = div_den<T>(s, den, rden);
        }
    }
    // equilibrium coefficients rho u^alpha (athermal, T0 = c_s^2), the order-0 one as rho - rho_ref
    template <typename T>
    __device__ static void eq_coeffs(T rho, T drho, T ux, T uy, T* a) {
        a[0] = drho;
        a[1] = rho * ux;
        a[2] = rho * uy;
        a[3] = rho * ux * ux;
        a[4] = rho * ux * uy;
        a[5] = rho * uy * uy;
        a[6] = rho * ux * ux * ux;
        a[7] = rho * ux * ux * uy;
        a[8] = rho * ux * uy * uy;
        a[9] = rho * uy * uy * uy;
    }
    template <typename T>
    __device__ static void feq_dev(T rho, T ux, T uy, T rho_ref, T* f) {
        T a[10];
        eq_coeffs<T>(rho, rho - rho_ref, ux, uy, a);
        expand<T>(a, f);
    }
    // BGK (Eq. CollisionStep) or RR (Eq. GenRegCollision) on deviations; omega = 1 / tau
    template <typename T>
    __device__ static void collide(T* f, T omega, T rho_ref) {
        T drho = 0, jx = 0, jy = 0, sxx = 0, sxy = 0, syy = 0;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const T v = f[q];
            const int x = cx(q), y = cy(q);
            drho += v;
            if (x) jx += T(x) * v;
            if (y) jy += T(y) * v;
            if (x) sxx += T(x * x) * v;
            if (x && y) sxy += T(x * y) * v;
            if (y) syy += T(y * y) * v;
        }
        const T rho = rho_ref + drho;
        const T ir = T(1) / rho;
        const T ux = jx * ir, uy = jy * ir;
        T a[10];
        eq_coeffs<T>(rho, drho, ux, uy, a);
        if constexpr (RR) {
            // Pi_ab = sum H^(2)_ab (f - f_eq); the weights' own H^(2) moments vanish, so with
            // deviations Pi_xx = sum (xi_x^2 - c_s^2) delta - rho u_x^2
            const T cs2 = T(2.0 / 3.0);
            const T keep = T(1) - omega;
            const T pxx = sxx - cs2 * drho - rho * ux * ux;
            const T pxy = sxy - rho * ux * uy;
            const T pyy = syy - cs2 * drho - rho * uy * uy;
            a[3] += keep * pxx;
            a[4] += keep * pxy;
            a[5] += keep * pyy;
            a[6] += keep * (T(3) * pxx * ux);
            a[7] += keep * (pxx * uy + T(2) * pxy * ux);
            a[8] += keep * (pyy * ux + T(2) * pxy * uy);
            a[9] += keep * (T(3) * pyy * uy);
            expand<T>(a, f);
        } else {
            T fe[Q];
            expand<T>(a, fe);
#pragma unroll
            for (int q = 0; q < Q; ++q) f[q] -= omega * (f[q] - fe[q]);
        }
    }
    __device__ static void init_guess(double, double, double, double*) {}
};

// the integer table reproduces the moments of the expansion: component k = (a, b) alone carries
// exactly the monomial moment xi_x^a xi_y^b (sum_i xi^(a,b) G(i, k) = 25920, orthonormality of
// the scaled Hermite basis under the weights) and no lower odd moment
namespace {
template <int K, int PX, int PY>
constexpr long moment21() {
    long s = 0;
    for (int q = 0; q < 21; ++q) {
        long t = D2Q21W<true>::G(q, K);
        for (int i = 0; i < PX; ++i) t *= D2Q21W<true>::cx(q);
        for (int i = 0; i < PY; ++i) t *= D2Q21W<true>::cy(q);
        s += t;
    }
    return s;
}
static_assert(moment21<0, 0, 0>() == 25920 && moment21<1, 1, 0>() == 25920 && moment21<2, 0, 1>() == 25920,
              "D2Q21 integer reconstruction table");
static_assert(moment21<3, 2, 0>() == 25920 && moment21<4, 1, 1>() == 25920 && moment21<6, 3, 0>() == 25920,
              "D2Q21 integer reconstruction table");
static_assert(moment21<0, 1, 0>() == 0 && moment21<3, 1, 0>() == 0 && moment21<7, 2, 1>() == 25920 &&
                  moment21<9, 0, 3>() == 25920,
              "D2Q21 integer reconstruction table");
}  // namespace

bool find_kernels_d2q21w(int model, int storage, const int* blk, KernelSet& out) {
    if (blk[0] != 16 || blk[1] != 16 || blk[2] != 1) return false;
    if (storage != ST_F64 && storage != ST_F32) return false;   // no binary16 form
    if (model == 1) return pick_storage<D2Q21W<false>, 16, 16, 1>(storage, out);
    if (model == 2) return pick_storage<D2Q21W<true>, 16, 16, 1>(storage, out);
    return false;
}

cudaError_t upload_tables_d2q21w(const double* w21, const double* H21) {
    cudaError_t e;
    if ((e = cudaMemcpyToSymbol(cw21w, w21, sizeof(double) * 21)) != cudaSuccess) return e;
    float wf[21], iwf[21], hf[21 * 10];
    for (int q = 0; q < 21; ++q) {
        wf[q] = (float)w21[q];
        iwf[q] = (float)(1.0 / w21[q]);
    }
    for (int i = 0; i < 21 * 10; ++i) hf[i] = (float)H21[i];
    if ((e = cudaMemcpyToSymbol(cw21wf, wf, sizeof(wf))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(cinvw21wf, iwf, sizeof(iwf))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(cH21wf, hf, sizeof(hf))) != cudaSuccess) return e;
    return cudaMemcpyToSymbol(cH21w, H21, sizeof(double) * 21 * 10);
}

}  // namespace lbm
