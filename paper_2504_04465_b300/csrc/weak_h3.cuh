// Weakly compressible BGK and recursive-regularized models on lattices whose Hermite basis is
// every tensor component up to order 3 (D2Q13 and D2Q21, Appendix A, Tab. lattices_hermite of
// arXiv 2504.04465): the equilibrium of Eq. GenEq about T0 = c_s^2 of the lattice and the
// regularized collision of Eq. GenRegCollision with the pair-sum non-equilibrium moments of
// orders 2 and 3 (reading R5).  Populations are stored as deviations f_i - w_i rho_ref.
//
// A lattice policy P gives the velocity set and an integer form of its weights and Hermite
// factors: P::G(i, k) = P::DEN w_i h_a(xi_x) h_b(xi_y) / (a! b! c_s^(2(a+b))) for component
// k = (a, b) in the order (0,0) (1,0) (0,1) (2,0) (1,1) (0,2) (3,0) (2,1) (1,2) (0,3), an exact
// integer, so that f_i = (sum_k G(i, k) a_k) / DEN carries no rounded weight or Hermite constant
// (an FP32 table scales the conserved moments by 1 + O(1e-8) every step, a drift that grows with
// the step count).
#pragma once
#include "kernels_impl.cuh"

namespace lbm {

// component k -> (a, b)
__host__ __device__ constexpr int h3_a(int k) { return k == 0 ? 0 : k <= 2 ? 2 - k : k <= 5 ? 5 - k : 9 - k; }
__host__ __device__ constexpr int h3_b(int k) { return k == 0 ? 0 : k <= 2 ? k - 1 : k <= 5 ? k - 3 : k - 6; }

template <class P, bool RR_>
struct WeakH3 {
    static constexpr int D = 2, Q = P::Q;
    // occupancy targets of the step kernels (simple / other blocks) in units of 128 resident
    // threads per SM: 4 is two resident 16x16 blocks (512 threads, at most 128 registers each)
    static constexpr int MINB_FAST = 4, MINB_GEN = 2;
    static constexpr bool TUNE = false, BATCH = false, DEV = true;
    static constexpr bool HAS_G = false, HAS_LAM = false, RR = RR_;
    static constexpr bool HERMITE_WEAK = true;   // equilibrium and collision by the tables below
    __host__ __device__ static constexpr int cx(int q) { return P::cx(q); }
    __host__ __device__ static constexpr int cy(int q) { return P::cy(q); }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr double w(int q) { return double(P::G(q, 0)) / double(P::DEN); }
    __host__ __device__ static constexpr float wf(int q) { return float(w(q)); }
    __host__ __device__ static constexpr float inv_wf(int q) { return float(1.0 / w(q)); }

    // deviations f_i - w_i rho_ref of the expansion with coefficients a (a[0] = rho - rho_ref),
    // one correctly rounded division per population
    template <typename T>
    __device__ static void expand(const T* a, T* f) {
        const T den = T(P::DEN), rden = T(1) / den;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            T s = T(0);
#pragma unroll
            for (int k = 0; k < 10; ++k)
                if (P::G(q, k) != 0) s += T(P::G(q, k)) * a[k];
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
            const T cs2 = T(P::CS2);
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

// sum over the lattice of G(i, K) xi_x^PX xi_y^PY (exact integers)
template <class P, int K, int PX, int PY>
constexpr long h3_moment() {
    long s = 0;
    for (int q = 0; q < P::Q; ++q) {
        long t = P::G(q, K);
        for (int i = 0; i < PX; ++i) t *= P::cx(q);
        for (int i = 0; i < PY; ++i) t *= P::cy(q);
        s += t;
    }
    return s;
}

// the moments the collision relies on: component k = (a, b) carries exactly the monomial moment
// xi_x^a xi_y^b for the conserved and stress components (orthonormality of the scaled basis
// under the weights), and no density or momentum of another order
template <class P>
constexpr bool h3_table_ok() {
    constexpr long N = P::DEN;
    return h3_moment<P, 0, 0, 0>() == N && h3_moment<P, 1, 1, 0>() == N && h3_moment<P, 2, 0, 1>() == N &&
           h3_moment<P, 3, 2, 0>() == N && h3_moment<P, 4, 1, 1>() == N && h3_moment<P, 5, 0, 2>() == N &&
           h3_moment<P, 3, 0, 0>() == 0 && h3_moment<P, 5, 0, 0>() == 0 && h3_moment<P, 6, 1, 0>() == 0 &&
           h3_moment<P, 8, 1, 0>() == 0 && h3_moment<P, 7, 0, 1>() == 0 && h3_moment<P, 9, 0, 1>() == 0;
}

}  // namespace lbm
