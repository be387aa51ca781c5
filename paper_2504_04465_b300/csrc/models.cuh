// Weakly compressible collision models of the CUDA path (Appendix A of arXiv 2504.04465).
//
// D2Q9 and D3Q27.  The Hermite basis of these lattices is the tensor product of the 1D set
// {1, xi, xi^2 - c_s^2} (Tab. lattices_hermite for D2Q9; every axis at most twice for D3Q27).
// Contracting Eq. GenEq over all index tuples gives, per component (a, b, c) in {0, 1, 2}^3,
//     f_i = w_i sum_{abc} h_a(xi_x) h_b(xi_y) h_c(xi_z) A_abc,   A_abc = a_abc / (a! b! c! c_s^2n)
// so the reconstruction is three separable 3-point transforms (x, then y, then z) instead of a
// Q x Q contraction.  Equilibrium moments: a_eq = rho u_x^a u_y^b u_z^c (Eq. RecursivityEquilibrium);
// RR non-equilibrium moments by the pair sum of the recursion of Eq. a1Rec,
//     a_neq = [a=2] Pi_xx u^(a-2,b,c) + ... + a b Pi_xy u^(a-1,b-1,c) + ...,
// with Pi_ab = sum_i xi_a xi_b f_i - rho u_a u_b - c_s^2 rho delta_ab (Appendix A, after Eq. a1Rec).
// BGK: f* = f + (f_eq - f)/tau (Eq. CollisionStep); RR: f* from a* = a_eq + (1 - 1/tau) a_neq
// (Eq. GenRegCollision).
#pragma once
#include "device_common.cuh"

namespace lbm {

__host__ __device__ constexpr double w1d(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
__host__ __device__ constexpr double h1d(int a, int c) {
    return a == 0 ? 1.0 : (a == 1 ? double(c) : double(c * c) - 1.0 / 3.0);
}
__host__ __device__ constexpr double inv_fact(int a) { return a == 2 ? 0.5 : 1.0; }
__host__ __device__ constexpr double pow3(int n) { return n == 0 ? 1.0 : 3.0 * pow3(n - 1); }

template <int D> struct TP;     // tensor-product lattices, same order as Lat<9> / Lat<27>
template <> struct TP<2> {
    static constexpr int Q = 9, NZ = 1;
    __host__ __device__ static constexpr int cx(int q) { return q % 3 - 1; }
    __host__ __device__ static constexpr int cy(int q) { return (q / 3) % 3 - 1; }
    __host__ __device__ static constexpr int cz(int) { return 0; }
};
template <> struct TP<3> {
    static constexpr int Q = 27, NZ = 3;
    __host__ __device__ static constexpr int cx(int q) { return q % 3 - 1; }
    __host__ __device__ static constexpr int cy(int q) { return (q / 3) % 3 - 1; }
    __host__ __device__ static constexpr int cz(int q) { return q / 9 - 1; }
};

template <int D> __host__ __device__ constexpr double tp_w(int q) {
    return w1d(TP<D>::cx(q)) * w1d(TP<D>::cy(q)) * (D == 3 ? w1d(TP<D>::cz(q)) : 1.0);
}

// f_i = w_i sum_abc h_a h_b h_c A[a + 3b + 9c], evaluated separably.  Per axis,
//     18 w(xi) (A_0 + xi A_1 + (xi^2 - 1/3) A_2) = 4 (3 A_0 - A_2) at xi = 0,
//                                                 3 A_0 +- 3 A_1 + 2 A_2 at xi = +-1,
// so every coefficient is an exact integer and the only inexact constant is the final division
// by 18^D.  Rounded constants such as fl(1/6) would scale the reconstructed mass and momentum by
// the same factor at every step (a bias that grows linearly in FP32).  The division is a
// multiplication by fl(1/18^D) followed by one residual correction q += (x - q d) r computed with
// FMAs, which leaves an error of order (rounding of 1/d)^2 instead of a systematic one.
template <typename T>
__device__ __forceinline__ T r1(int x, T a0, T a1, T a2) {
    return x == 0 ? T(4) * (T(3) * a0 - a2) : (T(3) * a0 + T(x) * T(3) * a1 + T(2) * a2);
}

template <int D, typename T>
__device__ __forceinline__ void tp_reconstruct(const T* A, T* f) {
    constexpr int NZ = TP<D>::NZ;
    T X[3][3][NZ];
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < NZ; ++c) X[x][b][c] = r1<T>(x - 1, A[3 * b + 9 * c], A[1 + 3 * b + 9 * c], A[2 + 3 * b + 9 * c]);
    T Y[3][3][NZ];
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int y = 0; y < 3; ++y)
#pragma unroll
            for (int c = 0; c < NZ; ++c) Y[x][y][c] = r1<T>(y - 1, X[x][0][c], X[x][1][c], X[x][2][c]);
    const T den = T(D == 2 ? 324.0 : 5832.0);
    const T rden = T(1) / den;                        // folded at compile time
#pragma unroll
    for (int q = 0; q < TP<D>::Q; ++q) {
        const int x = TP<D>::cx(q) + 1, y = TP<D>::cy(q) + 1, z = TP<D>::cz(q);
        T s;
        if constexpr (D == 2) s = Y[x][y][0];
        else s = r1<T>(z, Y[x][y][0], Y[x][y][NZ > 1 ? 1 : 0], Y[x][y][NZ > 2 ? 2 : 0]);
        const T qt = s * rden;
        f[q] = fma(fma(-qt, den, s), rden, qt);
    }
}

// Weakly compressible collision in place, on deviations d_i = f_i - w_i rho_ref.
// RR = true: recursive regularization, else BGK.  rho = rho_ref + sum d, j = sum xi d,
// sum xi_a xi_b f = rho_ref c_s^2 delta_ab + sum xi_a xi_b d; the reconstruction with
// A_000 = rho - rho_ref returns the post-collision deviations.
template <int D, bool RR, typename T>
__device__ __forceinline__ void weak_collide(T* f, T omega, T rho_ref) {
    constexpr int Q = TP<D>::Q;
    constexpr int NZ = TP<D>::NZ;
    T drho = 0, jx = 0, jy = 0, jz = 0, mxx = 0, myy = 0, mzz = 0, mxy = 0, mxz = 0, myz = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int x = TP<D>::cx(q), y = TP<D>::cy(q), z = TP<D>::cz(q);
        const T v = f[q];
        drho += v;
        if (x) { jx += x > 0 ? v : -v; mxx += v; }
        if (y) { jy += y > 0 ? v : -v; myy += v; }
        if (z) { jz += z > 0 ? v : -v; mzz += v; }
        if (x * y) mxy += x * y > 0 ? v : -v;
        if (x * z) mxz += x * z > 0 ? v : -v;
        if (y * z) myz += y * z > 0 ? v : -v;
    }
    const T rho = rho_ref + drho;
    const T ir = T(1) / rho;
    const T ux = jx * ir, uy = jy * ir, uz = jz * ir;
    const T px[3] = {T(1), ux, ux * ux}, py[3] = {T(1), uy, uy * uy}, pz[3] = {T(1), uz, uz * uz};
    T Pxx = 0, Pyy = 0, Pzz = 0, Pxy = 0, Pxz = 0, Pyz = 0;
    if constexpr (RR) {
        Pxx = mxx - drho / T(3) - rho * ux * ux;
        Pyy = myy - drho / T(3) - rho * uy * uy;
        Pxy = mxy - rho * ux * uy;
        if constexpr (D == 3) {
            Pzz = mzz - drho / T(3) - rho * uz * uz;
            Pxz = mxz - rho * ux * uz;
            Pyz = myz - rho * uy * uz;
        }
    }
    const T keep = T(1) - omega;
    T A[27];
#pragma unroll
    for (int c = 0; c < NZ; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const T eq = (a + b + c == 0) ? drho : rho * px[a] * py[b] * pz[c];
                T ne = 0;
                if (RR && a + b + c >= 2) {
                    if (a == 2) ne += Pxx * py[b] * pz[c];
                    if (b == 2) ne += Pyy * px[a] * pz[c];
                    if (c == 2) ne += Pzz * px[a] * py[b];
                    if (a && b) ne += T(a * b) * Pxy * px[a ? a - 1 : 0] * py[b ? b - 1 : 0] * pz[c];
                    if (a && c) ne += T(a * c) * Pxz * px[a ? a - 1 : 0] * py[b] * pz[c ? c - 1 : 0];
                    if (b && c) ne += T(b * c) * Pyz * px[a] * py[b ? b - 1 : 0] * pz[c ? c - 1 : 0];
                }
                const T scale = T(inv_fact(a) * inv_fact(b) * inv_fact(c) * pow3(a + b + c));
                A[a + 3 * b + 9 * c] = (RR ? (eq + keep * ne) : eq) * scale;
            }
    if constexpr (RR) {
        tp_reconstruct<D, T>(A, f);
    } else {
        T feq[Q];
        tp_reconstruct<D, T>(A, feq);
#pragma unroll
        for (int q = 0; q < Q; ++q) f[q] += omega * (feq[q] - f[q]);
    }
}

// Weakly compressible equilibrium as deviations f_eq,i - w_i rho_ref (boundary cells,
// initialisation)
template <int D, typename T>
__device__ __forceinline__ void weak_feq_dev(T rho, T ux, T uy, T uz, T rho_ref, T* f) {
    constexpr int NZ = TP<D>::NZ;
    const T px[3] = {T(1), ux, ux * ux}, py[3] = {T(1), uy, uy * uy}, pz[3] = {T(1), uz, uz * uz};
    T A[27];
#pragma unroll
    for (int c = 0; c < NZ; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a)
                A[a + 3 * b + 9 * c] = ((a + b + c == 0) ? rho - rho_ref : rho * px[a] * py[b] * pz[c]) *
                                       T(inv_fact(a) * inv_fact(b) * inv_fact(c) * pow3(a + b + c));
    tp_reconstruct<D, T>(A, f);
}

}  // namespace lbm
