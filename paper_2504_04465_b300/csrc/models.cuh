// Weakly compressible collision models of the CUDA path (Appendix A of arXiv 2504.04465).
//
// D2Q9 and D3Q27.  The Hermite basis of these lattices is the tensor product of the 1D set
// {1, xi, xi^2 - c_s^2} (Tab. lattices_hermite for D2Q9; every axis at most twice for D3Q27).
// Contracting Eq. GenEq over all index tuples gives, per component (a, b, c) in {0, 1, 2}^3,
//     f_i = w_i sum_{abc} h_a(xi_x) h_b(xi_y) h_c(xi_z) A_abc,   A_abc = a_abc / (a! b! c! c_s^2n)
// so the reconstruction factorises per axis (below) instead of a Q x Q contraction.  Equilibrium moments: a_eq = rho u_x^a u_y^b u_z^c (Eq. RecursivityEquilibrium);
// RR non-equilibrium moments by the pair sum of the recursion of Eq. a1Rec,
//     a_neq = [a=2] Pi_xx u^(a-2,b,c) + ... + a b Pi_xy u^(a-1,b-1,c) + ...,
// with Pi_ab = sum_i xi_a xi_b f_i - rho u_a u_b - c_s^2 rho delta_ab (Appendix A, after Eq. a1Rec).
// BGK: f* = f + (f_eq - f)/tau (Eq. CollisionStep); RR: f* from a* = a_eq + (1 - 1/tau) a_neq
// (Eq. GenRegCollision).
#pragma once
#include "device_common.cuh"

namespace lbm {

__host__ __device__ constexpr double w1d(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }

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

// ------------------------------------------------------------------ factorised form
// The D1Q3 tensor-product structure makes every term of Eq. GenRegCollision separable:
//   18^D f*_i = rho E_x E_y E_z + (1 - 1/tau) [Pi_xx X2_x E_y E_z + Pi_yy E_x X2_y E_z
//              + Pi_zz E_x E_y X2_z + Pi_xy X1_x X1_y E_z + Pi_xz X1_x E_y X1_z + Pi_yz E_x X1_y X1_z]
// with, per axis and velocity component c in {-1, 0, 1} (18 w(c) times the 1D Hermite sums):
//   E(c)  = 12 - 18 u^2 (c = 0),   3 + 9 c u + 9 u^2 (c = +-1)      equilibrium factor
//   X1(c) = -36 u       (c = 0),   9 c + 18 u       (c = +-1)        sum_a a h_a u^(a-1) 3^a/a!
//   X2(c) = -18         (c = 0),   9                (c = +-1)        h_2 3^2/2!
// (the a_eq = rho u u u and pair-sum a_neq of models.cuh's tensor-product basis, regrouped per
// axis).  Deviations from w rho_ref use E = W + e with W(c) = 18 w(c) = {12, 3, 3} and
// e = E - W, so E_x E_y E_z - W_x W_y W_z = (e_x E_y + W_x e_y) E_z + W_x W_y e_z stays small.
template <typename T>
struct Axis {
    T E[3], e[3], X1[3];
    __host__ __device__ __forceinline__ explicit Axis(T u) {
        const T u2 = u * u;
        e[1] = T(-18) * u2;
        e[0] = T(9) * u2 - T(9) * u;
        e[2] = T(9) * u2 + T(9) * u;
        E[1] = T(12) + e[1];
        E[0] = T(3) + e[0];
        E[2] = T(3) + e[2];
        X1[1] = T(-36) * u;
        X1[0] = T(18) * u - T(9);
        X1[2] = T(18) * u + T(9);
    }
};
__host__ __device__ constexpr double Wc(int i) { return i == 1 ? 12.0 : 3.0; }     // i = c + 1
__host__ __device__ constexpr double X2c(int i) { return i == 1 ? -18.0 : 9.0; }

// x / (18^D), correctly rounded up to a residual of order fl(1/d) error squared
template <typename T>
__host__ __device__ __forceinline__ T div_den(T x, T den, T rden) {
    const T qt = x * rden;
    return fma(fma(-qt, den, x), rden, qt);
}

// moments of deviations d (sum d, sum xi d, sum xi xi d) by a separable transform
template <int D, typename T>
__host__ __device__ __forceinline__ void tp_moments(const T* d, T& drho, T* j, T* m2 /* xx yy zz xy xz yz */) {
    constexpr int NZ = TP<D>::NZ;
    T s0[3][NZ], s1[3][NZ], s2[3][NZ];     // per (y, z): x-sums of d, x d, x^2 d
#pragma unroll
    for (int z = 0; z < NZ; ++z)
#pragma unroll
        for (int y = 0; y < 3; ++y) {
            const int b = 3 * y + 9 * z;
            const T dm = d[b], d0 = d[b + 1], dp = d[b + 2];
            s2[y][z] = dp + dm;
            s1[y][z] = dp - dm;
            s0[y][z] = s2[y][z] + d0;
        }
    T t00[NZ], t01[NZ], t02[NZ], t10[NZ], t11[NZ], t20[NZ];
#pragma unroll
    for (int z = 0; z < NZ; ++z) {
        const T a = s0[2][z] + s0[0][z];
        t02[z] = a;
        t00[z] = a + s0[1][z];
        t01[z] = s0[2][z] - s0[0][z];
        t10[z] = s1[0][z] + s1[1][z] + s1[2][z];
        t11[z] = s1[2][z] - s1[0][z];
        t20[z] = s2[0][z] + s2[1][z] + s2[2][z];
    }
    if constexpr (D == 2) {
        drho = t00[0]; j[0] = t10[0]; j[1] = t01[0]; j[2] = T(0);
        m2[0] = t20[0]; m2[1] = t02[0]; m2[2] = T(0); m2[3] = t11[0]; m2[4] = T(0); m2[5] = T(0);
    } else {
        const T a = t00[2] + t00[0];
        drho = a + t00[1];
        j[2] = t00[2] - t00[0];
        m2[2] = a;
        j[1] = t01[0] + t01[1] + t01[2];
        m2[5] = t01[2] - t01[0];
        m2[1] = t02[0] + t02[1] + t02[2];
        j[0] = t10[0] + t10[1] + t10[2];
        m2[4] = t10[2] - t10[0];
        m2[3] = t11[0] + t11[1] + t11[2];
        m2[0] = t20[0] + t20[1] + t20[2];
    }
}

// Weakly compressible collision in place, on deviations d_i = f_i - w_i rho_ref.
// RR = true: recursive regularization, else BGK (same equilibrium).
// REL (recursive regularization only): the result is written relative to the reference,
// f*_i / (w_i rho_ref) - 1, the binary16 storage value, with inv_rho_ref = 1 / rho_ref: the
// division by 18^D and by w_i rho_ref fold into one product by 1 / (W_x W_y W_z).
// VAR = WV_TRT (with RR = false): two-relaxation-time collision, the parts of f - f_eq even and
// odd under xi -> -xi relaxed with omega and omega_m (the opposite of q is Q - 1 - q).
// VAR = WV_TRACE (with RR = true): the trace of Pi equilibrated (Pi replaced by its deviatoric
// part, bulk relaxation time one; Appendix A, after Eq. a1Rec).
enum : int { WV_PLAIN = 0, WV_TRT = 1, WV_TRACE = 2 };
template <int D, bool RR, typename T, bool REL = false, int VAR = WV_PLAIN>
__host__ __device__ __forceinline__ void weak_collide(T* f, T omega, T rho_ref, T inv_rho_ref = T(1),
                                                      T omega_m = T(0)) {
    constexpr int NZ = TP<D>::NZ;
    constexpr int Q = TP<D>::Q;
    static_assert(!REL || RR, "relative output only for the regularized collision");
    static_assert(VAR == WV_PLAIN || (VAR == WV_TRT && !RR && !REL) || (VAR == WV_TRACE && RR && !REL),
                  "collision variant");
    T fe[VAR == WV_TRT ? Q : 1];
    T drho, j[3], m2[6];
    tp_moments<D, T>(f, drho, j, m2);
    const T rho = rho_ref + drho;
    const T ir = T(1) / rho;
    const T ux = j[0] * ir, uy = j[1] * ir, uz = j[2] * ir;
    const Axis<T> ax(ux), ay(uy), az(uz);
    const T den = T(D == 2 ? 324.0 : 5832.0);
    const T rden = T(1) / den;
    T kxx = 0, kyy = 0, kzz = 0, kxy = 0, kxz = 0, kyz = 0;
    if constexpr (RR) {
        // (1 - 1/tau) Pi_ab, Pi_ab = sum xi_a xi_b f - rho (u_a u_b + c_s^2 delta_ab)
        const T keep = REL ? (T(1) - omega) * inv_rho_ref : T(1) - omega;
        T pxx = m2[0] - drho / T(3) - rho * ux * ux;
        T pyy = m2[1] - drho / T(3) - rho * uy * uy;
        T pzz = D == 3 ? m2[2] - drho / T(3) - rho * uz * uz : T(0);
        if constexpr (VAR == WV_TRACE) {
            const T tr = (pxx + pyy + pzz) / T(D);
            pxx -= tr;
            pyy -= tr;
            if constexpr (D == 3) pzz -= tr;
        }
        kxx = keep * pxx;
        kyy = keep * pyy;
        kxy = keep * (m2[3] - rho * ux * uy);
        if constexpr (D == 3) {
            kzz = keep * pzz;
            kxz = keep * (m2[4] - rho * ux * uz);
            kyz = keep * (m2[5] - rho * uy * uz);
        }
    }
    if constexpr (REL) {                 // equilibrium part divided by rho_ref as well
        drho = drho * inv_rho_ref;
        rho_ref = T(1);
    }
#pragma unroll
    for (int ix = 0; ix < 3; ++ix)
#pragma unroll
        for (int iy = 0; iy < 3; ++iy) {
            const T Exy = ax.E[ix] * ay.E[iy];
            const T dExy = ax.e[ix] * ay.E[iy] + T(Wc(ix)) * ay.e[iy];
            const T A0 = drho * Exy + rho_ref * dExy;
            T N0 = 0, N1 = 0, N2 = 0;
            if constexpr (RR) {
                N0 = kxx * T(X2c(ix)) * ay.E[iy] + kyy * ax.E[ix] * T(X2c(iy)) + kxy * ax.X1[ix] * ay.X1[iy];
                if constexpr (D == 3) {
                    N1 = kzz * Exy;
                    N2 = kxz * ax.X1[ix] * ay.E[iy] + kyz * ax.E[ix] * ay.X1[iy];
                }
            }
            if constexpr (D == 2) {
                const int q = ix + 3 * iy;
                const T num = A0 + N0;
                if constexpr (REL) f[q] = num * T(1.0 / (Wc(ix) * Wc(iy)));
                else if constexpr (RR) f[q] = div_den<T>(num, den, rden);
                else if constexpr (VAR == WV_TRT) fe[q] = div_den<T>(A0, den, rden);
                else f[q] += omega * (div_den<T>(A0, den, rden) - f[q]);
            } else {
                const T B0 = rho_ref * T(Wc(ix) * Wc(iy));
#pragma unroll
                for (int iz = 0; iz < 3; ++iz) {
                    const int q = ix + 3 * iy + 9 * iz;
                    const T eq = A0 * az.E[iz] + B0 * az.e[iz];
                    if constexpr (RR) {
                        const T num = eq + N0 * az.E[iz] + N1 * T(X2c(iz)) + N2 * az.X1[iz];
                        if constexpr (REL) f[q] = num * T(1.0 / (Wc(ix) * Wc(iy) * Wc(iz)));
                        else f[q] = div_den<T>(num, den, rden);
                    } else if constexpr (VAR == WV_TRT) {
                        fe[q] = div_den<T>(eq, den, rden);
                    } else {
                        f[q] += omega * (div_den<T>(eq, den, rden) - f[q]);
                    }
                }
            }
        }
    if constexpr (VAR == WV_TRT) {
#pragma unroll
        for (int q = 0; q < Q / 2; ++q) {
            const int qb = Q - 1 - q;
            const T dq = f[q] - fe[q], db = f[qb] - fe[qb];
            const T ev = T(0.5) * (dq + db), od = T(0.5) * (dq - db);
            f[q] -= omega * ev + omega_m * od;
            f[qb] -= omega * ev - omega_m * od;
        }
        f[Q / 2] -= omega * (f[Q / 2] - fe[Q / 2]);
    }
    (void)NZ;
    (void)fe;
}

// Weakly compressible equilibrium as deviations f_eq,i - w_i rho_ref (boundary cells,
// initialisation)
template <int D, typename T>
__host__ __device__ __forceinline__ void weak_feq_dev(T rho, T ux, T uy, T uz, T rho_ref, T* f) {
    const Axis<T> ax(ux), ay(uy), az(uz);
    const T den = T(D == 2 ? 324.0 : 5832.0);
    const T rden = T(1) / den;
    const T drho = rho - rho_ref;
#pragma unroll
    for (int ix = 0; ix < 3; ++ix)
#pragma unroll
        for (int iy = 0; iy < 3; ++iy) {
            const T Exy = ax.E[ix] * ay.E[iy];
            const T dExy = ax.e[ix] * ay.E[iy] + T(Wc(ix)) * ay.e[iy];
            const T A0 = drho * Exy + rho_ref * dExy;
            if constexpr (D == 2) {
                f[ix + 3 * iy] = div_den<T>(A0, den, rden);
            } else {
                const T B0 = rho_ref * T(Wc(ix) * Wc(iy));
#pragma unroll
                for (int iz = 0; iz < 3; ++iz) f[ix + 3 * iy + 9 * iz] = div_den<T>(A0 * az.E[iz] + B0 * az.e[iz], den, rden);
            }
        }
}

}  // namespace lbm
