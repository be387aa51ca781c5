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

// ------------------------------------------------------------------ relative form, binary16 storage
// Scalar (float) or packed two-cell (F2: a float2 per value, fma.rn.f32x2 and friends) arithmetic
// for the collision of the binary16 interior kernel.
struct F2 {
    float2 v;
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return {__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v)}; }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return {__fmul2_rn(a.v, b.v)}; }
template <class V> struct Ar;
template <> struct Ar<float> {
    static __device__ __forceinline__ float c(float s) { return s; }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
    static __device__ __forceinline__ float rcp(float a) { return __frcp_rn(a); }
};
template <> struct Ar<F2> {
    static __device__ __forceinline__ F2 c(float s) { return {make_float2(s, s)}; }
    static __device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
    static __device__ __forceinline__ F2 rcp(F2 a) { return {make_float2(__frcp_rn(a.v.x), __frcp_rn(a.v.y))}; }
};

// D3Q27 recursive regularization (Eq. GenRegCollision with the a_neq of Eq. a1Rec) in the
// variables of the binary16 format: in h_q = f_q / (w_q rho_ref) - 1, out the same of f*_q
// (emit(q, value) receives each); keep = 1 - 1/tau.  With W18 = 18 w1d = {3, 12, 3} per axis and every factor of the
// factorised form above divided by W18 of its velocity component (E' = E / W18 = 1 + e', X1',
// X2' = {3, -1.5, 3}),
//   h*_q = (1 + R) E'_x E'_y E'_z - 1 + K_xx X2'_x E'_y E'_z + ... + K_yz E'_x X1'_y X1'_z
// with R = (rho - rho_ref) / rho_ref and K_ab = (1 - 1/tau) Pi_ab / rho_ref, and
//   (1 + R) E'E'E' - 1 = (R E'_x E'_y + e'_x E'_y + e'_y) E'_z + e'_z,
// so that a velocity costs three FMAs after nine products per (xi_x, xi_y) pair.  The moments
// of w_q h_q (w_q = W(xi_x) W(xi_y) W(xi_z) / 216, W = {1, 4, 1}) come from the same separable
// sums as tp_moments, scaled by 1/216 at the end.
template <class V, class Emit>
__device__ __forceinline__ void rr_rel_q27(const V* h, float keep, Emit&& emit) {
    using A = Ar<V>;
    const V four = A::c(4.0f);
    V s[3][3][3];     // [a][y][z]: sum_x W(x) x^a h
#pragma unroll
    for (int z = 0; z < 3; ++z)
#pragma unroll
        for (int y = 0; y < 3; ++y) {
            const int b = 3 * y + 9 * z;
            const V u = h[b + 2] + h[b];
            s[2][y][z] = u;
            s[1][y][z] = h[b + 2] - h[b];
            s[0][y][z] = A::fma(four, h[b + 1], u);
        }
    V t[3][3][3];     // [a][b][z]: sum_y W(y) y^b s[a][y][z], a + b <= 2
#pragma unroll
    for (int z = 0; z < 3; ++z)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const V u = s[a][2][z] + s[a][0][z];
            t[a][0][z] = A::fma(four, s[a][1][z], u);
            if (a <= 1) t[a][1][z] = s[a][2][z] - s[a][0][z];
            if (a == 0) t[a][2][z] = u;
        }
    // sum_z W(z) z^c t[a][b][z]
    auto z0 = [&](int a, int b) { return A::fma(four, t[a][b][1], t[a][b][2] + t[a][b][0]); };
    const V r216 = A::c(1.0f / 216.0f);
    const V R = z0(0, 0) * r216;
    const V Jx = z0(1, 0) * r216, Jy = z0(0, 1) * r216, Jz = (t[0][0][2] - t[0][0][0]) * r216;
    const V Mxx = z0(2, 0) * r216, Myy = z0(0, 2) * r216, Mzz = (t[0][0][2] + t[0][0][0]) * r216;
    const V Mxy = z0(1, 1) * r216, Mxz = (t[1][0][2] - t[1][0][0]) * r216, Myz = (t[0][1][2] - t[0][1][0]) * r216;
    const V ir = A::rcp(A::c(1.0f) + R);
    const V ux = Jx * ir, uy = Jy * ir, uz = Jz * ir;
    // K_ab = keep (M_ab - J_a u_b - delta_ab R / 3)
    const V kp = A::c(keep), r3 = R * A::c(1.0f / 3.0f);
    const V Kxx = kp * (Mxx - A::fma(Jx, ux, r3)), Kyy = kp * (Myy - A::fma(Jy, uy, r3)),
            Kzz = kp * (Mzz - A::fma(Jz, uz, r3));
    const V Kxy = kp * A::fma(A::c(0.0f) - Jx, uy, Mxy), Kxz = kp * A::fma(A::c(0.0f) - Jx, uz, Mxz),
            Kyz = kp * A::fma(A::c(0.0f) - Jy, uz, Myz);
    // per axis and component i = xi + 1: e', E' = 1 + e', X1' (the x axis one component at a
    // time, inside the loop below, which keeps fewer values live)
    auto axis_i = [&](V a, V t3, int i, V& e, V& E, V& X) {
        e = i == 0 ? a - t3 : (i == 1 ? a * A::c(-0.5f) : a + t3);
        E = A::c(1.0f) + e;
        X = i == 0 ? A::fma(A::c(2.0f), t3, A::c(-3.0f)) : (i == 1 ? A::c(0.0f) - t3 : A::fma(A::c(2.0f), t3, A::c(3.0f)));
    };
    const V ax = A::c(3.0f) * (ux * ux), tx = A::c(3.0f) * ux;
    const V ay = A::c(3.0f) * (uy * uy), t3y = A::c(3.0f) * uy;
    const V az = A::c(3.0f) * (uz * uz), t3z = A::c(3.0f) * uz;
    V ey[3], Ey[3], Xy[3], ez[3], Ez[3], Xz[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        axis_i(ay, t3y, i, ey[i], Ey[i], Xy[i]);
        axis_i(az, t3z, i, ez[i], Ez[i], Xz[i]);
    }
    // K with the X2' and X1' factors of one axis folded in
    const V ky2[2] = {Kyy * A::c(3.0f), Kyy * A::c(-1.5f)}, kz2[2] = {Kzz * A::c(3.0f), Kzz * A::c(-1.5f)};
    V kyz[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) kyz[i] = Kyz * Xy[i];
#pragma unroll
    for (int ix = 0; ix < 3; ++ix) {
        V exi, Exi, Xxi;
        axis_i(ax, tx, ix, exi, Exi, Xxi);
        const V kx2 = Kxx * A::c(ix == 1 ? -1.5f : 3.0f), kxy = Kxy * Xxi, kxz = Kxz * Xxi;
#pragma unroll
        for (int iy = 0; iy < 3; ++iy) {
            const V Exy = Exi * Ey[iy];
            const V dE = A::fma(exi, Ey[iy], ey[iy]);
            const V N0 = A::fma(kx2, Ey[iy], A::fma(ky2[iy == 1], Exi, kxy * Xy[iy]));
            const V P = A::fma(R, Exy, dE + N0);
            const V N2 = A::fma(kxz, Ey[iy], kyz[iy] * Exi);
#pragma unroll
            for (int iz = 0; iz < 3; ++iz)
                emit(ix + 3 * iy + 9 * iz, A::fma(P, Ez[iz], A::fma(Exy, kz2[iz == 1], A::fma(N2, Xz[iz], ez[iz]))));
        }
    }
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
