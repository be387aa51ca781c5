// Compressible double-distribution building blocks of the CUDA path (Appendix A of
// arXiv 2504.04465): thermal Hermite moments, the kinetic shock sensor and the FP64 Newton
// solver of the numerical (max-entropy) equilibrium.
//
// T from Eq. polyTemp, g_eq from Eq. gEq, sensor of Eqs. DeltaAvg/shock_function (alpha = 1
// below 0.01), BGK on f and g with the same tau.  The thermal expansion about theta adds, for
// every set of disjoint index pairs, a factor (T - theta) delta per pair.  Numerical equilibrium:
// Eq. exponential with the 8 constraints G0..G3yaa, solved with rho = 1 by Newton-Raphson in
// FP64, or FP32 when selected (step d = (sum e M M^T)^-1 G by Cholesky, backtracking halving of
// the step until ||G||_2 decreases, at most 30 halvings, stop when max |G| < tol).
#pragma once
#include <utility>
#include "device_common.cuh"

namespace lbm {

// math of the solver's own precision (no promotion of FP32 arguments to the FP64 routines)
__device__ __forceinline__ float r_exp(float x) { return expf(x); }
__device__ __forceinline__ double r_exp(double x) { return ::exp(x); }
__device__ __forceinline__ float r_log(float x) { return logf(x); }
__device__ __forceinline__ double r_log(double x) { return ::log(x); }
__device__ __forceinline__ float r_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double r_sqrt(double x) { return ::sqrt(x); }
__device__ __forceinline__ float r_fabs(float x) { return fabsf(x); }
__device__ __forceinline__ double r_fabs(double x) { return ::fabs(x); }
__device__ __forceinline__ float r_fmax(float x, float y) { return fmaxf(x, y); }
__device__ __forceinline__ double r_fmax(double x, double y) { return ::fmax(x, y); }
__device__ __forceinline__ bool r_finite(float x) { return __finitef(x) != 0; }
__device__ __forceinline__ bool r_finite(double x) { return isfinite(x); }

// thermal Hermite moments a_k, components ordered (0,0) (1,0) (0,1) (2,0) (1,1) (0,2) (3,0) (2,1)
// (1,2) (0,3) (4,0) (3,1) (2,2) (1,3) (0,4); dT = T - theta
template <typename T>
__device__ __forceinline__ void thermal_moments(T rho, T ux, T uy, T dT, int order, T* a) {
    const T ux2 = ux * ux, uy2 = uy * uy;
    a[0] = rho;
    a[1] = rho * ux;
    a[2] = rho * uy;
    a[3] = rho * (ux2 + dT);
    a[4] = rho * ux * uy;
    a[5] = rho * (uy2 + dT);
    a[6] = rho * ux * (ux2 + T(3) * dT);
    a[7] = rho * uy * (ux2 + dT);
    a[8] = rho * ux * (uy2 + dT);
    a[9] = rho * uy * (uy2 + T(3) * dT);
    if (order >= 4) {
        a[10] = rho * (ux2 * ux2 + T(6) * ux2 * dT + T(3) * dT * dT);
        a[11] = rho * ux * uy * (ux2 + T(3) * dT);
        a[12] = rho * (ux2 * uy2 + (ux2 + uy2) * dT + dT * dT);
        a[13] = rho * ux * uy * (uy2 + T(3) * dT);
        a[14] = rho * (uy2 * uy2 + T(6) * uy2 * dT + T(3) * dT * dT);
    }
}

// one term |f - f_eq| / f_eq of Eq. DeltaAvg: the FP32 kernels take the fast approximate
// division (a reciprocal and a product, a few ulps); the sensor only compares the mean with
// thresholds 0.01, 0.1 and 1, so a few ulps matter no more than the FP32 rounding of f itself
__device__ __forceinline__ float sensor_ratio(float num, float den) { return __fdividef(num, den); }
__device__ __forceinline__ double sensor_ratio(double num, double den) { return num / den; }

// Eq. shock_function with alpha = 1 below 0.01
template <typename T>
__device__ __forceinline__ T sensor_alpha(T eps, T tau, T A) {
    if (eps < T(0.01)) return T(1);
    if (eps < T(0.10)) return T(1.05);
    if (eps < T(1.00)) return A;
    return T(1) / tau;
}

// ------------------------------------------------------------------ Newton (FP64)
// f(integral_constant<int, 0>) ... f(integral_constant<int, N - 1>): the velocity index is a
// compile-time constant in every instance, so the monomials fold to constants and the
// per-velocity arrays stay in registers however large the body is
template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F& f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

template <int Q> struct MB {
    // raw monomials 1, x, y, xx, xy, yy, x r2, y r2 of velocity q
    __host__ __device__ static constexpr double m(int q, int a) {
        const double x = Lat<Q>::cx(q), y = Lat<Q>::cy(q), r2 = x * x + y * y;
        return a == 0 ? 1.0 : a == 1 ? x : a == 2 ? y : a == 3 ? x * x : a == 4 ? x * y : a == 5 ? y * y : a == 6 ? x * r2 : y * r2;
    }
};

// R: the arithmetic of the solve (double, or float for the single-precision variant)
template <int Q, typename R = double>
__device__ __forceinline__ void newton_eval(const R* lam, const R* tgt, R* e, R* G) {
#pragma unroll
    for (int a = 0; a < 8; ++a) G[a] = -tgt[a];
    static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        R s = R(1);
#pragma unroll
        for (int a = 0; a < 8; ++a) s += lam[a] * R(MB<Q>::m(q, a));
        e[q] = r_exp(-s);
#pragma unroll
        for (int a = 0; a < 8; ++a) G[a] += e[q] * R(MB<Q>::m(q, a));
    });
}

// Cholesky solve of the packed SPD system A d = G (A lower triangle, row-major packed)
template <typename R = double>
__device__ __forceinline__ void chol8_solve(R* A, const R* G, R* d) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        R s = A[j * (j + 1) / 2 + j];
#pragma unroll
        for (int k = 0; k < j; ++k) s -= A[j * (j + 1) / 2 + k] * A[j * (j + 1) / 2 + k];
        const R djj = r_sqrt(s);
        A[j * (j + 1) / 2 + j] = djj;
#pragma unroll
        for (int i = j + 1; i < 8; ++i) {
            R t = A[i * (i + 1) / 2 + j];
#pragma unroll
            for (int k = 0; k < j; ++k) t -= A[i * (i + 1) / 2 + k] * A[j * (j + 1) / 2 + k];
            A[i * (i + 1) / 2 + j] = t / djj;
        }
    }
    R y[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        R t = G[i];
#pragma unroll
        for (int k = 0; k < i; ++k) t -= A[i * (i + 1) / 2 + k] * y[k];
        y[i] = t / A[i * (i + 1) / 2 + i];
    }
#pragma unroll
    for (int i = 7; i >= 0; --i) {
        R t = y[i];
#pragma unroll
        for (int k = i + 1; k < 8; ++k) t -= A[k * (k + 1) / 2 + i] * d[k];
        d[i] = t / A[i * (i + 1) / 2 + i];
    }
}

template <int Q, typename R = double>
__device__ __forceinline__ void newton_dir(const R* e, const R* G, R* d) {
    R A[36];
#pragma unroll
    for (int k = 0; k < 36; ++k) A[k] = R(0);
    static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        int k = 0;
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b <= a; ++b) A[k++] += e[q] * R(MB<Q>::m(q, a) * MB<Q>::m(q, b));
    });
    chol8_solve<R>(A, G, d);
}

// Solve for lambda (in/out) at (u, T); e[] receives exp(-(1 + lambda.M)) (rho = 1).
// Returns the number of Newton steps; *conv = 1 if the residual is finite and max |G| < tol.
// A cell stops unconverged at its last finite iterate when the Jacobian's Cholesky
// factorisation meets a non-positive pivot (non-finite direction) or the line search ends on a
// non-finite trial.
template <int Q, typename R = double>
__device__ __noinline__ int newton_solve(R ux, R uy, R Tt, R* lam, R* e, R tol, int max_iter, int* conv) {
    const R u2 = ux * ux + uy * uy, t2 = u2 + R(4) * Tt;
    const R tgt[8] = {R(1), ux, uy, ux * ux + Tt, ux * uy, uy * uy + Tt, ux * t2, uy * t2};
    R G[8];
    newton_eval<Q, R>(lam, tgt, e, G);
    *conv = 0;
    int it = 0;
    for (;; ++it) {
        R gmax = R(0);
        bool fin = true;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            fin = fin && r_finite(G[a]);
            gmax = r_fmax(gmax, r_fabs(G[a]));
        }
        if (fin && gmax < tol) { *conv = 1; break; }
        if (!fin || it == max_iter) break;
        R d[8];
        newton_dir<Q, R>(e, G, d);
        bool dfin = true;
#pragma unroll
        for (int a = 0; a < 8; ++a) dfin = dfin && r_finite(d[a]);
        if (!dfin) break;
        R g0 = R(0);
#pragma unroll
        for (int a = 0; a < 8; ++a) g0 += G[a] * G[a];
        R t = R(1);
        R trial[8], Gt[8];
        bool take = false;
#pragma unroll 1
        for (int h = 0; h <= 30; ++h) {
#pragma unroll
            for (int a = 0; a < 8; ++a) trial[a] = lam[a] + t * d[a];
            newton_eval<Q, R>(trial, tgt, e, Gt);
            R g1 = R(0);
#pragma unroll
            for (int a = 0; a < 8; ++a) g1 += Gt[a] * Gt[a];
            if (g1 < g0 || (h == 30 && r_finite(g1))) { take = true; break; }
            t *= R(0.5);
        }
        if (!take) {                        // keep the current iterate (restore its e)
            newton_eval<Q, R>(lam, tgt, e, G);
            break;
        }
#pragma unroll
        for (int a = 0; a < 8; ++a) { lam[a] = trial[a]; G[a] = Gt[a]; }
    }
    return it;
}

// the same iteration inlined into the caller (the FP32 kernels keep its arrays in registers)
template <int Q, typename R = double>
__device__ __forceinline__ int newton_solve_inl(R ux, R uy, R Tt, R* lam, R* e, R tol, int max_iter, int* conv) {
    const R u2 = ux * ux + uy * uy, t2 = u2 + R(4) * Tt;
    const R tgt[8] = {R(1), ux, uy, ux * ux + Tt, ux * uy, uy * uy + Tt, ux * t2, uy * t2};
    R G[8];
    newton_eval<Q, R>(lam, tgt, e, G);
    *conv = 0;
    int it = 0;
    for (;; ++it) {
        R gmax = R(0);
        bool fin = true;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            fin = fin && r_finite(G[a]);
            gmax = r_fmax(gmax, r_fabs(G[a]));
        }
        if (fin && gmax < tol) { *conv = 1; break; }
        if (!fin || it == max_iter) break;
        R d[8];
        newton_dir<Q, R>(e, G, d);
        bool dfin = true;
#pragma unroll
        for (int a = 0; a < 8; ++a) dfin = dfin && r_finite(d[a]);
        if (!dfin) break;
        R g0 = R(0);
#pragma unroll
        for (int a = 0; a < 8; ++a) g0 += G[a] * G[a];
        R t = R(1);
        R trial[8], Gt[8];
        bool take = false;
#pragma unroll 1
        for (int h = 0; h <= 30; ++h) {
#pragma unroll
            for (int a = 0; a < 8; ++a) trial[a] = lam[a] + t * d[a];
            newton_eval<Q, R>(trial, tgt, e, Gt);
            R g1 = R(0);
#pragma unroll
            for (int a = 0; a < 8; ++a) g1 += Gt[a] * Gt[a];
            if (g1 < g0 || (h == 30 && r_finite(g1))) { take = true; break; }
            t *= R(0.5);
        }
        if (!take) {                        // keep the current iterate (restore its e)
            newton_eval<Q, R>(lam, tgt, e, G);
            break;
        }
#pragma unroll
        for (int a = 0; a < 8; ++a) { lam[a] = trial[a]; G[a] = Gt[a]; }
    }
    return it;
}

// Polynomial Newton guess: weighted least-squares fit of -1 - ln f_poly onto the eight basis
// functions over the populations with f_poly > 0 (weights w_i), kept only where it is finite and
// closer to the root than lambda = 0.  fpoly(q, &w) returns f_poly,i (rho = 1) and sets w = w_i.
template <int Q, typename R, typename FP>
__device__ __forceinline__ void poly_guess_fit(R ux, R uy, R Tt, FP fpoly, R* lam) {
    R A[36], b[8];
#pragma unroll
    for (int k = 0; k < 36; ++k) A[k] = R(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) b[k] = R(0);
    static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        R w;
        const R fp = fpoly(q, w);
        if (fp > R(0)) {
            const R y = R(-1) - r_log(fp);
            int k = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                b[i] += w * R(MB<Q>::m(q, i)) * y;
#pragma unroll
                for (int j = 0; j <= i; ++j) A[k++] += w * R(MB<Q>::m(q, i) * MB<Q>::m(q, j));
            }
        }
    });
    R fit[8];
    chol8_solve<R>(A, b, fit);
    const R u2 = ux * ux + uy * uy, t2 = u2 + R(4) * Tt;
    const R tgt[8] = {R(1), ux, uy, ux * ux + Tt, ux * uy, uy * uy + Tt, ux * t2, uy * t2};
    bool fin = true;
#pragma unroll
    for (int a = 0; a < 8; ++a) fin = fin && r_finite(fit[a]);
    R e[Q], G[8], gf = R(0), g0 = R(0);
    if (fin) {
        newton_eval<Q, R>(fit, tgt, e, G);
#pragma unroll
        for (int a = 0; a < 8; ++a) gf += G[a] * G[a];
        const R zero[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        newton_eval<Q, R>(zero, tgt, e, G);
#pragma unroll
        for (int a = 0; a < 8; ++a) g0 += G[a] * G[a];
    }
    const bool keep = fin && (gf < g0);
#pragma unroll
    for (int a = 0; a < 8; ++a) lam[a] = keep ? fit[a] : R(0);
}

}  // namespace lbm
