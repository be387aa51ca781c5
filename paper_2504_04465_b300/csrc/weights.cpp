// Lattice constants of the CUDA path that are not plain fractions.
//
// D2Q37 (Appendix A, Tab. lattices_structure of arXiv 2504.04465) prints its eight group weights
// and c_s^2 to 15 decimals only.  They are re-derived here in FP64 from the isotropy conditions of
// the lattice: the weighted moments <1>, <x^2>, <x^4>, <x^2 y^2>, <x^6>, <x^4 y^2>, <x^8>,
// <x^6 y^2>, <x^4 y^4> equal those of a 2D Gaussian of variance theta (1, th, 3th^2, th^2,
// 15th^3, 3th^3, 105th^4, 15th^4, 9th^4).  Newton's method on the 9 unknowns starts from the
// printed values.  D2Q21 uses the printed fractions.
//
// The Hermite tables hold h_a(xi_x) h_b(xi_y) / (a! b! theta^(a+b)) for the components (a, b)
// of the thermal expansion (order <= 4 for D2Q37, <= 3 for D2Q21), in the component order used by
// models_comp.cuh; h_n are the 1D Hermite polynomials of variance theta.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <utility>

#include "kernels.h"
#include "lattice_tables.h"

namespace lbm {
namespace {

const int kGroups37[8][2] = {{0, 0}, {1, 0}, {1, 1}, {2, 0}, {2, 1}, {2, 2}, {3, 0}, {3, 1}};
const double kPrinted37[9] = {0.233150669132352, 0.107306091542219, 0.057667859888794, 0.014208216158450,
                              0.005353049000513, 0.001011937592673, 0.000245301027757, 0.000283414252994,
                              0.697953322019683};

int group_of(int x, int y) {
    int a = std::abs(x), b = std::abs(y);
    if (a < b) std::swap(a, b);
    for (int g = 0; g < 8; ++g)
        if (kGroups37[g][0] == a && kGroups37[g][1] == b) return g;
    return -1;
}

// solve the 9x9 system J dz = F by Gaussian elimination with partial pivoting
void solve9(double J[9][9], double F[9], double dz[9]) {
    for (int c = 0; c < 9; ++c) {
        int best = c;
        for (int r = c + 1; r < 9; ++r)
            if (std::fabs(J[r][c]) > std::fabs(J[best][c])) best = r;
        for (int k = 0; k < 9; ++k) std::swap(J[c][k], J[best][k]);
        std::swap(F[c], F[best]);
        for (int r = c + 1; r < 9; ++r) {
            const double m = J[r][c] / J[c][c];
            for (int k = c; k < 9; ++k) J[r][k] -= m * J[c][k];
            F[r] -= m * F[c];
        }
    }
    for (int r = 8; r >= 0; --r) {
        double s = F[r];
        for (int k = r + 1; k < 9; ++k) s -= J[r][k] * dz[k];
        dz[r] = s / J[r][r];
    }
}

double herm1d(int n, double x, double th) {
    switch (n) {
        case 0: return 1.0;
        case 1: return x;
        case 2: return x * x - th;
        case 3: return x * x * x - 3.0 * th * x;
        default: return x * x * x * x - 6.0 * th * x * x + 3.0 * th * th;
    }
}

const int kComp[15][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}, {3, 0}, {2, 1},
                          {1, 2}, {0, 3}, {4, 0}, {3, 1}, {2, 2}, {1, 3}, {0, 4}};
const double kFact[5] = {1, 1, 2, 6, 24};

// ulp of a float (distance to the next float away from zero)
long double ulpf(float v) {
    const float a = std::fabs(v);
    return (long double)std::nextafter(a, 2.0f * a + 1.0f) - (long double)a;
}

}  // namespace

void lattice_constants(double w37[37], double H37[37 * 15], double* cs2_37, double w21[21], double H21[21 * 10]) {
    const int cond[9][4] = {{0, 0, 1, 0}, {2, 0, 1, 1}, {4, 0, 3, 2}, {2, 2, 1, 2}, {6, 0, 15, 3},
                            {4, 2, 3, 3}, {8, 0, 105, 4}, {6, 2, 15, 4}, {4, 4, 9, 4}};
    double R[9][8];
    std::memset(R, 0, sizeof(R));
    for (int q = 0; q < 37; ++q) {
        const int x = Lat<37>::cx(q), y = Lat<37>::cy(q), g = group_of(x, y);
        for (int c = 0; c < 9; ++c) R[c][g] += std::pow(double(x), cond[c][0]) * std::pow(double(y), cond[c][1]);
    }
    double z[9];
    for (int k = 0; k < 9; ++k) z[k] = kPrinted37[k];
    for (int it = 0; it < 50; ++it) {
        double F[9], J[9][9], dz[9];
        const double th = z[8];
        for (int c = 0; c < 9; ++c) {
            double s = 0;
            for (int g = 0; g < 8; ++g) { s += R[c][g] * z[g]; J[c][g] = R[c][g]; }
            const int k = cond[c][3];
            F[c] = s - cond[c][2] * std::pow(th, k);
            J[c][8] = k ? -cond[c][2] * k * std::pow(th, k - 1) : 0.0;
        }
        solve9(J, F, dz);
        double mx = 0;
        for (int k = 0; k < 9; ++k) { z[k] -= dz[k]; mx = std::fmax(mx, std::fabs(dz[k])); }
        if (mx < 1e-17) break;
    }
    *cs2_37 = z[8];
    for (int q = 0; q < 37; ++q) {
        w37[q] = z[group_of(Lat<37>::cx(q), Lat<37>::cy(q))];
        for (int k = 0; k < 15; ++k) {
            const int a = kComp[k][0], b = kComp[k][1];
            H37[q * 15 + k] = herm1d(a, Lat<37>::cx(q), z[8]) * herm1d(b, Lat<37>::cy(q), z[8]) /
                              (kFact[a] * kFact[b] * std::pow(z[8], a + b));
        }
    }
    for (int q = 0; q < 21; ++q) {
        int x = std::abs(Lat<21>::cx(q)), y = std::abs(Lat<21>::cy(q));
        if (x < y) std::swap(x, y);
        double w = 0;
        if (x == 0) w = 91.0 / 324.0;
        else if (x == 1 && y == 0) w = 1.0 / 12.0;
        else if (x == 1 && y == 1) w = 2.0 / 27.0;
        else if (x == 2 && y == 0) w = 7.0 / 360.0;
        else if (x == 2 && y == 2) w = 1.0 / 432.0;
        else if (x == 3 && y == 0) w = 1.0 / 1620.0;
        w21[q] = w;
        const double th = 2.0 / 3.0;
        for (int k = 0; k < 10; ++k) {
            const int a = kComp[k][0], b = kComp[k][1];
            H21[q * 10 + k] = herm1d(a, Lat<21>::cx(q), th) * herm1d(b, Lat<21>::cy(q), th) /
                              (kFact[a] * kFact[b] * std::pow(th, a + b));
        }
    }
}

// Class table of the D2Q37 thermal equilibrium.  The 37 velocities fall into the 13 classes
// (X, Y) = (|xi_x|, |xi_y|) of d2q37_class_x/y; a velocity (sx X, sy Y) of class c has the coefficient
// sx^a sy^b C[c][k] for component k = (a, b), with C[c][k] = w(X, Y) h_a(X) h_b(Y) / (a! b! th^(a+b))
// (h_n of odd n are odd functions).  C64 is that table in FP64 about th = c_s^2.  C32 is its FP32
// form about th32 = fl32(c_s^2), rounded so that the reconstruction conserves exactly: each entry
// is moved by whole ulps from the nearest float until the exact moments of every column, summed
// over the 37 velocities, match those of the expansion -- mass sum f = a_0, momentum
// sum xi f = (a_x, a_y), energy sum |xi|^2 f = 2 th32 a_0 + a_xx + a_yy -- to within the FP32
// granularity of the small entries (about 1e-11).  Plain rounding leaves errors of order 1e-8 in
// these moments, which the BGK relaxation turns into a drift of mass, momentum and energy that
// grows with every step.
void d2q37_class_tables(double C64[13 * 15], float C32[13 * 15], double* th64, float* th32, double* max_residual) {
    double w37[37], H37[37 * 15], cs2, w21[21], H21[21 * 10];
    lattice_constants(w37, H37, &cs2, w21, H21);
    double wc[13];
    for (int c = 0; c < 13; ++c) {
        wc[c] = 0;
        for (int q = 0; q < 37; ++q)
            if (Lat<37>::cx(q) == d2q37_class_x(c) && Lat<37>::cy(q) == d2q37_class_y(c)) wc[c] = w37[q];
    }
    const float thf = (float)cs2;
    *th64 = cs2;
    *th32 = thf;
    for (int c = 0; c < 13; ++c)
        for (int k = 0; k < 15; ++k) {
            const int a = kComp[k][0], b = kComp[k][1], X = d2q37_class_x(c), Y = d2q37_class_y(c);
            C64[c * 15 + k] = wc[c] * herm1d(a, X, cs2) * herm1d(b, Y, cs2) / (kFact[a] * kFact[b] * std::pow(cs2, a + b));
            const double v = wc[c] * herm1d(a, X, thf) * herm1d(b, Y, thf) / (kFact[a] * kFact[b] * std::pow((double)thf, a + b));
            C32[c * 15 + k] = (X == 0 && (a & 1)) || (Y == 0 && (b & 1)) ? 0.0f : (float)v;
        }
    // rows: mass, x momentum, y momentum, energy; D[c][r]: moment r of column k per unit of C[c][k]
    auto unit_moments = [&](int c, int k, long double* D) {
        const int a = kComp[k][0], b = kComp[k][1], X = d2q37_class_x(c), Y = d2q37_class_y(c);
        for (int r = 0; r < 4; ++r) D[r] = 0;
        for (int sx = -1; sx <= 1; sx += 2)
            for (int sy = -1; sy <= 1; sy += 2) {
                if ((X == 0 && sx < 0) || (Y == 0 && sy < 0)) continue;
                const long double sgn = ((a & 1) && sx < 0 ? -1 : 1) * ((b & 1) && sy < 0 ? -1 : 1);
                const long double x = sx * X, y = sy * Y;
                D[0] += sgn;
                D[1] += sgn * x;
                D[2] += sgn * y;
                D[3] += sgn * (x * x + y * y);
            }
    };
    double worst = 0;
    for (int k = 0; k < 15; ++k) {
        const long double tgt[4] = {k == 0 ? 1.0L : 0.0L, k == 1 ? 1.0L : 0.0L, k == 2 ? 1.0L : 0.0L,
                                    (k == 0 ? 2.0L * (long double)thf : 0.0L) + (k == 3 || k == 5 ? 1.0L : 0.0L)};
        auto residual = [&](long double* r) {
            for (int i = 0; i < 4; ++i) r[i] = -tgt[i];
            for (int c = 0; c < 13; ++c) {
                long double D[4];
                unit_moments(c, k, D);
                for (int i = 0; i < 4; ++i) r[i] += D[i] * (long double)C32[c * 15 + k];
            }
        };
        auto norm = [](const long double* r) { return r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3]; };
        // moves of one entry, or of two entries at once (mass and energy of a column tie every
        // single entry to a fixed ratio 1 : X^2 + Y^2, so some residuals need a pair), by whole
        // ulps; take the move that lowers the residual most until none does
        auto step = [&](int c, long double* d) {
            long double D[4];
            unit_moments(c, k, D);
            const long double u = ulpf(C32[c * 15 + k]);
            for (int i = 0; i < 4; ++i) d[i] = D[i] * u;
        };
        auto shift = [&](int c, long long n) {
            float& v = C32[c * 15 + k];
            const float dir = n > 0 ? INFINITY : -INFINITY;
            for (long long s2 = 0; s2 < (n > 0 ? n : -n); ++s2) v = std::nextafter(v, dir);
        };
        long double r[4];
        residual(r);
        for (int it = 0; it < 200; ++it) {
            long double best = norm(r);
            int bc[2] = {-1, -1};
            long long bn[2] = {0, 0};
            for (int c1 = 0; c1 < 13; ++c1) {
                if (C32[c1 * 15 + k] == 0.0f) continue;
                long double d1[4];
                step(c1, d1);
                long double a11 = 0, b1 = 0;
                for (int i = 0; i < 4; ++i) { a11 += d1[i] * d1[i]; b1 -= r[i] * d1[i]; }
                if (a11 > 0) {
                    const long double t = b1 / a11;
                    if (std::fabs((double)t) < 1e6) {
                        const long long n = std::llround((double)t);
                        long double rn[4];
                        for (int i = 0; i < 4; ++i) rn[i] = r[i] + n * d1[i];
                        if (n != 0 && norm(rn) < best) { best = norm(rn); bc[0] = c1; bc[1] = -1; bn[0] = n; }
                    }
                }
                for (int c2 = c1 + 1; c2 < 13; ++c2) {
                    if (C32[c2 * 15 + k] == 0.0f) continue;
                    long double d2[4];
                    step(c2, d2);
                    long double a12 = 0, a22 = 0, b2 = 0;
                    for (int i = 0; i < 4; ++i) { a12 += d1[i] * d2[i]; a22 += d2[i] * d2[i]; b2 -= r[i] * d2[i]; }
                    const long double det = a11 * a22 - a12 * a12;
                    if (!(std::fabs((double)det) > 1e-6 * (double)(a11 * a22))) continue;
                    const long double t1 = (b1 * a22 - b2 * a12) / det, t2 = (a11 * b2 - a12 * b1) / det;
                    if (std::fabs((double)t1) > 1e6 || std::fabs((double)t2) > 1e6) continue;
                    for (int f1 = 0; f1 < 2; ++f1)
                        for (int f2 = 0; f2 < 2; ++f2) {
                            const long long n1 = (long long)(f1 ? std::ceil((double)t1) : std::floor((double)t1));
                            const long long n2 = (long long)(f2 ? std::ceil((double)t2) : std::floor((double)t2));
                            long double rn[4];
                            for (int i = 0; i < 4; ++i) rn[i] = r[i] + n1 * d1[i] + n2 * d2[i];
                            if ((n1 != 0 || n2 != 0) && norm(rn) < best) {
                                best = norm(rn);
                                bc[0] = c1; bc[1] = c2; bn[0] = n1; bn[1] = n2;
                            }
                        }
                }
            }
            if (bc[0] < 0) break;
            shift(bc[0], bn[0]);
            if (bc[1] >= 0) shift(bc[1], bn[1]);
            residual(r);
        }
        for (int i = 0; i < 4; ++i) worst = std::fmax(worst, std::fabs((double)r[i]));
    }
    if (max_residual) *max_residual = worst;
}

}  // namespace lbm
