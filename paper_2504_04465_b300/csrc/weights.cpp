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

}  // namespace lbm
