// Velocity sets and cell types of the CUDA path (host and device).
//
// Appendix A, Tab. lattices_structure of arXiv 2504.04465 gives the symmetry groups of D2Q9,
// D2Q13, D2Q21 and D2Q37; D3Q27 is the tensor product of the 1D three-velocity set.  The CUDA path
// orders every 2D set row-major over (y, x) in [-r, r]^2 and D3Q27 as x + 3y + 9z with
// components in {-1, 0, 1}.  Both orders are point-symmetric, so the opposite of velocity q is
// Q - 1 - q.  Weights are not stored here: D2Q9/D2Q21/D3Q27 use the printed fractions and D2Q37
// re-derives its weights at start-up (weights.cpp).
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define LBM_HD __host__ __device__
#else
#define LBM_HD
#endif

namespace lbm {

// cell types of the layout (host builder and kernels)
enum CellType : unsigned char { C_ABSENT = 0, C_FLUID = 1, C_CGHOST = 2, C_FGHOST = 3, C_BC = 4, C_SOLID = 5 };

enum LatticeId { L_D2Q9 = 9, L_D2Q13 = 13, L_D2Q21 = 21, L_D2Q37 = 37, L_D3Q27 = 27 };

// membership of (x, y) in the 2D sets (|x|, |y| <= 3)
LBM_HD constexpr bool in_d2q13(int x, int y) {
    const int ax = x < 0 ? -x : x, ay = y < 0 ? -y : y;
    return ax + ay <= 2;                                // (0,0) (1,0) (1,1) (2,0)
}
LBM_HD constexpr bool in_d2q21(int x, int y) {
    int ax = x < 0 ? -x : x, ay = y < 0 ? -y : y;
    if (ax > 3 || ay > 3) return false;
    if (ax == 0 || ay == 0) return true;               // (0,0) (1,0) (2,0) (3,0)
    return ax == ay && ax <= 2;                         // (1,1) (2,2)
}
LBM_HD constexpr bool in_d2q37(int x, int y) {
    int ax = x < 0 ? -x : x, ay = y < 0 ? -y : y;
    if (ax > 3 || ay > 3) return false;
    if (ax == 3 && ay >= 2) return false;
    if (ay == 3 && ax >= 2) return false;
    return true;                                        // groups (a,b) with a,b <= 2 or (3,0),(3,1)
}

// component (x if want_y == 0, else y) of velocity q of a 2D set enumerated row-major over (y, x)
LBM_HD constexpr int enum13(int q, int want_y) {
    int k = 0;
    for (int y = -2; y <= 2; ++y)
        for (int x = -2; x <= 2; ++x)
            if (in_d2q13(x, y)) {
                if (k == q) return want_y ? y : x;
                ++k;
            }
    return 0;
}
LBM_HD constexpr int enum21(int q, int want_y) {
    int k = 0;
    for (int y = -3; y <= 3; ++y)
        for (int x = -3; x <= 3; ++x)
            if (in_d2q21(x, y)) {
                if (k == q) return want_y ? y : x;
                ++k;
            }
    return 0;
}
LBM_HD constexpr int enum37(int q, int want_y) {
    int k = 0;
    for (int y = -3; y <= 3; ++y)
        for (int x = -3; x <= 3; ++x)
            if (in_d2q37(x, y)) {
                if (k == q) return want_y ? y : x;
                ++k;
            }
    return 0;
}

// the same enumerations as switch tables: folded to constants where q is known at compile time
// (unrolled loops), a jump table otherwise
LBM_HD constexpr int d2q13_x(int q) {
    switch (q) { case 1: return -1; case 3: return 1; case 4: return -2; case 5: return -1; case 7: return 1; case 8: return 2; case 9: return -1; case 11: return 1; default: return 0; }
}
LBM_HD constexpr int d2q13_y(int q) {
    switch (q) { case 0: return -2; case 1: return -1; case 2: return -1; case 3: return -1; case 9: return 1; case 10: return 1; case 11: return 1; case 12: return 2; default: return 0; }
}
LBM_HD constexpr int d2q21_x(int q) {
    switch (q) { case 0: return 0; case 1: return -2; case 2: return 0; case 3: return 2; case 4: return -1; case 5: return 0; case 6: return 1; case 7: return -3; case 8: return -2; case 9: return -1; case 10: return 0; case 11: return 1; case 12: return 2; case 13: return 3; case 14: return -1; case 15: return 0; case 16: return 1; case 17: return -2; case 18: return 0; case 19: return 2; case 20: return 0; default: return 0; }
}
LBM_HD constexpr int d2q21_y(int q) {
    switch (q) { case 0: return -3; case 1: return -2; case 2: return -2; case 3: return -2; case 4: return -1; case 5: return -1; case 6: return -1; case 7: return 0; case 8: return 0; case 9: return 0; case 10: return 0; case 11: return 0; case 12: return 0; case 13: return 0; case 14: return 1; case 15: return 1; case 16: return 1; case 17: return 2; case 18: return 2; case 19: return 2; case 20: return 3; default: return 0; }
}
LBM_HD constexpr int d2q37_x(int q) {
    switch (q) { case 0: return -1; case 1: return 0; case 2: return 1; case 3: return -2; case 4: return -1; case 5: return 0; case 6: return 1; case 7: return 2; case 8: return -3; case 9: return -2; case 10: return -1; case 11: return 0; case 12: return 1; case 13: return 2; case 14: return 3; case 15: return -3; case 16: return -2; case 17: return -1; case 18: return 0; case 19: return 1; case 20: return 2; case 21: return 3; case 22: return -3; case 23: return -2; case 24: return -1; case 25: return 0; case 26: return 1; case 27: return 2; case 28: return 3; case 29: return -2; case 30: return -1; case 31: return 0; case 32: return 1; case 33: return 2; case 34: return -1; case 35: return 0; case 36: return 1; default: return 0; }
}
LBM_HD constexpr int d2q37_y(int q) {
    switch (q) { case 0: return -3; case 1: return -3; case 2: return -3; case 3: return -2; case 4: return -2; case 5: return -2; case 6: return -2; case 7: return -2; case 8: return -1; case 9: return -1; case 10: return -1; case 11: return -1; case 12: return -1; case 13: return -1; case 14: return -1; case 15: return 0; case 16: return 0; case 17: return 0; case 18: return 0; case 19: return 0; case 20: return 0; case 21: return 0; case 22: return 1; case 23: return 1; case 24: return 1; case 25: return 1; case 26: return 1; case 27: return 1; case 28: return 1; case 29: return 2; case 30: return 2; case 31: return 2; case 32: return 2; case 33: return 2; case 34: return 3; case 35: return 3; case 36: return 3; default: return 0; }
}

// the switch tables agree with the enumeration for every velocity (checked at compile time)
LBM_HD constexpr bool tables_match() {
    for (int q = 0; q < 13; ++q)
        if (d2q13_x(q) != enum13(q, 0) || d2q13_y(q) != enum13(q, 1)) return false;
    for (int q = 0; q < 21; ++q)
        if (d2q21_x(q) != enum21(q, 0) || d2q21_y(q) != enum21(q, 1)) return false;
    for (int q = 0; q < 37; ++q)
        if (d2q37_x(q) != enum37(q, 0) || d2q37_y(q) != enum37(q, 1)) return false;
    return true;
}
static_assert(tables_match(), "D2Q13/D2Q21/D2Q37 switch tables differ from the enumeration");

// The 13 classes (X, Y) = (|xi_x|, |xi_y|) of the D2Q37 velocities, the centre first, then the
// axis pairs (X, 0) and (0, Y), then the quadruples (+-X, +-Y)
LBM_HD constexpr int d2q37_class_x(int c) {
    constexpr int t[13] = {0, 1, 0, 2, 0, 3, 0, 1, 2, 1, 2, 3, 1};
    return t[c];
}
LBM_HD constexpr int d2q37_class_y(int c) {
    constexpr int t[13] = {0, 0, 1, 0, 2, 0, 3, 1, 1, 2, 2, 1, 3};
    return t[c];
}

template <int Q> struct Lat;

template <> struct Lat<9> {
    static constexpr int Q = 9, D = 2, R = 1;
    LBM_HD static constexpr int cx(int q) { return q % 3 - 1; }
    LBM_HD static constexpr int cy(int q) { return q / 3 - 1; }
    LBM_HD static constexpr int cz(int) { return 0; }
};

template <> struct Lat<27> {
    static constexpr int Q = 27, D = 3, R = 1;
    LBM_HD static constexpr int cx(int q) { return q % 3 - 1; }
    LBM_HD static constexpr int cy(int q) { return (q / 3) % 3 - 1; }
    LBM_HD static constexpr int cz(int q) { return q / 9 - 1; }
};

template <> struct Lat<13> {
    static constexpr int Q = 13, D = 2, R = 2;
    LBM_HD static constexpr int cx(int q) { return d2q13_x(q); }
    LBM_HD static constexpr int cy(int q) { return d2q13_y(q); }
    LBM_HD static constexpr int cz(int) { return 0; }
};

template <> struct Lat<21> {
    static constexpr int Q = 21, D = 2, R = 3;
    LBM_HD static constexpr int cx(int q) { return d2q21_x(q); }
    LBM_HD static constexpr int cy(int q) { return d2q21_y(q); }
    LBM_HD static constexpr int cz(int) { return 0; }
};

template <> struct Lat<37> {
    static constexpr int Q = 37, D = 2, R = 3;
    LBM_HD static constexpr int cx(int q) { return d2q37_x(q); }
    LBM_HD static constexpr int cy(int q) { return d2q37_y(q); }
    LBM_HD static constexpr int cz(int) { return 0; }
};

// runtime view (host builder)
struct LatticeDesc {
    int Q, D, R;
    int xi[37][3];
};

template <class L>
inline void fill_desc(LatticeDesc& d) {
    d.Q = L::Q; d.D = L::D; d.R = L::R;
    for (int q = 0; q < L::Q; ++q) { d.xi[q][0] = L::cx(q); d.xi[q][1] = L::cy(q); d.xi[q][2] = L::cz(q); }
}

inline LatticeDesc lattice_desc(int id) {
    LatticeDesc d{};
    switch (id) {
        case L_D2Q9: fill_desc<Lat<9>>(d); break;
        case L_D2Q13: fill_desc<Lat<13>>(d); break;
        case L_D2Q21: fill_desc<Lat<21>>(d); break;
        case L_D2Q37: fill_desc<Lat<37>>(d); break;
        case L_D3Q27: fill_desc<Lat<27>>(d); break;
        default: d.Q = 0;
    }
    return d;
}

}  // namespace lbm
