// D2Q21 weakly compressible BGK and recursive-regularized kernels (Appendix A.2 of arXiv
// 2504.04465): the order-3 Hermite models of weak_h3.cuh about c_s^2 = 2/3.
#include "weak_h3.cuh"

namespace lbm {

// 25920 w_i H[i][k] as an integer: 25920 w_i is 7280, 2160, 1920, 504, 60, 16 for the velocity
// classes (0,0), (1,0), (1,1), (2,0), (2,2), (3,0); per axis the factor h_a(xi) / (a! c_s^2a)
// with c_s^2 = 2/3 is 1, 3 xi / 2, 3 (3 xi^2 - 2) / 8 and 9 (xi^3 - 2 xi) / 16 for a = 0..3,
// and every product divides exactly.
struct P21 {
    static constexpr int Q = 21;
    static constexpr long DEN = 25920;
    static constexpr double CS2 = 2.0 / 3.0;
    __host__ __device__ static constexpr int cx(int q) { return Lat<21>::cx(q); }
    __host__ __device__ static constexpr int cy(int q) { return Lat<21>::cy(q); }
    __host__ __device__ static constexpr int wint(int x, int y) {
        const int a = x < 0 ? -x : x, b = y < 0 ? -y : y;
        const int m = a > b ? a : b, n = a > b ? b : a;
        return m == 0 ? 7280 : m == 1 ? (n == 0 ? 2160 : 1920) : m == 2 ? (n == 0 ? 504 : 60) : 16;
    }
    __host__ __device__ static constexpr int hnum(int a, int x) {
        return a == 0 ? 1 : a == 1 ? 3 * x : a == 2 ? 3 * (3 * x * x - 2) : 9 * (x * x * x - 2 * x);
    }
    __host__ __device__ static constexpr int hden(int a) { return a == 0 ? 1 : a == 1 ? 2 : a == 2 ? 8 : 16; }
    __host__ __device__ static constexpr int G(int q, int k) {
        return wint(cx(q), cy(q)) * hnum(h3_a(k), cx(q)) * hnum(h3_b(k), cy(q)) / (hden(h3_a(k)) * hden(h3_b(k)));
    }
};
static_assert(h3_table_ok<P21>(), "D2Q21 integer reconstruction table");
static_assert(h3_moment<P21, 6, 3, 0>() == P21::DEN && h3_moment<P21, 7, 2, 1>() == P21::DEN &&
                  h3_moment<P21, 9, 0, 3>() == P21::DEN,
              "D2Q21 reproduces the third-order moments exactly");

bool find_kernels_d2q21w(int model, int storage, const int* blk, KernelSet& out) {
    if (blk[0] != 16 || blk[1] != 16 || blk[2] != 1) return false;
    if (storage != ST_F64 && storage != ST_F32) return false;   // no binary16 form
    if (model == 1) return pick_storage<WeakH3<P21, false>, 16, 16, 1>(storage, out);
    if (model == 2) return pick_storage<WeakH3<P21, true>, 16, 16, 1>(storage, out);
    return false;
}

}  // namespace lbm
