// D2Q21 compressible double-distribution kernels with the numerical (max-entropy) equilibrium
// (Appendix A of arXiv 2504.04465): the kernel sets of the FP64 Newton, the batched equilibrium
// solve, and the lookup of every D2Q21 numerical kernel set.  The FP32-Newton sets are compiled
// in translation units of their own (k_d2q21_n32_*.cu, one per storage format).
#include "d2q21.cuh"

namespace lbm {

extern template KernelSet make_set<D2Q21M<true>, ST_F64, 16, 16, 1>();
extern template KernelSet make_set<D2Q21M<true>, ST_F32, 16, 16, 1>();
extern template KernelSet make_set<D2Q21M<true>, ST_F16DEV, 16, 16, 1>();
cudaError_t upload_tables_d2q21_n32_f64(const double*, const double*);
cudaError_t upload_tables_d2q21_n32_f32(const double*, const double*);
cudaError_t upload_tables_d2q21_n32_f16(const double*, const double*);

// batched equilibrium solve: samples (u_x, u_y, T), guess 1 zero, 2 polynomial, 3 network
__global__ void __launch_bounds__(128) k_newton_batch(const double* __restrict__ uT, long long n, ModelDev m,
                                                      double* __restrict__ lam_out, int* __restrict__ iters) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double ux = uT[3 * i], uy = uT[3 * i + 1], Tt = uT[3 * i + 2];
    double lam[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (m.guess == 2) poly_guess21<double>(ux, uy, Tt, lam);
    else if (m.guess == 3) mlp_guess<double>(m.mlp, m.T0, m.mlp_m, m.mlp_s, ux, uy, Tt, lam);
    double e[21];
    int conv = 0;
    const int it = newton_solve<21>(ux, uy, Tt, lam, e, m.newton_tol, m.newton_max_iter, &conv);
#pragma unroll
    for (int a = 0; a < 8; ++a) lam_out[8 * i + a] = lam[a];
    iters[i] = conv ? it : -1;
}

void launch_newton_batch_d2q21(const double* uT, long long n, const ModelDev& m, double* lam, int* iters, cudaStream_t s) {
    if (n) k_newton_batch<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(uT, n, m, lam, iters);
}

static bool fp32_newton_set(int storage, KernelSet& out) {
    switch (storage) {
        case ST_F64: out = make_set<D2Q21M<true>, ST_F64, 16, 16, 1>(); return true;
        case ST_F32: out = make_set<D2Q21M<true>, ST_F32, 16, 16, 1>(); return true;
        case ST_F16DEV: out = make_set<D2Q21M<true>, ST_F16DEV, 16, 16, 1>(); return true;
    }
    return false;
}

bool find_kernels_d2q21(int model, int storage, const int* blk, bool newton_fp32, KernelSet& out) {
    if (model != 4 || blk[0] != 16 || blk[1] != 16 || blk[2] != 1) return false;
    return newton_fp32 ? fp32_newton_set(storage, out) : pick_storage<D2Q21M<false>, 16, 16, 1>(storage, out);
}

cudaError_t upload_tables_d2q21(const double* w21, const double* H21) {
    cudaError_t e = upload21_here(w21, H21);
    if (e == cudaSuccess) e = upload_tables_d2q21_n32_f64(w21, H21);
    if (e == cudaSuccess) e = upload_tables_d2q21_n32_f32(w21, H21);
    if (e == cudaSuccess) e = upload_tables_d2q21_n32_f16(w21, H21);
    return e;
}

}  // namespace lbm
