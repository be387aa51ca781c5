// D2Q37 compressible double-distribution kernels (Appendix A of arXiv 2504.04465): the kernel
// sets of the thermal polynomial equilibrium, the batched equilibrium solve, and the lookup of
// every D2Q37 kernel set.  The Newton-solved sets are compiled in translation units of their
// own (k_d2q37_n64.cu: FP64 Newton; k_d2q37_n32_*.cu: FP32 Newton, one per storage format).
#include "d2q37.cuh"

namespace lbm {

extern template KernelSet make_set<D2Q37N<false>, ST_F64, 16, 16, 1>();
extern template KernelSet make_set<D2Q37N<false>, ST_F32, 16, 16, 1>();
extern template KernelSet make_set<D2Q37N<false>, ST_F16DEV, 16, 16, 1>();
extern template KernelSet make_set<D2Q37N<true>, ST_F64, 16, 16, 1>();
extern template KernelSet make_set<D2Q37N<true>, ST_F32, 16, 16, 1>();
extern template KernelSet make_set<D2Q37N<true>, ST_F16DEV, 16, 16, 1>();
cudaError_t upload_tables_d2q37_n64(const double*, const double*, double);
cudaError_t upload_tables_d2q37_n32_f64(const double*, const double*, double);
cudaError_t upload_tables_d2q37_n32_f32(const double*, const double*, double);
cudaError_t upload_tables_d2q37_n32_f16(const double*, const double*, double);

// batched equilibrium solve: samples (u_x, u_y, T), guess 1 zero, 2 polynomial, 3 network
__global__ void __launch_bounds__(128) k_newton_batch37(const double* __restrict__ uT, long long n, ModelDev m,
                                                        double* __restrict__ lam_out, int* __restrict__ iters) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double ux = uT[3 * i], uy = uT[3 * i + 1], Tt = uT[3 * i + 2];
    double lam[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (m.guess == 2) poly_guess37<double>(ux, uy, Tt, lam);
    else if (m.guess == 3) mlp_guess<double>(m.mlp, m.T0, m.mlp_m, m.mlp_s, ux, uy, Tt, lam);
    double e[37];
    int conv = 0;
    const int it = newton_solve<37>(ux, uy, Tt, lam, e, m.newton_tol, m.newton_max_iter, &conv);
#pragma unroll
    for (int a2 = 0; a2 < 8; ++a2) lam_out[8 * i + a2] = lam[a2];
    iters[i] = conv ? it : -1;
}

void launch_newton_batch_d2q37(const double* uT, long long n, const ModelDev& m, double* lam, int* iters, cudaStream_t s) {
    if (n) k_newton_batch37<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(uT, n, m, lam, iters);
}

template <bool N32>
static bool numerical_set(int storage, KernelSet& out) {
    switch (storage) {
        case ST_F64: out = make_set<D2Q37N<N32>, ST_F64, 16, 16, 1>(); return true;
        case ST_F32: out = make_set<D2Q37N<N32>, ST_F32, 16, 16, 1>(); return true;
        case ST_F16DEV: out = make_set<D2Q37N<N32>, ST_F16DEV, 16, 16, 1>(); return true;
    }
    return false;
}

bool find_kernels_d2q37(int model, int storage, const int* blk, bool newton_fp32, KernelSet& out) {
    if (blk[0] != 16 || blk[1] != 16 || blk[2] != 1) return false;
    if (model == 4) return newton_fp32 ? numerical_set<true>(storage, out) : numerical_set<false>(storage, out);
    if (model == 3) return pick_storage<D2Q37M, 16, 16, 1>(storage, out);
    return false;
}

cudaError_t upload_tables_d2q37(const double* w37, const double* H37, double cs2_37) {
    cudaError_t e = upload37_here(w37, H37, cs2_37);
    if (e == cudaSuccess) e = upload_tables_d2q37_n64(w37, H37, cs2_37);
    if (e == cudaSuccess) e = upload_tables_d2q37_n32_f64(w37, H37, cs2_37);
    if (e == cudaSuccess) e = upload_tables_d2q37_n32_f32(w37, H37, cs2_37);
    if (e == cudaSuccess) e = upload_tables_d2q37_n32_f16(w37, H37, cs2_37);
    return e;
}

}  // namespace lbm
