// D3Q27 weakly compressible BGK and recursive-regularized kernels (Appendix A of
// arXiv 2504.04465; the D3Q27 basis is every Hermite tensor with each axis at most twice).
#include "kernels_impl.cuh"

namespace lbm {

// RR_: recursive regularization, else BGK; VAR_: WV_TRT (two relaxation times, with BGK's
// equilibrium) or WV_TRACE (RR with the trace of Pi equilibrated), see models.cuh
template <bool RR_, int VAR_ = WV_PLAIN> struct D3Q27M {
    static constexpr int VAR = VAR_;
    static constexpr bool AA = VAR_ == WV_PLAIN;   // compile the AA-pattern (in-place) kernels
    static constexpr int D = 3, Q = 27;
    // resident 128-thread blocks per SM the step kernels are compiled for (simple / other blocks)
    static constexpr int MINB_FAST = 6, MINB_GEN = 6;
    static constexpr bool TUNE = VAR_ == WV_PLAIN;   // compile occupancy variants for the autotuner
    static constexpr int TUNE_V[3] = {88, 86, 66};   // their targets, 10 * interior + general
    static constexpr bool BATCH = false; // compile the batched multi-case launch
    static constexpr bool DEV = true;
    static constexpr bool HAS_G = false, HAS_LAM = false, RR = RR_;
    __host__ __device__ static constexpr int cx(int q) { return TP<3>::cx(q); }
    __host__ __device__ static constexpr int cy(int q) { return TP<3>::cy(q); }
    __host__ __device__ static constexpr int cz(int q) { return TP<3>::cz(q); }
    __host__ __device__ static constexpr double w(int q) { return tp_w<3>(q); }
    __host__ __device__ static constexpr float wf(int q) { return float(tp_w<3>(q)); }
    __host__ __device__ static constexpr float inv_wf(int q) { return float(1.0 / tp_w<3>(q)); }
};

bool find_kernels_d3q27(int model, int storage, const int* blk, KernelSet& out) {
    if (model == LBM_TRT || model == KMODEL_RR_TRACE) {
        // FP64 and FP32 storage, 8 x 4 x 4 blocks
        if (blk[0] != 8 || blk[1] != 4 || blk[2] != 4 || (storage != ST_F64 && storage != ST_F32)) return false;
        return model == LBM_TRT ? pick_storage<D3Q27M<false, WV_TRT>, 8, 4, 4>(storage, out)
                                : pick_storage<D3Q27M<true, WV_TRACE>, 8, 4, 4>(storage, out);
    }
    if (blk[0] == 8 && blk[1] == 4 && blk[2] == 4) {
        if (model == 1) return pick_storage<D3Q27M<false>, 8, 4, 4>(storage, out);
        if (model == 2) return pick_storage<D3Q27M<true>, 8, 4, 4>(storage, out);
    }
    if (blk[0] == 16 && blk[1] == 4 && blk[2] == 2 && model == 2) return pick_storage<D3Q27M<true>, 16, 4, 2>(storage, out);
    if (blk[0] == 8 && blk[1] == 8 && blk[2] == 2 && model == 2) return pick_storage<D3Q27M<true>, 8, 8, 2>(storage, out);
    return false;
}

}  // namespace lbm
