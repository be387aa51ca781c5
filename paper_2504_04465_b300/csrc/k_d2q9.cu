// D2Q9 weakly compressible BGK and recursive-regularized kernels (Appendix A of
// arXiv 2504.04465); see kernels_impl.cuh and models.cuh.
#include "kernels_impl.cuh"

namespace lbm {

// RR_: recursive regularization, else BGK; VAR_: WV_TRT (two relaxation times, with BGK's
// equilibrium) or WV_TRACE (RR with the trace of Pi equilibrated), see models.cuh
template <bool RR_, int VAR_ = WV_PLAIN> struct D2Q9M {
    static constexpr int VAR = VAR_;
    static constexpr bool AA = VAR_ == WV_PLAIN;   // compile the AA-pattern (in-place) kernels
    static constexpr int D = 2, Q = 9;
    // resident 128-thread blocks per SM the step kernels are compiled for (simple / other blocks)
    static constexpr int MINB_FAST = 12, MINB_GEN = 6;
    static constexpr bool TUNE = VAR_ == WV_PLAIN;   // compile occupancy variants for the autotuner
    static constexpr int TUNE_V[3] = {84, 86, 66};   // their targets, 10 * interior + general
    static constexpr bool BATCH = VAR_ == WV_PLAIN;  // compile the batched multi-case launch
    static constexpr bool DEV = true;
    static constexpr bool HAS_G = false, HAS_LAM = false, RR = RR_;
    __host__ __device__ static constexpr int cx(int q) { return TP<2>::cx(q); }
    __host__ __device__ static constexpr int cy(int q) { return TP<2>::cy(q); }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr double w(int q) { return tp_w<2>(q); }
    __host__ __device__ static constexpr float wf(int q) { return float(tp_w<2>(q)); }
    __host__ __device__ static constexpr float inv_wf(int q) { return float(1.0 / tp_w<2>(q)); }
};

bool find_kernels_d2q9(int model, int storage, const int* blk, KernelSet& out) {
    if (blk[2] != 1) return false;
    if (model == LBM_TRT || model == KMODEL_RR_TRACE) {
        // FP64 and FP32 storage, 16 x 16 blocks
        if (blk[0] != 16 || blk[1] != 16 || (storage != ST_F64 && storage != ST_F32)) return false;
        return model == LBM_TRT ? pick_storage<D2Q9M<false, WV_TRT>, 16, 16, 1>(storage, out)
                                : pick_storage<D2Q9M<true, WV_TRACE>, 16, 16, 1>(storage, out);
    }
    if (blk[0] == 16 && blk[1] == 16) {
        if (model == 1) return pick_storage<D2Q9M<false>, 16, 16, 1>(storage, out);
        if (model == 2) return pick_storage<D2Q9M<true>, 16, 16, 1>(storage, out);
    }
    if (blk[0] == 32 && blk[1] == 8) {
        if (model == 1) return pick_storage<D2Q9M<false>, 32, 8, 1>(storage, out);
        if (model == 2) return pick_storage<D2Q9M<true>, 32, 8, 1>(storage, out);
    }
    return false;
}

}  // namespace lbm
