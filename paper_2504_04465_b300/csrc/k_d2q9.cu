// D2Q9 weakly compressible BGK and recursive-regularized kernels (Appendix A of
// arXiv 2504.04465); see kernels_impl.cuh and models.cuh.
#include "kernels_impl.cuh"

namespace lbm {

template <bool RR_> struct D2Q9M {
    static constexpr int D = 2, Q = 9;
    // resident 128-thread blocks per SM the step kernels are compiled for (simple / other blocks)
    static constexpr int MINB_FAST = 12, MINB_GEN = 6;
    static constexpr bool TUNE = true;      // compile occupancy variants for the autotuner
    static constexpr int TUNE_V[3] = {84, 86, 66};   // their targets, 10 * interior + general
    static constexpr bool BATCH = true;  // compile the batched multi-case launch
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
