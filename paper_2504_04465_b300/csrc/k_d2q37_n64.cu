// D2Q37 kernel set of the numerical (max-entropy) equilibrium with the FP64 Newton, every storage format;
// see d2q37.cuh.
#include "d2q37.cuh"

namespace lbm {

template KernelSet make_set<D2Q37N<false>, ST_F64, 16, 16, 1>();
template KernelSet make_set<D2Q37N<false>, ST_F32, 16, 16, 1>();
template KernelSet make_set<D2Q37N<false>, ST_F16DEV, 16, 16, 1>();

cudaError_t upload_tables_d2q37_n64(const double* w37, const double* H37, double cs2_37) {
    return upload37_here(w37, H37, cs2_37);
}

}  // namespace lbm
