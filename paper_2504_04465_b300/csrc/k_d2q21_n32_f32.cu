// D2Q21 kernel set of the numerical (max-entropy) equilibrium with the FP32 Newton, FP32 populations;
// see d2q21.cuh.
#include "d2q21.cuh"

namespace lbm {

template KernelSet make_set<D2Q21M<true>, ST_F32, 16, 16, 1>();

cudaError_t upload_tables_d2q21_n32_f32(const double* w21, const double* H21) { return upload21_here(w21, H21); }

}  // namespace lbm
